// Kleinman-Bylander projector tables (paper Sec. 2.1: nonlocal pseudopotential applied through
// its "outer product nature").  For every atom a, the support of
//   beta_a(x) = sum_T exp(i k.T) chi(x - R_a - T),  chi(r) = (pi^1.5 r_p^3)^-1/2 exp(-r^2/(2 r_p^2)),
// restricted to r < r_c, is enumerated over the unwrapped grid box around R_a: box point I
// (integer, unwrapped) is grid point g = I mod n seen from image T = -floor(I/n) L.
// Two tables are built on the device:
//   * atom-major lists (idx, value) in box order, used by the projection C = beta^H Y;
//   * a per-grid-point slot table (atom, value) sorted by atom, used by the scatter inside
//     the stencil kernel, so that H Y needs no atomics.
#include "internal.cuh"

#include <algorithm>
#include <cmath>

namespace sdft {
namespace {

struct AtomBox {
    int lo[3];
    int dim[3];
    double pos[3];
    double rp, rc;
};

__global__ void atom_support_kernel(const AtomBox* __restrict__ boxes, int cap, int n1, int n2, int n3,
                                    double h1, double h2, double h3, double k1, double k2, double k3,
                                    int cplx, int* __restrict__ cnt, int* __restrict__ idx,
                                    int* __restrict__ img, double* __restrict__ val64,
                                    float* __restrict__ val32, int isolated) {
    const int a = blockIdx.x;
    const AtomBox B = boxes[a];
    const int total = B.dim[0] * B.dim[1] * B.dim[2];
    const double norm = rsqrt(pow(M_PI, 1.5) * B.rp * B.rp * B.rp);
    __shared__ int warp_tot[32];
    __shared__ int base;
    if (threadIdx.x == 0) base = 0;
    __syncthreads();
    for (int start = 0; start < total; start += blockDim.x) {
        const int p = start + threadIdx.x;
        bool keep = false;
        int I[3] = {0, 0, 0};
        double r2 = 0.0;
        if (p < total) {
            int rem = p;
            const int ix = rem % B.dim[0];
            rem /= B.dim[0];
            const int iy = rem % B.dim[1];
            const int iz = rem / B.dim[1];
            I[0] = B.lo[0] + ix;
            I[1] = B.lo[1] + iy;
            I[2] = B.lo[2] + iz;
            const double dx = I[0] * h1 - B.pos[0], dy = I[1] * h2 - B.pos[1], dz = I[2] * h3 - B.pos[2];
            r2 = dx * dx + dy * dy + dz * dz;
            keep = r2 < B.rc * B.rc;
            // an isolated cell has no periodic images: points beyond the grid are not wrapped back in
            if (isolated && (I[0] < 0 || I[0] >= n1 || I[1] < 0 || I[1] >= n2 || I[2] < 0 || I[2] >= n3)) keep = false;
        }
        // ordered compaction: warp ballot + prefix over warps
        const unsigned ballot = __ballot_sync(0xffffffffu, keep);
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        const int before = __popc(ballot & ((1u << lane) - 1u));
        if (lane == 0) warp_tot[warp] = __popc(ballot);
        __syncthreads();
        int off = 0, all = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            if (w < warp) off += warp_tot[w];
            all += warp_tot[w];
        }
        if (keep) {
            const int slot = base + off + before;
            int t[3], g[3];
            const int nn[3] = {n1, n2, n3};
            for (int d = 0; d < 3; ++d) {
                int q = I[d] / nn[d];
                int r = I[d] - q * nn[d];
                if (r < 0) { r += nn[d]; --q; }
                g[d] = r;
                t[d] = q;
            }
            const long long e = (long long)a * cap + slot;
            idx[e] = (int)(((long long)g[2] * n2 + g[1]) * n1 + g[0]);
            img[e] = ((t[0] + 512) & 1023) | (((t[1] + 512) & 1023) << 10) | (((t[2] + 512) & 1023) << 20);
            const double chi = norm * exp(-r2 / (2.0 * B.rp * B.rp));
            if (cplx) {
                // image T = -t L: phase exp(i k.T) = exp(-2 pi i kappa.t)
                const double ang = -2.0 * M_PI * (k1 * t[0] + k2 * t[1] + k3 * t[2]);
                double s, c;
                sincos(ang, &s, &c);
                val64[2 * e] = chi * c;
                val64[2 * e + 1] = chi * s;
                val32[2 * e] = (float)(chi * c);
                val32[2 * e + 1] = (float)(chi * s);
            } else {
                val64[e] = chi;
                val32[e] = (float)chi;
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) base += all;
        __syncthreads();
    }
    if (threadIdx.x == 0) cnt[a] = base;
}

__global__ void point_count_kernel(const int* __restrict__ cnt, const int* __restrict__ idx, int cap,
                                   int* __restrict__ pcnt) {
    const int a = blockIdx.x;
    for (int j = threadIdx.x; j < cnt[a]; j += blockDim.x) atomicAdd(&pcnt[idx[(long long)a * cap + j]], 1);
}

__global__ void point_fill_kernel(const int* __restrict__ cnt, const int* __restrict__ idx,
                                  const double* __restrict__ val64, const float* __restrict__ val32, int cap,
                                  int cplx, long long ng, int S, int* __restrict__ pfill,
                                  int* __restrict__ patom, double* __restrict__ pval64,
                                  float* __restrict__ pval32) {
    const int a = blockIdx.x;
    for (int j = threadIdx.x; j < cnt[a]; j += blockDim.x) {
        const long long e = (long long)a * cap + j;
        const int g = idx[e];
        const int s = atomicAdd(&pfill[g], 1);
        if (s >= S) continue;  // cannot happen: S is the counted maximum
        const long long q = (long long)s * ng + g;
        patom[q] = a;
        if (cplx) {
            pval64[2 * q] = val64[2 * e];
            pval64[2 * q + 1] = val64[2 * e + 1];
            pval32[2 * q] = val32[2 * e];
            pval32[2 * q + 1] = val32[2 * e + 1];
        } else {
            pval64[q] = val64[e];
            pval32[q] = val32[e];
        }
    }
}

// sort each point's slots by (atom, value) so the scatter sums in a fixed order
__global__ void point_sort_kernel(const int* __restrict__ pcnt, long long ng, int cplx,
                                  int* __restrict__ patom, double* __restrict__ pval64,
                                  float* __restrict__ pval32) {
    const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (g >= ng) return;
    const int m = pcnt[g];
    for (int i = 1; i < m; ++i) {
        for (int j = i; j > 0; --j) {
            const long long p = (long long)j * ng + g, q = (long long)(j - 1) * ng + g;
            const double vp = cplx ? pval64[2 * p] : pval64[p];
            const double vq = cplx ? pval64[2 * q] : pval64[q];
            const bool swap = patom[p] < patom[q] || (patom[p] == patom[q] && vp < vq);
            if (!swap) break;
            int ta = patom[p];
            patom[p] = patom[q];
            patom[q] = ta;
            if (cplx) {
                for (int k = 0; k < 2; ++k) {
                    double t = pval64[2 * p + k];
                    pval64[2 * p + k] = pval64[2 * q + k];
                    pval64[2 * q + k] = t;
                    float f = pval32[2 * p + k];
                    pval32[2 * p + k] = pval32[2 * q + k];
                    pval32[2 * q + k] = f;
                }
            } else {
                double t = pval64[p];
                pval64[p] = pval64[q];
                pval64[q] = t;
                float f = pval32[p];
                pval32[p] = pval32[q];
                pval32[q] = f;
            }
        }
    }
}

__global__ void max_kernel(const int* __restrict__ v, long long n, int* __restrict__ out) {
    int m = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        m = max(m, v[i]);
    for (int off = 16; off > 0; off >>= 1) m = max(m, __shfl_down_sync(0xffffffffu, m, off));
    if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

}  // namespace

void build_kb_tables(sdft_ctx* c, int kpt) {
    KBTables& T = c->kb[kpt];
    T.natom = c->natom;
    double kred[3] = {0, 0, 0};
    if (!c->kpts.empty())
        for (int d = 0; d < 3; ++d) kred[d] = c->kpts[3 * kpt + d];
    T.cplx = kred[0] != 0.0 || kred[1] != 0.0 || kred[2] != 0.0;
    std::vector<AtomBox> boxes(c->natom);
    int cap = 0;
    for (int a = 0; a < c->natom; ++a) {
        const sdft_pseudo& s = c->species[c->types[a]];
        AtomBox& B = boxes[a];
        for (int d = 0; d < 3; ++d) {
            B.pos[d] = c->pos[3 * a + d];
            B.lo[d] = (int)std::ceil((B.pos[d] - s.r_cut_proj) / c->h[d]);
            const int hi = (int)std::floor((B.pos[d] + s.r_cut_proj) / c->h[d]);
            B.dim[d] = std::max(0, hi - B.lo[d] + 1);
        }
        B.rp = s.r_proj;
        B.rc = s.r_cut_proj;
        cap = std::max(cap, B.dim[0] * B.dim[1] * B.dim[2]);
    }
    T.cap = std::max(cap, 1);
    const size_t ent = (size_t)c->natom * T.cap;
    const int vw = T.cplx ? 2 : 1;
    T.cnt = (int*)ctx_alloc(c, sizeof(int) * std::max(1, c->natom));
    T.idx = (int*)ctx_alloc(c, sizeof(int) * ent);
    T.img = (int*)ctx_alloc(c, sizeof(int) * ent);
    T.val64 = (double*)ctx_alloc(c, sizeof(double) * ent * vw);
    T.val32 = (float*)ctx_alloc(c, sizeof(float) * ent * vw);
    T.gamma = (double*)ctx_alloc(c, sizeof(double) * std::max(1, c->natom));
    std::vector<double> gam(c->natom);
    for (int a = 0; a < c->natom; ++a) gam[a] = c->species[c->types[a]].E_kb * c->dV;
    AtomBox* dboxes = (AtomBox*)ctx_alloc(c, sizeof(AtomBox) * std::max(1, c->natom));
    if (c->natom > 0) {
        SDFT_CUDA(cudaMemcpyAsync(T.gamma, gam.data(), sizeof(double) * c->natom, cudaMemcpyHostToDevice, c->stream));
        SDFT_CUDA(cudaMemcpyAsync(dboxes, boxes.data(), sizeof(AtomBox) * c->natom, cudaMemcpyHostToDevice, c->stream));
        atom_support_kernel<<<c->natom, 256, 0, c->stream>>>(dboxes, T.cap, c->n[0], c->n[1], c->n[2], c->h[0], c->h[1],
                                                            c->h[2], kred[0], kred[1], kred[2], T.cplx, T.cnt, T.idx,
                                                            T.img, T.val64, T.val32,
                                                            c->opt.boundary == SDFT_BC_DIRICHLET);
        SDFT_CUDA(cudaGetLastError());
        count_launch(c);
    }
    // per-point slot table
    T.pcnt = (int*)ctx_alloc(c, sizeof(int) * c->ng);
    SDFT_CUDA(cudaMemsetAsync(T.pcnt, 0, sizeof(int) * c->ng, c->stream));
    int S = 0;
    if (c->natom > 0) {
        point_count_kernel<<<c->natom, 256, 0, c->stream>>>(T.cnt, T.idx, T.cap, T.pcnt);
        int* dmax = (int*)c->scal;
        SDFT_CUDA(cudaMemsetAsync(dmax, 0, sizeof(int), c->stream));
        max_kernel<<<256, 256, 0, c->stream>>>(T.pcnt, c->ng, dmax);
        SDFT_CUDA(cudaGetLastError());
        count_launch(c, 2);
        SDFT_CUDA(cudaMemcpyAsync(&S, dmax, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
        SDFT_CUDA(cudaStreamSynchronize(c->stream));
    }
    T.S = S;
    if (S > 0) {
        const size_t ps = (size_t)S * c->ng;
        T.patom = (int*)ctx_alloc(c, sizeof(int) * ps);
        SDFT_CUDA(cudaMemsetAsync(T.patom, 0xff, sizeof(int) * ps, c->stream));  // unused slots: atom -1
        T.pval64 = (double*)ctx_alloc(c, sizeof(double) * ps * vw);
        T.pval32 = (float*)ctx_alloc(c, sizeof(float) * ps * vw);
        int* pfill = (int*)ctx_alloc(c, sizeof(int) * c->ng);
        SDFT_CUDA(cudaMemsetAsync(pfill, 0, sizeof(int) * c->ng, c->stream));
        point_fill_kernel<<<c->natom, 256, 0, c->stream>>>(T.cnt, T.idx, T.val64, T.val32, T.cap, T.cplx, c->ng, S,
                                                          pfill, T.patom, T.pval64, T.pval32);
        point_sort_kernel<<<(unsigned)((c->ng + 255) / 256), 256, 0, c->stream>>>(T.pcnt, c->ng, T.cplx, T.patom,
                                                                                  T.pval64, T.pval32);
        SDFT_CUDA(cudaGetLastError());
        count_launch(c, 2);
        ctx_release(c, pfill);
    }
    ctx_release(c, dboxes);
}

void release_kb_tables(sdft_ctx* c, int kpt) {
    KBTables& T = c->kb[kpt];
    for (void* p : {(void*)T.cnt, (void*)T.idx, (void*)T.img, (void*)T.val64, (void*)T.val32, (void*)T.gamma,
                    (void*)T.pcnt, (void*)T.patom, (void*)T.pval64, (void*)T.pval32})
        ctx_release(c, p);
    T = KBTables{};
}

}  // namespace sdft
