// Geometric multigrid V-cycle for the periodic Poisson problem: the preconditioner M ~ A^-1 of the
// FP32 AAR correction solves, A = -L_h the order-12 finite-difference Laplacian (paper Sec. 2.1:
// the electrostatic potential from a Poisson problem solved by AAR with matrix-free stencil
// Laplacian-vector products; the paper does not fix AAR's preconditioner, the plain choice being
// the Jacobi scaling 1 / diag A).
//
// M applies one V-cycle of the second-order (7-point) Laplacian A2 on a hierarchy of grids that
// halves every dimension while it is even: red-black Gauss-Seidel smoothing, full-weighting
// restriction of the residual, trilinear prolongation, and on the coarsest grid (at most 512
// points, or up to 16 384 when a dimension turns odd earlier) a fixed number of Chebyshev iterations for the known spectrum of A2 run by one CTA out
// of shared memory.  A2 and A share their low-frequency spectrum; at the highest grid frequency the
// order-12 symbol is about 2.5 times the second-order one, so the preconditioned operator M A
// keeps its eigenvalues in a small interval and AAR reaches a 1e-3 reduction in a few iterations
// instead of the hundreds the Jacobi scaling needs (its iteration count grows with the grid).
//
// Every grid is periodic, so A2 is singular with the constants as null space.  The right-hand
// sides the V-cycle sees have zero mean (residuals of a zero-mean problem; full weighting keeps
// the mean), and no smoothing or Chebyshev step adds a constant, so no projection is needed.
#include "internal.cuh"

#include <algorithm>
#include <cmath>
#include <cstdlib>

namespace sdft {
namespace {

struct MgDims {
    int n1, n2, n3;
    float w1, w2, w3;   // 1 / h_d^2 of the level
    float diag;         // 2 (w1 + w2 + w3)
};

__device__ __forceinline__ int wrapi(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// (A2 x)[i, j, k] on a periodic grid
__device__ __forceinline__ float apply_a2(const float* __restrict__ x, const MgDims& d, int i, int j, int k) {
    const int rowj = (k * d.n2 + j) * d.n1;
    const float xc = x[rowj + i];
    const float sx = x[rowj + wrapi(i + 1, d.n1)] + x[rowj + wrapi(i - 1, d.n1)];
    const float sy = x[(k * d.n2 + wrapi(j + 1, d.n2)) * d.n1 + i] + x[(k * d.n2 + wrapi(j - 1, d.n2)) * d.n1 + i];
    const float sz = x[(wrapi(k + 1, d.n3) * d.n2 + j) * d.n1 + i] + x[(wrapi(k - 1, d.n3) * d.n2 + j) * d.n1 + i];
    return d.diag * xc - (d.w1 * sx + d.w2 * sy + d.w3 * sz);
}

// red-black Gauss-Seidel half sweep over the points with (i + j + k) & 1 == color (n1, n2, n3 even,
// so the six neighbours of a point all have the other colour); zero != 0: x is taken as zero
// (the first half sweep of a cycle, which then needs no cleared buffer)
__global__ void __launch_bounds__(256) mg_rbgs_kernel(float* __restrict__ x, const float* __restrict__ b, MgDims d,
                                                      int color, int zero) {
    const int half = d.n1 >> 1;
    const int npts = half * d.n2 * d.n3;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < npts; t += gridDim.x * blockDim.x) {
        const int q = t % half, row = t / half;
        const int j = row % d.n2, k = row / d.n2;
        const int i = 2 * q + ((j + k + color) & 1);
        const int g = row * d.n1 + i;
        float s = b[g];
        if (!zero) {
            const int rowj = row * d.n1;
            s += d.w1 * (x[rowj + wrapi(i + 1, d.n1)] + x[rowj + wrapi(i - 1, d.n1)]);
            s += d.w2 * (x[(k * d.n2 + wrapi(j + 1, d.n2)) * d.n1 + i] + x[(k * d.n2 + wrapi(j - 1, d.n2)) * d.n1 + i]);
            s += d.w3 * (x[(wrapi(k + 1, d.n3) * d.n2 + j) * d.n1 + i] + x[(wrapi(k - 1, d.n3) * d.n2 + j) * d.n1 + i]);
        }
        x[g] = s / d.diag;
    }
}

// b_c[I, J, K] = sum over the 27 fine points (2I + a, 2J + b, 2K + c), a, b, c in {-1, 0, 1}, of
// w_a w_b w_c (b_f - A2 x_f), w_0 = 1/2, w_+-1 = 1/4 (full weighting; the weights sum to one)
__global__ void __launch_bounds__(256) mg_restrict_kernel(const float* __restrict__ xf, const float* __restrict__ bf,
                                                          MgDims f, float* __restrict__ bc, MgDims c) {
    const int npts = c.n1 * c.n2 * c.n3;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < npts; t += gridDim.x * blockDim.x) {
        const int I = t % c.n1, row = t / c.n1;
        const int J = row % c.n2, K = row / c.n2;
        float acc = 0.f;
        for (int dk = -1; dk <= 1; ++dk) {
            const int k = wrapi(2 * K + dk, f.n3);
            const float wk = dk == 0 ? 0.5f : 0.25f;
            for (int dj = -1; dj <= 1; ++dj) {
                const int j = wrapi(2 * J + dj, f.n2);
                const float wjk = wk * (dj == 0 ? 0.5f : 0.25f);
                for (int di = -1; di <= 1; ++di) {
                    const int i = wrapi(2 * I + di, f.n1);
                    const float r = bf[(k * f.n2 + j) * f.n1 + i] - apply_a2(xf, f, i, j, k);
                    acc += wjk * (di == 0 ? 0.5f : 0.25f) * r;
                }
            }
        }
        bc[t] = acc;
    }
}

// x_f += P x_c: trilinear interpolation, fine point 2I + 1 between coarse points I and I + 1
__global__ void __launch_bounds__(256) mg_prolong_kernel(float* __restrict__ xf, MgDims f, const float* __restrict__ xc,
                                                         MgDims c) {
    const int npts = f.n1 * f.n2 * f.n3;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < npts; t += gridDim.x * blockDim.x) {
        const int i = t % f.n1, row = t / f.n1;
        const int j = row % f.n2, k = row / f.n2;
        const int i0 = i >> 1, j0 = j >> 1, k0 = k >> 1;
        const int i1 = (i & 1) ? wrapi(i0 + 1, c.n1) : i0;
        const int j1 = (j & 1) ? wrapi(j0 + 1, c.n2) : j0;
        const int k1 = (k & 1) ? wrapi(k0 + 1, c.n3) : k0;
        auto at = [&](int a, int b_, int cc) { return xc[(cc * c.n2 + b_) * c.n1 + a]; };
        const float v = 0.125f * (at(i0, j0, k0) + at(i1, j0, k0) + at(i0, j1, k0) + at(i1, j1, k0) + at(i0, j0, k1) +
                                  at(i1, j0, k1) + at(i0, j1, k1) + at(i1, j1, k1));
        xf[t] += v;
    }
}

// coarsest grid: K Chebyshev iterations for A2 x = b from x = 0, for the spectrum [lmin, lmax] of A2
// without its zero eigenvalue (Saad, Iterative Methods for Sparse Linear Systems, Algorithm 12.1),
// one CTA, x and the step d in shared memory
__global__ void __launch_bounds__(1024) mg_coarse_kernel(float* __restrict__ x, const float* __restrict__ b, MgDims d,
                                                         float lmin, float lmax, int K) {
    extern __shared__ float sm[];
    const int n = d.n1 * d.n2 * d.n3;
    float* xs = sm;
    float* ds = sm + n;
    const float theta = 0.5f * (lmax + lmin), delta = 0.5f * (lmax - lmin);
    const float sigma1 = theta / delta;
    for (int p = threadIdx.x; p < n; p += blockDim.x) {
        ds[p] = b[p] / theta;
        xs[p] = ds[p];
    }
    float rho = 1.f / sigma1;
    for (int it = 1; it < K; ++it) {
        __syncthreads();
        const float rho1 = 1.f / (2.f * sigma1 - rho);
        for (int p = threadIdx.x; p < n; p += blockDim.x) {
            const int i = p % d.n1, row = p / d.n1;
            const int j = row % d.n2, k = row / d.n2;
            const float r = b[p] - apply_a2(xs, d, i, j, k);
            ds[p] = rho1 * rho * ds[p] + (2.f * rho1 / delta) * r;
        }
        __syncthreads();
        for (int p = threadIdx.x; p < n; p += blockDim.x) xs[p] += ds[p];
        rho = rho1;
    }
    __syncthreads();
    for (int p = threadIdx.x; p < n; p += blockDim.x) x[p] = xs[p];
}

MgDims dims_of(const MgLevel& L) {
    MgDims d;
    d.n1 = L.n[0];
    d.n2 = L.n[1];
    d.n3 = L.n[2];
    d.w1 = (float)L.w[0];
    d.w2 = (float)L.w[1];
    d.w3 = (float)L.w[2];
    d.diag = (float)(2.0 * (L.w[0] + L.w[1] + L.w[2]));
    return d;
}

unsigned mg_blocks(long long work) { return (unsigned)std::max<long long>(1, std::min<long long>((work + 255) / 256, 152LL * 8)); }

constexpr int MG_COARSE_STOP = 512;    // coarsening stops once a grid has at most this many points
constexpr int MG_COARSE_MAX = 16384;   // largest coarsest grid (x and d in shared memory)
constexpr int MG_NU = 1;               // red-black sweeps before and after the coarse correction

}  // namespace

// Level hierarchy of the context's grid: level 0 is the fine grid (its x and b are the V-cycle's
// output and input, supplied per call); each further level halves all three dimensions, until a
// grid has at most MG_COARSE_STOP points or a dimension is odd.  Returns false (no multigrid)
// unless there is at least one coarse level and the coarsest has at most MG_COARSE_MAX points.
bool mg_setup(sdft_ctx* c) {
    c->mg.clear();
    MgLevel L0;
    for (int d = 0; d < 3; ++d) {
        L0.n[d] = c->n[d];
        L0.w[d] = 1.0 / (c->h[d] * c->h[d]);
    }
    L0.np = c->ng;
    std::vector<MgLevel> lv{L0};
    while (true) {
        const MgLevel& f = lv.back();
        if (f.np <= MG_COARSE_STOP) break;
        bool even = true;
        for (int d = 0; d < 3; ++d) even = even && f.n[d] % 2 == 0 && f.n[d] >= 4;
        if (!even) break;
        MgLevel g;
        for (int d = 0; d < 3; ++d) {
            g.n[d] = f.n[d] / 2;
            g.w[d] = f.w[d] / 4.0;
        }
        g.np = (long long)g.n[0] * g.n[1] * g.n[2];
        lv.push_back(g);
    }
    if (lv.size() < 2 || lv.back().np > MG_COARSE_MAX || c->ng >= (1LL << 30)) return false;
    long long tot = 0;
    for (size_t l = 1; l < lv.size(); ++l) tot += 2 * lv[l].np;
    float* buf = (float*)ctx_alloc(c, sizeof(float) * (size_t)tot);
    for (size_t l = 1; l < lv.size(); ++l) {
        lv[l].x = buf;
        lv[l].b = buf + lv[l].np;
        buf += 2 * lv[l].np;
    }
    // coarsest grid: spectrum of the periodic 7-point operator, sum_d 4 w_d sin^2(pi m_d / n_d)
    MgLevel& cl = lv.back();
    double lmax = 0.0, lmin = 1e300;
    for (int d = 0; d < 3; ++d) {
        const double s = std::sin(M_PI * (cl.n[d] / 2) / cl.n[d]);
        lmax += 4.0 * cl.w[d] * s * s;
        const double s1 = std::sin(M_PI / cl.n[d]);
        if (cl.n[d] > 1) lmin = std::min(lmin, 4.0 * cl.w[d] * s1 * s1);
    }
    c->mg_lmin = lmin;
    c->mg_lmax = lmax;
    // iterations for a 1e-1 error bound, 2 q^K <= 1e-1 with q = (sqrt(k) - 1) / (sqrt(k) + 1): as a
    // preconditioner the V-cycle needs no accurate coarse solve (tighter bounds did not reduce the
    // AAR iteration count in a model of the solver)
    const double sk = std::sqrt(lmax / lmin), q = (sk - 1.0) / (sk + 1.0);
    c->mg_coarse_iters = q <= 0.0 ? 1 : std::min(64, std::max(2, (int)std::ceil(std::log(5e-2) / std::log(q))));
    // the attribute belongs to the kernel, not to this context: allow the largest coarsest grid of any
    // context, so that a context created later with a smaller one does not lower it for this one
    SDFT_CUDA(cudaFuncSetAttribute(mg_coarse_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)(sizeof(float) * 2 * MG_COARSE_MAX)));
    c->mg = lv;
    return true;
}

namespace {
// the V-cycle's launches (level 0 uses r and z in place of its own b and x)
void mg_enqueue(sdft_ctx* c, const float* r, float* z) {
    const int nl = (int)c->mg.size();
    SDFT_REQUIRE(nl >= 2, SDFT_ERR_INVALID_ARG, "multigrid V-cycle without a hierarchy");
    auto xb = [&](int l, float** x, const float** b) {
        *x = l == 0 ? z : c->mg[l].x;
        *b = l == 0 ? r : c->mg[l].b;
    };
    for (int l = 0; l + 1 < nl; ++l) {
        float* x;
        const float* b;
        xb(l, &x, &b);
        const MgDims d = dims_of(c->mg[l]);
        const unsigned nbh = mg_blocks(c->mg[l].np / 2);
        for (int s = 0; s < MG_NU; ++s) {
            mg_rbgs_kernel<<<nbh, 256, 0, c->stream>>>(x, b, d, 0, s == 0 ? 1 : 0);
            mg_rbgs_kernel<<<nbh, 256, 0, c->stream>>>(x, b, d, 1, 0);
        }
        mg_restrict_kernel<<<mg_blocks(c->mg[l + 1].np), 256, 0, c->stream>>>(x, b, d, c->mg[l + 1].b,
                                                                                 dims_of(c->mg[l + 1]));
        count_launch(c, 2 * MG_NU + 1);
    }
    {
        const MgLevel& cl = c->mg[nl - 1];
        const size_t smem = sizeof(float) * 2 * (size_t)cl.np;
        mg_coarse_kernel<<<1, 1024, smem, c->stream>>>(cl.x, cl.b, dims_of(cl), (float)c->mg_lmin, (float)c->mg_lmax,
                                                        c->mg_coarse_iters);
        count_launch(c);
    }
    for (int l = nl - 2; l >= 0; --l) {
        float* x;
        const float* b;
        xb(l, &x, &b);
        const MgDims d = dims_of(c->mg[l]);
        mg_prolong_kernel<<<mg_blocks(c->mg[l].np), 256, 0, c->stream>>>(x, d, c->mg[l + 1].x, dims_of(c->mg[l + 1]));
        const unsigned nbh = mg_blocks(c->mg[l].np / 2);
        for (int s = 0; s < MG_NU; ++s) {
            mg_rbgs_kernel<<<nbh, 256, 0, c->stream>>>(x, b, d, 1, 0);
            mg_rbgs_kernel<<<nbh, 256, 0, c->stream>>>(x, b, d, 0, 0);
        }
        count_launch(c, 2 * MG_NU + 1);
    }
    SDFT_CUDA(cudaGetLastError());
}
}  // namespace

// z = M r: one V-cycle from a zero start.  The V-cycle is some twenty small launches, most of them on
// grids of a few thousand points, so it is captured once into a CUDA graph (for the context's r and
// z buffers) and replayed; SDFT_MG_GRAPH=0 launches the kernels one by one.
void mg_vcycle(sdft_ctx* c, const float* r, float* z) {
    static const bool use_graph = [] {
        const char* env = getenv("SDFT_MG_GRAPH");
        return env == nullptr || atoi(env) != 0;
    }();
    if (!use_graph) {
        mg_enqueue(c, r, z);
        return;
    }
    if (c->mg_graph && (c->mg_graph_r != r || c->mg_graph_z != z)) {
        cudaGraphExecDestroy(c->mg_graph);
        c->mg_graph = nullptr;
    }
    if (!c->mg_graph) {
        const uint64_t l0 = c->launches;
        cudaGraph_t graph = nullptr;
        // capture on the private stream (the context's stream may be the legacy default stream)
        if (!c->cap_stream) SDFT_CUDA(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
        cudaStream_t user_stream = c->stream;
        c->stream = c->cap_stream;
        SDFT_CUDA(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
        try {
            mg_enqueue(c, r, z);
        } catch (...) {
            cudaStreamEndCapture(c->stream, &graph);
            if (graph) cudaGraphDestroy(graph);
            c->stream = user_stream;
            throw;
        }
        const cudaError_t ce = cudaStreamEndCapture(c->stream, &graph);
        c->stream = user_stream;
        SDFT_CUDA(ce);
        const cudaError_t ie = cudaGraphInstantiate(&c->mg_graph, graph, 0);
        cudaGraphDestroy(graph);
        SDFT_CUDA(ie);
        c->mg_graph_launches = (int)(c->launches - l0);
        c->launches = l0;
        c->mg_graph_r = r;
        c->mg_graph_z = z;
    }
    SDFT_CUDA(cudaGraphLaunch(c->mg_graph, c->stream));
    count_launch(c, c->mg_graph_launches);
}

}  // namespace sdft
