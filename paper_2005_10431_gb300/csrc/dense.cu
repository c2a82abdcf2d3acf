// Dense subspace steps of CheFSI's Rayleigh-Ritz (paper Sec. 2.1; Zhou et al. 2006):
//   M = Y^H Y, Hs = Y^H (H Y)          (split-K over the grid, deterministic reduction)
//   Hs q = lambda M q                  (FP64, diagonal equilibration + cuSOLVER sygvd/hegvd)
//   X = Y Q                            (rotation)
// The paper names this subspace diagonalisation as the step that limits scaling (Sec. 4).
#include "internal.cuh"

#include <algorithm>
#include <cmath>
#include <mutex>

namespace sdft {
namespace {

// storage kinds: 0 FP64 real, 1 FP64 complex (double2), 2 FP32 paired real, 3 FP32 complex (float2)
template <int KIND> struct KindT;
template <> struct KindT<0> { using A = double; static constexpr bool cplx = false; };
template <> struct KindT<1> { using A = double; static constexpr bool cplx = true; };
template <> struct KindT<2> { using A = float; static constexpr bool cplx = false; };
template <> struct KindT<3> { using A = float; static constexpr bool cplx = true; };

template <int KIND>
__device__ __forceinline__ void ld(const void* __restrict__ p, long long g, int n, long long ng,
                                   typename KindT<KIND>::A& re, typename KindT<KIND>::A& im) {
    if (KIND == 0) {
        re = ((const double*)p)[(long long)n * ng + g];
        im = 0;
    } else if (KIND == 1) {
        const double2 v = ((const double2*)p)[(long long)n * ng + g];
        re = v.x;
        im = v.y;
    } else if (KIND == 2) {
        re = ((const float*)p)[(((long long)(n >> 1)) * ng + g) * 2 + (n & 1)];
        im = 0;
    } else {
        const float2 v = ((const float2*)p)[(long long)n * ng + g];
        re = v.x;
        im = v.y;
    }
}

template <int KIND>
__device__ __forceinline__ void st(void* __restrict__ p, long long g, int n, long long ng,
                                   typename KindT<KIND>::A re, typename KindT<KIND>::A im) {
    if (KIND == 0) {
        ((double*)p)[(long long)n * ng + g] = re;
    } else if (KIND == 1) {
        ((double2*)p)[(long long)n * ng + g] = make_double2(re, im);
    } else if (KIND == 2) {
        ((float*)p)[(((long long)(n >> 1)) * ng + g) * 2 + (n & 1)] = re;
    } else {
        ((float2*)p)[(long long)n * ng + g] = make_float2(re, im);
    }
}

constexpr int GT = 32;   // output tile
constexpr int GK = 32;   // k step (16 for complex FP64 to stay within 48 KB of static smem)
template <int KIND> constexpr int gram_k() { return KIND == 1 ? 16 : GK; }

// partial Gram over grid chunk blockIdx.z: part[z][which][i + j*ncol] (complex: 2 doubles)
template <int KIND>
__global__ void __launch_bounds__(256)
gram_kernel(const void* __restrict__ Y, const void* __restrict__ HY, int ncol, long long ng, long long chunk,
            double* __restrict__ part) {
    using A = typename KindT<KIND>::A;
    constexpr bool C = KindT<KIND>::cplx;
    constexpr int KS = gram_k<KIND>();
    const int ti = blockIdx.x, tj = blockIdx.y;
    if (tj < ti) return;  // upper triangle of tiles only
    const int i0 = ti * GT, j0 = tj * GT;
    const long long g0 = blockIdx.z * chunk;
    const long long g1 = min(ng, g0 + chunk);
    __shared__ A Ar[KS][GT + 1], Ai[C ? KS : 1][GT + 1], Br[KS][GT + 1], Bi[C ? KS : 1][GT + 1], Hr[KS][GT + 1],
        Hi[C ? KS : 1][GT + 1];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    // each thread: outputs (i0 + ty + 16a, j0 + tx + 16b), a, b in {0,1}
    A mr[2][2] = {{0, 0}, {0, 0}}, mi[2][2] = {{0, 0}, {0, 0}};
    A hr[2][2] = {{0, 0}, {0, 0}}, hi[2][2] = {{0, 0}, {0, 0}};
    for (long long gb = g0; gb < g1; gb += KS) {
        // load KS x GT tiles, k fastest across threads (coalesced along the grid)
        for (int e = threadIdx.x; e < KS * GT; e += 256) {
            const int kk = e % KS;
            const int cc = e / KS;
            const long long g = gb + kk;
            A ar = 0, ai = 0, br = 0, bi = 0, hr_ = 0, hi_ = 0;
            if (g < g1) {
                if (i0 + cc < ncol) ld<KIND>(Y, g, i0 + cc, ng, ar, ai);
                if (j0 + cc < ncol) {
                    ld<KIND>(Y, g, j0 + cc, ng, br, bi);
                    ld<KIND>(HY, g, j0 + cc, ng, hr_, hi_);
                }
            }
            Ar[kk][cc] = ar;
            Br[kk][cc] = br;
            Hr[kk][cc] = hr_;
            if constexpr (C) {
                Ai[kk][cc] = ai;
                Bi[kk][cc] = bi;
                Hi[kk][cc] = hi_;
            }
        }
        __syncthreads();
#pragma unroll 8
        for (int k = 0; k < KS; ++k) {
            A ar[2], ai[2], br[2], bi[2], h_r[2], h_i[2];
            for (int a = 0; a < 2; ++a) {
                ar[a] = Ar[k][ty + 16 * a];
                ai[a] = A(0);
                if constexpr (C) ai[a] = Ai[k][ty + 16 * a];
            }
            for (int b = 0; b < 2; ++b) {
                br[b] = Br[k][tx + 16 * b];
                h_r[b] = Hr[k][tx + 16 * b];
                bi[b] = h_i[b] = A(0);
                if constexpr (C) {
                    bi[b] = Bi[k][tx + 16 * b];
                    h_i[b] = Hi[k][tx + 16 * b];
                }
            }
            for (int a = 0; a < 2; ++a)
                for (int b = 0; b < 2; ++b) {
                    // conj(a) * b
                    mr[a][b] = fma(ar[a], br[b], mr[a][b]);
                    hr[a][b] = fma(ar[a], h_r[b], hr[a][b]);
                    if (C) {
                        mr[a][b] = fma(ai[a], bi[b], mr[a][b]);
                        mi[a][b] = fma(ar[a], bi[b], fma(-ai[a], br[b], mi[a][b]));
                        hr[a][b] = fma(ai[a], h_i[b], hr[a][b]);
                        hi[a][b] = fma(ar[a], h_i[b], fma(-ai[a], h_r[b], hi[a][b]));
                    }
                }
        }
        __syncthreads();
    }
    const long long nn = (long long)ncol * ncol;
    const int w = C ? 2 : 1;
    double* pm = part + (long long)blockIdx.z * 2 * nn * w;
    double* ph = pm + nn * w;
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
            const int i = i0 + ty + 16 * a, j = j0 + tx + 16 * b;
            if (i < ncol && j < ncol && j >= i) {
                const long long o = (long long)i + (long long)j * ncol;
                if (C) {
                    pm[2 * o] = mr[a][b];
                    pm[2 * o + 1] = mi[a][b];
                    ph[2 * o] = hr[a][b];
                    ph[2 * o + 1] = hi[a][b];
                } else {
                    pm[o] = mr[a][b];
                    ph[o] = hr[a][b];
                }
            }
        }
}

// sum the split-K partials (upper triangle), mirror to a full Hermitian matrix
__global__ void gram_reduce_kernel(const double* __restrict__ part, int nsplit, int ncol, int cplx,
                                   double* __restrict__ M, double* __restrict__ Hs) {
    const long long nn = (long long)ncol * ncol;
    const int w = cplx ? 2 : 1;
    for (long long o = blockIdx.x * (long long)blockDim.x + threadIdx.x; o < nn; o += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(o % ncol), j = (int)(o / ncol);
        if (j < i) continue;
        double m[2] = {0, 0}, h[2] = {0, 0};
        for (int s = 0; s < nsplit; ++s) {
            const double* pm = part + (long long)s * 2 * nn * w;
            const double* ph = pm + nn * w;
            for (int q = 0; q < w; ++q) {
                m[q] += pm[w * o + q];
                h[q] += ph[w * o + q];
            }
        }
        const long long ot = (long long)j + (long long)i * ncol;
        if (cplx) {
            M[2 * o] = m[0];
            M[2 * o + 1] = m[1];
            M[2 * ot] = m[0];
            M[2 * ot + 1] = -m[1];
            Hs[2 * o] = h[0];
            Hs[2 * o + 1] = h[1];
            Hs[2 * ot] = h[0];
            Hs[2 * ot + 1] = -h[1];
            if (i == j) {
                M[2 * o + 1] = 0.0;
                Hs[2 * o + 1] = 0.0;
            }
        } else {
            M[o] = m[0];
            M[ot] = m[0];
            Hs[o] = h[0];
            Hs[ot] = h[0];
        }
    }
}

// D^-1/2 scaling of M and Hs with D = diag(M)
__global__ void diag_kernel(const double* __restrict__ M, double* __restrict__ d, int n, int cplx) {
    const int w = cplx ? 2 : 1;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        d[i] = rsqrt(M[w * ((long long)i + (long long)i * n)]);
}

__global__ void scale_kernel(double* __restrict__ M, double* __restrict__ Hs, const double* __restrict__ d, int n,
                             int cplx) {
    const int w = cplx ? 2 : 1;
    const long long nn = (long long)n * n;
    for (long long o = blockIdx.x * (long long)blockDim.x + threadIdx.x; o < nn; o += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(o % n), j = (int)(o / n);
        const double s = d[i] * d[j];
        for (int q = 0; q < w; ++q) {
            M[w * o + q] *= s;
            Hs[w * o + q] *= s;
        }
    }
}

// Q <- D^-1/2 Q (rows)
__global__ void unscale_rows_kernel(double* __restrict__ Q, const double* __restrict__ d, int n, int cplx) {
    const int w = cplx ? 2 : 1;
    const long long nn = (long long)n * n;
    for (long long o = blockIdx.x * (long long)blockDim.x + threadIdx.x; o < nn; o += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(o % n);
        for (int q = 0; q < w; ++q) Q[w * o + q] *= d[i];
    }
}

// X = Y Q: tile 64 grid points x 32 columns, k in steps of 32
template <int KIND>
__global__ void __launch_bounds__(256)
rotate_kernel(const void* __restrict__ Y, const void* __restrict__ Q, void* __restrict__ X, int ncol, long long ng) {
    using A = typename KindT<KIND>::A;
    constexpr bool C = KindT<KIND>::cplx;
    constexpr int TG = 64, TN = 32, TK = KIND == 1 ? 16 : 32;
    __shared__ A Yr[TG][TK + 1], Yi[C ? TG : 1][TK + 1];
    __shared__ A Qr[TK][TN], Qi[C ? TK : 1][TN];
    const long long g0 = blockIdx.x * (long long)TG;
    const int n0 = blockIdx.y * TN;
    const int gl = threadIdx.x % TG;
    const int nl = (threadIdx.x / TG) * 8;
    A accr[8], acci[8];
    for (int j = 0; j < 8; ++j) accr[j] = acci[j] = 0;
    const A* Qa = (const A*)Q;
    for (int k0 = 0; k0 < ncol; k0 += TK) {
        for (int e = threadIdx.x; e < TG * TK; e += 256) {
            const int gg = e % TG, kk = e / TG;
            A re = 0, im = 0;
            if (g0 + gg < ng && k0 + kk < ncol) ld<KIND>(Y, g0 + gg, k0 + kk, ng, re, im);
            Yr[gg][kk] = re;
            if constexpr (C) Yi[gg][kk] = im;
        }
        for (int e = threadIdx.x; e < TK * TN; e += 256) {
            const int nn = e % TN, kk = e / TN;
            A re = 0, im = 0;
            if (k0 + kk < ncol && n0 + nn < ncol) {
                const long long o = (long long)(k0 + kk) + (long long)(n0 + nn) * ncol;
                if (C) {
                    re = Qa[2 * o];
                    im = Qa[2 * o + 1];
                } else {
                    re = Qa[o];
                }
            }
            Qr[kk][nn] = re;
            if constexpr (C) Qi[kk][nn] = im;
        }
        __syncthreads();
#pragma unroll 4
        for (int k = 0; k < TK; ++k) {
            const A yr = Yr[gl][k];
            A yi = A(0);
            if constexpr (C) yi = Yi[gl][k];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const A qr = Qr[k][nl + j];
                accr[j] = fma(yr, qr, accr[j]);
                if constexpr (C) {
                    const A qi = Qi[k][nl + j];
                    accr[j] = fma(-yi, qi, accr[j]);
                    acci[j] = fma(yr, qi, fma(yi, qr, acci[j]));
                }
            }
        }
        __syncthreads();
    }
    if (g0 + gl < ng)
        for (int j = 0; j < 8; ++j)
            if (n0 + nl + j < ncol) st<KIND>(X, g0 + gl, n0 + nl + j, ng, accr[j], acci[j]);
}

__global__ void to_float_kernel(const double* __restrict__ a, float* __restrict__ b, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        b[i] = (float)a[i];
}

// block conversion between MIXED and FP64 storage
template <int FROM, int TO>
__global__ void convert_kernel(const void* __restrict__ src, void* __restrict__ dst, int ncol, long long ng) {
    const long long total = (long long)ncol * ng;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
        const int n = (int)(e / ng);
        const long long g = e - (long long)n * ng;
        typename KindT<FROM>::A re, im;
        ld<FROM>(src, g, n, ng, re, im);
        st<TO>(dst, g, n, ng, (typename KindT<TO>::A)re, (typename KindT<TO>::A)im);
    }
}

inline int kind_of(int precision, bool cplx) { return precision == SDFT_FP64 ? (cplx ? 1 : 0) : (cplx ? 3 : 2); }
inline unsigned nb(long long n) { return (unsigned)std::min<long long>((n + 255) / 256, 152LL * 16); }

// ---------------------------------------------------------------------------------------
// Fixed device scratch of the allocation-free Gram entry point: the split-K partial sums live
// in this file-scope array instead of memory from cudaMalloc.  Every device that loads the
// library holds it (32 MiB) until the process exits.  In host code the symbol is only a
// stand-in; its device address is looked up once per device with cudaGetSymbolAddress.
// ---------------------------------------------------------------------------------------
constexpr size_t kNoAllocGramDoubles = size_t(1) << 22;
static __device__ __align__(256) double g_noalloc_gram_scratch[kNoAllocGramDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
double* g_noalloc_ptr[kMaxDevices] = {};

// Device address of the scratch on the current device (set-up on the first call per device).
double* noalloc_scratch() {
    int dev = 0;
    SDFT_CUDA(cudaGetDevice(&dev));
    SDFT_REQUIRE(dev >= 0 && dev < kMaxDevices, SDFT_ERR_INVALID_ARG, "device index out of range");
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        SDFT_CUDA(cudaGetSymbolAddress(&p, g_noalloc_gram_scratch));
        g_noalloc_ptr[dev] = static_cast<double*>(p);
    }
    return g_noalloc_ptr[dev];
}

}  // namespace

// M = Y^H Y, Hs = Y^H HY with the split-K partials in the fixed scratch above, on `stream`, allocating
// nothing.  Always the CUDA-core gram_kernel of the storage kind: for real mixed blocks with ncol >= 32
// subspace_gram takes the BF16x3 tensor-core path instead, and the two agree to FP32 tolerance.
void subspace_gram_noalloc(int precision, bool cplx, const void* Y, const void* HY, long long ng, int ncol,
                           double* M, double* Hs, cudaStream_t stream) {
    const int w = cplx ? 2 : 1;
    const long long nn = (long long)ncol * ncol;
    const long long per_split = 2 * nn * w;
    SDFT_REQUIRE(per_split <= (long long)kNoAllocGramDoubles, SDFT_ERR_INVALID_ARG,
                 "ncol too large for the fixed scratch of the allocation-free Gram: 2*ncol^2*(2 if complex) must be "
                 "<= 4194304 (ncol <= 1448 real, <= 1024 complex)");
    double* part = noalloc_scratch();
    const int kind = kind_of(precision, cplx);
    const int tiles = (ncol + GT - 1) / GT;
    const long long tri = (long long)tiles * (tiles + 1) / 2;
    long long nsplit = std::max<long long>(1, (4LL * 152 * 4) / std::max<long long>(1, tri));
    nsplit = std::min<long long>(nsplit, (long long)kNoAllocGramDoubles / per_split);
    nsplit = std::max<long long>(1, std::min<long long>(nsplit, (ng + GK - 1) / GK));
    long long chunk = (ng + nsplit - 1) / nsplit;
    chunk = (chunk + GK - 1) / GK * GK;
    nsplit = (ng + chunk - 1) / chunk;
    dim3 grid(tiles, tiles, (unsigned)nsplit);
    switch (kind) {
        case 0: gram_kernel<0><<<grid, 256, 0, stream>>>(Y, HY, ncol, ng, chunk, part); break;
        case 1: gram_kernel<1><<<grid, 256, 0, stream>>>(Y, HY, ncol, ng, chunk, part); break;
        case 2: gram_kernel<2><<<grid, 256, 0, stream>>>(Y, HY, ncol, ng, chunk, part); break;
        default: gram_kernel<3><<<grid, 256, 0, stream>>>(Y, HY, ncol, ng, chunk, part); break;
    }
    gram_reduce_kernel<<<nb(nn), 256, 0, stream>>>(part, (int)nsplit, ncol, cplx, M, Hs);
    SDFT_CUDA(cudaGetLastError());
}

void subspace_gram(sdft_ctx* c, int precision, bool cplx, const void* Y, const void* HY, double* M, double* Hs,
                   int ncol) {
    if (gram_tc_supported(c, precision, cplx, ncol)) {
        subspace_gram_tc(c, Y, HY, M, Hs, ncol);
        return;
    }
    const int kind = kind_of(precision, cplx);
    const int tiles = (ncol + GT - 1) / GT;
    const int w = cplx ? 2 : 1;
    const long long nn = (long long)ncol * ncol;
    // split K so that the grid has ~4 waves of CTAs, bounded by the partial buffer
    const long long tri = (long long)tiles * (tiles + 1) / 2;
    long long nsplit = std::max<long long>(1, (4LL * 152 * 4) / std::max<long long>(1, tri));
    nsplit = std::min<long long>(nsplit, (long long)(c->part_elems / (2 * nn * w)));
    nsplit = std::max<long long>(1, std::min<long long>(nsplit, (c->ng + GK - 1) / GK));
    long long chunk = (c->ng + nsplit - 1) / nsplit;
    chunk = (chunk + GK - 1) / GK * GK;
    nsplit = (c->ng + chunk - 1) / chunk;
    SDFT_REQUIRE((size_t)(nsplit * 2 * nn * w) <= c->part_elems, SDFT_ERR_INVALID_ARG, "gram: partial buffer too small");
    dim3 grid(tiles, tiles, (unsigned)nsplit);
    // algorithmic flops: two full ngrid x ncol x ncol products (M and Hs), x4 for complex
    ScopedTimer timer(c, SDFT_K_GRAM, 0.0, 4.0 * (double)c->ng * ncol * ncol * (cplx ? 4.0 : 1.0));
    switch (kind) {
        case 0: gram_kernel<0><<<grid, 256, 0, c->stream>>>(Y, HY, ncol, c->ng, chunk, c->part); break;
        case 1: gram_kernel<1><<<grid, 256, 0, c->stream>>>(Y, HY, ncol, c->ng, chunk, c->part); break;
        case 2: gram_kernel<2><<<grid, 256, 0, c->stream>>>(Y, HY, ncol, c->ng, chunk, c->part); break;
        default: gram_kernel<3><<<grid, 256, 0, c->stream>>>(Y, HY, ncol, c->ng, chunk, c->part); break;
    }
    gram_reduce_kernel<<<nb(nn), 256, 0, c->stream>>>(c->part, (int)nsplit, ncol, cplx, M, Hs);
    SDFT_CUDA(cudaGetLastError());
    count_launch(c, 2);
}

void generalized_eig(sdft_ctx* c, bool cplx, double* M, double* Hs, double* eig, int ncol) {
    const long long nn = (long long)ncol * ncol;
    if (c->eig_method < 0 && batched_eig_supported(ncol)) {
        // small subspace: one-CTA Cholesky + Jacobi solver (no cuSOLVER latency)
        ensure_ptab(c, 1, 3);
        c->ptab_host.assign({(void*)M, (void*)Hs, (void*)eig});
        SDFT_CUDA(cudaMemcpyAsync(c->ptab_dev, c->ptab_host.data(), 3 * sizeof(void*), cudaMemcpyHostToDevice,
                                  c->stream));
        double* const* tab = reinterpret_cast<double* const*>(c->ptab_dev);
        batched_generalized_eig(c, cplx, tab, tab + 1, tab + 2, ncol, 1, c->pinfo_dev);
        int info = 0;
        SDFT_CUDA(cudaMemcpyAsync(&info, c->pinfo_dev, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
        SDFT_CUDA(cudaStreamSynchronize(c->stream));
        if (info != 0)
            throw Error{SDFT_ERR_CHOLESKY, "subspace overlap matrix not positive definite at column " +
                                               std::to_string(info - 1)};
        return;
    }
    if (!cplx && refined_eig_supported(ncol) &&
        (c->eig_method == 2 || (c->eig_method < 0 && c->opt.precision == SDFT_MIXED))) {
        // FP32 solve refined to FP64 accuracy; verified on the device, else redone by cuSOLVER
        if (refined_generalized_eig(c, M, Hs, Hs, eig, ncol)) {
            ++c->reig_accepted;
            return;
        }
        if (c->eig_method == 2)
            throw Error{(c->reig_last_status & 1) ? SDFT_ERR_CHOLESKY : SDFT_ERR_NONFINITE,
                        "refined subspace eigensolver rejected its result (status " +
                            std::to_string(c->reig_last_status) + ")"};
        ++c->reig_fallbacks;
    }
    ScopedTimer timer(c, SDFT_K_EIGEN);
    diag_kernel<<<nb(ncol), 256, 0, c->stream>>>(M, c->dscale, ncol, cplx);
    scale_kernel<<<nb(nn), 256, 0, c->stream>>>(M, Hs, c->dscale, ncol, cplx);
    count_launch(c, 2);
    cusolverStatus_t st;
    if (c->eig_method == 1 && !cplx) {
        st = cusolverDnDsygvj(c->solver, CUSOLVER_EIG_TYPE_1, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_UPPER, ncol, Hs,
                              ncol, M, ncol, eig, (double*)c->solver_work, c->solver_lwork, c->dinfo, c->syevj_params);
    } else if (cplx) {
        st = cusolverDnZhegvd(c->solver, CUSOLVER_EIG_TYPE_1, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_UPPER, ncol,
                              (cuDoubleComplex*)Hs, ncol, (cuDoubleComplex*)M, ncol, eig,
                              (cuDoubleComplex*)c->solver_work, c->solver_lwork, c->dinfo);
    } else {
        st = cusolverDnDsygvd(c->solver, CUSOLVER_EIG_TYPE_1, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_UPPER, ncol, Hs,
                              ncol, M, ncol, eig, (double*)c->solver_work, c->solver_lwork, c->dinfo);
    }
    SDFT_REQUIRE(st == CUSOLVER_STATUS_SUCCESS, SDFT_ERR_CUDA, "cuSOLVER generalized eigensolver failed to launch");
    unscale_rows_kernel<<<nb(nn), 256, 0, c->stream>>>(Hs, c->dscale, ncol, cplx);
    SDFT_CUDA(cudaGetLastError());
    count_launch(c);
    int info = 0;
    SDFT_CUDA(cudaMemcpyAsync(&info, c->dinfo, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    SDFT_CUDA(cudaStreamSynchronize(c->stream));
    if (info != 0)
        throw Error{SDFT_ERR_CHOLESKY, "subspace eigensolver info = " + std::to_string(info) +
                                           (info > ncol ? " (overlap matrix not positive definite)" : "")};
}

void rotate_block(sdft_ctx* c, int precision, bool cplx, const void* Y, const double* Q, void* X, int ncol) {
    const int kind = kind_of(precision, cplx);
    dim3 grid((unsigned)((c->ng + 63) / 64), (ncol + 31) / 32);
    const void* Qp = Q;
    if (precision != SDFT_FP64) {
        if (rotate_tc_supported(c, precision, cplx, ncol)) {
            rotate_tc(c, Y, Q, X, ncol);
            return;
        }
        const long long nq = (long long)ncol * ncol * (cplx ? 2 : 1);
        to_float_kernel<<<nb(nq), 256, 0, c->stream>>>(Q, (float*)c->Q32, nq);
        count_launch(c);
        Qp = c->Q32;
    }
    ScopedTimer timer(c, SDFT_K_ROTATE, 0.0, 2.0 * (double)c->ng * ncol * ncol * (cplx ? 4.0 : 1.0));
    switch (kind) {
        case 0: rotate_kernel<0><<<grid, 256, 0, c->stream>>>(Y, Qp, X, ncol, c->ng); break;
        case 1: rotate_kernel<1><<<grid, 256, 0, c->stream>>>(Y, Qp, X, ncol, c->ng); break;
        case 2: rotate_kernel<2><<<grid, 256, 0, c->stream>>>(Y, Qp, X, ncol, c->ng); break;
        default: rotate_kernel<3><<<grid, 256, 0, c->stream>>>(Y, Qp, X, ncol, c->ng); break;
    }
    SDFT_CUDA(cudaGetLastError());
    count_launch(c);
}

void convert_block(sdft_ctx* c, bool cplx, int from_precision, const void* src, void* dst, int ncol) {
    const unsigned g = nb((long long)ncol * c->ng);
    if (from_precision == SDFT_MIXED) {
        if (cplx) convert_kernel<3, 1><<<g, 256, 0, c->stream>>>(src, dst, ncol, c->ng);
        else convert_kernel<2, 0><<<g, 256, 0, c->stream>>>(src, dst, ncol, c->ng);
    } else {
        if (cplx) convert_kernel<1, 3><<<g, 256, 0, c->stream>>>(src, dst, ncol, c->ng);
        else convert_kernel<0, 2><<<g, 256, 0, c->stream>>>(src, dst, ncol, c->ng);
    }
    SDFT_CUDA(cudaGetLastError());
    count_launch(c);
}

}  // namespace sdft
