// Subspace generalized eigensolve Hs q = lambda M q of Rayleigh-Ritz (paper Sec. 2.1, the
// projected problem of CheFSI) for real blocks of 64 < n <= 1024: an FP32 solve (one CTA for
// n <= 160, cuSOLVER's FP32 sygvd above, where two n x n FP32 matrices no longer fit in one CTA's
// shared memory), refined to FP64 accuracy by FP64 matrix products that spread over the GPU.
//
// The GB300's FP64 pipes are few, so a one-CTA FP64 reduction to tridiagonal form is slow for
// these sizes (cuSOLVER's sygvd takes ~6.6 ms at n = 154).  This solver
//   1. equilibrates with D = diag(M)^-1/2, factors M' = L L^T, forms A = L^-1 H' L^-T and
//      diagonalises A by cyclic Jacobi in tournament order, all in FP32 in shared memory;
//      Q0 = D L^-T V in FP64, columns in ascending eigenvalue order;
//   2. refines Q twice by the Ogita-Aishima iteration (Ogita & Aishima 2018, written here for the
//      generalized problem): with G = Q^T M Q and S = Q^T Hs Q in FP64 and lambda_i = S_ii / G_ii,
//      Q <- Q (I + F), F_ii = (1 - G_ii) / 2, and for i != j
//          F_ij = (S_ij - lambda_j G_ij) / (lambda_j - lambda_i)   (eigenvalues farther apart
//                                                                    than omega),
//          F_ij = -G_ij / 2                                        (inside a cluster),
//      omega = 100 max_{i != j} |S_ij - lambda_j G_ij| of the FP32 solution, so |F_ij| <= 1/100
//      between clusters, and the same clusters in every step (a threshold that shrank with the
//      residual would release barely separated pairs with large first-order rotations);
//      this is the first-order solution of (I+F)^T G (I+F) = I, (I+F)^T S (I+F) diagonal, and
//      the error of Q is squared by each step;
//   3. solves each cluster's small eigenproblem S_cc w = mu w (FP64 Jacobi, one thread per
//      cluster, after normalising by diag(G)) on the refined Q, which fixes the basis inside
//      clusters of (near-)degenerate eigenvalues; Q <- Q T with T block diagonal, columns sorted.
// The host reads one status word: a failed FP32 Cholesky, a cluster larger than 32, a non-finite
// value, or a final off-cluster residual or orthonormality defect above 1e-10 (relative) makes
// the caller fall back to the FP64 cuSOLVER solver; M and Hs are not modified before success.
#include "internal.cuh"

#include <algorithm>

namespace sdft {
namespace {

constexpr int RE_MAX_N = 160;        // one-CTA FP32 solve (step 1)
constexpr int RE2_MAX_N = 1024;      // refinement (steps 2-3), FP32 start from cuSOLVER above RE_MAX_N
constexpr int RE_KMAX = 32;          // largest cluster solved by step 3
constexpr int RE_MAX_SWEEPS = 20;    // FP32 Jacobi
constexpr int RE_CL_SWEEPS = 40;     // FP64 cluster Jacobi

enum : int {
    ST_CHOLESKY = 1,
    ST_CLUSTER = 2,
    ST_RESIDUAL = 4,
    ST_ORTHO = 8,
    ST_NONFINITE = 16,
};

__device__ __forceinline__ int rr_pos(int i, int r, int m) { return i == 0 ? 0 : 1 + (i - 1 + r) % (m - 1); }

// rotation of the classical Jacobi method (Golub & Van Loan, sym.schur2): J = [[c, s], [-s, c]] in
// the (p, q) plane makes (J^T A J)_pq = 0
template <typename T>
__device__ __forceinline__ void jacobi_cs(T app, T aqq, T apq, T& c, T& s) {
    const T tau = (aqq - app) / (T(2) * apq);
    const T t = (tau >= T(0) ? T(1) : T(-1)) / (fabs(tau) + sqrt(T(1) + tau * tau));
    c = T(1) / sqrt(T(1) + t * t);
    s = t * c;
}

// step 1: one CTA; X (FP64, n x n column-major) <- Q0; status <- 0 or ST_CHOLESKY
__global__ void __launch_bounds__(1024, 1)
eig32_kernel(const double* __restrict__ M, const double* __restrict__ Hs, int n, double* __restrict__ X,
             float* __restrict__ Lg, int* __restrict__ status) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int P = n + 1;
    float* A = reinterpret_cast<float*>(smraw);   // H' -> A -> (after Jacobi) L again
    float* V = A + n * P;                         // M' -> L, then eigenvectors
    double* d = reinterpret_cast<double*>(V + n * P);
    float* lam = reinterpret_cast<float*>(d + n);
    int* order = reinterpret_cast<int*>(lam + n);
    __shared__ int rp[RE_MAX_N / 2], rq[RE_MAX_N / 2];
    __shared__ float rc[RE_MAX_N / 2], rs[RE_MAX_N / 2];
    __shared__ int s_fail, s_rot;
    __shared__ float s_scale;
#define AT(Z, i, j) Z[(i) + (j) * P]
    const int tid = threadIdx.x, NT = blockDim.x;
    if (tid == 0) {
        s_fail = 0;
        s_scale = 0.f;
    }
    for (int e = tid; e < n; e += NT) d[e] = rsqrt(M[e + (long long)e * n]);
    __syncthreads();
    for (int e = tid; e < n * n; e += NT) {
        const int i = e % n, j = e / n;
        const double s = d[i] * d[j];
        AT(V, i, j) = (float)(s * M[e]);
        AT(A, i, j) = (float)(s * Hs[e]);
    }
    __syncthreads();
    // Cholesky of M' in V (lower), right-looking
    for (int k = 0; k < n; ++k) {
        if (tid == 0) {
            const float akk = AT(V, k, k);
            if (!(akk > 0.f)) s_fail = k + 1;
            AT(V, k, k) = akk > 0.f ? sqrtf(akk) : 1.f;
        }
        __syncthreads();
        if (s_fail) break;
        const float inv = 1.f / AT(V, k, k);
        for (int i = k + 1 + tid; i < n; i += NT) AT(V, i, k) *= inv;
        __syncthreads();
        for (int j = k + 1 + (tid >> 5); j < n; j += NT >> 5) {
            const float ljk = AT(V, j, k);
            for (int i = j + (tid & 31); i < n; i += 32) AT(V, i, j) -= AT(V, i, k) * ljk;
        }
        __syncthreads();
    }
    if (s_fail) {
        if (tid == 0) *status = ST_CHOLESKY;
        return;
    }
    // A <- L^-1 A, transpose, A <- L^-1 A (= L^-1 H' L^-T), symmetrise
    for (int pass = 0; pass < 2; ++pass) {
        for (int j = tid; j < n; j += NT)
            for (int i = 0; i < n; ++i) {
                float s = AT(A, i, j);
                for (int k = 0; k < i; ++k) s -= AT(V, i, k) * AT(A, k, j);
                AT(A, i, j) = s / AT(V, i, i);
            }
        __syncthreads();
        for (int e = tid; e < n * n; e += NT) {
            const int i = e % n, j = e / n;
            if (i < j) {
                const float a = AT(A, i, j), b = AT(A, j, i);
                if (pass == 0) {
                    AT(A, i, j) = b;
                    AT(A, j, i) = a;
                } else {
                    AT(A, i, j) = AT(A, j, i) = 0.5f * (a + b);
                }
            }
        }
        __syncthreads();
    }
    // keep L in global memory for the back substitution; V <- I
    for (int e = tid; e < n * n; e += NT) {
        const int i = e % n, j = e / n;
        Lg[e] = i >= j ? AT(V, i, j) : 0.f;
        AT(V, i, j) = i == j ? 1.f : 0.f;
    }
    for (int i = tid; i < n; i += NT) atomicMax(reinterpret_cast<int*>(&s_scale), __float_as_int(fabsf(AT(A, i, i))));
    __syncthreads();
    // cyclic Jacobi, tournament order; a rotation is skipped below the FP32 noise of A
    const float scale = s_scale;
    const int m = n + (n & 1), npair = m / 2;
    const int warp = tid >> 5, lane = tid & 31, nwarp = NT >> 5;
    for (int sweep = 0; sweep < RE_MAX_SWEEPS; ++sweep) {
        if (tid == 0) s_rot = 0;
        __syncthreads();
        for (int r = 0; r < m - 1; ++r) {
            for (int k = tid; k < npair; k += NT) {
                int a = rr_pos(k, r, m), b = rr_pos(m - 1 - k, r, m);
                if (a > b) {
                    const int t = a;
                    a = b;
                    b = t;
                }
                rp[k] = a;
                rq[k] = b;
                rc[k] = 1.f;
                rs[k] = 0.f;
                if (b < n) {
                    const float apq = AT(A, a, b), app = AT(A, a, a), aqq = AT(A, b, b);
                    if (fabsf(apq) > 1e-7f * (fabsf(app) + fabsf(aqq)) + 4e-7f * scale) {
                        float c, s;
                        jacobi_cs(app, aqq, apq, c, s);
                        rc[k] = c;
                        rs[k] = s;
                        s_rot = 1;
                    }
                }
            }
            __syncthreads();
            // a warp per pair, a lane per row (column pass) or column (row pass)
            for (int k = warp; k < npair; k += nwarp) {   // columns: A <- A J, V <- V J
                const float s = rs[k];
                if (s == 0.f) continue;
                const float c = rc[k];
                const int a = rp[k], b = rq[k];
                for (int row = lane; row < n; row += 32) {
                    float x = AT(A, row, a), y = AT(A, row, b);
                    AT(A, row, a) = c * x - s * y;
                    AT(A, row, b) = s * x + c * y;
                    x = AT(V, row, a);
                    y = AT(V, row, b);
                    AT(V, row, a) = c * x - s * y;
                    AT(V, row, b) = s * x + c * y;
                }
            }
            __syncthreads();
            for (int k = warp; k < npair; k += nwarp) {   // rows: A <- J^T A
                const float s = rs[k];
                if (s == 0.f) continue;
                const float c = rc[k];
                const int a = rp[k], b = rq[k];
                for (int col = lane; col < n; col += 32) {
                    const float x = AT(A, a, col), y = AT(A, b, col);
                    AT(A, a, col) = c * x - s * y;
                    AT(A, b, col) = s * x + c * y;
                }
            }
            __syncthreads();
        }
        if (s_rot == 0) break;
        __syncthreads();
    }
    for (int i = tid; i < n; i += NT) {
        lam[i] = AT(A, i, i);
        order[i] = i;   // stays a valid index even if NaNs break the ranking (the refinement rejects those)
    }
    __syncthreads();
    for (int i = tid; i < n; i += NT) {
        int rank = 0;
        for (int j = 0; j < n; ++j) rank += (lam[j] < lam[i]) || (lam[j] == lam[i] && j < i);
        order[rank] = i;
    }
    // L back into A's storage, then V <- L^-T V in place (thread j owns column j)
    for (int e = tid; e < n * n; e += NT) AT(A, e % n, e / n) = Lg[e];
    __syncthreads();
    for (int j = tid; j < n; j += NT)
        for (int i = n - 1; i >= 0; --i) {
            float s = AT(V, i, j);
            for (int k = i + 1; k < n; ++k) s -= AT(A, k, i) * AT(V, k, j);
            AT(V, i, j) = s / AT(A, i, i);
        }
    __syncthreads();
    for (int e = tid; e < n * n; e += NT) {
        const int i = e % n, jo = e / n;
        X[e] = d[i] * (double)AT(V, i, order[jo]);
    }
    if (tid == 0) *status = 0;
#undef AT
}

size_t eig32_smem(int n) {
    return sizeof(float) * 2 * (size_t)n * (n + 1) + sizeof(double) * n + sizeof(float) * n + sizeof(int) * n;
}

// C = op(A) B for n x n column-major FP64 matrices, op(A) = A or A^T; blockIdx.z picks one of
// two products.  32 x 32 tile per CTA, 2 x 2 outputs per thread.
struct Prod2 {
    const double* A[2];
    const double* B[2];
    double* C[2];
};

template <bool TA>
__global__ void __launch_bounds__(256) gemm64_kernel(Prod2 g, int n, const int* __restrict__ status) {
    constexpr int T = 32, KT = 16;
    if (*status & ST_CHOLESKY) return;
    __shared__ double As[KT][T + 1];   // As[k][i] = op(A)(i0 + i, k0 + k)
    __shared__ double Bs[KT][T + 1];   // Bs[k][j] = B(k0 + k, j0 + j)
    const double* __restrict__ A = g.A[blockIdx.z];
    const double* __restrict__ B = g.B[blockIdx.z];
    double* __restrict__ C = g.C[blockIdx.z];
    const int i0 = blockIdx.x * T, j0 = blockIdx.y * T;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    double acc[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
    for (int k0 = 0; k0 < n; k0 += KT) {
        for (int e = threadIdx.x; e < KT * T; e += 256) {
            int i, k;
            if (TA) {
                k = e % KT;
                i = e / KT;
            } else {
                i = e % T;
                k = e / T;
            }
            const int gi = i0 + i, gk = k0 + k;
            double v = 0.0;
            if (gi < n && gk < n) v = TA ? A[gk + (long long)gi * n] : A[gi + (long long)gk * n];
            As[k][i] = v;
            const int kb = e % KT, jb = e / KT;
            const int gj = j0 + jb, gkb = k0 + kb;
            Bs[kb][jb] = (gj < n && gkb < n) ? B[gkb + (long long)gj * n] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < KT; ++k) {
            const double a0 = As[k][tx], a1 = As[k][tx + 16], b0 = Bs[k][ty], b1 = Bs[k][ty + 16];
            acc[0][0] = fma(a0, b0, acc[0][0]);
            acc[1][0] = fma(a1, b0, acc[1][0]);
            acc[0][1] = fma(a0, b1, acc[0][1]);
            acc[1][1] = fma(a1, b1, acc[1][1]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const int i = i0 + tx + 16 * a, j = j0 + ty + 16 * b;
            if (i < n && j < n) C[i + (long long)j * n] = acc[a][b];
        }
}

__device__ __forceinline__ void atomic_max_nonneg(unsigned long long* p, double v) {
    atomicMax(p, (unsigned long long)__double_as_longlong(v));   // order of non-negative doubles
}

__device__ double block_max(double v, unsigned long long* slot) {
    for (int off = 16; off > 0; off >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, off));
    if ((threadIdx.x & 31) == 0) atomic_max_nonneg(slot, v);
    return v;
}

// steps 2 (mode 0) and 3 (mode 1): T from G = Q^T M Q and S = Q^T Hs Q; mode 1 also writes the
// eigenvalues (ascending) and checks the final residuals.  ws: 2 * RE_KMAX * n doubles.
__global__ void __launch_bounds__(1024, 1)
refine_step_kernel(const double* __restrict__ G, const double* __restrict__ S, double* __restrict__ Tm,
                   double* __restrict__ eig, double* __restrict__ ws, int n, int step, int mode,
                   int* __restrict__ status, double* __restrict__ diag) {
    __shared__ double lam[RE2_MAX_N];
    __shared__ int ord[RE2_MAX_N], rnk[RE2_MAX_N], first[RE2_MAX_N], cstart[RE2_MAX_N], csize[RE2_MAX_N];
    __shared__ unsigned long long s_eta, s_scale, s_inter, s_orth;
    __shared__ int s_bad;
    if (*status & ST_CHOLESKY) return;
    const int tid = threadIdx.x, NT = blockDim.x;
    const int warp = tid >> 5, lane = tid & 31, nwarp = NT >> 5;
    const long long nn = (long long)n * n;
    if (tid == 0) {
        s_eta = s_scale = s_inter = s_orth = 0ull;
        s_bad = 0;
    }
    __syncthreads();
    for (int i = tid; i < n; i += NT) {
        double l = S[i + (long long)i * n] / G[i + (long long)i * n];
        if (!isfinite(l)) {
            s_bad = 1;
            l = 0.0;
        }
        lam[i] = l;
    }
    __syncthreads();
    double eta = 0.0, sc = 0.0;
    for (int j = warp; j < n; j += nwarp)
        for (int i = lane; i < n; i += 32) {
            const long long e = i + (long long)j * n;
            if (i != j) eta = fmax(eta, fabs(S[e] - lam[j] * G[e]));
            else sc = fmax(sc, fabs(lam[i]));
        }
    if (!isfinite(eta)) {
        s_bad = 1;
        eta = 0.0;
    }
    block_max(eta, &s_eta);
    block_max(sc, &s_scale);
    for (int i = tid; i < n; i += NT) {
        int r = 0;
        for (int j = 0; j < n; ++j) r += (lam[j] < lam[i]) || (lam[j] == lam[i] && j < i);
        rnk[i] = r;
        ord[r] = i;
    }
    __syncthreads();
    const double scale = __longlong_as_double((long long)s_scale);
    // cluster threshold: set by the first step, kept by the later ones (diag[8])
    const double omega = step == 0 ? fmax(100.0 * __longlong_as_double((long long)s_eta), 1e-14 * fmax(scale, 1e-300))
                                   : diag[8];
    for (int r = tid; r < n; r += NT) first[r] = r == 0 || lam[ord[r]] - lam[ord[r - 1]] > omega;
    __syncthreads();
    for (int r = tid; r < n; r += NT) {
        int s = r;
        while (!first[s]) --s;
        cstart[r] = s;
        if (first[r]) {
            int k = 1;
            while (r + k < n && !first[r + k]) ++k;
            csize[r] = k;
        }
    }
    __syncthreads();
    // off-cluster residual and orthonormality defect of the current Q
    double inter = 0.0, orth = 0.0;
    for (int j = warp; j < n; j += nwarp)
        for (int i = lane; i < n; i += 32) {
            const long long e = i + (long long)j * n;
            if (i != j && cstart[rnk[i]] != cstart[rnk[j]]) inter = fmax(inter, fabs(S[e] - lam[j] * G[e]));
            orth = fmax(orth, fabs(G[e] - (i == j ? 1.0 : 0.0)));
        }
    block_max(inter, &s_inter);
    block_max(orth, &s_orth);
    if (mode == 0) {
        for (int j = warp; j < n; j += nwarp)
            for (int i = lane; i < n; i += 32) {
            const long long e = i + (long long)j * n;
            double t;
            if (i == j) t = 1.0 + 0.5 * (1.0 - G[e]);
            else if (cstart[rnk[i]] == cstart[rnk[j]]) t = -0.5 * G[e];
            else t = (S[e] - lam[j] * G[e]) / (lam[j] - lam[i]);
            Tm[e] = t;
            }
    } else {
        for (long long e = tid; e < nn; e += NT) Tm[e] = 0.0;
        __syncthreads();
        for (int r0 = tid; r0 < n; r0 += NT) {
            if (!first[r0]) continue;
            const int k = csize[r0];
            if (k == 1) {
                const int i = ord[r0];
                Tm[i + (long long)r0 * n] = 1.0 / sqrt(G[i + (long long)i * n]);
                eig[r0] = lam[i];
                continue;
            }
            if (k > RE_KMAX) {
                atomicOr(status, ST_CLUSTER);
                continue;
            }
            double* Bm = ws + (size_t)2 * RE_KMAX * r0;   // k x k, then W (k x k)
            double* W = Bm + k * k;
            for (int b = 0; b < k; ++b)
                for (int a = 0; a < k; ++a) {
                    const int i = ord[r0 + a], j = ord[r0 + b];
                    const double gij = sqrt(G[i + (long long)i * n] * G[j + (long long)j * n]);
                    Bm[a + b * k] = 0.5 * (S[i + (long long)j * n] + S[j + (long long)i * n]) / gij;
                    W[a + b * k] = a == b ? 1.0 : 0.0;
                }
            for (int sweep = 0; sweep < RE_CL_SWEEPS; ++sweep) {
                int rot = 0;
                for (int p = 0; p < k - 1; ++p)
                    for (int q = p + 1; q < k; ++q) {
                        const double apq = Bm[p + q * k], app = Bm[p + p * k], aqq = Bm[q + q * k];
                        if (!(fabs(apq) > 1e-16 * (fabs(app) + fabs(aqq)) && fabs(apq) > 1e-300)) continue;
                        double c, s;
                        jacobi_cs(app, aqq, apq, c, s);
                        ++rot;
                        for (int x = 0; x < k; ++x) {
                            const double u = Bm[x + p * k], v = Bm[x + q * k];
                            Bm[x + p * k] = c * u - s * v;
                            Bm[x + q * k] = s * u + c * v;
                            const double wu = W[x + p * k], wv = W[x + q * k];
                            W[x + p * k] = c * wu - s * wv;
                            W[x + q * k] = s * wu + c * wv;
                        }
                        for (int x = 0; x < k; ++x) {
                            const double u = Bm[p + x * k], v = Bm[q + x * k];
                            Bm[p + x * k] = c * u - s * v;
                            Bm[q + x * k] = s * u + c * v;
                        }
                    }
                if (rot == 0) break;
            }
            for (int b = 0; b < k; ++b) {
                const double mu = Bm[b + b * k];
                int rb = 0;
                for (int a = 0; a < k; ++a) {
                    const double ma = Bm[a + a * k];
                    rb += (ma < mu) || (ma == mu && a < b);
                }
                eig[r0 + rb] = mu;
                for (int a = 0; a < k; ++a) {
                    const int i = ord[r0 + a];
                    Tm[i + (long long)(r0 + rb) * n] = W[a + b * k] / sqrt(G[i + (long long)i * n]);
                }
            }
        }
    }
    __syncthreads();
    if (tid == 0) {
        const double e = __longlong_as_double((long long)s_eta), in = __longlong_as_double((long long)s_inter),
                     o = __longlong_as_double((long long)s_orth);
        diag[4 * mode + 0] = e;
        diag[4 * mode + 1] = in;
        diag[4 * mode + 2] = o;
        diag[4 * mode + 3] = scale;
        if (step == 0) diag[8] = omega;
        int st = s_bad ? ST_NONFINITE : 0;
        if (mode == 1) {
            if (!(in <= 1e-10 * fmax(scale, 1.0))) st |= ST_RESIDUAL;
            if (!(o <= 1e-10)) st |= ST_ORTHO;
        }
        if (st) atomicOr(status, st);
    }
}

// FP32 start for n > RE_MAX_N: d = diag(M)^-1/2, M32 = D M D, H32 = D Hs D (FP32, column-major)
__global__ void equil32_kernel(const double* __restrict__ M, const double* __restrict__ Hs, int n,
                               double* __restrict__ d, float* __restrict__ M32, float* __restrict__ H32) {
    const long long nn = (long long)n * n;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nn; e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e % n), j = (int)(e / n);
        const double s = rsqrt(M[i + (long long)i * n]) * rsqrt(M[j + (long long)j * n]);
        M32[e] = (float)(s * M[e]);
        H32[e] = (float)(s * Hs[e]);
        if (j == 0) d[i] = rsqrt(M[i + (long long)i * n]);
    }
}
// X = D V in FP64 from cuSOLVER's FP32 eigenvectors (ascending); status = Cholesky failure or 0
__global__ void start32_kernel(const float* __restrict__ V, const double* __restrict__ d, int n,
                               const int* __restrict__ info, double* __restrict__ X, int* __restrict__ status) {
    const long long nn = (long long)n * n;
    const bool bad = *info != 0;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nn; e += (long long)gridDim.x * blockDim.x)
        X[e] = d[e % n] * (double)V[e];
    if (blockIdx.x == 0 && threadIdx.x == 0) *status = bad ? ST_CHOLESKY : 0;
}

}  // namespace

bool refined_eig_supported(int n) { return n >= 2 && n <= RE2_MAX_N; }

bool refined_generalized_eig(sdft_ctx* c, const double* M, const double* Hs, double* Q, double* eig, int n) {
    SDFT_REQUIRE(refined_eig_supported(n), SDFT_ERR_INVALID_ARG, "refined eigensolver supports 2 <= n <= 1024");
    const size_t nn = (size_t)n * n;
    // scratch sized for the context's widest Rayleigh-Ritz block (at least RE_MAX_N)
    const int nmax = std::max(RE_MAX_N, std::max(n, c->nfilt));
    if (!c->reig_buf || c->reig_nmax < nmax) {
        const size_t N2 = (size_t)nmax * nmax;
        // X, X', T, P1, P2, G, S (FP64 n x n each), ws, eig, diag, d; L / M32 / H32 (FP32); status, info
        c->reig_buf = (double*)ctx_alloc(c, sizeof(double) * (7 * N2 + 2 * RE_KMAX * nmax + 2 * nmax + 16) +
                                                sizeof(float) * (3 * N2 + nmax) + 64);
        c->reig_nmax = nmax;
    }
    const size_t N2 = (size_t)c->reig_nmax * c->reig_nmax;
    double* X = c->reig_buf;
    double* Xn = X + N2;
    double* Tm = Xn + N2;
    double* P1 = Tm + N2;
    double* P2 = P1 + N2;
    double* G = P2 + N2;
    double* S = G + N2;
    double* ws = S + N2;
    double* ev = ws + 2 * RE_KMAX * (size_t)c->reig_nmax;
    double* dsc = ev + c->reig_nmax;
    double* diag = dsc + c->reig_nmax;
    float* Lg = reinterpret_cast<float*>(diag + 16);
    float* M32 = Lg + N2;
    float* H32 = M32 + N2;
    float* w32 = H32 + N2;
    int* status = reinterpret_cast<int*>(w32 + c->reig_nmax);
    int* info = status + 1;
    ScopedTimer timer(c, SDFT_K_EIGEN);
    if (n <= RE_MAX_N) {
        const size_t sm = eig32_smem(n);
        SDFT_CUDA(cudaFuncSetAttribute(eig32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        eig32_kernel<<<1, 1024, sm, c->stream>>>(M, Hs, n, X, Lg, status);
    } else {
        // FP32 generalized eigensolve by cuSOLVER on the equilibrated problem (workspace on first use)
        if (c->reig_lwork32 < 0 || c->reig_work32_n < n) {
            int lw = 0;
            cusolverStatus_t cs = cusolverDnSsygvd_bufferSize(c->solver, CUSOLVER_EIG_TYPE_1, CUSOLVER_EIG_MODE_VECTOR,
                                                              CUBLAS_FILL_MODE_UPPER, n, H32, n, M32, n, w32, &lw);
            SDFT_REQUIRE(cs == CUSOLVER_STATUS_SUCCESS, SDFT_ERR_CUDA, "FP32 sygvd workspace query failed");
            c->reig_work32 = (float*)ctx_alloc(c, sizeof(float) * ((size_t)lw + 64));
            c->reig_lwork32 = lw;
            c->reig_work32_n = n;
        }
        const unsigned g = (unsigned)std::min<size_t>((nn + 255) / 256, 152 * 8);
        equil32_kernel<<<g, 256, 0, c->stream>>>(M, Hs, n, dsc, M32, H32);
        SDFT_CUDA(cudaGetLastError());
        const cusolverStatus_t cs = cusolverDnSsygvd(c->solver, CUSOLVER_EIG_TYPE_1, CUSOLVER_EIG_MODE_VECTOR,
                                                     CUBLAS_FILL_MODE_UPPER, n, H32, n, M32, n, w32, c->reig_work32,
                                                     c->reig_lwork32, info);
        SDFT_REQUIRE(cs == CUSOLVER_STATUS_SUCCESS, SDFT_ERR_CUDA, "FP32 sygvd failed to launch");
        start32_kernel<<<g, 256, 0, c->stream>>>(H32, dsc, n, info, X, status);
        SDFT_CUDA(cudaGetLastError());
    }
    const dim3 grid((n + 31) / 32, (n + 31) / 32, 2);
    for (int step = 0; step < 3; ++step) {
        gemm64_kernel<false><<<grid, 256, 0, c->stream>>>(Prod2{{M, Hs}, {X, X}, {P1, P2}}, n, status);
        gemm64_kernel<true><<<grid, 256, 0, c->stream>>>(Prod2{{X, X}, {P1, P2}, {G, S}}, n, status);
        refine_step_kernel<<<1, 1024, 0, c->stream>>>(G, S, Tm, ev, ws, n, step, step == 2 ? 1 : 0, status, diag);
        const dim3 g1(grid.x, grid.y, 1);
        gemm64_kernel<false><<<g1, 256, 0, c->stream>>>(Prod2{{X, nullptr}, {Tm, nullptr}, {Xn, nullptr}}, n, status);
        std::swap(X, Xn);
    }
    SDFT_CUDA(cudaGetLastError());
    count_launch(c, 13);
    int st = 0;
    SDFT_CUDA(cudaMemcpyAsync(&st, status, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    SDFT_CUDA(cudaStreamSynchronize(c->stream));
    c->reig_last_status = st;
    if (st != 0) return false;
    SDFT_CUDA(cudaMemcpyAsync(Q, X, sizeof(double) * nn, cudaMemcpyDeviceToDevice, c->stream));
    SDFT_CUDA(cudaMemcpyAsync(eig, ev, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->stream));
    return true;
}

}  // namespace sdft
