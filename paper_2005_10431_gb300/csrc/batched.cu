// Batched small generalized Hermitian eigensolver of Rayleigh-Ritz (paper Sec. 2.1: CheFSI's
// subspace projection; "orthogonalisation + subspace eigensolve"), for many (k-point, spin,
// cell) problems at once: Hs q = lambda M q, n <= 64, FP64, one CTA per problem.
//
//   1. equilibrate with D = diag(M)^-1/2 (M' = D M D, H' = D H D)
//   2. Cholesky M' = L L^H
//   3. A = L^-1 H' L^-H (two triangular solves, then symmetrised)
//   4. cyclic Jacobi on A with the round-robin (tournament) order: n/2 disjoint rotations per
//      round, applied as one column pass and one row pass; sweeps until no rotation is needed
//   5. eigenvalues ascending, Q = D L^-H V
// Q overwrites Hs (column-major, eigenvector j in column j), eig ascending; info[p] = 0, or k+1
// if the equilibrated M is not positive definite at column k.
#include "internal.cuh"

#include <algorithm>
#include <vector>

namespace sdft {
namespace {

struct Cx {
    double r, i;
};
__device__ __forceinline__ Cx cx(double r, double i = 0.0) { return Cx{r, i}; }
__device__ __forceinline__ Cx operator+(Cx a, Cx b) { return Cx{a.r + b.r, a.i + b.i}; }
__device__ __forceinline__ Cx operator-(Cx a, Cx b) { return Cx{a.r - b.r, a.i - b.i}; }
__device__ __forceinline__ Cx operator*(Cx a, Cx b) { return Cx{a.r * b.r - a.i * b.i, a.r * b.i + a.i * b.r}; }
__device__ __forceinline__ Cx operator*(double s, Cx a) { return Cx{s * a.r, s * a.i}; }
__device__ __forceinline__ Cx conj(Cx a) { return Cx{a.r, -a.i}; }
__device__ __forceinline__ double abs2(Cx a) { return a.r * a.r + a.i * a.i; }

constexpr int GEIG_MAX_N = 64;
constexpr int GEIG_MAX_SWEEPS = 30;

// element (i, j) of an n x n column-major matrix in global memory
template <bool CPLX>
__device__ __forceinline__ Cx gload(const double* p, int i, int j, int n) {
    const long long o = (long long)i + (long long)j * n;
    return CPLX ? cx(p[2 * o], p[2 * o + 1]) : cx(p[o]);
}
template <bool CPLX>
__device__ __forceinline__ void gstore(double* p, int i, int j, int n, Cx v) {
    const long long o = (long long)i + (long long)j * n;
    if (CPLX) {
        p[2 * o] = v.r;
        p[2 * o + 1] = v.i;
    } else {
        p[o] = v.r;
    }
}

// round-robin schedule: in round r, slot k pairs positions k and m-1-k of the list
// [0, 1 + (r) mod (m-1), 1 + (r+1) mod (m-1), ...]; m even
__device__ __forceinline__ int rr_pos(int i, int r, int m) { return i == 0 ? 0 : 1 + (i - 1 + r) % (m - 1); }

template <bool CPLX>
__global__ void __launch_bounds__(256)
batched_geig_kernel(double* const* __restrict__ Ms, double* const* __restrict__ Hss, double* const* __restrict__ eigs,
                    int n, int* __restrict__ info) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int P = n + 1;   // padded leading dimension
    Cx* L = reinterpret_cast<Cx*>(smraw);   // M -> L (lower)
    Cx* A = L + n * P;                      // H -> W -> A
    Cx* V = A + n * P;                      // Z, then eigenvectors
    double* d = reinterpret_cast<double*>(V + n * P);
    double* lam = d + n;
    int* order = reinterpret_cast<int*>(lam + n);
    __shared__ int s_fail, s_rot;
#define AT(X, i, j) X[(i) + (j) * P]
    const int p = blockIdx.x, tid = threadIdx.x, NT = blockDim.x;
    const double* M = Ms[p];
    double* Hs = Hss[p];
    double* eig = eigs[p];
    if (tid == 0) s_fail = 0;
    for (int e = tid; e < n; e += NT) d[e] = rsqrt(gload<CPLX>(M, e, e, n).r);
    __syncthreads();
    for (int e = tid; e < n * n; e += NT) {
        const int i = e % n, j = e / n;
        const double s = d[i] * d[j];
        AT(L, i, j) = s * gload<CPLX>(M, i, j, n);
        AT(A, i, j) = s * gload<CPLX>(Hs, i, j, n);
    }
    __syncthreads();
    // Cholesky, right-looking, lower triangle
    for (int k = 0; k < n; ++k) {
        if (tid == 0) {
            const double akk = AT(L, k, k).r;
            if (!(akk > 0.0)) s_fail = k + 1;
            AT(L, k, k) = cx(akk > 0.0 ? sqrt(akk) : 1.0);
        }
        __syncthreads();
        if (s_fail) break;
        const double inv = 1.0 / AT(L, k, k).r;
        for (int i = k + 1 + tid; i < n; i += NT) AT(L, i, k) = inv * AT(L, i, k);
        __syncthreads();
        const int m = n - k - 1;
        for (int e = tid; e < m * m; e += NT) {
            const int i = k + 1 + e % m, j = k + 1 + e / m;
            if (i >= j) AT(L, i, j) = AT(L, i, j) - AT(L, i, k) * conj(AT(L, j, k));
        }
        __syncthreads();
    }
    if (s_fail) {
        if (tid == 0) info[p] = s_fail;
        return;
    }
    // W = L^-1 H (column j by thread j), Z = L^-1 W^H, A = (Z + Z^H)/2
    for (int j = tid; j < n; j += NT)
        for (int i = 0; i < n; ++i) {
            Cx s = AT(A, i, j);
            for (int k = 0; k < i; ++k) s = s - AT(L, i, k) * AT(A, k, j);
            AT(A, i, j) = (1.0 / AT(L, i, i).r) * s;
        }
    __syncthreads();
    for (int j = tid; j < n; j += NT)
        for (int i = 0; i < n; ++i) {
            Cx s = conj(AT(A, j, i));
            for (int k = 0; k < i; ++k) s = s - AT(L, i, k) * AT(V, k, j);
            AT(V, i, j) = (1.0 / AT(L, i, i).r) * s;
        }
    __syncthreads();
    for (int e = tid; e < n * n; e += NT) {
        const int i = e % n, j = e / n;
        Cx a = 0.5 * (AT(V, i, j) + conj(AT(V, j, i)));
        if (i == j) a.i = 0.0;
        AT(A, i, j) = a;
    }
    __syncthreads();
    for (int e = tid; e < n * n; e += NT) {
        const int i = e % n, j = e / n;
        AT(V, i, j) = cx(i == j ? 1.0 : 0.0);
    }
    __syncthreads();
    // cyclic Jacobi, tournament order
    const int m = n + (n & 1);
    const int npair = m / 2;
    // per-pair rotation U = [[c, s], [-s conj(e), c conj(e)]] on (p, q), p < q
    double* rc = lam;                                  // reuse: c per pair (npair <= 32 <= n)
    __shared__ double rs[GEIG_MAX_N / 2];
    __shared__ Cx re[GEIG_MAX_N / 2];
    __shared__ int rp[GEIG_MAX_N / 2], rq[GEIG_MAX_N / 2];
    for (int sweep = 0; sweep < GEIG_MAX_SWEEPS; ++sweep) {
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
                rc[k] = 1.0;
                rs[k] = 0.0;
                re[k] = cx(1.0);
                if (b < n) {
                    const Cx apq = AT(A, a, b);
                    const double app = AT(A, a, a).r, aqq = AT(A, b, b).r;
                    const double g = sqrt(abs2(apq));
                    if (g > 1e-300 && g > 1e-15 * (fabs(app) + fabs(aqq))) {
                        const Cx e = cx(apq.r / g, apq.i / g);
                        const double tau = (aqq - app) / (2.0 * g);
                        const double t = (tau >= 0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                        const double c = 1.0 / sqrt(1.0 + t * t);
                        rc[k] = c;
                        rs[k] = t * c;
                        re[k] = e;
                        atomicAdd(&s_rot, 1);
                    }
                }
            }
            __syncthreads();
            // columns: A <- A U, V <- V U
            for (int e = tid; e < npair * n; e += NT) {
                const int k = e / n, row = e - k * n;
                if (rq[k] >= n || (rs[k] == 0.0)) continue;
                const int a = rp[k], b = rq[k];
                const double c = rc[k], s = rs[k];
                const Cx ce = conj(re[k]);
                const Cx upp = cx(c), upq = cx(s), uqp = (-s) * ce, uqq = c * ce;
                Cx x = AT(A, row, a), y = AT(A, row, b);
                AT(A, row, a) = x * upp + y * uqp;
                AT(A, row, b) = x * upq + y * uqq;
                x = AT(V, row, a);
                y = AT(V, row, b);
                AT(V, row, a) = x * upp + y * uqp;
                AT(V, row, b) = x * upq + y * uqq;
            }
            __syncthreads();
            // rows: A <- U^H A
            for (int e = tid; e < npair * n; e += NT) {
                const int k = e / n, col = e - k * n;
                if (rq[k] >= n || (rs[k] == 0.0)) continue;
                const int a = rp[k], b = rq[k];
                const double c = rc[k], s = rs[k];
                const Cx ce = conj(re[k]);
                const Cx upp = cx(c), upq = cx(s), uqp = (-s) * ce, uqq = c * ce;
                const Cx x = AT(A, a, col), y = AT(A, b, col);
                AT(A, a, col) = conj(upp) * x + conj(uqp) * y;
                AT(A, b, col) = conj(upq) * x + conj(uqq) * y;
            }
            __syncthreads();
        }
        if (s_rot == 0) break;
        __syncthreads();
    }
    // eigenvalues ascending (rank sort, ties by index)
    for (int i = tid; i < n; i += NT) lam[i] = AT(A, i, i).r;
    __syncthreads();
    for (int i = tid; i < n; i += NT) {
        int rank = 0;
        for (int j = 0; j < n; ++j) rank += (lam[j] < lam[i]) || (lam[j] == lam[i] && j < i);
        order[rank] = i;
    }
    __syncthreads();
    for (int j = tid; j < n; j += NT) eig[j] = lam[order[j]];
    // Q(:, j) = D L^-H V(:, order[j]) by back substitution; thread j owns column j
    for (int j = tid; j < n; j += NT) {
        const int src = order[j];
        Cx y[GEIG_MAX_N];
        for (int i = n - 1; i >= 0; --i) {
            Cx s = AT(V, i, src);
            for (int k = i + 1; k < n; ++k) s = s - conj(AT(L, k, i)) * y[k];
            y[i] = (1.0 / AT(L, i, i).r) * s;
        }
        for (int i = 0; i < n; ++i) gstore<CPLX>(Hs, i, j, n, d[i] * y[i]);
    }
    if (tid == 0) info[p] = 0;
#undef AT
}

size_t geig_smem(int n) {
    const int P = n + 1;
    return sizeof(Cx) * 3 * (size_t)n * P + sizeof(double) * 2 * n + sizeof(int) * n;
}

}  // namespace

bool batched_eig_supported(int n) { return n >= 1 && n <= GEIG_MAX_N; }

void ensure_ptab(sdft_ctx* c, int count, int width) {
    const int need = count * width;
    if (need <= c->ptab_cap && c->pinfo_dev) return;
    const int cap = std::max(need, 256);
    // the old tables stay owned by the context (released at destroy); all users synchronise
    // before a table is rewritten, so nothing in flight reads the replaced one
    c->ptab_dev = (void**)ctx_alloc(c, sizeof(void*) * (size_t)cap);
    c->pinfo_dev = (int*)ctx_alloc(c, sizeof(int) * (size_t)cap);
    c->ptab_cap = cap;
}

// Ms/Hss/eigs: device arrays of `count` device pointers; info: device int[count]
void batched_generalized_eig(sdft_ctx* c, bool cplx, double* const* Ms, double* const* Hss, double* const* eigs,
                             int n, int count, int* info) {
    SDFT_REQUIRE(batched_eig_supported(n), SDFT_ERR_INVALID_ARG, "batched eigensolver supports n <= 64");
    if (count <= 0) return;
    ScopedTimer timer(c, SDFT_K_EIGEN);
    const size_t sm = geig_smem(n);
    if (cplx) {
        SDFT_CUDA(cudaFuncSetAttribute(batched_geig_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        batched_geig_kernel<true><<<count, 256, sm, c->stream>>>(Ms, Hss, eigs, n, info);
    } else {
        SDFT_CUDA(cudaFuncSetAttribute(batched_geig_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        batched_geig_kernel<false><<<count, 256, sm, c->stream>>>(Ms, Hss, eigs, n, info);
    }
    SDFT_CUDA(cudaGetLastError());
    count_launch(c);
}

}  // namespace sdft
