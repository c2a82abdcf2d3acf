// Grid-level FP64 kernels of the SCF (paper Sec. 2.1): pseudocharges and the SAD guess,
// Perdew-Zunger LDA, the AAR Poisson solver, density from orbitals (Eq. 2), Fermi-Dirac
// occupations, Pulay mixing, reductions and Hellmann-Feynman forces.
#include "internal.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>

namespace sdft {
namespace {

constexpr int RB = 256;   // reduction block size

// ---------------------------------------------------------------------------------------
// set-up: pseudocharge b and SAD density, summed over periodic images within the cutoff
// ---------------------------------------------------------------------------------------
struct AtomG {
    double pos[3];
    double amp_b, w_b, cut_b;      // pseudocharge amplitude, width, cutoff
    double amp_s, w_s, cut_s;      // SAD
};

__device__ double image_sum(double x, double y, double z, const double* pos, double L1, double L2, double L3,
                            double amp, double w, double cut, int isolated) {
    double s = 0.0;
    const double L[3] = {L1, L2, L3};
    const double X[3] = {x, y, z};
    int tlo[3], thi[3];
    for (int d = 0; d < 3; ++d) {
        tlo[d] = isolated ? 0 : (int)ceil((X[d] - pos[d] - cut) / L[d]);   // isolated: the atom itself only
        thi[d] = isolated ? 0 : (int)floor((X[d] - pos[d] + cut) / L[d]);
    }
    const double inv = 1.0 / (2.0 * w * w);
    for (int t2 = tlo[2]; t2 <= thi[2]; ++t2)
        for (int t1 = tlo[1]; t1 <= thi[1]; ++t1)
            for (int t0 = tlo[0]; t0 <= thi[0]; ++t0) {
                const double dx = X[0] - pos[0] - t0 * L1, dy = X[1] - pos[1] - t1 * L2, dz = X[2] - pos[2] - t2 * L3;
                const double r2 = dx * dx + dy * dy + dz * dz;
                if (r2 <= cut * cut) s += amp * exp(-r2 * inv);
            }
    return s;
}

__global__ void setup_fields_kernel(const AtomG* __restrict__ at, int natom, int n1, int n2, int n3, double h1,
                                    double h2, double h3, double L1, double L2, double L3, double* __restrict__ b,
                                    double* __restrict__ sad, int isolated) {
    const long long ng = (long long)n1 * n2 * n3;
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < ng; g += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(g % n1), j = (int)((g / n1) % n2), k = (int)(g / ((long long)n1 * n2));
        const double x = i * h1, y = j * h2, z = k * h3;
        double sb = 0.0, ss = 0.0;
        for (int a = 0; a < natom; ++a) {
            sb += image_sum(x, y, z, at[a].pos, L1, L2, L3, at[a].amp_b, at[a].w_b, at[a].cut_b, isolated);
            ss += image_sum(x, y, z, at[a].pos, L1, L2, L3, at[a].amp_s, at[a].w_s, at[a].cut_s, isolated);
        }
        b[g] = sb;
        sad[g] = ss;
    }
}

// ---------------------------------------------------------------------------------------
// reductions: deterministic two-stage sums of several dot products
// ---------------------------------------------------------------------------------------
template <int K>
__global__ void multidot_kernel(const double* const* __restrict__ A, const double* const* __restrict__ B, long long n,
                                double* __restrict__ part) {
    double acc[K];
#pragma unroll
    for (int k = 0; k < K; ++k) acc[k] = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
#pragma unroll
        for (int k = 0; k < K; ++k)
            if (A[k]) acc[k] = fma(A[k][i], B[k][i], acc[k]);
    }
    __shared__ double sh[K][RB / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        double v = acc[k];
        for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
        if (lane == 0) sh[k][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x < K) {
        double v = 0.0;
        for (int w = 0; w < RB / 32; ++w) v += sh[threadIdx.x][w];
        part[(long long)blockIdx.x * K + threadIdx.x] = v;
    }
}

template <int K>
__global__ void multidot_finish_kernel(const double* __restrict__ part, int nblk, double* __restrict__ out) {
    const int k = threadIdx.x;
    if (k >= K) return;
    double v = 0.0;
    for (int b = 0; b < nblk; ++b) v += part[(long long)b * K + k];
    out[k] = v;
}

// ---------------------------------------------------------------------------------------
// LDA (Perdew & Zunger 1981): PZ81 correlation, Dirac exchange, von Barth-Hedin f(zeta)
// ---------------------------------------------------------------------------------------
struct PZ {
    double g, b1, b2, A, B, C, D;
};
__device__ __forceinline__ void pz_phase(double rs, const PZ& p, double& eps, double& mu) {
    if (rs >= 1.0) {
        const double s = sqrt(rs);
        const double den = 1.0 + p.b1 * s + p.b2 * rs;
        eps = p.g / den;
        mu = eps * (1.0 + 7.0 / 6.0 * p.b1 * s + 4.0 / 3.0 * p.b2 * rs) / den;
    } else {
        const double lr = log(rs);
        eps = p.A * lr + p.B + p.C * rs * lr + p.D * rs;
        mu = p.A * lr + (p.B - p.A / 3.0) + 2.0 / 3.0 * p.C * rs * lr + (2.0 * p.D - p.C) / 3.0 * rs;
    }
}

__global__ void lda_kernel(int nspin, const double* __restrict__ rho, double* __restrict__ exc,
                           double* __restrict__ vxc, long long n) {
    const PZ U{-0.1423, 1.0529, 0.3334, 0.0311, -0.048, 0.0020, -0.0116};
    const PZ P{-0.0843, 1.3981, 0.2611, 0.01555, -0.0269, 0.0007, -0.0048};
    const double floor_ = 1e-14;
    const double cx = -0.75 * cbrt(3.0 / M_PI);
    const double fden = pow(2.0, 4.0 / 3.0) - 2.0;
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < n; g += (long long)gridDim.x * blockDim.x) {
        if (nspin == 1) {
            const double r = fmax(rho[g], floor_);
            const double ex = cx * cbrt(r);
            const double rs = cbrt(3.0 / (4.0 * M_PI * r));
            double ec, vc;
            pz_phase(rs, U, ec, vc);
            exc[g] = ex + ec;
            vxc[g] = 4.0 / 3.0 * ex + vc;
        } else {
            const double ru = rho[g], rd = rho[n + g];
            const double r = fmax(ru + rd, floor_);
            const double z = fmin(1.0, fmax(-1.0, (ru - rd) / r));
            const double exu = cx * cbrt(r);
            const double opz = 1.0 + z, omz = 1.0 - z;
            const double c_opz = cbrt(opz), c_omz = cbrt(omz);
            const double ex = exu * 0.5 * (opz * c_opz + omz * c_omz);
            const double rs = cbrt(3.0 / (4.0 * M_PI * r));
            double eu, mu_u, ep, mu_p;
            pz_phase(rs, U, eu, mu_u);
            pz_phase(rs, P, ep, mu_p);
            const double f = (opz * c_opz + omz * c_omz - 2.0) / fden;
            const double df = 4.0 / 3.0 * (c_opz - c_omz) / fden;
            const double ec = eu + f * (ep - eu);
            const double vcc = mu_u + f * (mu_p - mu_u);
            exc[g] = ex + ec;
            vxc[g] = 4.0 / 3.0 * exu * c_opz + vcc + (ep - eu) * df * (1.0 - z);
            vxc[n + g] = 4.0 / 3.0 * exu * c_omz + vcc + (ep - eu) * df * (-1.0 - z);
        }
    }
}

__global__ void veff_kernel(int nspin, const double* __restrict__ phi, const double* __restrict__ vxc,
                            double* __restrict__ veff, float* __restrict__ veff32, long long n) {
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < n; g += (long long)gridDim.x * blockDim.x)
        for (int s = 0; s < nspin; ++s) {
            const double v = phi[g] + vxc[s * n + g];
            veff[s * n + g] = v;
            veff32[s * n + g] = (float)v;
        }
}

// ---------------------------------------------------------------------------------------
// elementwise helpers
// ---------------------------------------------------------------------------------------
template <typename T>
__global__ void axpby_kernel(T* __restrict__ y, const T* __restrict__ x, T a, T b, long long n) {
    // y = a*x + b*y
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = a * x[i] + b * y[i];
}
template <typename T, typename U>
__global__ void convert_add_kernel(T* __restrict__ y, const U* __restrict__ x, double a, double b, long long n) {
    // y = a*x + b*y with a type conversion (FP64 <-> FP32 vectors of the Poisson refinement)
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = (T)(a * (double)x[i] + b * (double)y[i]);
}
__global__ void to_float_grid_kernel(const double* __restrict__ a, float* __restrict__ b, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        b[i] = (float)a[i];
}
__global__ void add_scalar_kernel(double* __restrict__ y, const double* __restrict__ s, double scale, long long n) {
    const double v = scale * s[0];
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] += v;
}

// Anderson history push: X[slot] = x - xprev, F[slot] = c*f - fprev; xprev = x, fprev = c*f
template <typename T>
__global__ void anderson_push_kernel(const T* __restrict__ x, const T* __restrict__ f, T c, T* __restrict__ xprev,
                                     T* __restrict__ fprev, T* __restrict__ Xs, T* __restrict__ Fs, int have_prev,
                                     long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const T fi = c * f[i];
        if (have_prev) {
            Xs[i] = x[i] - xprev[i];
            Fs[i] = fi - fprev[i];
        }
        xprev[i] = x[i];
        fprev[i] = fi;
    }
}

// x += a*c*f - sum_j gamma_j (X_j + a F_j)   (gamma in device memory, m terms)
template <typename T>
__global__ void anderson_update_kernel(T* __restrict__ x, const T* __restrict__ f, T c, T a, const T* __restrict__ X,
                                       const T* __restrict__ F, const int* __restrict__ slots,
                                       const double* __restrict__ gamma, int m, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        T v = x[i] + a * c * f[i];
        for (int j = 0; j < m; ++j) {
            const long long o = (long long)slots[j] * n + i;
            v -= (T)gamma[j] * (X[o] + a * F[o]);
        }
        x[i] = v;
    }
}

// Gram of the history: G[i][j] = F_i . F_j (i <= j), r_i = F_i . (c f), plus f.f, for points
// [lo, hi) strided by `step`; C = history length at compile time keeps the accumulators in registers.
template <int C, typename T>
__device__ __forceinline__ void gram_accum(const T* __restrict__ F, const int* sl, const T* __restrict__ f, T c,
                                           long long n, long long lo, long long hi, long long step, double* out) {
    constexpr int ND = C * (C + 1) / 2 + C + 1;
    T acc[ND];
#pragma unroll
    for (int k = 0; k < ND; ++k) acc[k] = T(0);
    for (long long i = lo; i < hi; i += step) {
        T v[C > 0 ? C : 1];
#pragma unroll
        for (int j = 0; j < C; ++j) v[j] = F[(long long)sl[j] * n + i];
        const T fi = c * f[i];
        int k = 0;
#pragma unroll
        for (int a = 0; a < C; ++a)
#pragma unroll
            for (int b = a; b < C; ++b) acc[k++] += v[a] * v[b];
#pragma unroll
        for (int a = 0; a < C; ++a) acc[k++] += v[a] * fi;
        acc[k] += fi * fi;
    }
#pragma unroll
    for (int k = 0; k < ND; ++k) out[k] = (double)acc[k];
}

// per-thread partials of the history Gram for a runtime history length m <= 16
template <typename T>
__device__ void gram_accum_dispatch(int m, const T* F, const int* sl, const T* f, T c, long long n, long long lo,
                                    long long hi, long long step, double* out) {
    switch (m) {
#define SDFT_GRAM_CASE(CC) \
    case CC: gram_accum<CC, T>(F, sl, f, c, n, lo, hi, step, out); break;
        SDFT_GRAM_CASE(0) SDFT_GRAM_CASE(1) SDFT_GRAM_CASE(2) SDFT_GRAM_CASE(3) SDFT_GRAM_CASE(4) SDFT_GRAM_CASE(5)
        SDFT_GRAM_CASE(6) SDFT_GRAM_CASE(7) SDFT_GRAM_CASE(8) SDFT_GRAM_CASE(9) SDFT_GRAM_CASE(10) SDFT_GRAM_CASE(11)
        SDFT_GRAM_CASE(12) SDFT_GRAM_CASE(13) SDFT_GRAM_CASE(14) SDFT_GRAM_CASE(15) SDFT_GRAM_CASE(16)
#undef SDFT_GRAM_CASE
        default: break;
    }
}

// block-reduce nd per-thread values (in `vals`, one per thread slot) into part[blockIdx.x * nd + k]
template <int NW>
__device__ void block_reduce_partials(const double* vals, int nd, double* part_row, double (*sh)[NW]) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int k = 0; k < nd; ++k) {
        double v = vals[k];
        for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
        if (lane == 0) sh[k][warp] = v;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < nd; k += blockDim.x) {
        double v = 0.0;
        for (int w = 0; w < NW; ++w) v += sh[k][w];
        part_row[k] = v;
    }
}

constexpr int GRAM_MAXND = 16 * 17 / 2 + 16 + 1;

template <typename T>
__global__ void __launch_bounds__(RB) anderson_gram_kernel(const T* __restrict__ F, const int* __restrict__ slots,
                                                           int m, const T* __restrict__ f, T c, long long n,
                                                           double* __restrict__ part) {
    __shared__ double sh[GRAM_MAXND][RB / 32];
    int sl[16];
    for (int j = 0; j < m; ++j) sl[j] = slots[j];
    double vals[GRAM_MAXND];
    const long long step = (long long)gridDim.x * blockDim.x;
    gram_accum_dispatch<T>(m, F, sl, f, c, n, blockIdx.x * (long long)blockDim.x + threadIdx.x, n, step, vals);
    const int nd = m * (m + 1) / 2 + m + 1;
    block_reduce_partials<RB / 32>(vals, nd, part + (long long)blockIdx.x * nd, sh);
}

// sum partials (one thread per entry, in block order), then solve (F^T F) gamma = F^T f by
// Gaussian elimination with partial pivoting on one thread
__device__ void anderson_solve_block(const double* __restrict__ part, int nblk, int m, double* gamma, double* ff) {
    __shared__ double s[GRAM_MAXND];
    const int nd = m * (m + 1) / 2 + m + 1;
    for (int k = threadIdx.x; k < nd; k += blockDim.x) {
        double v = 0.0;
        for (int b = 0; b < nblk; ++b) v += part[(long long)b * nd + k];
        s[k] = v;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    double G[16][17];
    int k = 0;
    for (int a = 0; a < m; ++a)
        for (int b = a; b < m; ++b) {
            G[a][b] = s[k];
            G[b][a] = s[k];
            ++k;
        }
    for (int a = 0; a < m; ++a) G[a][m] = s[k++];
    *ff = s[k];
    for (int col = 0; col < m; ++col) {
        int piv = col;
        for (int r = col + 1; r < m; ++r)
            if (fabs(G[r][col]) > fabs(G[piv][col])) piv = r;
        if (piv != col)
            for (int q = 0; q <= m; ++q) {
                const double t = G[col][q];
                G[col][q] = G[piv][q];
                G[piv][q] = t;
            }
        const double d = G[col][col];
        for (int r = col + 1; r < m; ++r) {
            const double fct = d != 0.0 ? G[r][col] / d : 0.0;
            for (int q = col; q <= m; ++q) G[r][q] -= fct * G[col][q];
        }
    }
    for (int r = m - 1; r >= 0; --r) {
        double v = G[r][m];
        for (int q = r + 1; q < m; ++q) v -= G[r][q] * gamma[q];
        gamma[r] = G[r][r] != 0.0 ? v / G[r][r] : 0.0;
    }
}

__global__ void anderson_solve_kernel(const double* __restrict__ part, int nblk, int m, double* __restrict__ gamma,
                                      double* __restrict__ ff) {
    anderson_solve_block(part, nblk, m, gamma, ff);
}

// ---------------------------------------------------------------------------------------
// density from orbitals (Eq. 2): rho[g] += weight * sum_n occ[n] |X[g,n]|^2 / dV
// ---------------------------------------------------------------------------------------
template <int KIND>  // 0 FP64 real, 1 FP64 complex, 2 FP32 paired real, 3 FP32 complex
__global__ void density_kernel(const void* __restrict__ X, const double* __restrict__ occ, int ncol, double scale,
                               long long ng, double* __restrict__ rho) {
    // states past the last one with |occ| > 1e-14 change rho below FP64 rounding and are not read;
    // the FP32 kinds square and weight in FP32 (the orbitals carry FP32 rounding already) and add
    // groups of eight pairs into the FP64 sum, so that the few FP64 pipes of the GPU do not bound
    // a pass that should stream the block at HBM speed
    extern __shared__ float occf[];
    __shared__ int nlast;
    if (threadIdx.x == 0) nlast = 0;
    __syncthreads();
    for (int n = threadIdx.x; n < ncol; n += blockDim.x) {
        const double o = occ[n];
        if (KIND >= 2) occf[n] = (float)o;
        if (fabs(o) > 1e-14) atomicMax(&nlast, n + 1);
    }
    __syncthreads();
    const int nc = nlast;
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < ng; g += (long long)gridDim.x * blockDim.x) {
        double s = 0.0;
        if (KIND == 0) {
            const double* x = (const double*)X;
            for (int n = 0; n < nc; ++n) {
                const double v = x[(long long)n * ng + g];
                s += occ[n] * v * v;
            }
        } else if (KIND == 1) {
            const double2* x = (const double2*)X;
            for (int n = 0; n < nc; ++n) {
                const double2 v = x[(long long)n * ng + g];
                s += occ[n] * (v.x * v.x + v.y * v.y);
            }
        } else if (KIND == 2) {
            const float2* x = (const float2*)X;
            const int np = (nc + 1) / 2;
            for (int p0 = 0; p0 < np; p0 += 8) {
                float sf = 0.f;
                if (p0 + 8 <= np) {   // eight loads in flight
                    float2 v[8];
#pragma unroll
                    for (int i = 0; i < 8; ++i) v[i] = x[(long long)(p0 + i) * ng + g];
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        sf = fmaf(occf[2 * (p0 + i)], v[i].x * v[i].x, sf);
                        sf = fmaf(occf[2 * (p0 + i) + 1], v[i].y * v[i].y, sf);
                    }
                } else {
                    for (int p = p0; p < np; ++p) {
                        const float2 v = x[(long long)p * ng + g];
                        sf = fmaf(occf[2 * p], v.x * v.x, sf);
                        sf = fmaf(occf[2 * p + 1], v.y * v.y, sf);
                    }
                }
                s += (double)sf;
            }
        } else {
            const float2* x = (const float2*)X;
            for (int n0 = 0; n0 < nc; n0 += 8) {
                float sf = 0.f;
                const int n1 = min(nc, n0 + 8);
                for (int n = n0; n < n1; ++n) {
                    const float2 v = x[(long long)n * ng + g];
                    sf = fmaf(occf[n], v.x * v.x + v.y * v.y, sf);
                }
                s += (double)sf;
            }
        }
        rho[g] += scale * s;
    }
}

// ---------------------------------------------------------------------------------------
// Fermi level: bisection on sum_{s,k} w_k sum_n g = N_e, g = f_s / (1 + exp((e - mu)/kT))
// one CTA; writes occ, out[0] = mu, out[1] = -TS, out[2] = band energy sum w g e
// ---------------------------------------------------------------------------------------
__global__ void fermi_kernel(const double* __restrict__ eig, const double* __restrict__ kw, int nspin, int nk, int ns,
                             double nelec, double kT, double fs, double* __restrict__ occ, double* __restrict__ out) {
    __shared__ double red[1024 / 32];
    __shared__ double lo_s, hi_s;
    const int total = nspin * nk * ns;
    double emin = 1e300, emax = -1e300;
    for (int i = threadIdx.x; i < total; i += blockDim.x) {
        emin = fmin(emin, eig[i]);
        emax = fmax(emax, eig[i]);
    }
    auto block_reduce = [&](double v, int op) -> double {  // op 0 sum, 1 min, 2 max
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        for (int off = 16; off > 0; off >>= 1) {
            const double o = __shfl_down_sync(0xffffffffu, v, off);
            v = op == 0 ? v + o : (op == 1 ? fmin(v, o) : fmax(v, o));
        }
        __syncthreads();
        if (lane == 0) red[warp] = v;
        __syncthreads();
        double r = red[0];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
            r = op == 0 ? r + red[w] : (op == 1 ? fmin(r, red[w]) : fmax(r, red[w]));
        return r;
    };
    emin = block_reduce(emin, 1);
    emax = block_reduce(emax, 2);
    if (threadIdx.x == 0) {
        lo_s = emin - 50.0 * kT - 1.0;
        hi_s = emax + 50.0 * kT + 1.0;
    }
    __syncthreads();
    // safeguarded Newton on N(mu) = N_e: the bracket [lo, hi] shrinks every step (bisection
    // semantics as in the definition), the next trial point is the Newton step when it falls
    // inside the bracket, else the midpoint
    __shared__ double mu_s, red2[1024 / 32];
    __shared__ int done_s;
    if (threadIdx.x == 0) {
        mu_s = 0.5 * (lo_s + hi_s);
        done_s = 0;
    }
    __syncthreads();
    for (int it = 0; it < 200; ++it) {
        const double mid = mu_s;
        double cnt = 0.0, der = 0.0;
        for (int i = threadIdx.x; i < total; i += blockDim.x) {
            const int k = (i / ns) % nk;
            const double f = 0.5 * (1.0 - tanh(0.5 * (eig[i] - mid) / kT));
            cnt += kw[k] * fs * f;
            der += kw[k] * fs * f * (1.0 - f) / kT;
        }
        cnt = block_reduce(cnt, 0);
        {   // second sum through its own scratch row
            const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
            for (int off = 16; off > 0; off >>= 1) der += __shfl_down_sync(0xffffffffu, der, off);
            if (lane == 0) red2[warp] = der;
            __syncthreads();
            double r = red2[0];
            for (int w = 1; w < (int)(blockDim.x >> 5); ++w) r += red2[w];
            der = r;
        }
        if (threadIdx.x == 0) {
            if (cnt < nelec) lo_s = mid;
            else hi_s = mid;
            double next = 0.5 * (lo_s + hi_s);
            if (der > 0.0) {
                const double newton = mid + (nelec - cnt) / der;
                if (newton > lo_s && newton < hi_s) next = newton;
            }
            if (fabs(cnt - nelec) <= 1e-14 * fmax(1.0, nelec) || hi_s - lo_s < 1e-15 * fmax(1.0, fabs(mid))) {
                done_s = 1;
                next = mid;
            }
            mu_s = next;
        }
        __syncthreads();
        if (done_s) break;
    }
    const double mu = mu_s;
    double ts = 0.0, eb = 0.0;
    for (int i = threadIdx.x; i < total; i += blockDim.x) {
        const int k = (i / ns) % nk;
        const double g = fs * 0.5 * (1.0 - tanh(0.5 * (eig[i] - mu) / kT));
        occ[i] = g;
        const double f = g / fs;
        double t = 0.0;
        if (f > 0.0) t += f * log(f);
        if (f < 1.0) t += (1.0 - f) * log(1.0 - f);
        ts += kw[k] * fs * kT * t;
        eb += kw[k] * g * eig[i];
    }
    ts = block_reduce(ts, 0);
    eb = block_reduce(eb, 0);
    if (threadIdx.x == 0) {
        out[0] = mu;
        out[1] = ts;
        out[2] = eb;
    }
}

// ---------------------------------------------------------------------------------------
// forces
// ---------------------------------------------------------------------------------------
// local part per atom: -dV sum_x (x - R - T)/r_loc^2 b_a(x - R - T) phi(x); one CTA per atom
__global__ void force_local_kernel(const AtomG* __restrict__ at, int n1, int n2, int n3, double h1, double h2,
                                   double h3, double L1, double L2, double L3, double dV,
                                   const double* __restrict__ phi, double* __restrict__ F, int isolated) {
    const int a = blockIdx.x;
    const AtomG A = at[a];
    const double cut = A.cut_b;
    int lo[3], dim[3];
    const double h[3] = {h1, h2, h3};
    for (int d = 0; d < 3; ++d) {
        lo[d] = (int)ceil((A.pos[d] - cut) / h[d]);
        dim[d] = (int)floor((A.pos[d] + cut) / h[d]) - lo[d] + 1;
    }
    const long long total = (long long)dim[0] * dim[1] * dim[2];
    double acc[3] = {0, 0, 0};
    const double inv = 1.0 / (2.0 * A.w_b * A.w_b);
    for (long long p = threadIdx.x; p < total; p += blockDim.x) {
        const int ix = (int)(p % dim[0]), iy = (int)((p / dim[0]) % dim[1]), iz = (int)(p / ((long long)dim[0] * dim[1]));
        const int I[3] = {lo[0] + ix, lo[1] + iy, lo[2] + iz};
        const double dx = I[0] * h1 - A.pos[0], dy = I[1] * h2 - A.pos[1], dz = I[2] * h3 - A.pos[2];
        const double r2 = dx * dx + dy * dy + dz * dz;
        if (r2 > cut * cut) continue;
        if (isolated && (I[0] < 0 || I[0] >= n1 || I[1] < 0 || I[1] >= n2 || I[2] < 0 || I[2] >= n3)) continue;
        const int g0 = ((I[0] % n1) + n1) % n1, g1 = ((I[1] % n2) + n2) % n2, g2 = ((I[2] % n3) + n3) % n3;
        const double ph = phi[((long long)g2 * n2 + g1) * n1 + g0];
        const double bv = A.amp_b * exp(-r2 * inv);
        const double s = bv * ph / (A.w_b * A.w_b);
        acc[0] += dx * s;
        acc[1] += dy * s;
        acc[2] += dz * s;
    }
    __shared__ double sh[3][RB / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int d = 0; d < 3; ++d) {
        double v = acc[d];
        for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
        if (lane == 0) sh[d][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double v = 0.0;
        for (int w = 0; w < RB / 32; ++w) v += sh[threadIdx.x][w];
        F[3 * a + threadIdx.x] -= dV * v;
        (void)L1;
        (void)L2;
        (void)L3;
    }
}

// nonlocal part per atom: C_n = sum_j conj(beta_j) X[j,n], D_nd = sum_j conj(dbeta_j/dR_d) X[j,n]
// F_d -= w_k dV E_kb sum_n g_n 2 Re(conj(C_n) D_nd); FP64 blocks (real or complex)
template <bool CPLX>
__global__ void force_nl_kernel(const int* __restrict__ cnt, const int* __restrict__ idx, const int* __restrict__ img,
                                const double* __restrict__ val, int cap, const double* __restrict__ X, int ncol,
                                long long ng, const double* __restrict__ occ, double wk, const double* __restrict__ gamma,
                                const double* __restrict__ apos, const double* __restrict__ rp2, int n1, int n2,
                                double h1, double h2, double h3, double* __restrict__ F) {
    const int a = blockIdx.x;
    const int m = cnt[a];
    const double R[3] = {apos[3 * a], apos[3 * a + 1], apos[3 * a + 2]};
    double fsum[3] = {0, 0, 0};
    __shared__ double sh[8][RB / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int n = 0; n < ncol; ++n) {
        double c[2] = {0, 0}, d[3][2] = {{0, 0}, {0, 0}, {0, 0}};
        for (int j = threadIdx.x; j < m; j += blockDim.x) {
            const long long e = (long long)a * cap + j;
            const int g = idx[e];
            const int pk = img[e];
            const int t0 = (pk & 1023) - 512, t1 = ((pk >> 10) & 1023) - 512, t2 = ((pk >> 20) & 1023) - 512;
            const int gx = g % n1, gy = (g / n1) % n2, gz = g / (n1 * n2);
            // unwrapped box point I = g + t n;   displacement x_I - R
            const double disp[3] = {(gx + (double)t0 * n1) * h1 - R[0], (gy + (double)t1 * n2) * h2 - R[1],
                                    (gz + (double)t2 * (ng / ((long long)n1 * n2))) * h3 - R[2]};
            double br, bi;
            if (CPLX) {
                br = val[2 * e];
                bi = val[2 * e + 1];
            } else {
                br = val[e];
                bi = 0.0;
            }
            double xr, xi;
            if (CPLX) {
                xr = X[2 * ((long long)n * ng + g)];
                xi = X[2 * ((long long)n * ng + g) + 1];
            } else {
                xr = X[(long long)n * ng + g];
                xi = 0.0;
            }
            // conj(beta) * x
            const double pr = br * xr + bi * xi, pi = br * xi - bi * xr;
            c[0] += pr;
            c[1] += pi;
            for (int q = 0; q < 3; ++q) {
                const double s = disp[q] / rp2[a];
                d[q][0] += s * pr;
                d[q][1] += s * pi;
            }
        }
        double vals[8] = {c[0], c[1], d[0][0], d[0][1], d[1][0], d[1][1], d[2][0], d[2][1]};
        for (int k = 0; k < 8; ++k) {
            double v = vals[k];
            for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
            if (lane == 0) sh[k][warp] = v;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double s[8];
            for (int k = 0; k < 8; ++k) {
                s[k] = 0.0;
                for (int w = 0; w < RB / 32; ++w) s[k] += sh[k][w];
            }
            for (int q = 0; q < 3; ++q) fsum[q] += occ[n] * 2.0 * (s[0] * s[2 + 2 * q] + s[1] * s[3 + 2 * q]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int q = 0; q < 3; ++q) F[3 * a + q] -= wk * gamma[a] * fsum[q];
}

inline unsigned nblocks(long long n, int bs = 256) {
    return (unsigned)std::min<long long>((n + bs - 1) / bs, 152LL * 16);
}

std::vector<AtomG> atom_g(sdft_ctx* c) {
    std::vector<AtomG> at(c->natom);
    for (int a = 0; a < c->natom; ++a) {
        const sdft_pseudo& s = c->species[c->types[a]];
        for (int d = 0; d < 3; ++d) at[a].pos[d] = c->pos[3 * a + d];
        at[a].amp_b = -s.Z * std::pow(2.0 * M_PI * s.r_loc * s.r_loc, -1.5);
        at[a].w_b = s.r_loc;
        at[a].cut_b = 10.0 * s.r_loc;
        at[a].amp_s = s.Z * std::pow(2.0 * M_PI * s.sad_width * s.sad_width, -1.5);
        at[a].w_s = s.sad_width;
        at[a].cut_s = 10.0 * s.sad_width;
    }
    return at;
}

}  // namespace

// out[k] = a_k . b_k for k < count (<= 8), synchronously to host
void dots_host(sdft_ctx* c, int count, const double* const* a, const double* const* b, long long n, double* host_out) {
    SDFT_REQUIRE(count >= 1 && count <= 8, SDFT_ERR_INVALID_ARG, "dots_host: count");
    const double* pa[8] = {nullptr};
    const double* pb[8] = {nullptr};
    for (int k = 0; k < count; ++k) {
        pa[k] = a[k];
        pb[k] = b[k];
    }
    // pointer tables live in the small scalar area
    const double** dA = (const double**)(c->scal + 1024);
    const double** dB = (const double**)(c->scal + 1024 + 8);
    double* part = c->scal + 2048;
    double* out = c->scal + 1536;
    SDFT_CUDA(cudaMemcpyAsync((void*)dA, pa, sizeof(pa), cudaMemcpyHostToDevice, c->stream));
    SDFT_CUDA(cudaMemcpyAsync((void*)dB, pb, sizeof(pb), cudaMemcpyHostToDevice, c->stream));
    const int nblk = 128;  // 128 blocks x 8 dots fits in the 2048-double partial area
    multidot_kernel<8><<<nblk, RB, 0, c->stream>>>(dA, dB, n, part);
    multidot_finish_kernel<8><<<1, 32, 0, c->stream>>>(part, nblk, out);
    SDFT_CUDA(cudaGetLastError());
    count_launch(c, 2);
    SDFT_CUDA(cudaMemcpyAsync(c->hscal, out, sizeof(double) * 8, cudaMemcpyDeviceToHost, c->stream));
    SDFT_CUDA(cudaStreamSynchronize(c->stream));
    for (int k = 0; k < count; ++k) host_out[k] = c->hscal[k];
}

void build_pseudocharge_and_sad(sdft_ctx* c) {
    std::vector<AtomG> at = atom_g(c);
    AtomG* dat = (AtomG*)ctx_alloc(c, sizeof(AtomG) * std::max(1, c->natom));
    SDFT_CUDA(cudaMemcpyAsync(dat, at.data(), sizeof(AtomG) * c->natom, cudaMemcpyHostToDevice, c->stream));
    setup_fields_kernel<<<nblocks(c->ng), 256, 0, c->stream>>>(dat, c->natom, c->n[0], c->n[1], c->n[2], c->h[0],
                                                              c->h[1], c->h[2], c->L[0], c->L[1], c->L[2], c->b,
                                                              c->rho_sad, c->opt.boundary == SDFT_BC_DIRICHLET);
    SDFT_CUDA(cudaGetLastError());
    count_launch(c);
    // normalise the SAD density to N_e: sum rho = rho . 1
    double* ones = c->work64;
    SDFT_CUDA(cudaMemsetAsync(ones, 0, sizeof(double) * c->ng, c->stream));
    c->hscal[0] = 1.0;
    SDFT_CUDA(cudaMemcpyAsync(c->scal, c->hscal, sizeof(double), cudaMemcpyHostToDevice, c->stream));
    add_scalar_kernel<<<nblocks(c->ng), 256, 0, c->stream>>>(ones, c->scal, 1.0, c->ng);
    count_launch(c);
    const double* a[1] = {c->rho_sad};
    const double* b[1] = {ones};
    double s = 0.0;
    dots_host(c, 1, a, b, c->ng, &s);
    const double scale = c->nelec / (c->dV * s);
    axpby_kernel<double><<<nblocks(c->ng), 256, 0, c->stream>>>(c->rho_sad, c->rho_sad, 0.0, scale, c->ng);
    SDFT_CUDA(cudaGetLastError());
    count_launch(c);
    ctx_release(c, dat);
}

// ---------------------------------------------------------------------------------------
// PBE GGA, spin-unpolarized (paper Sec. 2.2 functionalities; Perdew, Burke & Ernzerhof 1996 with the
// Perdew-Wang 1992 correlation of the uniform gas).  On the grid: g_d = D_d rho with the order-12
// centred first-derivative stencil (periodic), sigma = sum_d g_d^2, f(rho, sigma) = rho eps_xc, and
// v_xc = f_rho - 2 sum_d D_d (f_sigma g_d), the exact derivative of E_xc = dV sum_g f (D_d^T = -D_d).
// ---------------------------------------------------------------------------------------
namespace {
struct D1Coef {
    double c[3][FD_RADIUS + 1];   // c_k / h_d, k = 1..6: (D_d u)(x) = sum_k c_k (u(x + k e_d) - u(x - k e_d))
};

// out_d = D_d u for the three axes (in0 == in1 == in2 == u), or out0 -= sum_d D_d in_d (accumulate)
template <bool DIV>
__global__ void __launch_bounds__(256) d1_kernel(const double* __restrict__ in0, const double* __restrict__ in1,
                                                 const double* __restrict__ in2, double* __restrict__ out0,
                                                 double* __restrict__ out1, double* __restrict__ out2, D1Coef K,
                                                 int n1, int n2, int n3) {
    const int plane = n1 * n2;
    const int ng = plane * n3;
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= ng) return;
    const int k = g / plane;
    const int rem = g - k * plane;
    const int j = rem / n1;
    const int i = rem - j * n1;
    const int row = g - i, col = g - j * n1, pl = g - k * plane;
    double dx = 0.0, dy = 0.0, dz = 0.0;
#pragma unroll
    for (int r = 1; r <= FD_RADIUS; ++r) {
        int ip = i + r, im = i - r, jp = j + r, jm = j - r, kp = k + r, km = k - r;
        ip -= ip >= n1 ? n1 : 0;
        im += im < 0 ? n1 : 0;
        jp -= jp >= n2 ? n2 : 0;
        jm += jm < 0 ? n2 : 0;
        kp -= kp >= n3 ? n3 : 0;
        km += km < 0 ? n3 : 0;
        dx += K.c[0][r] * (in0[row + ip] - in0[row + im]);
        dy += K.c[1][r] * (in1[col + jp * n1] - in1[col + jm * n1]);
        dz += K.c[2][r] * (in2[pl + kp * plane] - in2[pl + km * plane]);
    }
    if (DIV) {
        out0[g] -= dx + dy + dz;
    } else {
        out0[g] = dx;
        out1[g] = dy;
        out2[g] = dz;
    }
}

constexpr double PBE_KAPPA = 0.804;
constexpr double PBE_BETA = 0.06672455060314922;
constexpr double PW92_A = 0.031091, PW92_A1 = 0.21370, PW92_B1 = 7.5957, PW92_B2 = 3.5876, PW92_B3 = 1.6382,
                 PW92_B4 = 0.49294;

// eps_xc (per electron), f_rho and f_sigma of PBE at one point, analytic derivatives
__device__ void pbe_eval(double rho, double sigma, double& eps, double& frho, double& fsig) {
    const double pi = 3.14159265358979323846;
    const double mu = PBE_BETA * pi * pi / 3.0;
    const double gam = (1.0 - log(2.0)) / (pi * pi);
    const double r = fmax(rho, 1e-14);
    const double kf = cbrt(3.0 * pi * pi * r);
    const double exu = -3.0 * kf / (4.0 * pi);
    // exchange: f_x = r exu F_x(s2), s2 = sigma / (4 kf^2 r^2) ~ sigma r^(-8/3)
    const double s2den = 4.0 * kf * kf * r * r;
    const double s2 = sigma / s2den;
    const double den = PBE_KAPPA + mu * s2;
    const double Fx = 1.0 + PBE_KAPPA - PBE_KAPPA * PBE_KAPPA / den;
    const double dFx = mu * PBE_KAPPA * PBE_KAPPA / (den * den);   // dF_x / ds2
    const double fx = r * exu * Fx;
    const double fx_r = (4.0 / 3.0) * exu * Fx - (8.0 / 3.0) * exu * dFx * s2;
    const double fx_s = r * exu * dFx / s2den;
    // PW92 correlation of the uniform gas, eps_c(rs), rs = (3 / (4 pi r))^(1/3)
    const double rs = cbrt(3.0 / (4.0 * pi * r));
    const double sq = sqrt(rs);
    const double Q = 2.0 * PW92_A * (PW92_B1 * sq + PW92_B2 * rs + PW92_B3 * rs * sq + PW92_B4 * rs * rs);
    const double dQ = 2.0 * PW92_A * (0.5 * PW92_B1 / sq + PW92_B2 + 1.5 * PW92_B3 * sq + 2.0 * PW92_B4 * rs);
    const double Lq = log1p(1.0 / Q);
    const double ec = -2.0 * PW92_A * (1.0 + PW92_A1 * rs) * Lq;
    const double dec_drs = -2.0 * PW92_A * PW92_A1 * Lq + 2.0 * PW92_A * (1.0 + PW92_A1 * rs) * dQ / (Q * (1.0 + Q));
    const double dec_dr = -dec_drs * rs / (3.0 * r);
    // gradient correction H(ec, t2), t2 = sigma / (4 ks^2 r^2) ~ sigma r^(-7/3), ks^2 = 4 kf / pi
    const double t2den = 16.0 * kf * r * r / pi;
    const double t2 = sigma / t2den;
    const double E = exp(-ec / gam);
    const double A = (PBE_BETA / gam) / (E - 1.0);
    const double dA_dec = (PBE_BETA / (gam * gam)) * E / ((E - 1.0) * (E - 1.0));
    const double y = A * t2;
    const double Dn = 1.0 + y + y * y;
    const double Z = (PBE_BETA / gam) * t2 * (1.0 + y) / Dn;
    const double H = gam * log1p(Z);
    const double dH_dt2 = PBE_BETA * (1.0 + 2.0 * y) / ((1.0 + Z) * Dn * Dn);
    const double dH_dA = -PBE_BETA * t2 * t2 * y * (2.0 + y) / ((1.0 + Z) * Dn * Dn);
    const double fc = r * (ec + H);
    const double fc_r = ec + H + r * dec_dr * (1.0 + dH_dA * dA_dec) - (7.0 / 3.0) * dH_dt2 * t2;
    const double fc_s = r * dH_dt2 / t2den;
    eps = (fx + fc) / r;
    frho = fx_r + fc_r;
    fsig = fx_s + fc_s;
}

// exc = eps_xc, vxc = f_rho, w_d = 2 f_sigma g_d  (the divergence kernel then subtracts sum_d D_d w_d)
__global__ void pbe_point_kernel(const double* __restrict__ rho, const double* __restrict__ g0,
                                 const double* __restrict__ g1, const double* __restrict__ g2,
                                 double* __restrict__ exc, double* __restrict__ vxc, double* __restrict__ w0,
                                 double* __restrict__ w1, double* __restrict__ w2, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double a = g0[i], b = g1[i], cc = g2[i];
        double eps, fr, fs;
        pbe_eval(rho[i], a * a + b * b + cc * cc, eps, fr, fs);
        exc[i] = eps;
        vxc[i] = fr;
        w0[i] = 2.0 * fs * a;
        w1[i] = 2.0 * fs * b;
        w2[i] = 2.0 * fs * cc;
    }
}
}  // namespace

static void gga_pbe_device(sdft_ctx* c, const double* rho, double* exc, double* vxc) {
    const long long n = c->ng;
    if (!c->gga_ws) c->gga_ws = (double*)ctx_alloc(c, sizeof(double) * 6 * (size_t)n);
    double* g = c->gga_ws;
    double* w = c->gga_ws + 3 * n;
    // first-derivative weights c_k = (-1)^(k+1) (p!)^2 / (k (p-k)! (p+k)!), p = 6
    D1Coef K;
    {
        auto fact = [](int m) {
            double f = 1.0;
            for (int q = 2; q <= m; ++q) f *= q;
            return f;
        };
        const int p = FD_RADIUS;
        for (int d = 0; d < 3; ++d) {
            K.c[d][0] = 0.0;
            for (int k = 1; k <= p; ++k)
                K.c[d][k] = ((k % 2) ? 1.0 : -1.0) * fact(p) * fact(p) / (k * fact(p - k) * fact(p + k)) / c->h[d];
        }
    }
    const unsigned nbk = (unsigned)((n + 255) / 256);
    d1_kernel<false><<<nbk, 256, 0, c->stream>>>(rho, rho, rho, g, g + n, g + 2 * n, K, c->n[0], c->n[1], c->n[2]);
    pbe_point_kernel<<<nblocks(n), 256, 0, c->stream>>>(rho, g, g + n, g + 2 * n, exc, vxc, w, w + n, w + 2 * n, n);
    d1_kernel<true><<<nbk, 256, 0, c->stream>>>(w, w + n, w + 2 * n, vxc, nullptr, nullptr, K, c->n[0], c->n[1],
                                                 c->n[2]);
    SDFT_CUDA(cudaGetLastError());
    count_launch(c, 3);
}

void lda_device(sdft_ctx* c, int nspin, const double* rho, double* exc, double* vxc, size_t n) {
    if (c->opt.xc == SDFT_XC_GGA_PBE) {
        SDFT_REQUIRE(nspin == 1 && (long long)n == c->ng, SDFT_ERR_INVALID_ARG,
                     "PBE: spin-unpolarized densities on the context's grid only");
        gga_pbe_device(c, rho, exc, vxc);
        return;
    }
    lda_kernel<<<nblocks((long long)n), 256, 0, c->stream>>>(nspin, rho, exc, vxc, (long long)n);
    SDFT_CUDA(cudaGetLastError());
    count_launch(c);
}

// V_eff^s = phi + v_xc^s from rho_in (Poisson solved by the caller into c->phi)
void veff_assemble(sdft_ctx* c) {
    const int ns = c->opt.nspin;
    double* vxc = c->work64 + 2 * c->ng;  // [nspin][ng]
    lda_device(c, ns, c->rho_in, c->exc, vxc, (size_t)c->ng);
    veff_kernel<<<nblocks(c->ng), 256, 0, c->stream>>>(ns, c->phi, vxc, c->veff, c->veff32, c->ng);
    SDFT_CUDA(cudaGetLastError());
    count_launch(c);
}

void veff_to_float(sdft_ctx* c, int spin) {
    const long long n = c->ng;
    to_float_grid_kernel<<<nblocks(n), 256, 0, c->stream>>>(c->veff + spin * n, c->veff32 + spin * n, n);
    SDFT_CUDA(cudaGetLastError());
    count_launch(c);
}

// ---------------------------------------------------------------------------------------
// Single-vector Laplacian step for the Poisson solver: out = -2 alpha (-1/2 L x) - beta b, i.e.
// with alpha = -2, beta = -1:  out = b + L x (the residual of -L x = b).  One thread per grid
// point with direct neighbour loads: the vector is a few MB and stays in L2, so a flat grid of
// short independent threads beats the z-marching tile kernel built for orbital blocks.
// ---------------------------------------------------------------------------------------
struct LapCoef {
    double c[3][FD_RADIUS + 1];  // -1/2 w_r / h_d^2
    double c0;
};

template <typename T>
__global__ void __launch_bounds__(256) laplacian_residual_kernel(const T* __restrict__ x, const T* __restrict__ b,
                                                                 T* __restrict__ out, LapCoef K, int n1, int n2,
                                                                 int n3, T shift, int dirichlet) {
    // 32-bit indices: the grid has < 2^31 points
    const int plane = n1 * n2;
    const int ng = plane * n3;
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= ng) return;
    const int k = g / plane;
    const int rem = g - k * plane;
    const int j = rem / n1;
    const int i = rem - j * n1;
    const int row = g - i, col = g - j * n1, pl = g - k * plane;
    T acc = (T)K.c0 * x[g];
#pragma unroll
    for (int r = 1; r <= FD_RADIUS; ++r) {
        int ip = i + r, im = i - r, jp = j + r, jm = j - r, kp = k + r, km = k - r;
        ip -= ip >= n1 ? n1 : 0;
        im += im < 0 ? n1 : 0;
        jp -= jp >= n2 ? n2 : 0;
        jm += jm < 0 ? n2 : 0;
        kp -= kp >= n3 ? n3 : 0;
        km += km < 0 ? n3 : 0;
        if (dirichlet) {   // zero beyond the grid (isolated systems: ghost values enter through b)
            acc += (T)K.c[0][r] * ((i + r < n1 ? x[row + ip] : (T)0) + (i - r >= 0 ? x[row + im] : (T)0));
            acc += (T)K.c[1][r] * ((j + r < n2 ? x[col + jp * n1] : (T)0) + (j - r >= 0 ? x[col + jm * n1] : (T)0));
            acc += (T)K.c[2][r] * ((k + r < n3 ? x[pl + kp * plane] : (T)0) + (k - r >= 0 ? x[pl + km * plane] : (T)0));
        } else {
            acc += (T)K.c[0][r] * (x[row + ip] + x[row + im]);
            acc += (T)K.c[1][r] * (x[col + jp * n1] + x[col + jm * n1]);
            acc += (T)K.c[2][r] * (x[pl + kp * plane] + x[pl + km * plane]);
        }
    }
    // -L x = 2 * (-1/2 L x): out = b + L x - shift x = b - 2 acc - shift x  (residual of (-L + shift) x = b)
    out[g] = b[g] - (T)2 * acc - shift * x[g];
}

template <typename T>
void laplacian_residual(sdft_ctx* c, const T* x, const T* b, T* out, T shift = T(0)) {
    LapCoef K;
    for (int r = 0; r <= FD_RADIUS; ++r) {
        K.c[0][r] = c->coef.cx[r];
        K.c[1][r] = c->coef.cy[r];
        K.c[2][r] = c->coef.cz[r];
    }
    K.c0 = c->coef.c0;
    laplacian_residual_kernel<T><<<(unsigned)((c->ng + 255) / 256), 256, 0, c->stream>>>(
        x, b, out, K, c->n[0], c->n[1], c->n[2], shift, c->opt.boundary == SDFT_BC_DIRICHLET ? 1 : 0);
    SDFT_CUDA(cudaGetLastError());
    count_launch(c);
}

// ---------------------------------------------------------------------------------------
// Isolated systems (paper Sec. 2, 2.1: Dirichlet boundary conditions with multipole boundary values).
// q_lm = dV sum_g f_g r^l Y_lm about the centre of the grid box (l <= 6, real orthonormal Y_lm), and in
// the 6 ghost layers phi = sum 4 pi / (2l + 1) q_lm Y_lm / r^(l+1); inside -L0 phi = 4 pi f + G with
// L0 the zero-padded Laplacian and G the ghost values' share of the stencil.
// ---------------------------------------------------------------------------------------
namespace {
constexpr int MP_LMAX = 6, MP_NLM = (MP_LMAX + 1) * (MP_LMAX + 1);

// real orthonormal spherical harmonics of the direction (x, y, z), index l^2 + l + m (associated Legendre
// functions by the standard three-term recurrence; any real orthonormal basis gives the same potential)
__device__ void real_sh(double x, double y, double z, double* Y) {
    const double r = sqrt(x * x + y * y + z * z);
    double ct = 1.0, st = 0.0, cp = 1.0, sp = 0.0;
    if (r > 0.0) {
        ct = z / r;
        const double rxy = sqrt(x * x + y * y);
        st = rxy / r;
        if (rxy > 0.0) {
            cp = x / rxy;
            sp = y / rxy;
        }
    }
    double P[MP_LMAX + 1][MP_LMAX + 1];
    P[0][0] = 1.0;
    for (int m = 1; m <= MP_LMAX; ++m) P[m][m] = P[m - 1][m - 1] * (2 * m - 1) * st;
    for (int m = 0; m < MP_LMAX; ++m) P[m + 1][m] = ct * (2 * m + 1) * P[m][m];
    for (int m = 0; m <= MP_LMAX; ++m)
        for (int l = m + 2; l <= MP_LMAX; ++l)
            P[l][m] = ((2 * l - 1) * ct * P[l - 1][m] - (l + m - 1) * P[l - 2][m]) / (l - m);
    double cm[MP_LMAX + 1], sm[MP_LMAX + 1];
    cm[0] = 1.0;
    sm[0] = 0.0;
    for (int m = 1; m <= MP_LMAX; ++m) {
        cm[m] = cm[m - 1] * cp - sm[m - 1] * sp;
        sm[m] = sm[m - 1] * cp + cm[m - 1] * sp;
    }
    for (int l = 0; l <= MP_LMAX; ++l) {
        double ratio = 1.0;   // (l - m)! / (l + m)!
        for (int m = 0; m <= l; ++m) {
            if (m > 0) ratio /= (double)((l + m) * (l - m + 1));
            const double N = sqrt((2 * l + 1) / (4.0 * 3.14159265358979323846) * ratio);
            if (m == 0) {
                Y[l * l + l] = N * P[l][0];
            } else {
                Y[l * l + l + m] = 1.4142135623730951 * N * P[l][m] * cm[m];
                Y[l * l + l - m] = 1.4142135623730951 * N * P[l][m] * sm[m];
            }
        }
    }
}

// per-block partial moments part[block][lm] of f about the centre (c0, c1, c2)
__global__ void __launch_bounds__(256) multipole_kernel(const double* __restrict__ f, int n1, int n2, int n3,
                                                        double h1, double h2, double h3, double c0, double c1,
                                                        double c2, double* __restrict__ part) {
    __shared__ double sh[MP_NLM][8];
    double acc[MP_NLM];
    for (int k = 0; k < MP_NLM; ++k) acc[k] = 0.0;
    const long long ng = (long long)n1 * n2 * n3;
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < ng; g += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(g % n1), j = (int)((g / n1) % n2), k = (int)(g / ((long long)n1 * n2));
        const double x = i * h1 - c0, y = j * h2 - c1, z = k * h3 - c2;
        const double r = sqrt(x * x + y * y + z * z);
        double Y[MP_NLM];
        real_sh(x, y, z, Y);
        double rl = f[g];
        for (int l = 0; l <= MP_LMAX; ++l) {
            for (int m = -l; m <= l; ++m) acc[l * l + l + m] += rl * Y[l * l + l + m];
            rl *= r;
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int k = 0; k < MP_NLM; ++k) {
        double v = acc[k];
        for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
        if (lane == 0) sh[k][warp] = v;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < MP_NLM; k += blockDim.x) {
        double v = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += sh[k][w];
        part[(long long)blockIdx.x * MP_NLM + k] = v;
    }
}

__device__ double multipole_phi(const double* q, double x, double y, double z) {
    double Y[MP_NLM];
    real_sh(x, y, z, Y);
    const double r = sqrt(x * x + y * y + z * z);
    const double ir = 1.0 / r;
    double irl = ir, v = 0.0;   // r^-(l+1)
    for (int l = 0; l <= MP_LMAX; ++l) {
        double s = 0.0;
        for (int m = -l; m <= l; ++m) s += q[l * l + l + m] * Y[l * l + l + m];
        v += 4.0 * 3.14159265358979323846 / (2 * l + 1) * s * irl;
        irl *= ir;
    }
    return v;
}

// rhs = 4 pi f + G, G = sum over stencil neighbours beyond the grid of (w_r / h_d^2) phi_ghost
// (K.c = -1/2 w_r / h_d^2, so G = -2 sum K.c phi_ghost)
__global__ void __launch_bounds__(256) dirichlet_rhs_kernel(const double* __restrict__ f, double* __restrict__ rhs,
                                                            const double* __restrict__ q, LapCoef K, int n1, int n2,
                                                            int n3, double h1, double h2, double h3, double c0,
                                                            double c1, double c2) {
    const long long ng = (long long)n1 * n2 * n3;
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < ng; g += (long long)gridDim.x * blockDim.x) {
        const int I[3] = {(int)(g % n1), (int)((g / n1) % n2), (int)(g / ((long long)n1 * n2))};
        const int n[3] = {n1, n2, n3};
        const double h[3] = {h1, h2, h3}, cc[3] = {c0, c1, c2};
        double v = 4.0 * 3.14159265358979323846 * f[g];
        for (int d = 0; d < 3; ++d)
            for (int r = 1; r <= FD_RADIUS; ++r)
                for (int sgn = -1; sgn <= 1; sgn += 2) {
                    const int id = I[d] + sgn * r;
                    if (id >= 0 && id < n[d]) continue;
                    double X[3];
                    for (int e = 0; e < 3; ++e) X[e] = (e == d ? id : I[e]) * h[e] - cc[e];
                    v += -2.0 * K.c[d][r] * multipole_phi(q, X[0], X[1], X[2]);
                }
        rhs[g] = v;
    }
}
}  // namespace

// rhs of the isolated Poisson problem for charge f (device [ngrid])
static void isolated_poisson_rhs(sdft_ctx* c, const double* f, double* rhs) {
    const int nblk = 128;
    double* part = c->work64 + 27 * c->ng;   // nblk * 49 doubles (the grid's last scratch vector)
    SDFT_REQUIRE((long long)nblk * MP_NLM <= c->ng, SDFT_ERR_INVALID_ARG, "isolated Poisson: grid too small");
    double cen[3];
    for (int d = 0; d < 3; ++d) cen[d] = 0.5 * (c->n[d] - 1) * c->h[d];
    multipole_kernel<<<nblk, 256, 0, c->stream>>>(f, c->n[0], c->n[1], c->n[2], c->h[0], c->h[1], c->h[2], cen[0], cen[1],
                                                  cen[2], part);
    SDFT_CUDA(cudaGetLastError());
    count_launch(c);
    std::vector<double> hp((size_t)nblk * MP_NLM);
    SDFT_CUDA(cudaMemcpyAsync(hp.data(), part, sizeof(double) * hp.size(), cudaMemcpyDeviceToHost, c->stream));
    SDFT_CUDA(cudaStreamSynchronize(c->stream));
    double q[MP_NLM];
    for (int k = 0; k < MP_NLM; ++k) {
        double s = 0.0;
        for (int b = 0; b < nblk; ++b) s += hp[(size_t)b * MP_NLM + k];
        q[k] = c->dV * s;
    }
    double* dq = c->scal + 1700;   // [1700, 1749): multipole moments (free part of the scalar area)
    std::memcpy(c->hscal + 1700, q, sizeof(q));
    SDFT_CUDA(cudaMemcpyAsync(dq, c->hscal + 1700, sizeof(q), cudaMemcpyHostToDevice, c->stream));
    LapCoef K;
    for (int r = 0; r <= FD_RADIUS; ++r) {
        K.c[0][r] = c->coef.cx[r];
        K.c[1][r] = c->coef.cy[r];
        K.c[2][r] = c->coef.cz[r];
    }
    K.c0 = c->coef.c0;
    dirichlet_rhs_kernel<<<nblocks(c->ng), 256, 0, c->stream>>>(f, rhs, dq, K, c->n[0], c->n[1], c->n[2], c->h[0],
                                                               c->h[1], c->h[2], cen[0], cen[1], cen[2]);
    SDFT_CUDA(cudaGetLastError());
    count_launch(c);
}

// ---------------------------------------------------------------------------------------
// AAR Poisson (Pratapa, Suryanarayana & Pask 2016; Suryanarayana et al. 2019):
// A = -L_h, Jacobi preconditioner, Richardson steps with omega, Anderson every p-th step.
// ---------------------------------------------------------------------------------------
int poisson_aar(sdft_ctx* c, const double* f, double* phi, double tol, int max_iter) {
    const long long n = c->ng;
    ScopedTimer timer(c, SDFT_K_POISSON);
    const double omega = 0.6, beta = 0.6;
    const int m = 7, p = 6;
    // workspace: rhs, r, xprev, fprev, X[m], F[m]
    double* rhs = c->work64 + 0 * n;
    double* r = c->work64 + 1 * n;
    double* xprev = c->work64 + 4 * n;
    double* fprev = c->work64 + 5 * n;
    double* hist = c->work64 + 6 * n;  // 2*m vectors
    double* Xs = hist;
    double* Fs = hist + (long long)m * n;
    double* gam = c->scal + 64;
    int* slots = (int*)(c->scal + 96);
    double* ffv = c->scal + 128;
    double* part = c->scal + 4096;
    const bool isolated = c->opt.boundary == SDFT_BC_DIRICHLET;
    // rhs = 4 pi (f - mean f); phi -= mean(phi)   (isolated: rhs = 4 pi f + ghost term, no gauge)
    if (isolated) {
        isolated_poisson_rhs(c, f, rhs);
    } else {
        double* ones = c->work64 + 3 * n;
        SDFT_CUDA(cudaMemsetAsync(ones, 0, sizeof(double) * n, c->stream));
        c->hscal[0] = 1.0;
        SDFT_CUDA(cudaMemcpyAsync(c->scal, c->hscal, sizeof(double), cudaMemcpyHostToDevice, c->stream));
        add_scalar_kernel<<<nblocks(n), 256, 0, c->stream>>>(ones, c->scal, 1.0, n);
        const double* A[2] = {f, phi};
        const double* B[2] = {ones, ones};
        double s[2];
        dots_host(c, 2, A, B, n, s);
        SDFT_CUDA(cudaMemcpyAsync(rhs, f, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->stream));
        c->hscal[0] = -s[0] / n;
        c->hscal[1] = -s[1] / n;
        SDFT_CUDA(cudaMemcpyAsync(c->scal, c->hscal, 2 * sizeof(double), cudaMemcpyHostToDevice, c->stream));
        add_scalar_kernel<<<nblocks(n), 256, 0, c->stream>>>(rhs, c->scal, 1.0, n);
        add_scalar_kernel<<<nblocks(n), 256, 0, c->stream>>>(phi, c->scal + 1, 1.0, n);
        axpby_kernel<double><<<nblocks(n), 256, 0, c->stream>>>(rhs, rhs, 0.0, 4.0 * M_PI, n);
        SDFT_CUDA(cudaGetLastError());
        count_launch(c, 5);
    }
    double bnorm2;
    {
        const double* A[1] = {rhs};
        dots_host(c, 1, A, A, n, &bnorm2);
    }
    if (bnorm2 == 0.0) {
        SDFT_CUDA(cudaMemsetAsync(phi, 0, sizeof(double) * n, c->stream));
        return 0;
    }
    // Jacobi: diag(-L) = -(sum_d w0/h_d^2) = 2*c0 (c0 = -1/2 sum_d w0/h^2 > 0)
    const double cj = 1.0 / (2.0 * c->coef.c0);
    int count = 0, head = 0, it = 0;
    int hslots[16];
    for (it = 0; it < max_iter; ++it) {
        // r = rhs - A phi = rhs + L phi  (stencil: alpha=-2 on -1/2 L, beta=-1 on rhs)
        laplacian_residual<double>(c, phi, rhs, r);
        // history push with f = cj * r
        const int slot = head;
        anderson_push_kernel<double><<<nblocks(n), 256, 0, c->stream>>>(phi, r, cj, xprev, fprev, Xs + (long long)slot * n,
                                                                Fs + (long long)slot * n, it > 0, n);
        count_launch(c);
        if (it > 0) {
            head = (head + 1) % m;
            count = std::min(count + 1, m);
        }
        const bool anderson = ((it + 1) % p == 0) && count > 0;
        if (anderson) {
            for (int j = 0; j < count; ++j) hslots[j] = ((head - count + j) % m + m) % m;
            std::memcpy(c->hscal + 512, hslots, sizeof(int) * 16);
            SDFT_CUDA(cudaMemcpyAsync(slots, c->hscal + 512, sizeof(int) * count, cudaMemcpyHostToDevice, c->stream));
            const int nblk = 64;
            anderson_gram_kernel<double><<<nblk, RB, 0, c->stream>>>(Fs, slots, count, r, cj, n, part);
            anderson_solve_kernel<<<1, 256, 0, c->stream>>>(part, nblk, count, gam, ffv);
            anderson_update_kernel<double><<<nblocks(n), 256, 0, c->stream>>>(phi, r, cj, beta, Xs, Fs, slots, gam, count, n);
            SDFT_CUDA(cudaGetLastError());
            count_launch(c, 3);
            // convergence: ||r||^2 = ffv / cj^2
            SDFT_CUDA(cudaMemcpyAsync(c->hscal, ffv, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
            SDFT_CUDA(cudaStreamSynchronize(c->stream));
            const double rn2 = c->hscal[0] / (cj * cj);
            if (!std::isfinite(rn2)) throw Error{SDFT_ERR_NONFINITE, "Poisson residual is not finite"};
            if (rn2 <= tol * tol * bnorm2) {
                ++it;
                break;
            }
        } else {
            // Richardson: phi += omega * cj * r
            axpby_kernel<double><<<nblocks(n), 256, 0, c->stream>>>(phi, r, omega * cj, 1.0, n);
            SDFT_CUDA(cudaGetLastError());
            count_launch(c);
        }
    }
    if (it >= max_iter) return -it;
    return it;
}

// ---------------------------------------------------------------------------------------
// Mixed-precision Poisson: FP64 residuals with FP32 AAR correction solves (iterative refinement).
//   r = rhs + L phi (FP64);  A delta = r solved approximately in FP32 by AAR;  phi += delta.
// Each refinement gains ~4-5 digits, so FP64-level residuals cost a few FP32 solves.
// ---------------------------------------------------------------------------------------
static int aar_fp32(sdft_ctx* c, const float* b, float* x, double tol_rel, int max_iter, double* final_rel) {
    const long long n = c->ng;
    const float omega = 0.6f, beta = 0.6f;
    const int m = 7, p = 6;
    float* r = c->work32 + 1 * n;
    float* xprev = c->work32 + 2 * n;
    float* fprev = c->work32 + 3 * n;
    float* Xs = c->work32 + 4 * n;
    float* Fs = Xs + (long long)m * n;
    double* gam = c->scal + 64;
    int* slots = (int*)(c->scal + 96);
    double* ffv = c->scal + 128;
    double* part = c->scal + 4096;
    const float cj = (float)(1.0 / (2.0 * c->coef.c0));
    double bnorm2;
    {
        // ||b||^2 through the history Gram with m = 0 (its last entry is (c f).(c f))
        anderson_gram_kernel<float><<<64, RB, 0, c->stream>>>(Fs, slots, 0, b, 1.0f, n, part);
        anderson_solve_kernel<<<1, 256, 0, c->stream>>>(part, 64, 0, gam, ffv);
        count_launch(c, 2);
        SDFT_CUDA(cudaMemcpyAsync(c->hscal, ffv, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        SDFT_CUDA(cudaStreamSynchronize(c->stream));
        bnorm2 = c->hscal[0];
    }
    SDFT_CUDA(cudaMemsetAsync(x, 0, sizeof(float) * n, c->stream));
    if (bnorm2 == 0.0) {
        *final_rel = 0.0;
        return 0;
    }
    int count = 0, head = 0, it = 0;
    int hslots[16];
    double rel = 1.0;
    for (it = 0; it < max_iter; ++it) {
        laplacian_residual<float>(c, x, b, r);
        const int slot = head;
        anderson_push_kernel<float><<<nblocks(n), 256, 0, c->stream>>>(x, r, cj, xprev, fprev, Xs + (long long)slot * n,
                                                                       Fs + (long long)slot * n, it > 0, n);
        count_launch(c);
        if (it > 0) {
            head = (head + 1) % m;
            count = std::min(count + 1, m);
        }
        const bool anderson = ((it + 1) % p == 0) && count > 0;
        if (anderson) {
            for (int j = 0; j < count; ++j) hslots[j] = ((head - count + j) % m + m) % m;
            std::memcpy(c->hscal + 512, hslots, sizeof(int) * 16);
            SDFT_CUDA(cudaMemcpyAsync(slots, c->hscal + 512, sizeof(int) * count, cudaMemcpyHostToDevice, c->stream));
            const int nblk = 64;
            anderson_gram_kernel<float><<<nblk, RB, 0, c->stream>>>(Fs, slots, count, r, cj, n, part);
            anderson_solve_kernel<<<1, 256, 0, c->stream>>>(part, nblk, count, gam, ffv);
            anderson_update_kernel<float><<<nblocks(n), 256, 0, c->stream>>>(x, r, cj, beta, Xs, Fs, slots, gam, count, n);
            SDFT_CUDA(cudaGetLastError());
            count_launch(c, 3);
            SDFT_CUDA(cudaMemcpyAsync(c->hscal, ffv, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
            SDFT_CUDA(cudaStreamSynchronize(c->stream));
            rel = std::sqrt(c->hscal[0] / ((double)cj * cj) / bnorm2);
            if (!std::isfinite(rel)) throw Error{SDFT_ERR_NONFINITE, "Poisson residual is not finite"};
            if (rel <= tol_rel) {
                ++it;
                break;
            }
        } else {
            axpby_kernel<float><<<nblocks(n), 256, 0, c->stream>>>(x, r, omega * cj, 1.0f, n);
            SDFT_CUDA(cudaGetLastError());
            count_launch(c);
        }
    }
    *final_rel = rel;
    return it;
}

// FP32 AAR with the multigrid preconditioner M (one V-cycle, poisson_mg.cu) in place of the Jacobi
// scaling: f_k = M r_k enters the Richardson steps x += omega f and the Anderson extrapolation every
// p-th step exactly where c r_k does in aar_fp32; convergence is tested on the true residual
// ||r_k|| / ||b|| at the Anderson steps.  With M A well conditioned a short history and frequent
// Anderson steps suffice.
static int aar_fp32_mg(sdft_ctx* c, const float* b, float* x, double tol_rel, int max_iter, double* final_rel) {
    const long long n = c->ng;
    const float omega = 0.7f, beta = 0.7f;
    const int m = 5, p = 3;
    // reduction grids: the history Gram's partials (m (m + 1) / 2 + m + 1 = 21 per block) fill 64 * 21
    // of the 12 288 doubles from scal + 4096, the single dot's 64 of the 1 024 from scal + 2048 (more
    // blocks did not shorten the Gram, and the one-CTA solve then sums more partials)
    constexpr int NB_G = 64, NB_R = 64;
    float* r = c->work32 + 1 * n;
    float* xprev = c->work32 + 2 * n;
    float* fprev = c->work32 + 3 * n;
    float* Xs = c->work32 + 4 * n;
    float* Fs = Xs + (long long)m * n;
    float* z = c->work32 + 19 * n;
    double* gam = c->scal + 64;
    int* slots = (int*)(c->scal + 96);
    double* ffv = c->scal + 128;
    double* rrv = c->scal + 136;
    double* part = c->scal + 4096;
    double* part_r = c->scal + 2048;
    double bnorm2;
    {
        anderson_gram_kernel<float><<<NB_R, RB, 0, c->stream>>>(Fs, slots, 0, b, 1.0f, n, part_r);
        anderson_solve_kernel<<<1, 256, 0, c->stream>>>(part_r, NB_R, 0, gam, rrv);
        count_launch(c, 2);
        SDFT_CUDA(cudaMemcpyAsync(c->hscal, rrv, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        SDFT_CUDA(cudaStreamSynchronize(c->stream));
        bnorm2 = c->hscal[0];
    }
    SDFT_CUDA(cudaMemsetAsync(x, 0, sizeof(float) * n, c->stream));
    if (bnorm2 == 0.0) {
        *final_rel = 0.0;
        return 0;
    }
    int count = 0, head = 0, it = 0;
    int hslots[16];
    double rel = 1.0;
    for (it = 0; it < max_iter; ++it) {
        laplacian_residual<float>(c, x, b, r);
        mg_vcycle(c, r, z);
        const int slot = head;
        anderson_push_kernel<float><<<nblocks(n), 256, 0, c->stream>>>(x, z, 1.0f, xprev, fprev, Xs + (long long)slot * n,
                                                                       Fs + (long long)slot * n, it > 0, n);
        count_launch(c);
        if (it > 0) {
            head = (head + 1) % m;
            count = std::min(count + 1, m);
        }
        const bool anderson = ((it + 1) % p == 0) && count > 0;
        if (anderson) {
            for (int j = 0; j < count; ++j) hslots[j] = ((head - count + j) % m + m) % m;
            std::memcpy(c->hscal + 512, hslots, sizeof(int) * 16);
            SDFT_CUDA(cudaMemcpyAsync(slots, c->hscal + 512, sizeof(int) * count, cudaMemcpyHostToDevice, c->stream));
            anderson_gram_kernel<float><<<NB_G, RB, 0, c->stream>>>(Fs, slots, count, z, 1.0f, n, part);
            anderson_solve_kernel<<<1, 256, 0, c->stream>>>(part, NB_G, count, gam, ffv);
            // ||r||^2 of the residual this step was taken from
            anderson_gram_kernel<float><<<NB_R, RB, 0, c->stream>>>(Fs, slots, 0, r, 1.0f, n, part_r);
            anderson_solve_kernel<<<1, 256, 0, c->stream>>>(part_r, NB_R, 0, gam + 16, rrv);
            anderson_update_kernel<float><<<nblocks(n), 256, 0, c->stream>>>(x, z, 1.0f, beta, Xs, Fs, slots, gam, count, n);
            SDFT_CUDA(cudaGetLastError());
            count_launch(c, 5);
            SDFT_CUDA(cudaMemcpyAsync(c->hscal, rrv, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
            SDFT_CUDA(cudaStreamSynchronize(c->stream));
            rel = std::sqrt(c->hscal[0] / bnorm2);
            if (!std::isfinite(rel)) throw Error{SDFT_ERR_NONFINITE, "Poisson residual is not finite"};
            if (rel <= tol_rel) {
                ++it;
                break;
            }
        } else {
            axpby_kernel<float><<<nblocks(n), 256, 0, c->stream>>>(x, z, omega, 1.0f, n);
            SDFT_CUDA(cudaGetLastError());
            count_launch(c);
        }
    }
    *final_rel = rel;
    return it;
}

// ---------------------------------------------------------------------------------------
// Persistent FP32 AAR: the whole correction solve A d = b (A = -L_h) in one cooperative launch.
// CTA k owns points [k*per, (k+1)*per).  Per iteration: residual r = b + L x_cur on own points
// (neighbours read from L2), history push, then Richardson x_next = x_cur + w c r or, every p-th
// iteration, Anderson x_next = x_cur + beta c r - sum gamma (X + beta F) with the small Gram
// reduced through per-block partials (every CTA sums them in the same order and solves the same
// m x m system).  x is double-buffered, so one grid barrier per iteration separates the reads of
// x_cur from the writes of x_next (two on Anderson steps).  The barrier spin is bounded: on
// timeout the kernel records an error status and every CTA returns.
// ---------------------------------------------------------------------------------------
struct AarPersistArgs {
    const float* b;
    float* x0;       // x buffers (double-buffered)
    float* x1;
    float* r;
    float* xprev;
    float* fprev;
    float* Xs;       // [m][n]
    float* Fs;       // [m][n]
    double* part;    // [gridDim][ND]
    unsigned* bar;   // [2]: arrival count, generation
    int* status;     // [4]: 0 ok / 1 barrier timeout, iterations, final buffer index
    double* rel_out;
    LapCoef K;
    int n1, n2, n3;
    long long n;
    float cj, omega, beta;
    double bnorm2, tol_rel;
    int max_iter;
    unsigned expected_blocks;   // arrivals the barrier waits for (== gridDim.x)
    long long spin_limit;
};

constexpr int AAR_M = 7, AAR_P = 6, AAR_ND = AAR_M * (AAR_M + 1) / 2 + AAR_M + 1;

__device__ bool grid_barrier(unsigned* bar, unsigned expected, long long limit, int* flag) {
    __shared__ int ok_s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        volatile unsigned* gen = bar + 1;
        const unsigned g = *gen;
        __threadfence();
        const unsigned arrived = atomicAdd(bar, 1u);
        if (arrived == expected - 1) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            long long i = 0;
            while (*gen == g) {
                if (++i > limit || *(volatile int*)flag != 0) {
                    ok = 0;
                    break;
                }
            }
        }
        __threadfence();
        if (!ok) atomicExch(flag, 1);
        ok_s = ok;
    }
    __syncthreads();
    return ok_s != 0;
}

constexpr int AAR_BS = 256;    // threads per CTA of the persistent solver (one CTA per SM)

__global__ void __launch_bounds__(AAR_BS) aar_persistent_kernel(AarPersistArgs A) {
    __shared__ double red[AAR_ND][AAR_BS / 32];
    __shared__ double gam_s[AAR_M];
    __shared__ double ff_s;
    const long long per = (A.n + gridDim.x - 1) / gridDim.x;
    const long long lo = blockIdx.x * per, hi = min(A.n, lo + per);
    int head = 0, count = 0;
    int cur = 0;
    int it;
    double rel = 1.0;
    for (it = 0; it < A.max_iter; ++it) {
        float* xc = cur ? A.x1 : A.x0;
        float* xn = cur ? A.x0 : A.x1;
        const int slot = head;
        // residual and history push on own points.  Grid coordinates advance incrementally in
        // 32-bit arithmetic (the points of a thread are blockDim apart), so no division per point.
        {
            const int n1 = A.n1, n2 = A.n2, n3 = A.n3;
            const int pl32 = n1 * n2;
            int g = (int)lo + (int)threadIdx.x;
            int i = g % n1, row = g / n1;
            int j = row % n2, k = row / n2;
            const int di = (int)(blockDim.x % (unsigned)n1), drow = (int)(blockDim.x / (unsigned)n1);
            const int dj = drow % n2, dk = drow / n2;
            for (; g < (int)hi; g += (int)blockDim.x) {
                const int rowbase = g - i;              // (k n2 + j) n1
                const int colbase = g - j * n1;         // k n1 n2 + i
                const int plbase = g - k * pl32;        // j n1 + i
                float acc = (float)A.K.c0 * xc[g];
#pragma unroll
                for (int rr = 1; rr <= FD_RADIUS; ++rr) {
                    int ip = i + rr, im = i - rr, jp = j + rr, jm = j - rr, kp = k + rr, km = k - rr;
                    ip -= ip >= n1 ? n1 : 0;
                    im += im < 0 ? n1 : 0;
                    jp -= jp >= n2 ? n2 : 0;
                    jm += jm < 0 ? n2 : 0;
                    kp -= kp >= n3 ? n3 : 0;
                    km += km < 0 ? n3 : 0;
                    acc += (float)A.K.c[0][rr] * (xc[rowbase + ip] + xc[rowbase + im]);
                    acc += (float)A.K.c[1][rr] * (xc[colbase + jp * n1] + xc[colbase + jm * n1]);
                    acc += (float)A.K.c[2][rr] * (xc[plbase + kp * pl32] + xc[plbase + km * pl32]);
                }
                const float r = A.b[g] - 2.f * acc;
                A.r[g] = r;
                const float fi = A.cj * r;
                if (it > 0) {
                    A.Xs[(long long)slot * A.n + g] = xc[g] - A.xprev[g];
                    A.Fs[(long long)slot * A.n + g] = fi - A.fprev[g];
                }
                A.xprev[g] = xc[g];
                A.fprev[g] = fi;
                // next point of this thread: blockDim further along x, then y, then z
                i += di;
                j += dj;
                k += dk;
                if (i >= n1) {
                    i -= n1;
                    ++j;
                }
                if (j >= n2) {
                    j -= n2;
                    ++k;
                }
            }
        }
        if (it > 0) {
            head = (head + 1) % AAR_M;
            count = min(count + 1, AAR_M);
        }
        const bool anderson = ((it + 1) % AAR_P == 0) && count > 0;
        if (!anderson) {
            for (long long g = lo + threadIdx.x; g < hi; g += blockDim.x) xn[g] = xc[g] + A.omega * A.cj * A.r[g];
        } else {
            // partial Gram of the history (slots in age order) and F.(c r), (c r).(c r)
            int sl[AAR_M];
            for (int jj = 0; jj < count; ++jj) sl[jj] = ((head - count + jj) % AAR_M + AAR_M) % AAR_M;
            const int nd = count * (count + 1) / 2 + count + 1;
            double vals[AAR_ND];
            switch (count) {
#define SDFT_AAR_CASE(CC) \
    case CC: gram_accum<CC, float>(A.Fs, sl, A.r, A.cj, A.n, lo + threadIdx.x, hi, blockDim.x, vals); break;
                SDFT_AAR_CASE(1) SDFT_AAR_CASE(2) SDFT_AAR_CASE(3) SDFT_AAR_CASE(4) SDFT_AAR_CASE(5) SDFT_AAR_CASE(6)
                SDFT_AAR_CASE(7)
#undef SDFT_AAR_CASE
                default: break;
            }
            block_reduce_partials<AAR_BS / 32>(vals, nd, A.part + (long long)blockIdx.x * nd, red);
            if (!grid_barrier(A.bar, A.expected_blocks, A.spin_limit, A.status)) return;
            anderson_solve_block(A.part, gridDim.x, count, gam_s, &ff_s);
            __syncthreads();
            rel = sqrt(ff_s / ((double)A.cj * A.cj) / A.bnorm2);
            for (long long g = lo + threadIdx.x; g < hi; g += blockDim.x) {
                float v = xc[g] + A.beta * A.cj * A.r[g];
                for (int jj = 0; jj < count; ++jj) {
                    const long long o = (long long)sl[jj] * A.n + g;
                    v -= (float)gam_s[jj] * (A.Xs[o] + A.beta * A.Fs[o]);
                }
                xn[g] = v;
            }
        }
        if (!grid_barrier(A.bar, A.expected_blocks, A.spin_limit, A.status)) return;
        cur ^= 1;
        if (anderson && !(rel > A.tol_rel)) {   // converged (also stops on NaN)
            ++it;
            break;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        A.status[1] = it;
        A.status[2] = cur;
        *A.rel_out = rel;
    }
}

// FP32 correction solve by the persistent kernel; x (work32 slot) receives the solution.
static int aar_fp32_persistent(sdft_ctx* c, const float* b, float* x, double tol_rel, int max_iter,
                               double* final_rel) {
    const long long n = c->ng;
    AarPersistArgs A;
    A.b = b;
    A.x0 = x;
    A.x1 = c->work32 + 19 * n;
    A.r = c->work32 + 1 * n;
    A.xprev = c->work32 + 2 * n;
    A.fprev = c->work32 + 3 * n;
    A.Xs = c->work32 + 4 * n;
    A.Fs = A.Xs + (long long)AAR_M * n;
    A.part = c->scal + 4096;
    A.bar = reinterpret_cast<unsigned*>(c->scal + 40);
    A.status = reinterpret_cast<int*>(c->scal + 42);
    A.rel_out = c->scal + 44;
    for (int r = 0; r <= FD_RADIUS; ++r) {
        A.K.c[0][r] = c->coef.cx[r];
        A.K.c[1][r] = c->coef.cy[r];
        A.K.c[2][r] = c->coef.cz[r];
    }
    A.K.c0 = c->coef.c0;
    A.n1 = c->n[0];
    A.n2 = c->n[1];
    A.n3 = c->n[2];
    A.n = n;
    A.cj = (float)(1.0 / (2.0 * c->coef.c0));
    A.omega = 0.6f;
    A.beta = 0.6f;
    A.tol_rel = tol_rel;
    A.max_iter = max_iter;
    A.spin_limit = 1LL << 24;   // volatile polls of the barrier generation (~0.1-1 s)
    // ||b||^2
    {
        double* part = c->scal + 2048;
        anderson_gram_kernel<float><<<64, RB, 0, c->stream>>>(A.Fs, nullptr, 0, b, 1.0f, n, part);
        anderson_solve_kernel<<<1, 256, 0, c->stream>>>(part, 64, 0, c->scal + 64, c->scal + 128);
        count_launch(c, 2);
        SDFT_CUDA(cudaMemcpyAsync(c->hscal, c->scal + 128, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        SDFT_CUDA(cudaStreamSynchronize(c->stream));
        A.bnorm2 = c->hscal[0];
    }
    SDFT_CUDA(cudaMemsetAsync(x, 0, sizeof(float) * n, c->stream));
    if (A.bnorm2 == 0.0) {
        *final_rel = 0.0;
        return 0;
    }
    // grid: co-resident CTAs (cooperative launch), at most one per 2048 points, <= 12288 partial slots
    int dev = 0, nsm = 0, per_sm = 0;
    SDFT_CUDA(cudaGetDevice(&dev));
    SDFT_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    SDFT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, aar_persistent_kernel, AAR_BS, 0));
    if (per_sm < 1) {
        c->aar_persistent = false;
        return aar_fp32(c, b, x, tol_rel, max_iter, final_rel);
    }
    // every co-resident CTA (latency hiding for the stencil's scattered loads), fewer for small grids
    SDFT_REQUIRE(n < (1LL << 31) - 4096, SDFT_ERR_INVALID_ARG, "persistent Poisson solver: grid too large");
    long long nblk = std::min<long long>((long long)nsm * per_sm, (n + 1023) / 1024);
    nblk = std::max<long long>(1, std::min<long long>(nblk, 12288 / AAR_ND));
    A.expected_blocks = (unsigned)nblk + (c->test_barrier_extra ? 1u : 0u);
    if (c->test_barrier_extra) A.spin_limit = 200000;
    SDFT_CUDA(cudaMemsetAsync(A.bar, 0, 2 * sizeof(unsigned), c->stream));
    SDFT_CUDA(cudaMemsetAsync(A.status, 0, 4 * sizeof(int), c->stream));
    void* args[] = {&A};
    const cudaError_t le = cudaLaunchCooperativeKernel((const void*)aar_persistent_kernel, dim3((unsigned)nblk),
                                                       dim3(AAR_BS), args, 0, c->stream);
    if (le != cudaSuccess) {
        // no co-residency guarantee available: fall back to one launch per iteration
        cudaGetLastError();
        c->aar_persistent = false;
        return aar_fp32(c, b, x, tol_rel, max_iter, final_rel);
    }
    count_launch(c);
    int st[4];
    SDFT_CUDA(cudaMemcpyAsync(st, A.status, sizeof(st), cudaMemcpyDeviceToHost, c->stream));
    SDFT_CUDA(cudaMemcpyAsync(c->hscal, A.rel_out, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    SDFT_CUDA(cudaStreamSynchronize(c->stream));
    if (st[0] != 0) throw Error{SDFT_ERR_DEVICE_TIMEOUT, "persistent Poisson solver: grid barrier timed out"};
    if (st[2] == 1) SDFT_CUDA(cudaMemcpyAsync(x, A.x1, sizeof(float) * n, cudaMemcpyDeviceToDevice, c->stream));
    *final_rel = c->hscal[0];
    return st[1];
}

int poisson_mixed(sdft_ctx* c, const double* f, double* phi, double tol, int max_iter) {
    const long long n = c->ng;
    ScopedTimer timer(c, SDFT_K_POISSON);
    double* rhs = c->work64 + 0 * n;
    double* r = c->work64 + 1 * n;
    double* ones = c->work64 + 3 * n;
    float* b32 = c->work32;
    float* d32 = c->work32 + 18 * n;
    // rhs = 4 pi (f - mean f); phi -= mean(phi)
    SDFT_CUDA(cudaMemsetAsync(ones, 0, sizeof(double) * n, c->stream));
    c->hscal[0] = 1.0;
    SDFT_CUDA(cudaMemcpyAsync(c->scal, c->hscal, sizeof(double), cudaMemcpyHostToDevice, c->stream));
    add_scalar_kernel<<<nblocks(n), 256, 0, c->stream>>>(ones, c->scal, 1.0, n);
    {
        const double* A[2] = {f, phi};
        const double* B[2] = {ones, ones};
        double s[2];
        dots_host(c, 2, A, B, n, s);
        SDFT_CUDA(cudaMemcpyAsync(rhs, f, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->stream));
        c->hscal[0] = -s[0] / n;
        c->hscal[1] = -s[1] / n;
        SDFT_CUDA(cudaMemcpyAsync(c->scal, c->hscal, 2 * sizeof(double), cudaMemcpyHostToDevice, c->stream));
        add_scalar_kernel<<<nblocks(n), 256, 0, c->stream>>>(rhs, c->scal, 1.0, n);
        add_scalar_kernel<<<nblocks(n), 256, 0, c->stream>>>(phi, c->scal + 1, 1.0, n);
        axpby_kernel<double><<<nblocks(n), 256, 0, c->stream>>>(rhs, rhs, 0.0, 4.0 * M_PI, n);
        SDFT_CUDA(cudaGetLastError());
        count_launch(c, 4);
    }
    double bnorm2;
    {
        const double* A[1] = {rhs};
        dots_host(c, 1, A, A, n, &bnorm2);
    }
    if (bnorm2 == 0.0) {
        SDFT_CUDA(cudaMemsetAsync(phi, 0, sizeof(double) * n, c->stream));
        return 0;
    }
    // zero-mean gauge: FP32 corrections drift along the constant null vector of L, which the
    // residual cannot see, so the mean is removed from phi at the end
    auto remove_mean = [&]() {
        const double* A[1] = {phi};
        const double* B[1] = {ones};
        double sphi;
        dots_host(c, 1, A, B, n, &sphi);
        c->hscal[0] = -sphi / n;
        SDFT_CUDA(cudaMemcpyAsync(c->scal, c->hscal, sizeof(double), cudaMemcpyHostToDevice, c->stream));
        add_scalar_kernel<<<nblocks(n), 256, 0, c->stream>>>(phi, c->scal, 1.0, n);
        count_launch(c);
    };
    int total = 0;
    for (int refine = 0; refine < 16; ++refine) {
        // FP64 residual r = rhs + L phi
        laplacian_residual<double>(c, phi, rhs, r);
        double rn2;
        {
            const double* A[1] = {r};
            dots_host(c, 1, A, A, n, &rn2);
        }
        const double rel = std::sqrt(rn2 / bnorm2);
        if (!std::isfinite(rel)) throw Error{SDFT_ERR_NONFINITE, "Poisson residual is not finite"};
        if (rel <= tol) {
            remove_mean();
            return std::max(total, 1);
        }
        if (total >= max_iter) break;
        // FP32 correction A d = r: a relative reduction of 1e-3 per refinement stays above the
        // FP32 rounding floor of the residual (~ cond(L) * 2^-24)
        convert_add_kernel<float, double><<<nblocks(n), 256, 0, c->stream>>>(b32, r, 1.0, 0.0, n);
        count_launch(c);
        double inner_rel = 1.0;
        const double want = std::max(1e-3, 0.3 * tol / rel);
        const int budget = std::min(400, max_iter - total);
        total += !c->mg.empty()       ? aar_fp32_mg(c, b32, d32, want, budget, &inner_rel)
                 : c->aar_persistent ? aar_fp32_persistent(c, b32, d32, want, budget, &inner_rel)
                                     : aar_fp32(c, b32, d32, want, budget, &inner_rel);
        convert_add_kernel<double, float><<<nblocks(n), 256, 0, c->stream>>>(phi, d32, 1.0, 1.0, n);
        count_launch(c);
    }
    remove_mean();
    return -std::max(total, 1);
}

void density_accumulate(sdft_ctx* c, int precision, bool cplx, const void* X, const double* occ, int ncol,
                        double weight, double* rho) {
    const double scale = weight / c->dV;
    const unsigned nb = nblocks(c->ng);
    ScopedTimer timer(c, SDFT_K_DENSITY, (double)block_elems_bytes(c, precision, cplx, ncol));
    const size_t sm32 = sizeof(float) * (size_t)ncol;   // FP32 copy of the occupations
    SDFT_REQUIRE(sm32 <= 48 * 1024, SDFT_ERR_INVALID_ARG, "density: too many states for one block's occupations");
    if (precision == SDFT_FP64) {
        if (cplx) density_kernel<1><<<nb, 256, 0, c->stream>>>(X, occ, ncol, scale, c->ng, rho);
        else density_kernel<0><<<nb, 256, 0, c->stream>>>(X, occ, ncol, scale, c->ng, rho);
    } else {
        if (cplx) density_kernel<3><<<nb, 256, sm32, c->stream>>>(X, occ, ncol, scale, c->ng, rho);
        else density_kernel<2><<<nb, 256, sm32, c->stream>>>(X, occ, ncol, scale, c->ng, rho);
    }
    SDFT_CUDA(cudaGetLastError());
    count_launch(c);
}

void fermi_device(sdft_ctx* c, const double* eig, double* occ, double* out) {
    const int nk = c->opt.nkpt;
    double* kw = c->scal + 256;
    SDFT_CUDA(cudaMemcpyAsync(kw, c->kw.data(), sizeof(double) * nk, cudaMemcpyHostToDevice, c->stream));
    const double fs = c->opt.nspin == 1 ? 2.0 : 1.0;
    fermi_kernel<<<1, 256, 0, c->stream>>>(eig, kw, c->opt.nspin, nk, c->opt.nstates, c->nelec, c->opt.kT, fs, occ,
                                           out);
    SDFT_CUDA(cudaGetLastError());
    count_launch(c);
}

// ---------------------------------------------------------------------------------------
// Kerker preconditioner of the mixing (paper Sec. 2.1: periodic Pulay with a real-space
// preconditioner of Kerker type): P f = (-L_h)(-L_h + k0^2)^-1 f = f - k0^2 y, (-L_h + k0^2) y = f.
// The screened operator is positive definite, so y comes from the same AAR iteration as the
// Poisson solve (Jacobi-preconditioned Richardson steps, Anderson extrapolation every p-th step),
// with the diagonal shift k0^2 in the residual and in the Jacobi factor; no gauge is involved.
// ---------------------------------------------------------------------------------------
namespace {
constexpr int KERKER_M = 7, KERKER_P = 6;
constexpr double KERKER_TOL = 1e-10;    // relative residual of the screened solve inside the SCF

// x_k ← x_k - sum_j gamma_j X_j and f ← beta (f - sum_j gamma_j F_j): the optimal residual form of a
// Pulay step, whose linear part is then preconditioned
__global__ void pulay_residual_kernel(double* __restrict__ x, double* __restrict__ f, const double* __restrict__ X,
                                      const double* __restrict__ F, const int* __restrict__ slots,
                                      const double* __restrict__ gamma, int m, double beta, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        double xv = x[i], fv = f[i];
        for (int j = 0; j < m; ++j) {
            const long long o = (long long)slots[j] * n + i;
            xv -= gamma[j] * X[o];
            fv -= gamma[j] * F[o];
        }
        x[i] = xv;
        f[i] = beta * fv;
    }
}
}  // namespace

static double* kerker_workspace(sdft_ctx* c) {
    // rhs copy, solution, AAR residual, previous iterate and residual, X[m], F[m]
    if (!c->kerker_ws) c->kerker_ws = (double*)ctx_alloc(c, sizeof(double) * (size_t)(5 + 2 * KERKER_M) * c->ng);
    return c->kerker_ws;
}

int kerker_apply(sdft_ctx* c, const double* f, double* out, double k0, double tol, int max_iter) {
    const long long n = c->ng;
    SDFT_REQUIRE(k0 > 0.0 && tol > 0.0 && max_iter >= 1, SDFT_ERR_INVALID_ARG, "Kerker: k0 > 0, tol > 0 required");
    double* ws = kerker_workspace(c);
    double* y = ws + 1 * n;
    double* r = ws + 2 * n;
    double* xprev = ws + 3 * n;
    double* fprev = ws + 4 * n;
    double* Xs = ws + 5 * n;
    double* Fs = Xs + (long long)KERKER_M * n;
    double* gam = c->scal + 64;
    int* slots = (int*)(c->scal + 96);
    double* ffv = c->scal + 128;
    double* part = c->scal + 4096;
    const double k2 = k0 * k0;
    const double cj = 1.0 / (2.0 * c->coef.c0 + k2);   // Jacobi: diag(-L_h + k0^2)
    const double omega = 0.6, beta = 0.6;
    double bnorm2;
    {
        const double* A[1] = {f};
        dots_host(c, 1, A, A, n, &bnorm2);
    }
    SDFT_CUDA(cudaMemsetAsync(y, 0, sizeof(double) * n, c->stream));
    int it = 0;
    if (bnorm2 > 0.0) {
        int count = 0, head = 0;
        int hslots[16];
        bool done = false;
        for (it = 0; it < max_iter; ++it) {
            laplacian_residual<double>(c, y, f, r, k2);
            anderson_push_kernel<double><<<nblocks(n), 256, 0, c->stream>>>(y, r, cj, xprev, fprev,
                                                                            Xs + (long long)head * n,
                                                                            Fs + (long long)head * n, it > 0, n);
            count_launch(c);
            if (it > 0) {
                head = (head + 1) % KERKER_M;
                count = std::min(count + 1, KERKER_M);
            }
            if (((it + 1) % KERKER_P == 0) && count > 0) {
                for (int j = 0; j < count; ++j) hslots[j] = ((head - count + j) % KERKER_M + KERKER_M) % KERKER_M;
                std::memcpy(c->hscal + 512, hslots, sizeof(int) * 16);
                SDFT_CUDA(cudaMemcpyAsync(slots, c->hscal + 512, sizeof(int) * count, cudaMemcpyHostToDevice, c->stream));
                anderson_gram_kernel<double><<<64, RB, 0, c->stream>>>(Fs, slots, count, r, cj, n, part);
                anderson_solve_kernel<<<1, 256, 0, c->stream>>>(part, 64, count, gam, ffv);
                anderson_update_kernel<double><<<nblocks(n), 256, 0, c->stream>>>(y, r, cj, beta, Xs, Fs, slots, gam,
                                                                                  count, n);
                SDFT_CUDA(cudaGetLastError());
                count_launch(c, 3);
                SDFT_CUDA(cudaMemcpyAsync(c->hscal, ffv, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
                SDFT_CUDA(cudaStreamSynchronize(c->stream));
                const double rn2 = c->hscal[0] / (cj * cj);
                if (!std::isfinite(rn2)) throw Error{SDFT_ERR_NONFINITE, "Kerker solve residual is not finite"};
                if (rn2 <= tol * tol * bnorm2) {
                    ++it;
                    done = true;
                    break;
                }
            } else {
                axpby_kernel<double><<<nblocks(n), 256, 0, c->stream>>>(y, r, omega * cj, 1.0, n);
                SDFT_CUDA(cudaGetLastError());
                count_launch(c);
            }
        }
        if (!done) return -it;
    }
    // out = f - k0^2 y
    SDFT_CUDA(cudaMemcpyAsync(out, f, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->stream));
    axpby_kernel<double><<<nblocks(n), 256, 0, c->stream>>>(out, y, -k2, 1.0, n);
    SDFT_CUDA(cudaGetLastError());
    count_launch(c);
    return std::max(it, 1);
}

// Pulay mixing on rho_in (paper Sec. 2.1; Banerjee et al. 2016, Pratapa & Suryanarayana 2015):
// f = rho_out - rho_in; linear step rho += beta f, or Pulay every period-th iteration.
void pulay_update(sdft_ctx* c) {
    const long long n = (long long)c->opt.nspin * c->ng;
    const int m = c->opt.mix_hist;
    double* f = c->work64;  // needs nspin*ng <= 2 ng: use work64[0 .. 2ng)
    // f = rho_out - rho_in
    SDFT_CUDA(cudaMemcpyAsync(f, c->rho_out, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->stream));
    axpby_kernel<double><<<nblocks(n), 256, 0, c->stream>>>(f, c->rho_in, -1.0, 1.0, n);
    count_launch(c);
    const int slot = c->mix_head;
    anderson_push_kernel<double><<<nblocks(n), 256, 0, c->stream>>>(c->rho_in, f, 1.0, c->mix_xprev, c->mix_fprev,
                                                            c->mix_dx + (long long)slot * n,
                                                            c->mix_df + (long long)slot * n, c->mix_k > 0, n);
    count_launch(c);
    if (c->mix_k > 0) {
        c->mix_head = (c->mix_head + 1) % m;
        c->mix_count = std::min(c->mix_count + 1, m);
    }
    const bool pulay = c->mix_k > 0 && c->mix_count > 0 && ((c->mix_k + 1) % c->opt.pulay_period == 0);
    if (c->opt.kerker_k0 > 0.0) {
        // Kerker-preconditioned form: x <- x - X gamma + P(beta (f - F gamma)), P channel by channel
        if (pulay) {
            int hslots[16];
            const int cnt = c->mix_count;
            for (int j = 0; j < cnt; ++j) hslots[j] = ((c->mix_head - cnt + j) % m + m) % m;
            int* slots = (int*)(c->scal + 160);
            double* gam = c->scal + 192;
            double* ffv = c->scal + 224;
            double* part = c->scal + 4096;
            std::memcpy(c->hscal + 640, hslots, sizeof(int) * 16);
            SDFT_CUDA(cudaMemcpyAsync(slots, c->hscal + 640, sizeof(int) * cnt, cudaMemcpyHostToDevice, c->stream));
            const int nblk = 32;
            anderson_gram_kernel<double><<<nblk, RB, 0, c->stream>>>(c->mix_df, slots, cnt, f, 1.0, n, part);
            anderson_solve_kernel<<<1, 256, 0, c->stream>>>(part, nblk, cnt, gam, ffv);
            pulay_residual_kernel<<<nblocks(n), 256, 0, c->stream>>>(c->rho_in, f, c->mix_dx, c->mix_df, slots, gam, cnt,
                                                                     c->opt.mix_beta, n);
            count_launch(c, 3);
            if (c->opt.pulay_restart) c->mix_count = 0;
        } else {
            axpby_kernel<double><<<nblocks(n), 256, 0, c->stream>>>(f, f, 0.0, c->opt.mix_beta, n);
            count_launch(c);
        }
        SDFT_CUDA(cudaGetLastError());
        double* pf = c->work64 + 2 * c->ng;   // P of one channel
        for (int sp = 0; sp < c->opt.nspin; ++sp) {
            const int it = kerker_apply(c, f + (long long)sp * c->ng, pf, c->opt.kerker_k0, KERKER_TOL, 4000);
            if (it < 0) throw Error{SDFT_ERR_NOT_CONVERGED, "Kerker screened-Poisson solve did not converge"};
            axpby_kernel<double><<<nblocks(c->ng), 256, 0, c->stream>>>(c->rho_in + (long long)sp * c->ng, pf, 1.0, 1.0,
                                                                        c->ng);
            count_launch(c);
        }
        SDFT_CUDA(cudaGetLastError());
        c->mix_k += 1;
        return;
    }
    if (pulay) {
        int hslots[16];
        const int cnt = c->mix_count;
        for (int j = 0; j < cnt; ++j) hslots[j] = ((c->mix_head - cnt + j) % m + m) % m;
        int* slots = (int*)(c->scal + 160);
        double* gam = c->scal + 192;
        double* ffv = c->scal + 224;
        double* part = c->scal + 4096;
        std::memcpy(c->hscal + 640, hslots, sizeof(int) * 16);
        SDFT_CUDA(cudaMemcpyAsync(slots, c->hscal + 640, sizeof(int) * cnt, cudaMemcpyHostToDevice, c->stream));
        const int nblk = 32;  // 32 x (m(m+1)/2 + m + 1) <= 12288 partials for m <= 16
        anderson_gram_kernel<double><<<nblk, RB, 0, c->stream>>>(c->mix_df, slots, cnt, f, 1.0, n, part);
        anderson_solve_kernel<<<1, 256, 0, c->stream>>>(part, nblk, cnt, gam, ffv);
        anderson_update_kernel<double><<<nblocks(n), 256, 0, c->stream>>>(c->rho_in, f, 1.0, c->opt.mix_beta, c->mix_dx,
                                                                  c->mix_df, slots, gam, cnt, n);
        count_launch(c, 3);
        if (c->opt.pulay_restart) {
            c->mix_count = 0;
        }
    } else {
        axpby_kernel<double><<<nblocks(n), 256, 0, c->stream>>>(c->rho_in, f, c->opt.mix_beta, 1.0, n);
        count_launch(c);
    }
    SDFT_CUDA(cudaGetLastError());
    c->mix_k += 1;
}

void forces_compute(sdft_ctx* c) {
    const int na = c->natom;
    c->forces.assign(3 * na, 0.0);
    double* dF = c->scal + 3072;  // up to 341 atoms
    SDFT_REQUIRE(3 * na <= 1024, SDFT_ERR_INVALID_ARG, "forces: too many atoms for the scalar area");
    for (int i = 0; i < 3 * na; ++i) c->hscal[i] = -c->dEsc[i];
    SDFT_CUDA(cudaMemcpyAsync(dF, c->hscal, sizeof(double) * 3 * na, cudaMemcpyHostToDevice, c->stream));
    std::vector<AtomG> at = atom_g(c);
    AtomG* dat = (AtomG*)ctx_alloc(c, sizeof(AtomG) * std::max(1, na));
    SDFT_CUDA(cudaMemcpyAsync(dat, at.data(), sizeof(AtomG) * na, cudaMemcpyHostToDevice, c->stream));
    force_local_kernel<<<na, RB, 0, c->stream>>>(dat, c->n[0], c->n[1], c->n[2], c->h[0], c->h[1], c->h[2], c->L[0],
                                                 c->L[1], c->L[2], c->dV, c->phi, dF,
                                                 c->opt.boundary == SDFT_BC_DIRICHLET);
    count_launch(c);
    std::vector<double> rp2(na);
    for (int a = 0; a < na; ++a) rp2[a] = std::pow(c->species[c->types[a]].r_proj, 2);
    double* d_rp2 = (double*)ctx_alloc(c, sizeof(double) * std::max(1, na));
    double* d_pos = (double*)ctx_alloc(c, sizeof(double) * 3 * std::max(1, na));
    SDFT_CUDA(cudaMemcpyAsync(d_rp2, rp2.data(), sizeof(double) * na, cudaMemcpyHostToDevice, c->stream));
    SDFT_CUDA(cudaMemcpyAsync(d_pos, c->pos.data(), sizeof(double) * 3 * na, cudaMemcpyHostToDevice, c->stream));
    for (const Problem& P : c->probs) {
        const KBTables& T = c->kb[P.kpt];
        const void* X = c->opt.precision == SDFT_FP64 ? P.X : P.X64;
        SDFT_REQUIRE(X != nullptr, SDFT_ERR_INVALID_ARG, "forces need FP64 orbitals");
        const double wk = c->kw[P.kpt];
        if (T.cplx)
            force_nl_kernel<true><<<na, RB, 0, c->stream>>>(T.cnt, T.idx, T.img, T.val64, T.cap, (const double*)X,
                                                           c->opt.nstates, c->ng, P.occ, wk, T.gamma, d_pos, d_rp2,
                                                           c->n[0], c->n[1], c->h[0], c->h[1], c->h[2], dF);
        else
            force_nl_kernel<false><<<na, RB, 0, c->stream>>>(T.cnt, T.idx, T.img, T.val64, T.cap, (const double*)X,
                                                            c->opt.nstates, c->ng, P.occ, wk, T.gamma, d_pos, d_rp2,
                                                            c->n[0], c->n[1], c->h[0], c->h[1], c->h[2], dF);
        count_launch(c);
    }
    SDFT_CUDA(cudaGetLastError());
    SDFT_CUDA(cudaMemcpyAsync(c->hscal, dF, sizeof(double) * 3 * na, cudaMemcpyDeviceToHost, c->stream));
    SDFT_CUDA(cudaStreamSynchronize(c->stream));
    for (int i = 0; i < 3 * na; ++i) c->forces[i] = c->hscal[i];
    ctx_release(c, dat);   // per-call tables: released so that repeated SCFs (MD steps) do not accumulate them
    ctx_release(c, d_rp2);
    ctx_release(c, d_pos);
}

}  // namespace sdft
