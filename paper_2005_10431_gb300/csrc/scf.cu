// CheFSI inside the SCF loop (paper Sec. 2.1):
//  * spectrum bounds by Lanczos, then per SCF iteration a degree-m Chebyshev filter and a
//    Rayleigh-Ritz step for every (spin, k) problem, several filter passes in the first
//    SCF iteration;
//  * Fermi level, density (Eq. 2), Harris-Foulkes free energy, SCF error, Pulay mixing;
//  * for SDFT_MIXED, an optional FP64 filter + Rayleigh-Ritz pass at the end.
// Host code drives the iteration; every grid- or block-sized step runs in this library's
// kernels on the context's stream.
#include "internal.cuh"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <type_traits>

namespace sdft {

// ---------------------------------------------------------------------------------------
// counter-based initial orbitals: splitmix64 (Steele, Lea & Flood 2014), uniform in [-0.5, 0.5)
// value (g, n) of stream s = top 53 bits of splitmix64(s * 2^32 + n*ngrid + g)
// ---------------------------------------------------------------------------------------
namespace {
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long x) {
    unsigned long long z = x + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
__device__ __forceinline__ double uniform_counter(unsigned long long seed, unsigned long long i) {
    const unsigned long long z = splitmix64(((seed & 0xffffffffULL) << 32) + i);
    return (double)(z >> 11) * (1.0 / 9007199254740992.0) - 0.5;
}

__global__ void seed_kernel(int kind, void* __restrict__ X, int ncol, long long ng, unsigned long long seed) {
    const long long total = (long long)ncol * ng;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
        const int n = (int)(e / ng);
        const long long g = e - (long long)n * ng;
        const double re = uniform_counter(seed, (unsigned long long)e);
        if (kind == 0) {
            ((double*)X)[e] = re;
        } else if (kind == 1) {
            const double im = uniform_counter(seed + 0x5BD1, (unsigned long long)e);
            ((double2*)X)[e] = make_double2(re, im);
        } else if (kind == 2) {
            ((float*)X)[(((long long)(n >> 1)) * ng + g) * 2 + (n & 1)] = (float)re;
        } else {
            const double im = uniform_counter(seed + 0x5BD1, (unsigned long long)e);
            ((float2*)X)[e] = make_float2((float)re, (float)im);
        }
    }
}

__global__ void spin_split_kernel(const double* __restrict__ rho, int nspin, double moment, double* __restrict__ out,
                                  long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        if (nspin == 1) {
            out[i] = rho[i];
        } else {
            out[i] = 0.5 * rho[i] * (1.0 + moment);
            out[n + i] = 0.5 * rho[i] * (1.0 - moment);
        }
    }
}

__global__ void lincomb_kernel(double* __restrict__ y, const double* __restrict__ x, const double* __restrict__ z,
                               double a, double b, double cc, long long n) {
    // y = a*y + b*x + cc*z
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        double v = a * y[i] + b * x[i];
        if (z) v += cc * z[i];
        y[i] = v;
    }
}

__global__ void sum_spins_kernel(const double* __restrict__ rho, int nspin, const double* __restrict__ add,
                                 double* __restrict__ out, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        double s = add ? add[i] : 0.0;
        for (int k = 0; k < nspin; ++k) s += rho[k * n + i];
        out[i] = s;
    }
}

inline unsigned nb(long long n) { return (unsigned)std::min<long long>((n + 255) / 256, 152LL * 16); }
inline int kind_of(int precision, bool cplx) { return precision == SDFT_FP64 ? (cplx ? 1 : 0) : (cplx ? 3 : 2); }
inline double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// ---- typed filter / H application -------------------------------------------------------
template <typename E>
void filter_typed(sdft_ctx* c, int kpt, const E* X, E* Y, E* T1, E* T2, int ncolE, int m, double a, double b,
                  double a0, const typename Elem<E>::S* V, E* C) {
    const double e = 0.5 * (b - a), cc = 0.5 * (b + a);
    const double sigma1 = e / (a0 - cc);
    double sigma = sigma1;
    E* ring[3] = {T1, T2, Y};
    auto slot = [&](int k) -> E* { return ring[(((2 - (m - k)) % 3) + 3) % 3]; };
    const bool kb = c->kb[kpt].S > 0;
    // FP32 real blocks: a slab-tile step may also produce the KB coefficients of its output (into the
    // other coefficient buffer), which then replace the next step's projection pass
    E* Cb[2] = {C, C};
    if constexpr (std::is_same<E, float2>::value)
        if (C == reinterpret_cast<E*>(c->C32) && !c->kb[kpt].cplx && c->fuse_kb_projection) Cb[1] = reinterpret_cast<E*>(c->C32b);
    int ci = 0;
    bool have = false;
    for (int k = 1; k <= m; ++k) {
        const E* cur = k == 1 ? X : slot(k - 1);
        const E* prev = k == 1 ? nullptr : (k == 2 ? X : slot(k - 2));
        if (kb && !have) launch_kb_project<E>(c, kpt, cur, Cb[ci], ncolE);
        double alpha, beta = 0.0;
        if (k == 1) {
            alpha = sigma1 / e;
        } else {
            const double sigma2 = 1.0 / (2.0 / sigma1 - sigma);
            alpha = 2.0 * sigma2 / e;
            beta = sigma * sigma2;
            sigma = sigma2;
        }
        if constexpr (std::is_same<E, float2>::value) {
            c->kb_next = (kb && k < m && Cb[1] != Cb[0]) ? reinterpret_cast<float2*>(Cb[ci ^ 1]) : nullptr;
            c->kb_next_done = false;
        }
        launch_cheb_step<E>(c, kpt, cur, prev, slot(k), ncolE, V, kb ? Cb[ci] : nullptr, alpha, beta, cc);
        have = false;
        if constexpr (std::is_same<E, float2>::value) {
            have = c->kb_next != nullptr && c->kb_next_done;
            c->kb_next = nullptr;
            c->kb_next_done = false;
        }
        if (have) ci ^= 1;
    }
}

template <typename E>
void apply_h_typed(sdft_ctx* c, int kpt, const E* X, E* Y, int ncolE, const typename Elem<E>::S* V, E* C) {
    const bool kb = c->kb[kpt].S > 0;
    if (kb) launch_kb_project<E>(c, kpt, X, C, ncolE);
    launch_cheb_step<E>(c, kpt, X, nullptr, Y, ncolE, V, kb ? C : nullptr, 1.0, 0.0, 0.0);
}

// pick the two filter temporaries among the context's block buffers, distinct from Y/X
void pick_temps(sdft_ctx* c, const void* X, const void* Y, void** t1, void** t2) {
    int got = 0;
    for (int i = 0; i < 4 && got < 2; ++i) {
        if (c->blk[i] == X || c->blk[i] == Y) continue;
        if (got == 0) *t1 = c->blk[i];
        else *t2 = c->blk[i];
        ++got;
    }
    SDFT_REQUIRE(got == 2, SDFT_ERR_INVALID_ARG, "no free block buffers for the filter");
}

// tridiagonal (alpha, beta) extreme eigenvalues by Sturm-sequence bisection
double sturm_count(const std::vector<double>& al, const std::vector<double>& be, double x) {
    int cnt = 0;
    double q = 1.0;
    for (size_t i = 0; i < al.size(); ++i) {
        const double b2 = i > 0 ? be[i - 1] * be[i - 1] : 0.0;
        q = al[i] - x - (i > 0 ? b2 / q : 0.0);
        if (q == 0.0) q = -1e-300;
        if (q < 0) ++cnt;
    }
    return cnt;
}
double tridiag_eig(const std::vector<double>& al, const std::vector<double>& be, int which) {
    // which-th smallest eigenvalue (0-based)
    double lo = 1e300, hi = -1e300;
    for (size_t i = 0; i < al.size(); ++i) {
        const double r = (i > 0 ? std::fabs(be[i - 1]) : 0.0) + (i + 1 < al.size() ? std::fabs(be[i]) : 0.0);
        lo = std::min(lo, al[i] - r);
        hi = std::max(hi, al[i] + r);
    }
    for (int it = 0; it < 200; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (sturm_count(al, be, mid) > which) hi = mid;
        else lo = mid;
        if (hi - lo < 1e-15 * std::max(1.0, std::fabs(mid))) break;
    }
    return 0.5 * (lo + hi);
}

}  // namespace

// ---------------------------------------------------------------------------------------
void axpby_dev(sdft_ctx* c, double* y, const double* x, double a, double b, long long n) {
    lincomb_kernel<<<nb(n), 256, 0, c->stream>>>(y, x, nullptr, b, a, 0.0, n);
    SDFT_CUDA(cudaGetLastError());
    count_launch(c);
}

void seed_orbitals(sdft_ctx* c, int precision, bool cplx, void* X, int ncol, uint64_t seed) {
    seed_kernel<<<nb((long long)ncol * c->ng), 256, 0, c->stream>>>(kind_of(precision, cplx), X, ncol, c->ng, seed);
    SDFT_CUDA(cudaGetLastError());
    count_launch(c);
}

uint64_t problem_seed(const sdft_ctx* c, int s, int k) {
    return c->opt.seed * 4099ULL + (uint64_t)s * (uint64_t)c->opt.nkpt + (uint64_t)k;
}

void chebyshev_filter(sdft_ctx* c, int kpt, int precision, const void* X, void* Y, int ncol, int degree, double a,
                      double b, double a0, const double* veff64, const float* veff32) {
    SDFT_REQUIRE(degree >= 1, SDFT_ERR_INVALID_ARG, "degree must be >= 1");
    SDFT_REQUIRE(b > a && a > a0, SDFT_ERR_INVALID_ARG, "filter bounds must satisfy a0 < a < b");
    void *t1 = nullptr, *t2 = nullptr;
    pick_temps(c, X, Y, &t1, &t2);
    const bool cplx = c->kb[kpt].cplx;
    if (precision == SDFT_FP64) {
        if (cplx)
            filter_typed<double2>(c, kpt, (const double2*)X, (double2*)Y, (double2*)t1, (double2*)t2, ncol, degree, a,
                                  b, a0, veff64, (double2*)c->C64);
        else
            filter_typed<double>(c, kpt, (const double*)X, (double*)Y, (double*)t1, (double*)t2, ncol, degree, a, b,
                                 a0, veff64, c->C64);
    } else {
        const int ncolE = cplx ? ncol : ncol / 2;
        filter_typed<float2>(c, kpt, (const float2*)X, (float2*)Y, (float2*)t1, (float2*)t2, ncolE, degree, a, b, a0,
                             veff32, (float2*)c->C32);
    }
}

void apply_h(sdft_ctx* c, int kpt, int precision, const void* X, void* Y, int ncol, const double* veff64,
             const float* veff32) {
    const bool cplx = c->kb[kpt].cplx;
    if (precision == SDFT_FP64) {
        if (cplx) apply_h_typed<double2>(c, kpt, (const double2*)X, (double2*)Y, ncol, veff64, (double2*)c->C64);
        else apply_h_typed<double>(c, kpt, (const double*)X, (double*)Y, ncol, veff64, c->C64);
    } else {
        const int ncolE = cplx ? ncol : ncol / 2;
        apply_h_typed<float2>(c, kpt, (const float2*)X, (float2*)Y, ncolE, veff32, (float2*)c->C32);
    }
}

void rayleigh_ritz(sdft_ctx* c, int kpt, int precision, const void* Y, void* X, double* eig, int ncol,
                   const double* veff64, const float* veff32) {
    const bool cplx = c->kb[kpt].cplx;
    void* HY = nullptr;
    for (int i = 0; i < 4; ++i)
        if (c->blk[i] != Y && c->blk[i] != X) {
            HY = c->blk[i];
            break;
        }
    SDFT_REQUIRE(HY != nullptr, SDFT_ERR_INVALID_ARG, "no free block buffer for H Y");
    apply_h(c, kpt, precision, Y, HY, ncol, veff64, veff32);
    subspace_gram(c, precision, cplx, Y, HY, c->Ms, c->Hs, ncol);
    generalized_eig(c, cplx, c->Ms, c->Hs, eig, ncol);
    rotate_block(c, precision, cplx, Y, c->Hs, X, ncol);
}

// Lanczos on one FP64 vector started from the problem's first seeded orbital
void lanczos(sdft_ctx* c, int spin, int kpt, int steps, double* lower, double* upper) {
    const bool cplx = c->kb[kpt].cplx;
    const long long len = c->ng * (cplx ? 2 : 1);
    double* v = c->work64 + 0 * 2 * c->ng;
    double* vp = c->work64 + 1 * 2 * c->ng;
    double* w = c->work64 + 2 * 2 * c->ng;
    seed_orbitals(c, SDFT_FP64, cplx, v, 1, problem_seed(c, spin, kpt));
    SDFT_CUDA(cudaMemsetAsync(vp, 0, sizeof(double) * len, c->stream));
    const double* veff = c->veff + (long long)spin * c->ng;
    double nrm;
    {
        const double* A[1] = {v};
        dots_host(c, 1, A, A, len, &nrm);
    }
    axpby_dev(c, v, v, 1.0 / std::sqrt(nrm), 0.0, len);
    std::vector<double> al, be;
    double beta = 0.0;
    for (int j = 0; j < steps; ++j) {
        apply_h(c, kpt, SDFT_FP64, v, w, 1, veff, nullptr);
        double alpha;
        {
            const double* A[1] = {v};
            const double* B[1] = {w};
            dots_host(c, 1, A, B, len, &alpha);
        }
        lincomb_kernel<<<nb(len), 256, 0, c->stream>>>(w, v, vp, 1.0, -alpha, -beta, len);
        count_launch(c);
        double bn2;
        {
            const double* A[1] = {w};
            dots_host(c, 1, A, A, len, &bn2);
        }
        const double bnext = std::sqrt(bn2);
        al.push_back(alpha);
        be.push_back(bnext);
        // vp = v; v = w / bnext
        SDFT_CUDA(cudaMemcpyAsync(vp, v, sizeof(double) * len, cudaMemcpyDeviceToDevice, c->stream));
        lincomb_kernel<<<nb(len), 256, 0, c->stream>>>(v, w, nullptr, 0.0, 1.0 / bnext, 0.0, len);
        count_launch(c);
        beta = bnext;
    }
    std::vector<double> off(be.begin(), be.end() - 1);
    *lower = tridiag_eig(al, off, 0);
    *upper = tridiag_eig(al, off, (int)al.size() - 1) + be.back();
}

void reset_state(sdft_ctx* c) {
    const long long ng = c->ng;
    const int ns = c->opt.nspin;
    if (c->user_density) {
        SDFT_CUDA(cudaMemcpyAsync(c->rho_in, c->rho_user, sizeof(double) * ns * ng, cudaMemcpyDeviceToDevice, c->stream));
    } else {
        spin_split_kernel<<<nb(ng), 256, 0, c->stream>>>(c->rho_sad, ns, c->opt.initial_moment, c->rho_in, ng);
        count_launch(c);
    }
    SDFT_CUDA(cudaMemsetAsync(c->phi, 0, sizeof(double) * ng, c->stream));
    for (Problem& P : c->probs) {
        seed_orbitals(c, c->opt.precision, P.cplx, P.X, c->nfilt, problem_seed(c, P.spin, P.kpt));
        P.have_bounds = false;
    }
    c->warm_start = false;
    c->mix_k = 0;
    c->mix_count = 0;
    c->mix_head = 0;
    c->log.clear();
    SDFT_CUDA(cudaGetLastError());
}

// the occupied set's Ritz values (the lowest nstates) from the filtered block's (with buffer states)
static void keep_lowest_ritz_values(sdft_ctx* c, Problem& P) {
    if (P.eigf != P.eig)
        SDFT_CUDA(cudaMemcpyAsync(P.eig, P.eigf, sizeof(double) * c->opt.nstates, cudaMemcpyDeviceToDevice, c->stream));
}

// Rayleigh-Ritz of problem P on the filtered block Y into X, and the new filter bounds
static void rr_pass(sdft_ctx* c, Problem& P, int precision, void* Y, void* X) {
    const int nf = c->nfilt;
    const double* v64 = c->veff + (long long)P.spin * c->ng;
    const float* v32 = c->veff32 + (long long)P.spin * c->ng;
    rayleigh_ritz(c, P.kpt, precision, Y, X, P.eigf, nf, v64, v32);
    keep_lowest_ritz_values(c, P);
    double e2[2];
    SDFT_CUDA(cudaMemcpyAsync(&e2[0], P.eigf, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    SDFT_CUDA(cudaMemcpyAsync(&e2[1], P.eigf + nf - 1, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    SDFT_CUDA(cudaStreamSynchronize(c->stream));
    check_stencil_flag(c);
    if (!std::isfinite(e2[0]) || !std::isfinite(e2[1])) throw Error{SDFT_ERR_NONFINITE, "Ritz values are not finite"};
    P.lower = e2[0];
    P.cutoff = e2[1];
}

// one CheFSI pass of problem P at the current V_eff in `precision`
static void chefsi_pass(sdft_ctx* c, Problem& P, int precision, void* X) {
    const double* v64 = c->veff + (long long)P.spin * c->ng;
    const float* v32 = c->veff32 + (long long)P.spin * c->ng;
    void* Y = c->blk[0];
    chebyshev_filter(c, P.kpt, precision, X, Y, c->nfilt, c->opt.cheb_degree, P.cutoff, P.upper, P.lower, v64, v32);
    rr_pass(c, P, precision, Y, X);
}

// ---- batched CheFSI: all problems of one storage kind in grouped launches -------------------
// Per Chebyshev step one grouped KB projection and one grouped row-tile stencil launch cover every
// problem; the H Y of Rayleigh-Ritz likewise; then Gram matrices per problem, one batched
// eigensolve for all problems, rotations per problem, and one host read of all Ritz bounds.
static void ensure_group_buffers(sdft_ctx* c, int nprob, bool cplx) {
    const int ns = c->nfilt;
    if ((int)c->g_M.size() >= nprob) return;
    const size_t bytes = block_elems_bytes(c, SDFT_MIXED, cplx, ns);
    const int w2 = cplx ? 2 : 1;
    for (int p = (int)c->g_M.size(); p < nprob; ++p) {
        for (int i = 0; i < 3; ++i) c->g_blk.push_back(ctx_alloc(c, bytes));
        c->g_M.push_back((double*)ctx_alloc(c, sizeof(double) * ns * ns * w2));
        c->g_H.push_back((double*)ctx_alloc(c, sizeof(double) * ns * ns * w2));
        c->g_C.push_back(ctx_alloc(c, sizeof(float2) * (size_t)std::max(1, c->natom) * ns));
    }
}

static void chefsi_pass_group(sdft_ctx* c, const std::vector<Problem*>& G, int variant) {
    const int ns = c->nfilt, m = c->opt.cheb_degree;   // filtered block width
    const int np = (int)G.size();
    const bool cplx = G[0]->cplx;
    const int ncolE = cplx ? ns : ns / 2;
    const long long ng = c->ng;
    ensure_group_buffers(c, np, cplx);
    const int ntab = (m + 1) * np;
    if (c->g_tab_cap < ntab) {
        c->g_rtab = (RowProblem*)ctx_alloc(c, sizeof(RowProblem) * ntab);
        c->g_ktab = (KBProblem*)ctx_alloc(c, sizeof(KBProblem) * ntab);
        c->g_tab_cap = ntab;
    }
    c->g_rtab_h.assign(ntab, RowProblem{});
    c->g_ktab_h.assign(ntab, KBProblem{});
    bool haskb = false;
    for (int p = 0; p < np; ++p) {
        const Problem& P = *G[p];
        const double a = P.cutoff, b = P.upper, a0 = P.lower;
        SDFT_REQUIRE(b > a && a > a0, SDFT_ERR_INVALID_ARG, "filter bounds must satisfy a0 < a < b");
        const KBTables& kb = c->kb[P.kpt];
        haskb = haskb || kb.S > 0;
        float2* ring[3] = {(float2*)c->g_blk[3 * p], (float2*)c->g_blk[3 * p + 1], (float2*)c->g_blk[3 * p + 2]};
        auto slot = [&](int k) -> float2* { return ring[(((2 - (m - k)) % 3) + 3) % 3]; };
        const float2* X = (const float2*)P.X;
        float2* Cp = (float2*)c->g_C[p];
        RowProblem base{};
        base.V = c->veff32 + (long long)P.spin * ng;
        base.C = Cp;
        base.patom = kb.patom;
        base.pval = kb.pval32;
        base.nslot = kb.S;
        for (int d = 0; d < 3; ++d) {
            const double kd = c->kpts.empty() ? 0.0 : c->kpts[3 * P.kpt + d];
            base.phr[d] = (float)cos(2.0 * M_PI * kd);
            base.phi[d] = (float)sin(2.0 * M_PI * kd);
        }
        KBProblem kbase{nullptr, Cp, kb.cnt, kb.idx, kb.val32, kb.gamma, kb.cap, kb.natom, ncolE, ng};
        const double e = 0.5 * (b - a), cc = 0.5 * (b + a);
        const double sigma1 = e / (a0 - cc);
        double sigma = sigma1;
        for (int k = 1; k <= m; ++k) {
            RowProblem r = base;
            r.Y = k == 1 ? X : slot(k - 1);
            r.Yprev = k == 1 ? nullptr : (k == 2 ? X : slot(k - 2));
            r.Ynext = slot(k);
            double alpha, beta = 0.0;
            if (k == 1) {
                alpha = sigma1 / e;
            } else {
                const double sigma2 = 1.0 / (2.0 / sigma1 - sigma);
                alpha = 2.0 * sigma2 / e;
                beta = sigma * sigma2;
                sigma = sigma2;
            }
            r.alpha = (float)alpha;
            r.beta = (float)beta;
            r.shift = (float)cc;
            c->g_rtab_h[(k - 1) * np + p] = r;
            KBProblem kp = kbase;
            kp.Y = r.Y;
            c->g_ktab_h[(k - 1) * np + p] = kp;
        }
        // H Y of Rayleigh-Ritz: Y = slot(m) -> HY in the first free ring buffer
        RowProblem r = base;
        r.Y = slot(m);
        r.Yprev = nullptr;
        r.Ynext = slot(m - 1) == slot(m) ? slot(m - 2) : slot(m - 1);
        r.alpha = 1.f;
        r.beta = 0.f;
        r.shift = 0.f;
        c->g_rtab_h[m * np + p] = r;
        KBProblem kp = kbase;
        kp.Y = r.Y;
        c->g_ktab_h[m * np + p] = kp;
    }
    // first grouped pass of this context: time the row tiles on the H Y launch (its output buffer
    // is rewritten below), keep the fastest
    int& gch = c->group_choice[cplx ? 1 : 0];
    if (gch < 0) {
        SDFT_CUDA(cudaMemcpyAsync(c->g_rtab, c->g_rtab_h.data(), sizeof(RowProblem) * ntab, cudaMemcpyHostToDevice,
                                  c->stream));
        SDFT_CUDA(cudaMemcpyAsync(c->g_ktab, c->g_ktab_h.data(), sizeof(KBProblem) * ntab, cudaMemcpyHostToDevice,
                                  c->stream));
        if (haskb) launch_group_project_f32(c, cplx, c->g_ktab + (size_t)m * np, np, ncolE);
        gch = autotune_group_f32(c, cplx, c->g_rtab + (size_t)m * np, np, ncolE, haskb);
    }
    if (gch >= 0) variant = gch;
    // the filter (m steps) and H Y, every problem per launch, after uploading this pass's tables
    auto enqueue = [&](const RowProblem* rsrc, const KBProblem* ksrc) {
        SDFT_CUDA(cudaMemcpyAsync(c->g_rtab, rsrc, sizeof(RowProblem) * ntab, cudaMemcpyHostToDevice, c->stream));
        SDFT_CUDA(cudaMemcpyAsync(c->g_ktab, ksrc, sizeof(KBProblem) * ntab, cudaMemcpyHostToDevice, c->stream));
        for (int k = 0; k <= m; ++k) {
            if (haskb) launch_group_project_f32(c, cplx, c->g_ktab + (size_t)k * np, np, ncolE);
            launch_group_step_f32(c, cplx, variant, c->g_rtab + (size_t)k * np, np, ncolE, k > 0 && k < m, haskb);
        }
    };
    if (c->opt.use_graphs && !c->timing) {
        // CUDA graph of the grouped filter: captured once, replayed every pass; the replay copies
        // this pass's coefficients from the pinned tables, so only the host copy below changes
        if (c->g_pin_cap < ntab) {
            if (c->g_rtab_pin) cudaFreeHost(c->g_rtab_pin);
            if (c->g_ktab_pin) cudaFreeHost(c->g_ktab_pin);
            c->g_rtab_pin = nullptr;
            c->g_ktab_pin = nullptr;
            SDFT_CUDA(cudaMallocHost((void**)&c->g_rtab_pin, sizeof(RowProblem) * ntab));
            SDFT_CUDA(cudaMallocHost((void**)&c->g_ktab_pin, sizeof(KBProblem) * ntab));
            c->g_pin_cap = ntab;
            if (c->g_graph) cudaGraphExecDestroy(c->g_graph);
            c->g_graph = nullptr;
        }
        SDFT_CUDA(cudaStreamSynchronize(c->stream));   // the previous replay has read the pinned tables
        std::memcpy(c->g_rtab_pin, c->g_rtab_h.data(), sizeof(RowProblem) * ntab);
        std::memcpy(c->g_ktab_pin, c->g_ktab_h.data(), sizeof(KBProblem) * ntab);
        // a graph bakes in the launch shapes and the block pointers; recapture when they change
        std::vector<long long> key = {np, variant, (long long)cplx, m, (long long)haskb, ncolE};
        for (int p = 0; p < np; ++p) key.push_back((long long)(uintptr_t)G[p]->X);
        if (!c->g_graph || key != c->g_graph_key) {
            if (c->g_graph) cudaGraphExecDestroy(c->g_graph);
            c->g_graph = nullptr;
            const uint64_t l0 = c->launches;
            cudaGraph_t graph = nullptr;
            // capture on a private stream (the context's stream may be the legacy default stream,
            // which cannot be captured); the graph is then launched on the context's stream
            if (!c->cap_stream) SDFT_CUDA(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
            cudaStream_t user_stream = c->stream;
            c->stream = c->cap_stream;
            SDFT_CUDA(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
            try {
                enqueue(c->g_rtab_pin, c->g_ktab_pin);
            } catch (...) {
                cudaStreamEndCapture(c->stream, &graph);
                if (graph) cudaGraphDestroy(graph);
                c->stream = user_stream;
                throw;
            }
            const cudaError_t ce = cudaStreamEndCapture(c->stream, &graph);
            c->stream = user_stream;
            SDFT_CUDA(ce);
            const cudaError_t ie = cudaGraphInstantiate(&c->g_graph, graph, 0);
            cudaGraphDestroy(graph);
            SDFT_CUDA(ie);
            c->g_graph_launches = (int)(c->launches - l0);
            c->launches = l0;
            c->g_graph_key = key;
        }
        SDFT_CUDA(cudaGraphLaunch(c->g_graph, c->stream));
        count_launch(c, c->g_graph_launches);
    } else {
        enqueue(c->g_rtab_h.data(), c->g_ktab_h.data());
    }
    // Gram matrices per problem, one batched eigensolve, rotations per problem
    for (int p = 0; p < np; ++p) {
        const RowProblem& r = c->g_rtab_h[m * np + p];
        subspace_gram(c, SDFT_MIXED, cplx, r.Y, r.Ynext, c->g_M[p], c->g_H[p], ns);
    }
    if (batched_eig_supported(ns)) {
        ensure_ptab(c, np, 3);
        c->ptab_host.resize(3 * np);
        for (int p = 0; p < np; ++p) {
            c->ptab_host[p] = c->g_M[p];
            c->ptab_host[np + p] = c->g_H[p];
            c->ptab_host[2 * np + p] = G[p]->eigf;
        }
        SDFT_CUDA(cudaMemcpyAsync(c->ptab_dev, c->ptab_host.data(), sizeof(void*) * 3 * np, cudaMemcpyHostToDevice,
                                  c->stream));
        double* const* tab = reinterpret_cast<double* const*>(c->ptab_dev);
        batched_generalized_eig(c, cplx, tab, tab + np, tab + 2 * np, ns, np, c->pinfo_dev);
        std::vector<int> info(np);
        SDFT_CUDA(cudaMemcpyAsync(info.data(), c->pinfo_dev, sizeof(int) * np, cudaMemcpyDeviceToHost, c->stream));
        SDFT_CUDA(cudaStreamSynchronize(c->stream));
        for (int p = 0; p < np; ++p)
            if (info[p] != 0) throw Error{SDFT_ERR_CHOLESKY, "subspace overlap matrix not positive definite"};
    } else {
        for (int p = 0; p < np; ++p) generalized_eig(c, cplx, c->g_M[p], c->g_H[p], G[p]->eigf, ns);
    }
    for (int p = 0; p < np; ++p) {
        const RowProblem& r = c->g_rtab_h[m * np + p];
        rotate_block(c, SDFT_MIXED, cplx, r.Y, c->g_H[p], G[p]->X, ns);
    }
    std::vector<double> e2(2 * np);
    for (int p = 0; p < np; ++p) {
        keep_lowest_ritz_values(c, *G[p]);
        SDFT_CUDA(cudaMemcpyAsync(&e2[2 * p], G[p]->eigf, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        SDFT_CUDA(cudaMemcpyAsync(&e2[2 * p + 1], G[p]->eigf + ns - 1, sizeof(double), cudaMemcpyDeviceToHost,
                                  c->stream));
    }
    SDFT_CUDA(cudaStreamSynchronize(c->stream));
    for (int p = 0; p < np; ++p) {
        if (!std::isfinite(e2[2 * p]) || !std::isfinite(e2[2 * p + 1]))
            throw Error{SDFT_ERR_NONFINITE, "Ritz values are not finite"};
        G[p]->lower = e2[2 * p];
        G[p]->cutoff = e2[2 * p + 1];
    }
}

struct Energies {
    double F, mu, ts, eband;
};

// Harris-Foulkes free energy from rho_in quantities and the band energy (all on device)
static Energies energy_hf(sdft_ctx* c, const double* rho_in, const double* veff, const double* exc,
                          const double* phi, double* rho_tot_tmp) {
    const int ns = c->opt.nspin;
    const long long ng = c->ng;
    double mu_ts_eb[3];
    SDFT_CUDA(cudaMemcpyAsync(mu_ts_eb, c->scal + 8, 3 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    sum_spins_kernel<<<nb(ng), 256, 0, c->stream>>>(rho_in, ns, nullptr, rho_tot_tmp, ng);
    count_launch(c);
    double* rb = rho_tot_tmp + ng;  // rho_tot + b
    sum_spins_kernel<<<nb(ng), 256, 0, c->stream>>>(rho_in, ns, c->b, rb, ng);
    count_launch(c);
    const double* A[3] = {veff, exc, rb};
    const double* B[3] = {rho_in, rho_tot_tmp, phi};
    double d[3];
    // veff . rho_in over all spins (nspin*ng contiguous)
    double vr;
    {
        const double* a1[1] = {veff};
        const double* b1[1] = {rho_in};
        dots_host(c, 1, a1, b1, ns * ng, &vr);
    }
    dots_host(c, 3, A, B, ng, d);
    Energies E;
    E.mu = mu_ts_eb[0];
    E.ts = mu_ts_eb[1];
    E.eband = mu_ts_eb[2];
    E.F = E.eband - c->dV * vr + c->dV * d[1] + 0.5 * c->dV * d[2] - c->E_self + c->E_sc + E.ts;
    return E;
}

static void density_all(sdft_ctx* c, int precision, bool fp64_copy) {
    const int ns = c->opt.nstates;
    SDFT_CUDA(cudaMemsetAsync(c->rho_out, 0, sizeof(double) * c->opt.nspin * c->ng, c->stream));
    for (Problem& P : c->probs) {
        const void* X = fp64_copy ? P.X64 : P.X;
        density_accumulate(c, precision, P.cplx, X, P.occ, ns, c->kw[P.kpt], c->rho_out + (long long)P.spin * c->ng);
    }
}

// One SCF run of a context, in stages, so that several contexts can be stepped in lockstep
// (sdft_batch_scf) as well as alone (run_scf).
struct ScfRun {
    sdft_ctx* c;
    long long ng = 0, nv = 0;
    int nsp = 1, prec = SDFT_FP64;
    double *ftmp = nullptr, *etmp = nullptr, *diff = nullptr;
    double t_filter = 0, t_rr = 0, t_pois = 0, t0 = 0;
    cudaEvent_t ev_start = nullptr, ev_it = nullptr;
    bool converged = false, done = false;
    double last_err = 1.0;
    int it = 0, niter = 0;
    int last_pit = 0;          // AAR iterations and requested tolerance of the last Poisson solve
    double last_ptol = 0.0;
    Energies E{};
    // batched CheFSI: problems of one storage kind that a grouped row-tile launch fits
    std::vector<Problem*> groups[2], single;
    int group_var[2] = {-1, -1};
    bool batched = false;
    // mixed run finishing in FP64 (fp64_switch_tol): CheFSI passes on the FP64 copies of the orbitals
    bool tail64 = false;

    explicit ScfRun(sdft_ctx* c_) : c(c_) {}
    ScfRun(const ScfRun&) = delete;
    ScfRun& operator=(const ScfRun&) = delete;
    ~ScfRun() {
        if (ev_start) cudaEventDestroy(ev_start);
        if (ev_it) cudaEventDestroy(ev_it);
    }

    // several filter passes at the first V_eff (paper Sec. 2.1), one when the orbitals of the previous
    // MD step start the run
    int passes() const { return (it == 0 && !warm) ? std::max(1, c->opt.first_scf_filter_passes) : 1; }
    bool warm = false;

    void begin() {
        ng = c->ng;
        nsp = c->opt.nspin;
        nv = nsp * ng;
        prec = c->opt.precision;
        c->gemm_fp32 = false;
        warm = c->warm_start;
        c->warm_start = false;
        c->log.clear();
        ftmp = c->work64 + 20 * ng;   // rho_tot + b
        etmp = c->work64 + 21 * ng;   // two grid vectors for energies
        diff = c->work64 + 18 * ng;   // rho_out - rho_in (2 ng)
        t0 = now_s();
        // device-side clock of the run: an event at the start and one at the end of each iteration
        SDFT_CUDA(cudaEventCreate(&ev_start));
        SDFT_CUDA(cudaEventCreate(&ev_it));
        SDFT_CUDA(cudaEventRecord(ev_start, c->stream));
        if (prec == SDFT_MIXED && c->opt.batch_problems && c->probs.size() > 1) {
            for (int k = 0; k < 2; ++k) {
                const int ncolE = k ? c->nfilt : c->nfilt / 2;
                group_var[k] = group_variant_f32(c, k == 1, ncolE);
            }
            for (Problem& P : c->probs) {
                const int k = P.cplx ? 1 : 0;
                if (group_var[k] >= 0) groups[k].push_back(&P);
                else single.push_back(&P);
            }
            batched = !groups[0].empty() || !groups[1].empty();
        }
        done = c->opt.max_scf <= 0;
    }

    // potentials from rho_in (paper Sec. 2.1: Poisson by AAR, then V_eff = phi + V_xc), and the
    // Lanczos bounds of problems that have none yet
    void potential() {
        const double ta = now_s();
        sum_spins_kernel<<<nb(ng), 256, 0, c->stream>>>(c->rho_in, nsp, c->b, ftmp, ng);
        count_launch(c);
        // the potential only needs to be as accurate as the current SCF error allows: a relative
        // residual of 1e-2 x the last SCF error, at most 1e-4, and always two orders of magnitude
        // below the SCF target itself (a looser factor, 1e-1, stalls the Pulay mixing)
        const double pfloor = std::min(c->opt.poisson_tol, 1e-2 * c->opt.scf_tol);
        const double ptol = std::max(pfloor, std::min(1e-4, 1e-2 * last_err));
        const int pit = prec == SDFT_MIXED ? poisson_mixed(c, ftmp, c->phi, ptol, 4000)
                                           : poisson_aar(c, ftmp, c->phi, ptol, 4000);
        if (pit < 0) throw Error{SDFT_ERR_NOT_CONVERGED, "Poisson AAR did not converge"};
        last_pit = pit;
        last_ptol = ptol;
        veff_assemble(c);
        SDFT_CUDA(cudaStreamSynchronize(c->stream));
        t_pois += now_s() - ta;
        for (Problem& P : c->probs) {
            if (P.have_bounds) continue;
            double lo, up;
            lanczos(c, P.spin, P.kpt, c->opt.lanczos_steps, &lo, &up);
            P.lower = lo;
            P.upper = up;
            P.cutoff = lo + 0.1 * (up - lo);
            P.have_bounds = true;
        }
    }

    // this iteration's CheFSI passes of every problem of the context
    void filter_all() {
        const double ta = now_s();
        for (int p = 0; p < passes(); ++p) {
            if (tail64) {
                for (Problem& P : c->probs) chefsi_pass(c, P, SDFT_FP64, P.X64);
            } else if (batched) {
                for (int k = 0; k < 2; ++k)
                    if (!groups[k].empty()) chefsi_pass_group(c, groups[k], group_var[k]);
                for (Problem* P : single) chefsi_pass(c, *P, prec, P->X);
            } else {
                for (Problem& P : c->probs) chefsi_pass(c, P, prec, P.X);
            }
        }
        t_filter += now_s() - ta;
    }

    // occupations, density, energy, error, log; Pulay update unless finished.  Returns done.
    bool end_iteration() {
        fermi_device(c, c->probs[0].eig, c->probs[0].occ, c->scal + 8);
        density_all(c, tail64 ? SDFT_FP64 : prec, tail64);
        E = energy_hf(c, c->rho_in, c->veff, c->exc, c->phi, etmp);
        SDFT_CUDA(cudaMemcpyAsync(diff, c->rho_out, sizeof(double) * nv, cudaMemcpyDeviceToDevice, c->stream));
        axpby_dev(c, diff, c->rho_in, -1.0, 1.0, nv);
        double nn[2];
        {
            const double* A[2] = {diff, c->rho_out};
            const double* B[2] = {diff, c->rho_out};
            dots_host(c, 2, A, B, nv, nn);
        }
        const double err = std::sqrt(nn[0] / nn[1]);
        SDFT_CUDA(cudaEventRecord(ev_it, c->stream));
        SDFT_CUDA(cudaEventSynchronize(ev_it));
        float dev_ms = 0.f;
        SDFT_CUDA(cudaEventElapsedTime(&dev_ms, ev_start, ev_it));
        if (!std::isfinite(err) || !std::isfinite(E.F)) throw Error{SDFT_ERR_NONFINITE, "SCF produced non-finite values"};
        sdft_iter_record rec{};
        rec.iter = it;
        rec.energy = E.F;
        rec.scf_error = err;
        rec.mu = E.mu;
        rec.seconds = 1e-3 * dev_ms;
        last_err = err;
        rec.lower = c->probs[0].lower;
        rec.cutoff = c->probs[0].cutoff;
        rec.upper = c->probs[0].upper;
        rec.poisson_iters = last_pit;
        rec.poisson_tol = last_ptol;
        c->log.push_back(rec);
        niter = it + 1;
        if (err < c->opt.scf_tol) {
            converged = true;
            done = true;
            return true;
        }
        if (prec == SDFT_MIXED && c->opt.gemm_fp32_switch_tol > 0.0 && err < c->opt.gemm_fp32_switch_tol)
            c->gemm_fp32 = true;   // FP32 CUDA-core Gram and rotation from the next pass on
        if (!tail64 && prec == SDFT_MIXED && c->opt.fp64_switch_tol > 0.0 && err < c->opt.fp64_switch_tol) {
            // the next passes continue from FP64 copies of the current orbitals
            for (Problem& P : c->probs) convert_block(c, P.cplx, SDFT_MIXED, P.X, P.X64, c->nfilt);
            tail64 = true;
        }
        if (it + 1 < c->opt.max_scf) pulay_update(c);
        ++it;
        done = it >= c->opt.max_scf;
        return done;
    }

    sdft_status finish(sdft_result* out) {
        const sdft_status status = converged ? SDFT_OK : SDFT_ERR_NOT_CONVERGED;
        // final FP64 pass for the mixed path, at the last V_eff
        c->gemm_fp32 = false;   // the step-level calls after the SCF use the tensor cores again
        bool have64 = prec == SDFT_FP64 || tail64;
        if (tail64) {
            // keep the mixed-storage orbitals current for a following run (molecular dynamics)
            for (Problem& P : c->probs) convert_block(c, P.cplx, SDFT_FP64, P.X64, P.X, c->nfilt);
        }
        if (prec == SDFT_MIXED && c->opt.final_fp64_pass && !tail64) {
            for (Problem& P : c->probs) {
                convert_block(c, P.cplx, SDFT_MIXED, P.X, P.X64, c->nfilt);
                chefsi_pass(c, P, SDFT_FP64, P.X64);
            }
            fermi_device(c, c->probs[0].eig, c->probs[0].occ, c->scal + 8);
            density_all(c, SDFT_FP64, true);
            E = energy_hf(c, c->rho_in, c->veff, c->exc, c->phi, etmp);
            have64 = true;
        }
        // Kohn-Sham form at rho_out: phi[rho_out], eps_xc[rho_out]
        double Fks = 0.0;
        {
            double* phi_o = c->work64 + 23 * ng;
            double* exc_o = c->work64 + 24 * ng;
            SDFT_CUDA(cudaMemcpyAsync(phi_o, c->phi, sizeof(double) * ng, cudaMemcpyDeviceToDevice, c->stream));
            sum_spins_kernel<<<nb(ng), 256, 0, c->stream>>>(c->rho_out, nsp, c->b, ftmp, ng);
            count_launch(c);
            const double ptol_o = std::min(c->opt.poisson_tol, 1e-2 * c->opt.scf_tol);
            const int pit = prec == SDFT_MIXED ? poisson_mixed(c, ftmp, phi_o, ptol_o, 4000)
                                               : poisson_aar(c, ftmp, phi_o, ptol_o, 4000);
            if (pit < 0) throw Error{SDFT_ERR_NOT_CONVERGED, "Poisson AAR did not converge"};
            double* vxc_o = c->work64 + 25 * ng;  // [nspin][ng]
            lda_device(c, nsp, c->rho_out, exc_o, vxc_o, (size_t)ng);
            sum_spins_kernel<<<nb(ng), 256, 0, c->stream>>>(c->rho_out, nsp, nullptr, etmp, ng);
            sum_spins_kernel<<<nb(ng), 256, 0, c->stream>>>(c->rho_out, nsp, c->b, etmp + ng, ng);
            count_launch(c, 2);
            double vr, d[2];
            const double* a1[1] = {c->veff};
            const double* b1[1] = {c->rho_out};
            dots_host(c, 1, a1, b1, nv, &vr);
            const double* A[2] = {exc_o, etmp + ng};
            const double* B[2] = {etmp, phi_o};
            dots_host(c, 2, A, B, ng, d);
            Fks = E.eband - c->dV * vr + c->dV * d[0] + 0.5 * c->dV * d[1] - c->E_self + c->E_sc + E.ts;
        }
        // results to host
        const int ns = c->opt.nstates;
        const size_t ne = c->probs.size() * ns;
        c->eig_host.resize(ne);
        c->occ_host.resize(ne);
        SDFT_CUDA(cudaMemcpyAsync(c->eig_host.data(), c->probs[0].eig, sizeof(double) * ne, cudaMemcpyDeviceToHost,
                                  c->stream));
        SDFT_CUDA(cudaMemcpyAsync(c->occ_host.data(), c->probs[0].occ, sizeof(double) * ne, cudaMemcpyDeviceToHost,
                                  c->stream));
        SDFT_CUDA(cudaStreamSynchronize(c->stream));
        c->mu = E.mu;
        c->ts = E.ts;
        if (!have64)
            for (Problem& P : c->probs) convert_block(c, P.cplx, SDFT_MIXED, P.X, P.X64, c->nfilt);
        forces_compute(c);
        push_scf_history(c);
        resolve_timing(c);
        if (out) {
            out->energy = E.F;
            out->energy_ks = Fks;
            out->mu = E.mu;
            out->entropy_term = E.ts;
            out->niter = niter;
            out->converged = converged ? 1 : 0;
            out->t_total = now_s() - t0;
            out->t_filter = t_filter;
            out->t_rr = t_rr;
            out->t_poisson = t_pois;
            out->t_other = out->t_total - t_filter - t_pois;
        }
        return status;
    }
};

sdft_status run_scf(sdft_ctx* c, sdft_result* out) {
    ScfRun r(c);
    r.begin();
    while (!r.done) {
        r.potential();
        r.filter_all();
        r.end_iteration();
    }
    return r.finish(out);
}

// Several contexts' SCFs in lockstep.  Each iteration: the potentials of every running context,
// then the CheFSI passes, where the cells that the multi-cell filter takes (mixed precision, one
// real Gamma-point problem, one shared stream, the same degree and pass count) are filtered
// together -- one grouped KB projection and one stencil launch per Chebyshev step for all of
// them -- followed by each cell's Rayleigh-Ritz; then every context's density, energy and mixing.
// A context leaves the lockstep when it converges or reaches its max_scf.  The results are
// those of running each context alone with the column-tile stencil.
sdft_status run_batch_scf(const std::vector<sdft_ctx*>& ctxs, sdft_result* out) {
    const int n = (int)ctxs.size();
    std::vector<std::unique_ptr<ScfRun>> runs;
    for (sdft_ctx* c : ctxs) runs.emplace_back(new ScfRun(c));
    for (auto& r : runs) r->begin();
    auto multi_ok = [&](const ScfRun& r) {
        const sdft_ctx* c = r.c;
        return r.prec == SDFT_MIXED && !r.tail64 && c->probs.size() == 1 && !c->probs[0].cplx &&
               c->stream == ctxs[0]->stream;
    };
    for (;;) {
        std::vector<ScfRun*> live;
        for (auto& r : runs)
            if (!r->done) live.push_back(r.get());
        if (live.empty()) break;
        for (ScfRun* r : live) r->potential();
        // cells for the multi-cell filter, grouped by (degree, passes), at most MULTI_MAX per launch
        std::vector<ScfRun*> rest;
        std::vector<std::vector<ScfRun*>> sets;
        for (ScfRun* r : live) {
            if (!multi_ok(*r)) {
                rest.push_back(r);
                continue;
            }
            bool placed = false;
            for (auto& g : sets)
                if (g.size() < (size_t)MULTI_MAX && g[0]->c->opt.cheb_degree == r->c->opt.cheb_degree &&
                    g[0]->passes() == r->passes()) {
                    g.push_back(r);
                    placed = true;
                    break;
                }
            if (!placed) sets.push_back({r});
        }
        for (auto& g : sets) {
            if (g.size() == 1) {
                rest.push_back(g[0]);
                continue;
            }
            const double ta = now_s();
            std::vector<sdft_ctx*> cs;
            std::vector<const void*> xs;
            std::vector<void*> ys;
            for (ScfRun* r : g) {
                cs.push_back(r->c);
                xs.push_back(r->c->probs[0].X);
                ys.push_back(r->c->blk[0]);
            }
            std::vector<double> a(g.size()), b(g.size()), a0(g.size());
            for (int p = 0; p < g[0]->passes(); ++p) {
                for (size_t i = 0; i < g.size(); ++i) {
                    const Problem& P = g[i]->c->probs[0];
                    a[i] = P.cutoff;
                    b[i] = P.upper;
                    a0[i] = P.lower;
                }
                chebyshev_filter_multi(cs, xs, ys, g[0]->c->opt.cheb_degree, a.data(), b.data(), a0.data());
                for (ScfRun* r : g) rr_pass(r->c, r->c->probs[0], SDFT_MIXED, r->c->blk[0], r->c->probs[0].X);
            }
            const double share = (now_s() - ta) / (double)g.size();
            for (ScfRun* r : g) r->t_filter += share;
        }
        for (ScfRun* r : rest) r->filter_all();
        for (ScfRun* r : live) r->end_iteration();
    }
    sdft_status status = SDFT_OK;
    for (int i = 0; i < n; ++i) {
        const sdft_status s = runs[i]->finish(out ? out + i : nullptr);
        if (s != SDFT_OK && status == SDFT_OK) status = s;
    }
    return status;
}

}  // namespace sdft
