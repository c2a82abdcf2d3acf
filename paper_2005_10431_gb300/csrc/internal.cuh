// Internal declarations of the sdft library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <cusolverDn.h>

#include <cstdint>
#include <string>
#include <vector>

#include "sdft.h"

namespace sdft {

constexpr int FD_RADIUS = 6;
constexpr int SCAL_DOUBLES = 16384;
constexpr int MAX_KPT = 256;

// ---------------------------------------------------------------------------------------
// error handling
// ---------------------------------------------------------------------------------------
struct Error {
    sdft_status code;
    std::string msg;
};

#define SDFT_CUDA(call)                                                                     \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess)                                                              \
            throw ::sdft::Error{SDFT_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)}; \
    } while (0)

#define SDFT_REQUIRE(cond, code, text)                                                      \
    do {                                                                                    \
        if (!(cond)) throw ::sdft::Error{(code), (text)};                                   \
    } while (0)

// ---------------------------------------------------------------------------------------
// element types of orbital blocks
// ---------------------------------------------------------------------------------------
// E = float2 : SDFT_MIXED.  Real problems store two orbitals per element ("paired"),
//              complex problems store (re, im) of one orbital.
// E = double : SDFT_FP64 real.      E = double2 : SDFT_FP64 complex.
template <typename E> struct Elem;
template <> struct Elem<float2> { using S = float; static constexpr int lanes = 2; };
template <> struct Elem<double> { using S = double; static constexpr int lanes = 1; };
template <> struct Elem<float> { using S = float; static constexpr int lanes = 1; };  // Poisson FP32 correction
template <> struct Elem<double2> { using S = double; static constexpr int lanes = 2; };

struct StencilCoef {
    // -1/2 w_r / h_d^2 for r = 1..6 per axis; c0 = -1/2 sum_d w_0 / h_d^2
    double cx[FD_RADIUS + 1], cy[FD_RADIUS + 1], cz[FD_RADIUS + 1];
    double c0;
};

// Per-point KB scatter table and per-atom projection lists of one k-point.
struct KBTables {
    int natom = 0;
    int cap = 0;              // entries reserved per atom
    int* cnt = nullptr;       // [natom] support size
    int* idx = nullptr;       // [natom*cap] grid index, ascending (z, y, x box order)
    int* img = nullptr;       // [natom*cap] packed image vector t (3 x 10 bits, biased by 512)
    double* val64 = nullptr;  // [natom*cap] real chi (double)  or [2*natom*cap] complex beta
    float* val32 = nullptr;   // same in float
    int S = 0;                // slots per grid point
    int* pcnt = nullptr;      // [ng]
    int* patom = nullptr;     // [S*ng] atom of slot s at point g, -1 if unused (sorted by atom)
    double* pval64 = nullptr; // [S*ng] (x2 complex)
    float* pval32 = nullptr;
    double* gamma = nullptr;  // [natom] E_kb * dV
    bool cplx = false;
};

// One grid of the multigrid hierarchy that preconditions the FP32 Poisson corrections
// (poisson_mg.cu): dimensions, 1 / h_d^2, and its correction and right-hand side (levels >= 1).
struct MgLevel {
    int n[3] = {0, 0, 0};
    double w[3] = {0, 0, 0};
    long long np = 0;
    float* x = nullptr;
    float* b = nullptr;
};

struct PendingTiming {
    cudaEvent_t a, b;
    int fam;
    double bytes, flops;
};

// one problem of a grouped row-tile stencil launch (same grid, column count and tile for all)
struct RowProblem {
    const float2* Y;
    const float2* Yprev;
    float2* Ynext;
    const float* V;
    const float2* C;
    const int* patom;
    const void* pval;
    int nslot;
    float alpha, beta, shift;
    float phr[3], phi[3];
};
// one problem of a grouped KB projection C = gamma beta^H Y
constexpr int MULTI_MAX = 64;   // cells per multi-cell filter launch

struct KBProblem {
    const void* Y;
    void* C;
    const int* cnt;
    const int* idx;
    const void* val;
    const double* gamma;
    int cap;
    int natom;      // atoms (rows of C per column)
    int ncolE;      // block columns (paired columns in the real FP32 layout)
    long long ng;   // grid points per column
};

struct Problem {              // one (spin, k) eigenproblem
    int spin = 0, kpt = 0;
    bool cplx = false;
    void* X = nullptr;        // current orbitals (FP64 or MIXED storage)
    void* X64 = nullptr;      // FP64 copy used by the final FP64 pass (MIXED)
    double* eig = nullptr;    // [nstates] lowest Ritz values (occupations, energies, results)
    double* eigf = nullptr;   // [nstates + nbuffer] Ritz values of the filtered block (== eig if no buffer)
    double* occ = nullptr;    // [nstates]
    double lower = 0, cutoff = 0, upper = 0;
    bool have_bounds = false;
};

}  // namespace sdft

struct sdft_ctx {
    // geometry and options
    int n[3] = {0, 0, 0};
    double L[3] = {0, 0, 0}, h[3] = {0, 0, 0}, dV = 0;
    long long ng = 0;
    int natom = 0;
    std::vector<double> pos;
    std::vector<int> types;
    std::vector<sdft_pseudo> species;
    sdft_options opt{};
    int nfilt = 0;                // filtered block width: nstates + nbuffer
    bool gemm_fp32 = false;       // Rayleigh-Ritz GEMMs on CUDA cores in FP32 (set by the SCF's precise tail)
    std::vector<double> kpts, kw;
    double nelec = 0;
    sdft::StencilCoef coef{};

    cudaStream_t stream = nullptr;
    sdft_alloc_fn alloc = nullptr;
    sdft_free_fn release = nullptr;
    void* alloc_user = nullptr;
    std::vector<void*> owned;
    cusolverDnHandle_t solver = nullptr;
    syevjInfo_t syevj_params = nullptr;
    int eig_method = -1;          // -1: batched Jacobi for n <= 64, FP32 + FP64 refinement for real mixed-precision
                                  //     n <= 1024, else sygvd/hegvd; 0: sygvd/hegvd; 1: sygvj (real);
                                  //  2: FP32 + refinement wherever it applies, without fallback
    double* reig_buf = nullptr;   // scratch of the refined eigensolver (allocated on first use)
    int reig_nmax = 0;            // the largest n that scratch holds
    float* reig_work32 = nullptr; // cuSOLVER FP32 sygvd workspace (refined solve above n = 160)
    int reig_lwork32 = -1, reig_work32_n = 0;
    int reig_last_status = 0;     // its last status word (0 = accepted)
    int reig_fallbacks = 0;       // refined solves rejected and redone by cuSOLVER
    int reig_accepted = 0;        // refined solves accepted
    // device pointer tables of batched launches (grown on demand) and their host staging copy
    void** ptab_dev = nullptr;
    int* pinfo_dev = nullptr;
    int ptab_cap = 0;
    std::vector<void*> ptab_host;
    uint64_t launches = 0;
    bool timing = false;
    int stencil_choice[4] = {-1, -1, -1, -1};  // autotuned variant per storage kind
    int stencil_last[4] = {-1, -1, -1, -1};    // variant of the last launch per storage kind
    int group_choice[2] = {-1, -1};            // autotuned row variant of grouped launches (real, complex)
    const char* stencil_last_name[4] = {nullptr, nullptr, nullptr, nullptr};
    bool aar_persistent = true;   // FP32 Poisson corrections in one cooperative launch
    bool aar_mg = true;           // FP32 Poisson corrections by multigrid-preconditioned AAR (when the grid coarsens)
    std::vector<sdft::MgLevel> mg;   // multigrid hierarchy (empty: none)
    double mg_lmin = 0.0, mg_lmax = 0.0;   // spectrum bounds of the coarsest grid's operator
    int mg_coarse_iters = 0;              // Chebyshev iterations on the coarsest grid
    cudaGraphExec_t mg_graph = nullptr;   // the V-cycle's launches for (mg_graph_r, mg_graph_z)
    const float* mg_graph_r = nullptr;
    float* mg_graph_z = nullptr;
    int mg_graph_launches = 0;
    bool test_barrier_extra = false;  // test hook: the persistent barrier waits for one CTA too many
    std::vector<cudaEvent_t> ev_free;
    std::vector<sdft::PendingTiming> pending;
    sdft_kernel_stats kstat[SDFT_K_COUNT] = {};

    // grid fields (FP64)
    double* b = nullptr;          // pseudocharge
    double* rho_sad = nullptr;    // SAD density (total)
    double* rho_user = nullptr;   // user guess [nspin][ng]
    double* rho_in = nullptr;     // [nspin][ng]
    double* rho_out = nullptr;    // [nspin][ng]
    double* phi = nullptr;        // electrostatic potential
    double* veff = nullptr;       // [nspin][ng]
    float* veff32 = nullptr;      // [nspin][ng]
    double* exc = nullptr;        // eps_xc
    double* work64 = nullptr;     // [28*ng] grid scratch (Poisson, mixing, energies, Lanczos)
    float* work32 = nullptr;      // [20*ng] FP32 scratch of the mixed-precision Poisson solver
    // small device scalars / reductions [SCAL_DOUBLES], regions:
    //   [0,8) temporaries  [8,16) Fermi (mu, -TS, band energy)  [64,256) Anderson/Pulay small data
    //   [256,512) k-weights  [1024,1040) dot pointer tables  [1536,1544) dot results
    //   [2048,3072) dot partials  [3072,4096) forces  [4096,16384) Anderson Gram partials
    double* scal = nullptr;
    double* hscal = nullptr;      // pinned host mirror [SCAL_DOUBLES]

    std::vector<sdft::KBTables> kb;   // per k-point
    std::vector<sdft::Problem> probs; // [spin*nkpt + k]

    // block scratch (largest storage kind): 3 filter buffers + H Y
    size_t block_bytes = 0;
    void* blk[4] = {nullptr, nullptr, nullptr, nullptr};
    double* Ms = nullptr;         // nstates^2 (x2 complex)
    double* Hs = nullptr;
    double* part = nullptr;       // split-K partials
    size_t part_elems = 0;
    double* dscale = nullptr;     // equilibration
    double* eigtmp = nullptr;
    void* solver_work = nullptr;
    int solver_lwork = 0;
    int* dinfo = nullptr;
    void* Q32 = nullptr;          // rotation matrix in the block precision
    void* Qsplit = nullptr;       // bf16 hi/lo rows of Q^T for the tensor-core rotation
    size_t qsplit_bytes = 0;
    float* C32 = nullptr;         // KB coefficients [ncol * natom] (x2)
    long long c32_elems = 0;      // float2 elements of the C32 allocation (block plus padding)
    float* C32b = nullptr;        // second FP32 KB coefficient buffer (c32_elems float2): fused projections
    float2* kb_next = nullptr;    // set around one FP32 step launch: where a slab step may also write the KB
    bool kb_next_done = false;    //   coefficients of its output (kb_next_done: it did)
    bool fuse_kb_projection = true;   // SDFT_FUSE_KB=0: always the separate projection pass
    bool stencil_fuse = true;         // the autotuner's finding: fused projection (where offered) faster
    double* C64 = nullptr;

    // mixing history
    double* mix_dx = nullptr;     // [hist][nspin*ng]
    double* mix_df = nullptr;
    double* mix_xprev = nullptr;
    double* mix_fprev = nullptr;
    int mix_k = 0, mix_count = 0, mix_head = 0;
    double* kerker_ws = nullptr;  // screened-Poisson AAR workspace of the Kerker preconditioner (first use)
    double* gga_ws = nullptr;     // PBE: density gradient and f_sigma-weighted gradient, 6 ng (first use)
    // atom moves (QMD): the last three SCFs' positions and rho_out - rho_SAD (ring, newest at head - 1)
    double* hist_drho = nullptr;  // [3][nspin * ng] (first use)
    std::vector<double> hist_pos[3];
    int hist_count = 0, hist_head = 0;
    bool warm_start = false;      // the next SCF starts from kept orbitals (one filter pass first)
    double last_alfe[2] = {0.0, 0.0};
    bool user_density = false;
    void* mlp_scratch = nullptr;  // learned guess: features [ng][32] bf16 + output [ng] (allocated on first use)

    // batched CheFSI (allocated on first use): per problem 3 filter blocks, M, Hs, KB coefficients;
    // device step tables of the grouped launches and their host copies
    std::vector<void*> g_blk;
    std::vector<double*> g_M, g_H;
    std::vector<void*> g_C;
    sdft::RowProblem* g_rtab = nullptr;
    sdft::KBProblem* g_ktab = nullptr;
    int g_tab_cap = 0;
    std::vector<sdft::RowProblem> g_rtab_h;
    std::vector<sdft::KBProblem> g_ktab_h;
    // pinned copies of the step tables (sources of the graph's upload) and the captured filter
    sdft::RowProblem* g_rtab_pin = nullptr;
    sdft::KBProblem* g_ktab_pin = nullptr;
    sdft::KBProblem* m_ktab = nullptr;   // multi-cell filter: KB tables of every (step, cell)
    int m_ktab_cap = 0;
    int g_pin_cap = 0;
    cudaGraphExec_t g_graph = nullptr;
    cudaStream_t cap_stream = nullptr;   // private stream for graph capture
    std::vector<long long> g_graph_key;
    int g_graph_launches = 0;

    // results
    std::vector<sdft_iter_record> log;
    std::vector<double> forces;
    std::vector<double> eig_host, occ_host;
    double mu = 0, ts = 0;
    double E_self = 0, E_sc = 0;
    std::vector<double> dEsc;     // natom*3

    std::string last_error;
};

namespace sdft {

// allocation through the context's callbacks
void* ctx_alloc(sdft_ctx* c, size_t bytes);
// release one allocation made by ctx_alloc (stream-ordered through the callbacks, else cudaFree)
void ctx_release(sdft_ctx* c, void* p);
void ctx_free_all(sdft_ctx* c);
inline void count_launch(sdft_ctx* c, int n = 1) { c->launches += n; }
inline size_t block_elems_bytes(const sdft_ctx* c, int precision, bool cplx, int ncol) {
    // bytes of an ngrid x ncol block in the storage kind of (precision, cplx)
    size_t per = precision == SDFT_FP64 ? (cplx ? 16 : 8) : (cplx ? 8 : 4);
    return per * (size_t)c->ng * (size_t)ncol;
}

// CUDA-event timing of one kernel family over the scope (no-op unless c->timing)
struct ScopedTimer {
    sdft_ctx* c;
    int fam;
    double bytes, flops;
    cudaEvent_t a = nullptr, b = nullptr;
    ScopedTimer(sdft_ctx* c_, int fam_, double bytes_ = 0, double flops_ = 0);  // c_ null: no-op
    ~ScopedTimer();
};
// accumulate finished event pairs into c->kstat (synchronises the stream)
void resolve_timing(sdft_ctx* c);

// ---- stencil.cu ----------------------------------------------------------------------
// Ynext = alpha*(H Y - c Y) - beta*Yprev  for `ncolE` element-columns (see Elem).
// Yprev may be null (beta ignored).  V null: no local potential.  kbC null: no KB term.
// kb must hold the per-point table of this k-point; kbC is [ncolE][natom] elements of the
// (gamma-scaled) projection coefficients of Y.
template <typename E>
void launch_cheb_step(sdft_ctx* c, int kpt, const E* Y, const E* Yprev, E* Ynext, int ncolE,
                      const typename Elem<E>::S* V, const E* kbC, double alpha, double beta,
                      double shift, bool with_kinetic = true);
template <>
void launch_cheb_step<float>(sdft_ctx* c, int kpt, const float* Y, const float* Yprev, float* Ynext, int ncolE,
                             const float* V, const float* kbC, double alpha, double beta, double shift,
                             bool with_kinetic);
// KB projection C[col][a] = gamma_a * sum_j conj(beta_a(j)) Y[j, col]
template <typename E>
void launch_kb_project(sdft_ctx* c, int kpt, const E* Y, E* C, int ncolE);

// ---- stencil_tma.cu: TMA-fed slab tile (FP32 real paired blocks) -----------------------
template <int N1, int TY, int NP, int S, int D>
bool slab_variant_ok(const sdft_ctx* c, int ncolE);
template <int N1, int TY, int NP, int RY, int S, int D, int MINB>
void launch_slab_variant(sdft_ctx* c, int kpt, const float2* Y, const float2* Yprev, float2* Ynext, int ncolE,
                         const float* V, const float2* kbC, double alpha, double beta, double shift, bool kin,
                         bool timed);
// sticky device flag (int) set by a stencil launch whose bounded mbarrier wait gave up
int* stencil_error_flag(sdft_ctx* c);
// throws SDFT_ERR_DEVICE_TIMEOUT if that flag is set (reads it after the stream's work so far)
void check_stencil_flag(sdft_ctx* c);

// ---- kb.cu ---------------------------------------------------------------------------
void build_kb_tables(sdft_ctx* c, int kpt);
void release_kb_tables(sdft_ctx* c, int kpt);

// ---- qmd.cu: atom moves and the extrapolated start of the next SCF ----------------------
void push_scf_history(sdft_ctx* c);
void move_atoms(sdft_ctx* c, const double* pos, int guess);
void host_energy_constants(sdft_ctx* c);

// ---- gridops.cu ----------------------------------------------------------------------
void build_pseudocharge_and_sad(sdft_ctx* c);
void lda_device(sdft_ctx* c, int nspin, const double* rho, double* exc, double* vxc, size_t n);
void veff_assemble(sdft_ctx* c);
void veff_to_float(sdft_ctx* c, int spin);
void axpby_dev(sdft_ctx* c, double* y, const double* x, double a, double b, long long n);
int poisson_aar(sdft_ctx* c, const double* f, double* phi, double tol, int max_iter);
// same problem, FP64 residuals + FP32 AAR corrections; returns inner iterations (negative: failed)
int poisson_mixed(sdft_ctx* c, const double* f, double* phi, double tol, int max_iter);
// multigrid preconditioner of the FP32 Poisson corrections (poisson_mg.cu): build the hierarchy
// (false: the grid does not coarsen far enough), and z = M r by one V-cycle
bool mg_setup(sdft_ctx* c);
void mg_vcycle(sdft_ctx* c, const float* r, float* z);
// reductions: out[i] = sum_g a_i[g] * b_i[g] (device scal), returned synchronously to host
void dots_host(sdft_ctx* c, int count, const double* const* a, const double* const* b, long long n,
               double* host_out);
void fermi_device(sdft_ctx* c, const double* eig, double* occ, double* mu_ts_dev);
void density_accumulate(sdft_ctx* c, int precision, bool cplx, const void* X, const double* occ,
                        int ncol, double weight, double* rho);
void pulay_update(sdft_ctx* c);
// Kerker preconditioner out = (-L)(-L + k0^2)^-1 f of one grid vector by a screened AAR solve to relative
// residual tol; returns the iteration count (negative: not converged)
int kerker_apply(sdft_ctx* c, const double* f, double* out, double k0, double tol, int max_iter);
void forces_compute(sdft_ctx* c);

// ---- dense.cu ------------------------------------------------------------------------
// M = Y^H Y, Hs = Y^H HY (FP64 results, column-major ncol x ncol, x2 for complex)
void subspace_gram(sdft_ctx* c, int precision, bool cplx, const void* Y, const void* HY,
                   double* M, double* Hs, int ncol);
// tcgen05 BF16x3 path of subspace_gram for FP32 real blocks (gemm_tc.cu)
bool gram_tc_supported(const sdft_ctx* c, int precision, bool cplx, int ncol);
void subspace_gram_tc(sdft_ctx* c, const void* Y, const void* HY, double* M, double* Hs, int ncol);
bool rotate_tc_supported(const sdft_ctx* c, int precision, bool cplx, int ncol);
size_t qsplit_bytes(int ncol);
void rotate_tc(sdft_ctx* c, const void* Y, const double* Q, void* X, int ncol);
// allocation-free variant: partials in a fixed file-scope device array (no context needed)
void subspace_gram_noalloc(int precision, bool cplx, const void* Y, const void* HY, long long ng, int ncol,
                           double* M, double* Hs, cudaStream_t stream);
// solve Hs q = lambda M q (FP64); Q overwrites Hs; eig ascending; throws CHOLESKY on failure
void generalized_eig(sdft_ctx* c, bool cplx, double* M, double* Hs, double* eig, int ncol);
bool refined_eig_supported(int n);
bool refined_generalized_eig(sdft_ctx* c, const double* M, const double* Hs, double* Q, double* eig, int n);
// X = Y Q (Q FP64 column-major)
void rotate_block(sdft_ctx* c, int precision, bool cplx, const void* Y, const double* Q, void* X,
                  int ncol);
void convert_block(sdft_ctx* c, bool cplx, int from_precision, const void* src, void* dst, int ncol);

// ---- scf.cu --------------------------------------------------------------------------
void chebyshev_filter(sdft_ctx* c, int kpt, int precision, const void* X, void* Y, int ncol,
                      int degree, double a, double b, double a0, const double* veff64,
                      const float* veff32);
void apply_h(sdft_ctx* c, int kpt, int precision, const void* X, void* Y, int ncol,
             const double* veff64, const float* veff32);
void rayleigh_ritz(sdft_ctx* c, int kpt, int precision, const void* Y, void* X, double* eig,
                   int ncol, const double* veff64, const float* veff32);
void lanczos(sdft_ctx* c, int spin, int kpt, int steps, double* lower, double* upper);
sdft_status run_scf(sdft_ctx* c, sdft_result* out);
sdft_status run_batch_scf(const std::vector<sdft_ctx*>& ctxs, sdft_result* out);
void reset_state(sdft_ctx* c);
void seed_orbitals(sdft_ctx* c, int precision, bool cplx, void* X, int ncol, uint64_t seed);

// grouped FP32 stencil / KB projection over problems sharing the grid (stencil_f32.cu);
// grp: device tables.  group_variant_f32 returns -1 when no row tile fits the grid.
int group_variant_f32(sdft_ctx* c, bool cplx, int ncolE);
void launch_group_step_f32(sdft_ctx* c, bool cplx, int variant, const RowProblem* grp, int nprob, int ncolE,
                           bool prev, bool haskb);
void launch_group_project_f32(sdft_ctx* c, bool cplx, const KBProblem* grp, int nprob, int ncolE);
void launch_multi_project_f32(sdft_ctx* c, const KBProblem* grp, int nprob, int max_natom, int max_ncolE);
int autotune_group_f32(sdft_ctx* c, bool cplx, const RowProblem* grp, int nprob, int ncolE, bool haskb);
// Chebyshev filter of the FP32 real blocks of several cells (contexts with their own grids) with
// one column-tile stencil launch per step (scf.cu; kernels in stencil_f32.cu)
void chebyshev_filter_multi(const std::vector<sdft_ctx*>& ctxs, const std::vector<const void*>& X,
                            const std::vector<void*>& Y, int degree, const double* a, const double* b,
                            const double* a0);

// ---- batched.cu ----------------------------------------------------------------------
bool batched_eig_supported(int n);
// Ms/Hss/eigs: device arrays of `count` device pointers; info: device int[count]
void batched_generalized_eig(sdft_ctx* c, bool cplx, double* const* Ms, double* const* Hss, double* const* eigs,
                             int n, int count, int* info);
// device pointer table with room for `count` entries of `width` pointers (+ count ints of info)
void ensure_ptab(sdft_ctx* c, int count, int width);

// ---- mlp.cu --------------------------------------------------------------------------
int mlp_nparam();
void mlp_dataset(sdft_ctx* c, void* feat, float* target);
void mlp_loss_grad(const void* feat, const float* target, long long npts, long long batch, long long start,
                   const float* params, float* grad, double* loss, cudaStream_t st);
void mlp_forward(const void* feat, long long npts, const float* params, float* y, cudaStream_t st);
void mlp_adam(float* p, const float* g, float* m, float* v, int step, double lr, cudaStream_t st);
void mlp_train(const void* feat, const float* target, long long npts, long long batch, float* params, float* grad,
               float* m, float* v, int first_step, int nsteps, double lr, double* loss_dev, cudaStream_t st);
void mlp_guess(sdft_ctx* c, const float* params);

}  // namespace sdft
