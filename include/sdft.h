/*
 * sdft.h -- C ABI of a single-GPU (GB300, sm_103a) real-space Kohn-Sham DFT solver:
 * Chebyshev-filtered subspace iteration (CheFSI) inside the SCF loop, after the SPARC
 * method (Xu et al., arXiv 2005.10431).
 *
 * Problem statement (paper Sec. 2, Eq. 1 and Eq. 2): for each spin s and k-point,
 *     ( -1/2 Laplacian + V_eff^s[rho_up, rho_dn; R] ) psi_n = lambda_n psi_n,
 *     rho^s(x) = sum_n g_n |psi_n(x)|^2,  g_n Fermi-Dirac,
 * discretised on a uniform periodic grid with a 12th-order centred finite-difference
 * Laplacian, a Gaussian-pseudocharge local pseudopotential with the Poisson problem for the
 * electrostatic potential, and Kleinman-Bylander nonlocal projectors (paper Sec. 2.1).
 *
 * Conventions (all entry points):
 *  - Atomic units (bohr, hartree).  Grid point (i,j,k) is at (i h1, j h2, k h3), h_d = L_d/n_d,
 *    flat index g = i + n1 (j + n2 k).  dV = h1 h2 h3.
 *  - Every function returns sdft_status: 0 on success, a negative SDFT_ERR_* code otherwise.
 *    On error nothing is written to caller buffers unless stated; sdft_last_error() gives a
 *    message (owned by the library, valid until the next call on that context/thread).
 *  - Input arrays are owned by the caller and copied (host) or read (device) during the call.
 *    Device buffers allocated by the library belong to the context and are released by
 *    sdft_destroy().  The library never calls exit().
 *  - "device" pointers are CUDA device addresses on the context's device; kernels run on the
 *    stream given to sdft_create (NULL = legacy default stream).  Calls taking device output
 *    pointers are asynchronous w.r.t. the host unless stated; calls writing host memory
 *    synchronise the stream first.
 *  - Orbital blocks on the device ("blocks") come in three storage kinds, selected by the
 *    precision and the k-point:
 *      SDFT_FP64, real (Gamma)   : double,  column-major ngrid x ncol  (column n at n*ngrid)
 *      SDFT_FP64, complex (k!=0) : double2 (re,im), column-major ngrid x ncol
 *      SDFT_MIXED, real (Gamma)  : float, "paired" layout: columns 2p and 2p+1 interleaved,
 *                                  element (g, n) at ((n/2)*ngrid + g)*2 + (n%2); ncol even
 *      SDFT_MIXED, complex       : float2 (re,im), column-major ngrid x ncol
 *    Euclidean normalisation: the continuum orbital is X / sqrt(dV).
 */
#ifndef SDFT_H
#define SDFT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int sdft_status;

#define SDFT_OK 0
#define SDFT_ERR_INVALID_ARG (-1)   /* bad size, pointer, option, short output buffer */
#define SDFT_ERR_OOM (-2)           /* allocation callback or cudaMalloc failed */
#define SDFT_ERR_CUDA (-3)          /* a CUDA runtime / cuSOLVER call failed */
#define SDFT_ERR_NOT_CONVERGED (-4) /* SCF or Poisson did not reach its tolerance */
#define SDFT_ERR_CHOLESKY (-5)      /* subspace overlap matrix not positive definite */
#define SDFT_ERR_DEVICE_TIMEOUT (-6)/* a bounded device-side wait gave up */
#define SDFT_ERR_NONFINITE (-7)     /* NaN/Inf in an input or produced by the iteration */

enum { SDFT_FP64 = 0, SDFT_MIXED = 1 };
enum { SDFT_GUESS_SAD = 0, SDFT_GUESS_USER = 1 };
enum { SDFT_XC_LDA_PZ = 0, SDFT_XC_GGA_PBE = 1 };
enum { SDFT_BC_PERIODIC = 0, SDFT_BC_DIRICHLET = 1 };

typedef struct sdft_ctx sdft_ctx;

/* Periodic orthorhombic cell (paper Sec. 2: Bloch-periodic BCs on orbitals, periodic on phi). */
typedef struct {
    double L[3];          /* edge lengths, bohr, > 0 */
} sdft_cell;

/* Uniform grid (paper Sec. 2.1).  fd_order must be 12 (radius 6). Each n[d] >= 6. */
typedef struct {
    int n[3];
    int fd_order;
} sdft_grid;

/* Atoms: natom >= 1 positions (bohr, natom*3, x y z per atom) and species index per atom. */
typedef struct {
    int natom;
    const double* pos;
    const int* type;
} sdft_atoms;

/* Synthetic pseudo-atom (stands in for the paper's psp8 pseudopotentials, Sec. 2.2):
 * pseudocharge b(r) = -Z (2 pi r_loc^2)^(-3/2) exp(-r^2/(2 r_loc^2)), r <= 10 r_loc;
 * KB projector chi(r) = (pi^(3/2) r_proj^3)^(-1/2) exp(-r^2/(2 r_proj^2)), r < r_cut_proj,
 * V_nl = sum_a E_kb |beta_a><beta_a|; SAD density Z (2 pi s^2)^(-3/2) exp(-r^2/(2 s^2)),
 * r <= 10 s, s = sad_width. */
typedef struct {
    double Z, r_loc, r_proj, E_kb, r_cut_proj, sad_width;
} sdft_pseudo;

typedef struct {
    int nspin;                 /* 1 (unpolarized, occupation factor 2) or 2 */
    int nkpt;                  /* >= 1 */
    const double* kpts;        /* nkpt*3 reduced coordinates (k.L/(2 pi)); NULL = Gamma */
    const double* kw;          /* nkpt weights, sum 1; NULL = uniform */
    int nstates;               /* orbitals per (spin, k) problem; even for SDFT_MIXED */
    int cheb_degree;           /* Chebyshev filter degree m >= 1 */
    int first_scf_filter_passes; /* CheFSI passes in the first SCF iteration (paper Sec. 2.1) */
    int lanczos_steps;         /* Lanczos steps for the spectrum bounds */
    double kT;                 /* Fermi-Dirac smearing, Ha */
    int mix_hist;              /* Pulay history length (<= 16) */
    double mix_beta;           /* mixing parameter */
    int pulay_period;          /* Pulay extrapolation every pulay_period-th iteration */
    int pulay_restart;         /* 1: clear the history after each Pulay step */
    double scf_tol;            /* ||rho_out - rho_in|| / ||rho_out|| */
    int max_scf;
    int precision;             /* SDFT_FP64 or SDFT_MIXED */
    int final_fp64_pass;       /* MIXED: one FP64 filter + Rayleigh-Ritz pass after the SCF */
    double poisson_tol;        /* relative residual of the AAR Poisson solve */
    int init_guess;            /* SDFT_GUESS_SAD or SDFT_GUESS_USER (see sdft_set_density) */
    double initial_moment;     /* nspin=2: SAD split rho (1 +- m)/2 */
    uint64_t seed;             /* counter-based generator seed for the initial orbitals */
    int batch_problems;        /* 1: SDFT_MIXED runs the CheFSI passes of all (spin, k) problems of one
                                  storage kind together (grouped stencil / KB launches, batched
                                  eigensolve); 0: one problem after another */
    int use_graphs;            /* 1: the grouped filter of a batched pass (table upload, m KB projections
                                  and stencil steps, and the H Y of Rayleigh-Ritz) is captured once as a
                                  CUDA graph and replayed every pass (not while kernel timing is on) */
    double kerker_k0;          /* > 0: Kerker-preconditioned Pulay mixing (paper Sec. 2.1, preconditioned
                                  periodic Pulay) with screening wavevector k0 (1/bohr): the linear part of
                                  every update is P(beta r), P = (-L_h)(-L_h + k0^2)^-1 applied channel by
                                  channel through a screened-Poisson AAR solve; 0: plain Pulay */
    int xc;                    /* exchange-correlation: SDFT_XC_LDA_PZ (Perdew-Zunger LDA, paper Sec. 3) or
                                  SDFT_XC_GGA_PBE (PBE GGA, paper Sec. 2.2; nspin = 1 only) */
    int boundary;              /* SDFT_BC_PERIODIC, or SDFT_BC_DIRICHLET for an isolated system (paper Sec. 2,
                                  2.1): orbitals zero outside the grid, no periodic images of the atoms, and the
                                  electrostatic potential in the 6 ghost layers beyond each face given by the
                                  multipole expansion (l <= 6, about the centre of the grid box) of rho + b.
                                  Gamma point and SDFT_FP64 only */
    int nbuffer;               /* >= 0 extra orbitals per problem that are filtered and enter Rayleigh-Ritz
                                  but are never occupied (occupations, density, energy and forces use the
                                  lowest nstates).  The filter cutoff then sits at the top Ritz value of the
                                  wider block, away from the partially occupied states at the top of the
                                  nstates block, which the Chebyshev filter otherwise barely separates
                                  (CheFSI buffer states; the fixed point is unchanged).  nstates + nbuffer
                                  is even for SDFT_MIXED.  sdft_set/get_orbitals move the lowest nstates;
                                  the step-level calls accept blocks of up to nstates + nbuffer columns */
    double fp64_switch_tol;    /* SDFT_MIXED, > 0: once the SCF error falls below this, the remaining SCF
                                  iterations run FP64 CheFSI passes on FP64 copies of the orbitals (with FP32
                                  orbitals the density residual of the mixed path levels off near 1e-6), and
                                  the final FP64 pass is not needed; 0: the whole SCF in mixed precision */
    double gemm_fp32_switch_tol; /* SDFT_MIXED, > 0: once the SCF error falls below this, the Rayleigh-Ritz
                                  GEMMs (Gram, rotation) change from BF16x3 tensor-core products (about 17
                                  significant bits, which hold the mixed density residual near 1e-6) to FP32
                                  CUDA-core products for the rest of the SCF; 0: tensor cores throughout */
} sdft_options;

/* Per-iteration record of the SCF (paper Sec. 2.1 ".out" progress). */
typedef struct {
    int iter;
    double energy;     /* Harris-Foulkes free energy at rho_in, Ha */
    double scf_error;  /* ||rho_out - rho_in|| / ||rho_out|| */
    double mu;         /* Fermi level */
    double seconds;    /* device time (CUDA events) from the start of sdft_scf to the end of this iteration */
    double lower, cutoff, upper; /* filter bounds a0, a, b of the first problem */
    int poisson_iters;  /* AAR iterations of this iteration's Poisson solve (FP32 correction
                           iterations summed over the refinement rounds on the mixed path) */
    double poisson_tol; /* the relative residual that solve was asked for */
} sdft_iter_record;

typedef struct {
    double energy;        /* free energy (Harris-Foulkes form), Ha */
    double energy_ks;     /* Kohn-Sham form at the output density, Ha */
    double mu;
    double entropy_term;  /* -TS */
    int niter;
    int converged;
    double t_total, t_filter, t_rr, t_poisson, t_other;  /* seconds */
} sdft_result;

typedef void* (*sdft_alloc_fn)(size_t bytes, void* user);
typedef void (*sdft_free_fn)(void* ptr, void* user);

/* Fill *opt with the defaults: nspin 1, Gamma, nstates 8, degree 12, 4 first-step passes,
 * 20 Lanczos steps, kT 0.01, Pulay hist 7 / beta 0.3 / period 1 / no restart, scf_tol 1e-6,
 * max_scf 100, FP64, no final pass, poisson_tol 1e-10, SAD, moment 0.125, seed 0. */
void sdft_default_options(sdft_options* opt);

/* Create a context: copies all inputs, builds the pseudocharge, projector tables and the SAD
 * density on the device (paper Sec. 2.1 set-up).  alloc/free may be NULL (cudaMalloc/cudaFree);
 * memory from alloc must be 256-byte aligned (the TMA copies need 16-byte aligned bases), else
 * the allocation is handed back to free and the call fails with INVALID_ARG.
 * stream is a cudaStream_t (NULL = default stream).  Errors: INVALID_ARG (sizes, nonfinite
 * positions -> NONFINITE, misaligned allocations), OOM, CUDA. */
sdft_status sdft_create(const sdft_cell* cell, const sdft_grid* grid, const sdft_atoms* atoms,
                        int ntypes, const sdft_pseudo* pseudo, const sdft_options* opt,
                        sdft_alloc_fn alloc, sdft_free_fn free_fn, void* alloc_user,
                        void* cuda_stream, sdft_ctx** out);
void sdft_destroy(sdft_ctx* ctx);
/* Message of the last error on ctx; with ctx NULL, of the last failed sdft_create or
 * context-free call on this thread. */
const char* sdft_last_error(const sdft_ctx* ctx);

/* ---- full SCF (paper Sec. 2.1) ------------------------------------------------------ */

/* Run the SCF from the current guess (SAD, or the density given by sdft_set_density) and the
 * current orbitals (seeded, or given by sdft_set_orbitals).  Returns NOT_CONVERGED with the
 * partial result filled in if max_scf is reached, CHOLESKY if the overlap matrix breaks down. */
sdft_status sdft_scf(sdft_ctx* ctx, sdft_result* out);

/* The SCFs of n distinct contexts in lockstep (paper Sec. 2.1's SCF, batched over independent
 * cells; the paper runs such problems in separate groups of processes).  Per iteration every
 * running context computes its potential, then the CheFSI passes: cells in mixed precision with
 * one real Gamma-point problem, sharing one stream, with equal degree and pass count are filtered
 * together (sdft_chebyshev_filter_multi: one KB projection and one stencil launch per Chebyshev
 * step for all of them, column-tile stencil), each followed by its own Rayleigh-Ritz; other
 * contexts run their passes alone.  A context stops at its own convergence or max_scf.
 * out: host array of n results, filled for every context.  Returns the first non-OK status in
 * context order (NOT_CONVERGED if a context did not converge); an error inside any context
 * aborts the batch and is reported on ctxs[0] (and copied to the others' sdft_last_error).  Two
 * batches must not run at the same time (see the shared table of sdft_chebyshev_filter_multi). */
sdft_status sdft_batch_scf(sdft_ctx* const* ctxs, int n, sdft_result* out);
/* Re-seed the initial orbitals of every problem from opt.seed (as at create) and reset the
 * density guess to the SAD (or last user) density, so that sdft_scf can be repeated. */
sdft_status sdft_reset(sdft_ctx* ctx);

/* Move the atoms (pos: natom*3 bohr, host; same species and count) and prepare the next sdft_scf (paper
 * Sec. 2.1: in quantum molecular dynamics the density guess of later steps is extrapolated from earlier
 * ones, after D. Alfe, Comput. Phys. Commun. 118 (1999) 31).  The pseudocharge, SAD density, KB tables
 * and overlap energies are rebuilt for the new positions and the mixing history is cleared.
 *   guess = 0: start from the SAD density and seeded orbitals, as a new context would.
 *   guess = 1: start from the extrapolated density
 *       rho = rho_SAD(R) + (1 + alpha) D_0 + (beta - alpha) D_1 - beta D_2,
 *     D_i = rho_out - rho_SAD(R_i) of this context's i-th most recent SCF (positions R_i), where alpha,
 *     beta fit R - R_0 ~ alpha (R_0 - R_1) + beta (R_1 - R_2) in the least-squares sense (minimum-image
 *     differences; with two past SCFs beta = 0, with one alpha = beta = 0, with none guess 0 is used),
 *     clamped at 0 and renormalised to N_e; the orbitals and filter bounds of the last SCF are kept
 *     (the upper bound refreshed by Lanczos) and the first SCF iteration filters once.
 * coef (host, 2 doubles, may be NULL) receives alpha, beta.  Synchronises the stream. */
sdft_status sdft_move_atoms(sdft_ctx* ctx, const double* pos, int guess, double* coef);
/* The density the next sdft_scf starts from, [spin][ngrid] (host or device). */
sdft_status sdft_get_input_density(sdft_ctx* ctx, double* dst, size_t n, int on_device);

/* Eigenvalues [spin][k][state], n >= nspin*nkpt*nstates. Host. */
sdft_status sdft_get_eigenvalues(sdft_ctx* ctx, double* host, size_t n);
/* Occupations g (same layout), host. */
sdft_status sdft_get_occupations(sdft_ctx* ctx, double* host, size_t n);
/* Output density of the last SCF iteration, [spin][ngrid]; dst on host or device. */
sdft_status sdft_get_density(sdft_ctx* ctx, double* dst, size_t n, int on_device);
/* Set the input density guess [spin][ngrid] (used when init_guess = SDFT_GUESS_USER). */
sdft_status sdft_set_density(sdft_ctx* ctx, const double* src, size_t n, int on_device);
/* Hellmann-Feynman forces after sdft_scf, natom*3, Ha/bohr, host. */
sdft_status sdft_get_forces(sdft_ctx* ctx, double* host, size_t n);
/* Per-iteration records of the last sdft_scf; *count receives the number available. */
sdft_status sdft_get_scf_log(sdft_ctx* ctx, sdft_iter_record* host, size_t cap, size_t* count);
/* Pseudocharge b [ngrid] and SAD density [ngrid] as built at create (host or device). */
sdft_status sdft_get_pseudocharge(sdft_ctx* ctx, double* dst, size_t n, int on_device);
sdft_status sdft_get_sad_density(sdft_ctx* ctx, double* dst, size_t n, int on_device);
/* Orbitals of problem (spin, k) in the storage kind of `precision` (see header notes):
 * copy from/to a caller device buffer of the block's size. */
sdft_status sdft_set_orbitals(sdft_ctx* ctx, int spin, int kpt, const void* dev, size_t bytes);
sdft_status sdft_get_orbitals(sdft_ctx* ctx, int spin, int kpt, void* dev, size_t bytes);

/* ---- hot-path steps, exposed one by one (paper Sec. 2.1 CheFSI) ---------------------- */

/* Set V_eff^spin [ngrid] (FP64, host or device); the FP32 copy used by SDFT_MIXED is updated. */
sdft_status sdft_set_veff(sdft_ctx* ctx, int spin, const double* v, int on_device);

/* Y = H X for ncol columns of problem (spin, kpt) in `precision` (device blocks; paper Eq. 1,
 * matrix-free: 12th-order FD stencil + V_eff + KB projectors). */
sdft_status sdft_apply_h(sdft_ctx* ctx, int spin, int kpt, int precision,
                         const void* x, void* y, int ncol);

/* Degree-m scaled Chebyshev filter (Zhou-Saad): Y = p_m(H) X with the interval [a, b] mapped
 * to [-1, 1] and p_m(a0) = 1.  x is not modified; y receives the result (device blocks). */
sdft_status sdft_chebyshev_filter(sdft_ctx* ctx, int spin, int kpt, int precision,
                                  const void* x, void* y, int ncol, int degree,
                                  double a, double b, double a0);

/* Rayleigh-Ritz on the block y (device): M = Y^H Y, Hs = Y^H H Y, Hs q = lambda M q,
 * x = Y Q.  eig receives ncol eigenvalues ascending (device, FP64). */
sdft_status sdft_rayleigh_ritz(sdft_ctx* ctx, int spin, int kpt, int precision,
                               const void* y, void* x, double* eig, int ncol);

/* Chebyshev filter of several independent cells at once (the paper's filter, Sec. 2.1, applied to
 * n cells of different grids and sizes): cell i is the context ctxs[i] (SDFT_MIXED, Gamma point,
 * spin 0 V_eff as set for it), x[i] -> y[i] its FP32 paired block of nstates columns (device),
 * degree m with the cell's own bounds a0[i] < a[i] < b[i] (host arrays).  Each Chebyshev step is
 * ONE column-tile stencil launch over all cells (per-cell grid, coefficients and recurrence scalars
 * in a constant-memory table) after the cells' KB projections; every cell computes exactly what
 * sdft_chebyshev_filter computes for it with the column tile.  1 <= n <= 64; all contexts must use
 * the same CUDA stream.  Returns after the work is enqueued and completed (synchronises).  The
 * per-cell table is ONE constant-memory array of the library, rewritten before every step: two
 * multi-cell filters (this call or sdft_batch_scf) running at the same time on different streams or
 * host threads overwrite each other's table and give wrong results; serialise them. */
sdft_status sdft_chebyshev_filter_multi(sdft_ctx* const* ctxs, int n, const void* const* x, void* const* y,
                                        int degree, const double* a, const double* b, const double* a0);

/* Subspace matrices only: M = Y^H Y and Hs = Y^H (H Y) as FP64 ncol x ncol (device,
 * column-major; complex problems write double2).  hy is the device block H Y. */
sdft_status sdft_subspace_matrices(sdft_ctx* ctx, int kpt, int precision, const void* y,
                                   const void* hy, void* m, void* hs, int ncol);

/* Allocation-free variant of sdft_subspace_matrices, for callers that must not allocate device
 * memory: code that runs while a CUDA graph is being captured in global mode (cudaMalloc fails
 * then), hosts whose device memory is owned by their own pool allocator, and latency-critical
 * loops where an allocation (which can synchronise the device) is not acceptable.  The paper has
 * no counterpart; this is an interface convenience of this library.
 *
 * Computes the same M = Y^H Y and Hs = Y^H (H Y) (FP64 ncol x ncol, column-major, double2 for
 * complex) from device blocks y, hy of ngrid x ncol in the storage kind of (precision,
 * is_complex), enqueued on cuda_stream (a cudaStream_t, NULL = default stream); no context is
 * needed and nothing is allocated.  It always runs the CUDA-core Gram of the storage kind, so for
 * real SDFT_MIXED blocks with ncol >= 32 (where sdft_subspace_matrices runs the BF16x3 tensor-core
 * Gram) the two agree to FP32 tolerance, not bit for bit.  The split-K partial sums use a fixed
 * 32 MiB device array inside the library, so 2*ncol^2*(2 if complex) must not exceed 4194304
 * doubles (ncol <= 1448 real, <= 1024 complex); larger ncol returns SDFT_ERR_INVALID_ARG before
 * anything is launched.  The first call on each device looks up that array's device address
 * (cudaGetSymbolAddress) with the device current; make it before any stream capture.  All calls
 * share the one array per device and it keeps the last call's contents (every partial sum a call
 * reads is written by that call first): calls whose kernels overlap on the GPU (other streams,
 * other host threads) race and give wrong results.  Asynchronous; errors are reported by
 * sdft_last_error(NULL). */
sdft_status sdft_subspace_matrices_noalloc(int precision, int is_complex, const void* y, const void* hy,
                                           int64_t ngrid, int ncol, double* m, double* hs,
                                           void* cuda_stream);

/* Generalized Hermitian eigensolve of Rayleigh-Ritz (paper Sec. 2.1): Hs q = lambda M q, FP64,
 * column-major ncol x ncol device matrices (double2 for is_complex).  M must be positive definite.
 * On return Hs holds Q (Q^H M Q = I, eigenvector j in column j), eig (device, ncol) ascending; M is
 * overwritten (scratch).  ncol <= 64 uses the library's one-CTA Cholesky + Jacobi solver (unless
 * SDFT_EIGEN=0 selects cuSOLVER); a real problem with 64 < ncol <= 1024 on an SDFT_MIXED context
 * uses an FP32 solve (one CTA up to 160, cuSOLVER's FP32 sygvd above) refined to FP64 accuracy
 * (Ogita-Aishima steps + Rayleigh-Ritz inside clusters of near-degenerate eigenvalues), accepted
 * only if its FP64 residual and M-orthonormality
 * defect are below 1e-10 relative, else redone by cuSOLVER (SDFT_EIGEN=2 forces it on any context
 * and reports a rejection as an error instead); otherwise cuSOLVER sygvd/hegvd.  All after diagonal
 * equilibration.  SDFT_ERR_CHOLESKY if M is not positive definite. */
sdft_status sdft_subspace_eig(sdft_ctx* ctx, int is_complex, double* m, double* hs, double* eig, int ncol);

/* Rotation x = y Q for an FP64 ncol x ncol column-major Q (double2 for complex), device. */
sdft_status sdft_rotate(sdft_ctx* ctx, int kpt, int precision, const void* y, const void* q,
                        void* x, int ncol);

/* Poisson: -L phi = 4 pi (f - mean f), zero-mean phi, by AAR (paper Sec. 2.1; Pratapa,
 * Suryanarayana & Pask 2016).  For SDFT_BC_DIRICHLET contexts: -L phi = 4 pi f inside the grid with the
 * multipole boundary values of f in the ghost layers (no mean removal, phi -> 0 far away).  f, phi: device FP64 [ngrid]; phi is also the initial guess.
 * tol bounds the FP64 relative residual.  FP64 contexts iterate in FP64; SDFT_MIXED contexts use
 * FP64 residuals with FP32 AAR correction solves (iterative refinement), same tolerance.
 * *iters receives the (inner) iteration count.  NOT_CONVERGED if the tolerance is not reached. */
sdft_status sdft_poisson(sdft_ctx* ctx, const double* f, double* phi, double tol, int max_iter,
                         int* iters);

/* Exchange-correlation of the context's functional (opt.xc): rho [nspin][n] -> eps_xc [n] (per electron),
 * v_xc [nspin][n]; device FP64.  LDA: Perdew-Zunger (paper Sec. 3), pointwise.  GGA: PBE (paper Sec. 2.2),
 * nspin = 1 and n = ngrid: the gradient is the order-12 centred first-derivative stencil of the grid
 * (periodic), sigma = |D rho|^2, and v_xc = f_rho - 2 sum_d D_d (f_sigma D_d rho) is the exact derivative of
 * the discrete energy E_xc = dV sum rho eps_xc.  The density is floored at 1e-14 inside. */
sdft_status sdft_lda(sdft_ctx* ctx, int nspin, const double* rho, double* exc, double* vxc,
                     size_t n);

/* Kerker preconditioner of the density mixing (paper Sec. 2.1): out = P f = f - k0^2 y with
 * (-L_h + k0^2) y = f solved by AAR (FP64, Jacobi-preconditioned Richardson steps with Anderson
 * extrapolation) to a relative residual of tol, for nchan channels of ngrid points each (device FP64,
 * [nchan][ngrid]; f and out may not overlap).  On a plane wave of FD eigenvalue -lambda this multiplies
 * by lambda / (lambda + k0^2): the uniform component is removed and short waves pass.  k0 > 0, tol > 0.
 * NOT_CONVERGED if the solve does not reach tol in max_iter iterations. */
sdft_status sdft_kerker(sdft_ctx* ctx, const double* f, double* out, int nchan, double k0, double tol,
                        int max_iter);

/* One step of the context's density mixer (paper Sec. 2.1: periodic Pulay, Kerker-preconditioned when
 * opt.kerker_k0 > 0), exactly as sdft_scf applies it between iterations: from the input density x_in and
 * the output density x_out ([nspin][ngrid], device FP64) it pushes the history and writes the next input
 * x_next (device, may alias neither x_in nor x_out).  The history is the context's own: sdft_reset clears
 * it, and sdft_scf uses and then clears it. */
sdft_status sdft_mix_step(sdft_ctx* ctx, const double* x_in, const double* x_out, double* x_next);

/* Fermi level by bisection on sum_k w_k sum_n g = N_e; eig [nspin][nkpt][nstates] (device);
 * occ receives g (device), mu/ts written to host scalars. */
sdft_status sdft_fermi(sdft_ctx* ctx, const double* eig, double* occ, double* mu, double* ts);

/* Spectrum bounds by Lanczos on problem (spin, kpt): lower Ritz value, upper bound. Host out. */
sdft_status sdft_lanczos_bounds(sdft_ctx* ctx, int spin, int kpt, int steps, double* lower,
                                double* upper);

/* Counts of the refined subspace eigensolves (FP32 solve + FP64 refinement, see sdft_subspace_eig) on this
 * context since creation: accepted, and rejected by the device-side check and redone by cuSOLVER. */
sdft_status sdft_get_eig_stats(const sdft_ctx* ctx, int* refined_accepted, int* refined_rejected);

/* Number of kernel launches the library has issued on this context (for benchmarks). */
sdft_status sdft_launch_count(const sdft_ctx* ctx, uint64_t* count);

/* Stencil tile variant used by the last fused H Y + Chebyshev step on FP32 blocks of the given
 * kind (is_complex 0: paired real, 1: complex); *index = -1 and name "" if none ran yet.  The
 * variant is chosen once per context by timing every compiled tile shape on the first large
 * filter call (environment SDFT_STENCIL_VARIANT=k forces variant k where it fits the grid).
 * name (host, cap bytes) receives the variant's name. */
sdft_status sdft_get_stencil_variant(const sdft_ctx* ctx, int is_complex, int* index, char* name, size_t cap);

/* ---- tracing: per-kernel-family device time (paper Sec. 2.1 ".out ... various timings") -- */
enum {
    SDFT_K_STENCIL = 0,    /* fused H Y + Chebyshev step, FP32 blocks (bytes: Y, Yprev read + Ynext write) */
    SDFT_K_KB_PROJECT = 1, /* KB projection C = beta^H Y */
    SDFT_K_GRAM = 2,       /* M = Y^H Y, Hs = Y^H HY (flops: 4 ngrid ncol^2, complex x4) */
    SDFT_K_EIGEN = 3,      /* equilibration + generalized eigensolve */
    SDFT_K_ROTATE = 4,     /* X = Y Q (flops: 2 ngrid ncol^2, complex x4) */
    SDFT_K_POISSON = 5,    /* AAR Poisson solve (whole solve) */
    SDFT_K_DENSITY = 6,    /* density from orbitals */
    SDFT_K_STENCIL64 = 7,  /* the same step on FP64 blocks (FP64 path, final FP64 pass, Lanczos) */
    SDFT_K_COUNT = 8
};
typedef struct {
    uint64_t launches;     /* timed launches (or solves) */
    double seconds;        /* summed device time between CUDA events around each launch */
    double bytes;          /* summed algorithmic bytes moved (0 where not defined) */
    double flops;          /* summed algorithmic flops (0 where not defined) */
} sdft_kernel_stats;
/* on != 0: record a CUDA event pair around every launch of the families above (adds ~2 us per
 * launch); statistics accumulate until sdft_reset_kernel_stats. */
sdft_status sdft_set_timing(sdft_ctx* ctx, int on);
sdft_status sdft_get_kernel_stats(sdft_ctx* ctx, int family, sdft_kernel_stats* out);
sdft_status sdft_reset_kernel_stats(sdft_ctx* ctx);

/* ---- learned initial density -------------------------------------------------------------
 * The paper starts the SCF from a superposition of atomic densities (Sec. 2.1) and names machine
 * learning as a way to improve efficiency (Sec. 4).  Here a small network predicts the correction
 * rho* - rho_SAD at each grid point; only the SCF's starting point (hence its iteration count)
 * changes, the converged answer does not.
 *   Descriptors (Behler-Parrinello radial symmetry functions), j = 0..31:
 *     G_j(x) = sum_atoms sum_images exp(-(r - mu_j)^2 / (2 eta^2)) (cos(pi r / 6.5) + 1) / 2,
 *     r = |x - R_a - T| <= 6.5 bohr, mu_j = 6 j / 31, eta = 6 / 31 (bohr).
 *   Network: h1 = silu(W1 G + b1), h2 = silu(W2 h1 + b2), y = w3 . h2 + b3 (widths 32-64-64-1).
 *   Parameters: one FP32 vector of SDFT_MLP_NPARAM: W1 [64 x 32] row-major, b1 [64],
 *     W2 [64 x 64] row-major, b2 [64], w3 [64], b3.  Kernels round the parameters to BF16 and
 *     compute in FP32 (training keeps the FP32 vector as the master copy).
 *   Features: device BF16 (uint16 bit patterns) [npts][32], point-major.
 *   Loss: mean over the batch of (y - t)^2.
 *   Mini-batches: the batch of size B starting at s visits points perm((s + i) mod npts), i < B,
 *     with perm(j) = j * P mod npts, P = 1000003 (999983 when 1000003 divides npts).
 * All pointers below are device pointers unless named *_host; calls are asynchronous on
 * cuda_stream (a cudaStream_t) or on the context's stream; errors without a context are
 * reported by sdft_last_error(NULL). */
#define SDFT_MLP_NFEAT 32
#define SDFT_MLP_NPARAM 6337

/* Descriptors of every grid point of the context's cell -> feat [ngrid][32]; if target is not
 * NULL, also target [ngrid] (FP32) = sum over spins of the last SCF's output density minus the
 * SAD density (the training target once the SCF has converged).  Synchronises the stream. */
sdft_status sdft_mlp_dataset(sdft_ctx* ctx, uint16_t* feat, float* target);

/* Loss and gradient of one mini-batch: grad [NPARAM] is overwritten with d(loss)/d(params)
 * (FP32, BF16-rounded parameters in the forward pass); the batch loss is ADDED to *loss (device
 * double, so that several batches can share one accumulator).  1 <= batch <= npts. */
sdft_status sdft_mlp_loss_grad(const uint16_t* feat, const float* target, int64_t npts, int64_t batch,
                               int64_t start, const float* params, float* grad, double* loss,
                               void* cuda_stream);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected, step >= 1) on params, with
 * FP32 moments m, v [NPARAM] (zero before step 1). */
sdft_status sdft_mlp_adam(float* params, const float* grad, float* m, float* v, int step, double lr,
                          void* cuda_stream);

/* nsteps Adam steps; step first_step + k uses the batch starting at (first_step + k - 1) * batch
 * (mod npts) and writes its loss (before the update) to loss[k] (device double [nsteps]).
 * grad [NPARAM] is scratch. */
sdft_status sdft_mlp_train(const uint16_t* feat, const float* target, int64_t npts, int64_t batch,
                           float* params, float* grad, float* m, float* v, int first_step, int nsteps,
                           double lr, double* loss, void* cuda_stream);

/* Inference: y [npts] = network(feat). */
sdft_status sdft_mlp_forward(const uint16_t* feat, int64_t npts, const float* params, float* y,
                             void* cuda_stream);

/* Learned guess for the next sdft_scf of this context: rho0 = max(rho_SAD + y, 0) renormalised to
 * N_e, split over spins as the SAD guess is; it replaces the SAD start like sdft_set_density.
 * The first call allocates 68 bytes per grid point of scratch (kept until sdft_destroy).
 * Synchronises the stream. */
sdft_status sdft_mlp_predict(sdft_ctx* ctx, const float* params);

#ifdef __cplusplus
}
#endif
#endif /* SDFT_H */
