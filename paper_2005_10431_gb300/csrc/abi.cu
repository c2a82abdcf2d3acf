// extern "C" entry points of libsdft (declared in include/sdft.h).  Every entry point
// converts internal exceptions into an sdft_status and keeps the message for sdft_last_error.
#include "internal.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>

namespace sdft {

void* ctx_alloc(sdft_ctx* c, size_t bytes) {
    if (bytes == 0) bytes = 16;
    void* p = nullptr;
    if (c->alloc) {
        p = c->alloc(bytes, c->alloc_user);
        SDFT_REQUIRE(p != nullptr, SDFT_ERR_OOM, "allocation callback returned NULL for " + std::to_string(bytes) + " bytes");
        if (((uintptr_t)p & 255) != 0) {
            if (c->release) c->release(p, c->alloc_user);
            throw Error{SDFT_ERR_INVALID_ARG, "allocation callback returned memory that is not 256-byte aligned"};
        }
    } else {
        cudaError_t e = cudaMalloc(&p, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            throw Error{SDFT_ERR_OOM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed"};
        }
    }
    c->owned.push_back(p);
    SDFT_CUDA(cudaMemsetAsync(p, 0, bytes, c->stream));
    return p;
}

void ctx_release(sdft_ctx* c, void* p) {
    if (!p) return;
    auto it = std::find(c->owned.begin(), c->owned.end(), p);
    if (it == c->owned.end()) return;
    c->owned.erase(it);
    if (c->release) {
        c->release(p, c->alloc_user);
    } else {
        cudaStreamSynchronize(c->stream);
        cudaFree(p);
    }
}

void ctx_free_all(sdft_ctx* c) {
    if (c->stream || true) cudaStreamSynchronize(c->stream);
    for (void* p : c->owned) {
        if (c->release) c->release(p, c->alloc_user);
        else cudaFree(p);
    }
    c->owned.clear();
    for (const PendingTiming& p : c->pending) {
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
    }
    c->pending.clear();
    for (cudaEvent_t e : c->ev_free) cudaEventDestroy(e);
    c->ev_free.clear();
    if (c->hscal) {
        cudaFreeHost(c->hscal);
        c->hscal = nullptr;
    }
    if (c->g_graph) {
        cudaGraphExecDestroy(c->g_graph);
        c->g_graph = nullptr;
    }
    if (c->mg_graph) {
        cudaGraphExecDestroy(c->mg_graph);
        c->mg_graph = nullptr;
    }
    if (c->cap_stream) {
        cudaStreamDestroy(c->cap_stream);
        c->cap_stream = nullptr;
    }
    if (c->g_rtab_pin) cudaFreeHost(c->g_rtab_pin);
    if (c->g_ktab_pin) cudaFreeHost(c->g_ktab_pin);
    c->g_rtab_pin = nullptr;
    c->g_ktab_pin = nullptr;
}

static cudaEvent_t take_event(sdft_ctx* c) {
    if (!c->ev_free.empty()) {
        cudaEvent_t e = c->ev_free.back();
        c->ev_free.pop_back();
        return e;
    }
    cudaEvent_t e;
    SDFT_CUDA(cudaEventCreate(&e));
    return e;
}

ScopedTimer::ScopedTimer(sdft_ctx* c_, int fam_, double bytes_, double flops_)
    : c(c_), fam(fam_), bytes(bytes_), flops(flops_) {
    if (!c || !c->timing) return;
    a = take_event(c);
    b = take_event(c);
    cudaEventRecord(a, c->stream);
}

ScopedTimer::~ScopedTimer() {
    if (!a) return;
    cudaEventRecord(b, c->stream);
    c->pending.push_back(PendingTiming{a, b, fam, bytes, flops});
}

void resolve_timing(sdft_ctx* c) {
    if (c->pending.empty()) return;
    SDFT_CUDA(cudaStreamSynchronize(c->stream));
    for (const PendingTiming& p : c->pending) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
            sdft_kernel_stats& k = c->kstat[p.fam];
            k.launches += 1;
            k.seconds += 1e-3 * ms;
            k.bytes += p.bytes;
            k.flops += p.flops;
        }
        c->ev_free.push_back(p.a);
        c->ev_free.push_back(p.b);
    }
    c->pending.clear();
}

namespace {

bool finite_all(const double* p, size_t n) {
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(p[i])) return false;
    return true;
}

}  // namespace

void host_energy_constants(sdft_ctx* c) {
    // E_self = sum Z^2 / (2 sqrt(pi) r_loc); E_sc = 1/2 sum' Z Z' erfc(d/s)/d, s = sqrt(2(r^2 + r'^2))
    c->E_self = 0.0;
    for (int a = 0; a < c->natom; ++a) {
        const sdft_pseudo& s = c->species[c->types[a]];
        c->E_self += s.Z * s.Z / (2.0 * std::sqrt(M_PI) * s.r_loc);
    }
    c->E_sc = 0.0;
    c->dEsc.assign(3 * c->natom, 0.0);
    const double rmax = 30.0;
    int nimg[3];
    for (int d = 0; d < 3; ++d) nimg[d] = c->opt.boundary == SDFT_BC_DIRICHLET ? 0 : (int)std::ceil(rmax / c->L[d]) + 1;
    for (int a = 0; a < c->natom; ++a) {
        const sdft_pseudo& sa = c->species[c->types[a]];
        for (int b = 0; b < c->natom; ++b) {
            const sdft_pseudo& sb = c->species[c->types[b]];
            const double s = std::sqrt(2.0 * (sa.r_loc * sa.r_loc + sb.r_loc * sb.r_loc));
            for (int t0 = -nimg[0]; t0 <= nimg[0]; ++t0)
                for (int t1 = -nimg[1]; t1 <= nimg[1]; ++t1)
                    for (int t2 = -nimg[2]; t2 <= nimg[2]; ++t2) {
                        if (a == b && t0 == 0 && t1 == 0 && t2 == 0) continue;
                        const double v[3] = {c->pos[3 * a] - c->pos[3 * b] - t0 * c->L[0],
                                             c->pos[3 * a + 1] - c->pos[3 * b + 1] - t1 * c->L[1],
                                             c->pos[3 * a + 2] - c->pos[3 * b + 2] - t2 * c->L[2]};
                        const double d = std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
                        if (d > rmax) continue;
                        c->E_sc += 0.5 * sa.Z * sb.Z * std::erfc(d / s) / d;
                        if (a != b) {
                            const double f = sa.Z * sb.Z *
                                             (-2.0 / (s * std::sqrt(M_PI)) * std::exp(-(d / s) * (d / s)) / d -
                                              std::erfc(d / s) / (d * d));
                            for (int q = 0; q < 3; ++q) c->dEsc[3 * a + q] += f * v[q] / d;
                        }
                    }
        }
    }
}

namespace {


void build_context(sdft_ctx* c) {
    const sdft_options& o = c->opt;
    const long long ng = c->ng;
    const int ns = o.nstates;    // occupied set: eigenvalues and occupations reported per problem
    const int nf = c->nfilt;      // filtered block: orbitals, Rayleigh-Ritz matrices and workspaces
    SDFT_CUDA(cudaMallocHost(&c->hscal, sizeof(double) * SCAL_DOUBLES));
    cusolverStatus_t cs = cusolverDnCreate(&c->solver);
    SDFT_REQUIRE(cs == CUSOLVER_STATUS_SUCCESS, SDFT_ERR_CUDA, "cusolverDnCreate failed");
    cusolverDnSetStream(c->solver, c->stream);
    c->scal = (double*)ctx_alloc(c, sizeof(double) * SCAL_DOUBLES);
    c->b = (double*)ctx_alloc(c, sizeof(double) * ng);
    c->rho_sad = (double*)ctx_alloc(c, sizeof(double) * ng);
    c->rho_user = (double*)ctx_alloc(c, sizeof(double) * o.nspin * ng);
    c->rho_in = (double*)ctx_alloc(c, sizeof(double) * o.nspin * ng);
    c->rho_out = (double*)ctx_alloc(c, sizeof(double) * o.nspin * ng);
    c->phi = (double*)ctx_alloc(c, sizeof(double) * ng);
    c->veff = (double*)ctx_alloc(c, sizeof(double) * o.nspin * ng);
    c->veff32 = (float*)ctx_alloc(c, sizeof(float) * o.nspin * ng);
    c->exc = (double*)ctx_alloc(c, sizeof(double) * ng);
    c->work64 = (double*)ctx_alloc(c, sizeof(double) * 28 * ng);
    c->work32 = (float*)ctx_alloc(c, sizeof(float) * 20 * ng);
    // FD coefficients of -1/2 L_h
    const double w[7] = {-5369.0 / 1800.0, 12.0 / 7.0, -15.0 / 56.0, 10.0 / 189.0, -1.0 / 112.0, 2.0 / 1925.0,
                         -1.0 / 16632.0};
    double c0 = 0.0;
    for (int r = 0; r <= FD_RADIUS; ++r) {
        c->coef.cx[r] = -0.5 * w[r] / (c->h[0] * c->h[0]);
        c->coef.cy[r] = -0.5 * w[r] / (c->h[1] * c->h[1]);
        c->coef.cz[r] = -0.5 * w[r] / (c->h[2] * c->h[2]);
    }
    c0 = c->coef.cx[0] + c->coef.cy[0] + c->coef.cz[0];
    c->coef.c0 = c0;
    // geometry set-up on the device
    build_pseudocharge_and_sad(c);
    c->kb.resize(o.nkpt);
    bool any_cplx = false;
    for (int k = 0; k < o.nkpt; ++k) {
        build_kb_tables(c, k);
        any_cplx = any_cplx || c->kb[k].cplx;
    }
    host_energy_constants(c);
    // problems
    const int np = o.nspin * o.nkpt;
    double* eig_all = (double*)ctx_alloc(c, sizeof(double) * np * ns);
    double* occ_all = (double*)ctx_alloc(c, sizeof(double) * np * ns);
    c->probs.resize(np);
    size_t maxblock = 0;
    for (int s = 0; s < o.nspin; ++s)
        for (int k = 0; k < o.nkpt; ++k) {
            Problem& P = c->probs[s * o.nkpt + k];
            P.spin = s;
            P.kpt = k;
            P.cplx = c->kb[k].cplx;
            const size_t bytes = block_elems_bytes(c, o.precision, P.cplx, nf);
            P.X = ctx_alloc(c, bytes);
            if (o.precision == SDFT_MIXED) P.X64 = ctx_alloc(c, block_elems_bytes(c, SDFT_FP64, P.cplx, nf));
            P.eig = eig_all + (long long)(s * o.nkpt + k) * ns;
            P.eigf = nf > ns ? (double*)ctx_alloc(c, sizeof(double) * nf) : P.eig;
            P.occ = occ_all + (long long)(s * o.nkpt + k) * ns;
            maxblock = std::max(maxblock, bytes);
            if (o.precision == SDFT_MIXED) maxblock = std::max(maxblock, block_elems_bytes(c, SDFT_FP64, P.cplx, nf));
        }
    c->block_bytes = maxblock;
    for (int i = 0; i < 4; ++i) c->blk[i] = ctx_alloc(c, maxblock);
    const int w2 = any_cplx ? 2 : 1;
    c->Ms = (double*)ctx_alloc(c, sizeof(double) * nf * nf * w2);
    c->Hs = (double*)ctx_alloc(c, sizeof(double) * nf * nf * w2);
    c->part_elems = std::max<size_t>((size_t)2 * nf * nf * w2 * 64, 1 << 20);
    c->part = (double*)ctx_alloc(c, sizeof(double) * c->part_elems);
    c->dscale = (double*)ctx_alloc(c, sizeof(double) * nf);
    c->Q32 = ctx_alloc(c, sizeof(float) * nf * nf * w2);
    c->qsplit_bytes = sdft::qsplit_bytes(nf);
    c->Qsplit = ctx_alloc(c, c->qsplit_bytes);
    // FP32 KB coefficients, padded by two pair columns and two elements: the slab stencil copies a
    // 16-byte aligned window of a pair group's coefficients that may pass the block's end
    c->c32_elems = (long long)std::max(1, c->natom) * (nf + 2) + 2;
    c->C32 = (float*)ctx_alloc(c, sizeof(float2) * (size_t)c->c32_elems);
    c->C32b = (float*)ctx_alloc(c, sizeof(float2) * (size_t)c->c32_elems);
    c->C64 = (double*)ctx_alloc(c, sizeof(double) * 2 * std::max(1, c->natom) * nf);
    c->dinfo = (int*)ctx_alloc(c, sizeof(int) * 4);
    // cuSOLVER workspace for the generalized eigenproblem of size nf
    int lw = 0;
    if (any_cplx) {
        cs = cusolverDnZhegvd_bufferSize(c->solver, CUSOLVER_EIG_TYPE_1, CUSOLVER_EIG_MODE_VECTOR,
                                         CUBLAS_FILL_MODE_UPPER, nf, (cuDoubleComplex*)c->Hs, nf,
                                         (cuDoubleComplex*)c->Ms, nf, c->dscale, &lw);
        SDFT_REQUIRE(cs == CUSOLVER_STATUS_SUCCESS, SDFT_ERR_CUDA, "hegvd workspace query failed");
        c->solver_lwork = lw;
    }
    cs = cusolverDnDsygvd_bufferSize(c->solver, CUSOLVER_EIG_TYPE_1, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_UPPER,
                                     nf, c->Hs, nf, c->Ms, nf, c->dscale, &lw);
    SDFT_REQUIRE(cs == CUSOLVER_STATUS_SUCCESS, SDFT_ERR_CUDA, "sygvd workspace query failed");
    c->solver_lwork = std::max(c->solver_lwork, lw);
    if (const char* env = getenv("SDFT_EIGEN")) c->eig_method = atoi(env);
    if (const char* env = getenv("SDFT_AAR_PERSISTENT")) c->aar_persistent = atoi(env) != 0;
    // multigrid-preconditioned FP32 Poisson corrections (periodic mixed-precision path only)
    if (const char* env = getenv("SDFT_AAR_MG")) c->aar_mg = atoi(env) != 0;
    if (const char* env = getenv("SDFT_FUSE_KB")) c->fuse_kb_projection = atoi(env) != 0;
    if (c->aar_mg && c->opt.precision == SDFT_MIXED && c->opt.boundary != SDFT_BC_DIRICHLET) mg_setup(c);
    if (const char* env = getenv("SDFT_TEST_BARRIER_EXTRA")) c->test_barrier_extra = atoi(env) != 0;
    cs = cusolverDnCreateSyevjInfo(&c->syevj_params);
    SDFT_REQUIRE(cs == CUSOLVER_STATUS_SUCCESS, SDFT_ERR_CUDA, "syevj info");
    cusolverDnXsyevjSetTolerance(c->syevj_params, 1e-14);
    cusolverDnXsyevjSetMaxSweeps(c->syevj_params, 30);
    cs = cusolverDnDsygvj_bufferSize(c->solver, CUSOLVER_EIG_TYPE_1, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_UPPER,
                                     nf, c->Hs, nf, c->Ms, nf, c->dscale, &lw, c->syevj_params);
    SDFT_REQUIRE(cs == CUSOLVER_STATUS_SUCCESS, SDFT_ERR_CUDA, "sygvj workspace query failed");
    c->solver_lwork = std::max(c->solver_lwork, lw);
    c->solver_work = ctx_alloc(c, (size_t)c->solver_lwork * 16 + 256);
    // mixing history
    const long long nv = (long long)o.nspin * ng;
    c->mix_dx = (double*)ctx_alloc(c, sizeof(double) * nv * o.mix_hist);
    c->mix_df = (double*)ctx_alloc(c, sizeof(double) * nv * o.mix_hist);
    c->mix_xprev = (double*)ctx_alloc(c, sizeof(double) * nv);
    c->mix_fprev = (double*)ctx_alloc(c, sizeof(double) * nv);
    reset_state(c);
    SDFT_CUDA(cudaStreamSynchronize(c->stream));
}

sdft_status fail(sdft_ctx* c, const Error& e) {
    if (c) c->last_error = e.msg;
    return e.code;
}

thread_local std::string g_create_error;

}  // namespace
}  // namespace sdft

using sdft::Error;

#define SDFT_TRY(ctx, ...)                                                     \
    try {                                                                      \
        if (!(ctx)) return SDFT_ERR_INVALID_ARG;                               \
        (ctx)->last_error.clear();                                             \
        __VA_ARGS__;                                                               \
        return SDFT_OK;                                                        \
    } catch (const Error& e) {                                                 \
        return sdft::fail((ctx), e);                                           \
    } catch (const std::exception& e) {                                        \
        (ctx)->last_error = e.what();                                          \
        return SDFT_ERR_CUDA;                                                  \
    }

extern "C" {

void sdft_default_options(sdft_options* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->nspin = 1;
    o->nkpt = 1;
    o->nstates = 8;
    o->cheb_degree = 12;
    o->first_scf_filter_passes = 4;
    o->lanczos_steps = 20;
    o->kT = 0.01;
    o->mix_hist = 7;
    o->mix_beta = 0.3;
    o->pulay_period = 1;
    o->pulay_restart = 0;
    o->scf_tol = 1e-6;
    o->max_scf = 100;
    o->precision = SDFT_FP64;
    o->final_fp64_pass = 0;
    o->poisson_tol = 1e-10;
    o->init_guess = SDFT_GUESS_SAD;
    o->initial_moment = 0.125;
    o->seed = 0;
    o->batch_problems = 1;
    o->use_graphs = 1;
}

sdft_status sdft_create(const sdft_cell* cell, const sdft_grid* grid, const sdft_atoms* atoms, int ntypes,
                        const sdft_pseudo* pseudo, const sdft_options* opt, sdft_alloc_fn alloc, sdft_free_fn free_fn,
                        void* alloc_user, void* cuda_stream, sdft_ctx** out) {
    if (!out) return SDFT_ERR_INVALID_ARG;
    *out = nullptr;
    sdft_ctx* c = new sdft_ctx();
    try {
        SDFT_REQUIRE(cell && grid && atoms && pseudo && opt, SDFT_ERR_INVALID_ARG, "null argument");
        SDFT_REQUIRE(grid->fd_order == 12, SDFT_ERR_INVALID_ARG, "fd_order must be 12");
        SDFT_REQUIRE(ntypes >= 1, SDFT_ERR_INVALID_ARG, "ntypes must be >= 1");
        SDFT_REQUIRE(atoms->natom >= 1 && atoms->pos && atoms->type, SDFT_ERR_INVALID_ARG, "atoms");
        SDFT_REQUIRE(sdft::finite_all(atoms->pos, 3 * (size_t)atoms->natom), SDFT_ERR_NONFINITE,
                     "atom positions contain NaN/Inf");
        SDFT_REQUIRE(sdft::finite_all(cell->L, 3), SDFT_ERR_NONFINITE, "cell contains NaN/Inf");
        for (int d = 0; d < 3; ++d) {
            SDFT_REQUIRE(cell->L[d] > 0, SDFT_ERR_INVALID_ARG, "cell edges must be positive");
            SDFT_REQUIRE(grid->n[d] >= 6, SDFT_ERR_INVALID_ARG, "grid points per edge must be >= 6");
        }
        for (int t = 0; t < ntypes; ++t) {
            const sdft_pseudo& p = pseudo[t];
            const double v[6] = {p.Z, p.r_loc, p.r_proj, p.E_kb, p.r_cut_proj, p.sad_width};
            SDFT_REQUIRE(sdft::finite_all(v, 6), SDFT_ERR_NONFINITE, "pseudopotential contains NaN/Inf");
            SDFT_REQUIRE(p.Z > 0 && p.r_loc > 0 && p.r_proj > 0 && p.r_cut_proj > 0 && p.sad_width > 0,
                         SDFT_ERR_INVALID_ARG, "pseudopotential parameters must be positive");
        }
        for (int a = 0; a < atoms->natom; ++a)
            SDFT_REQUIRE(atoms->type[a] >= 0 && atoms->type[a] < ntypes, SDFT_ERR_INVALID_ARG, "atom type out of range");
        const sdft_options& o = *opt;
        SDFT_REQUIRE(o.nspin == 1 || o.nspin == 2, SDFT_ERR_INVALID_ARG, "nspin must be 1 or 2");
        SDFT_REQUIRE(o.nkpt >= 1 && o.nkpt <= sdft::MAX_KPT, SDFT_ERR_INVALID_ARG, "nkpt must be in [1, 256]");
        SDFT_REQUIRE(o.nstates >= 2, SDFT_ERR_INVALID_ARG, "nstates must be >= 2");
        SDFT_REQUIRE(o.precision == SDFT_FP64 || o.precision == SDFT_MIXED, SDFT_ERR_INVALID_ARG, "precision");
        SDFT_REQUIRE(o.precision == SDFT_FP64 || o.nstates % 2 == 0, SDFT_ERR_INVALID_ARG,
                     "SDFT_MIXED needs an even number of states");
        SDFT_REQUIRE(o.cheb_degree >= 1 && o.lanczos_steps >= 2, SDFT_ERR_INVALID_ARG, "degree / lanczos steps");
        SDFT_REQUIRE(o.kT > 0 && std::isfinite(o.kT), SDFT_ERR_INVALID_ARG, "kT must be positive");
        SDFT_REQUIRE(o.mix_hist >= 1 && o.mix_hist <= 16, SDFT_ERR_INVALID_ARG, "mix_hist must be in [1, 16]");
        SDFT_REQUIRE(std::isfinite(o.kerker_k0) && o.kerker_k0 >= 0.0, SDFT_ERR_INVALID_ARG,
                     "kerker_k0 must be finite and >= 0");
        SDFT_REQUIRE(o.xc == SDFT_XC_LDA_PZ || (o.xc == SDFT_XC_GGA_PBE && o.nspin == 1), SDFT_ERR_INVALID_ARG,
                     "xc must be SDFT_XC_LDA_PZ, or SDFT_XC_GGA_PBE with nspin = 1");
        SDFT_REQUIRE(o.boundary == SDFT_BC_PERIODIC ||
                         (o.boundary == SDFT_BC_DIRICHLET && o.precision == SDFT_FP64 && o.nkpt == 1 &&
                          (!o.kpts || (o.kpts[0] == 0.0 && o.kpts[1] == 0.0 && o.kpts[2] == 0.0))),
                     SDFT_ERR_INVALID_ARG, "boundary: SDFT_BC_DIRICHLET needs SDFT_FP64 and the Gamma point only");
        SDFT_REQUIRE(o.pulay_period >= 1, SDFT_ERR_INVALID_ARG, "pulay_period must be >= 1");
        SDFT_REQUIRE(o.max_scf >= 1, SDFT_ERR_INVALID_ARG, "max_scf must be >= 1");
        SDFT_REQUIRE(o.nbuffer >= 0 && (o.precision == SDFT_FP64 || o.nbuffer % 2 == 0), SDFT_ERR_INVALID_ARG,
                     "nbuffer must be >= 0, and even for SDFT_MIXED");
        SDFT_REQUIRE(std::isfinite(o.fp64_switch_tol) && o.fp64_switch_tol >= 0.0, SDFT_ERR_INVALID_ARG,
                     "fp64_switch_tol must be finite and >= 0");
        SDFT_REQUIRE(std::isfinite(o.gemm_fp32_switch_tol) && o.gemm_fp32_switch_tol >= 0.0, SDFT_ERR_INVALID_ARG,
                     "gemm_fp32_switch_tol must be finite and >= 0");
        c->opt = o;
        c->nfilt = o.nstates + o.nbuffer;
        c->stream = (cudaStream_t)cuda_stream;
        c->alloc = alloc;
        c->release = free_fn;
        c->alloc_user = alloc_user;
        for (int d = 0; d < 3; ++d) {
            c->n[d] = grid->n[d];
            c->L[d] = cell->L[d];
            c->h[d] = cell->L[d] / grid->n[d];
        }
        c->dV = c->h[0] * c->h[1] * c->h[2];
        c->ng = (long long)c->n[0] * c->n[1] * c->n[2];
        c->natom = atoms->natom;
        c->pos.assign(atoms->pos, atoms->pos + 3 * atoms->natom);
        c->types.assign(atoms->type, atoms->type + atoms->natom);
        c->species.assign(pseudo, pseudo + ntypes);
        c->nelec = 0.0;
        for (int a = 0; a < c->natom; ++a) c->nelec += c->species[c->types[a]].Z;
        c->kpts.assign(3 * o.nkpt, 0.0);
        if (o.kpts) {
            SDFT_REQUIRE(sdft::finite_all(o.kpts, 3 * (size_t)o.nkpt), SDFT_ERR_NONFINITE, "k-points contain NaN/Inf");
            c->kpts.assign(o.kpts, o.kpts + 3 * o.nkpt);
        }
        c->kw.assign(o.nkpt, 1.0 / o.nkpt);
        if (o.kw) c->kw.assign(o.kw, o.kw + o.nkpt);
        c->opt.kpts = nullptr;
        c->opt.kw = nullptr;
        const double nfill = c->nelec / (o.nspin == 1 ? 2.0 : 1.0) / (o.nspin == 1 ? 1.0 : 2.0);
        SDFT_REQUIRE(o.nstates >= (int)std::ceil(nfill), SDFT_ERR_INVALID_ARG, "nstates below the occupied count");
        sdft::build_context(c);
        *out = c;
        return SDFT_OK;
    } catch (const Error& e) {
        sdft::g_create_error = e.msg;
        sdft::ctx_free_all(c);
        if (c->solver) cusolverDnDestroy(c->solver);
        delete c;
        return e.code;
    }
}

void sdft_destroy(sdft_ctx* c) {
    if (!c) return;
    sdft::ctx_free_all(c);
    if (c->syevj_params) cusolverDnDestroySyevjInfo(c->syevj_params);
    if (c->solver) cusolverDnDestroy(c->solver);
    delete c;
}

const char* sdft_last_error(const sdft_ctx* c) {
    if (!c) return sdft::g_create_error.c_str();
    return c->last_error.c_str();
}

sdft_status sdft_scf(sdft_ctx* c, sdft_result* out) {
    try {
        if (!c) return SDFT_ERR_INVALID_ARG;
        c->last_error.clear();
        const sdft_status s = sdft::run_scf(c, out);
        if (s == SDFT_ERR_NOT_CONVERGED) c->last_error = "SCF did not reach scf_tol within max_scf iterations";
        return s;
    } catch (const Error& e) {
        return sdft::fail(c, e);
    }
}

sdft_status sdft_batch_scf(sdft_ctx* const* ctxs, int n, sdft_result* out) {
    if (!ctxs || n < 1) return SDFT_ERR_INVALID_ARG;
    for (int i = 0; i < n; ++i) {
        if (!ctxs[i]) return SDFT_ERR_INVALID_ARG;
        for (int j = 0; j < i; ++j)
            if (ctxs[j] == ctxs[i]) {
                ctxs[i]->last_error = "a context appears twice in the batch";
                return SDFT_ERR_INVALID_ARG;
            }
        ctxs[i]->last_error.clear();
    }
    try {
        const sdft_status s = sdft::run_batch_scf(std::vector<sdft_ctx*>(ctxs, ctxs + n), out);
        if (s == SDFT_ERR_NOT_CONVERGED)
            for (int i = 0; i < n; ++i)
                if (out && !out[i].converged)
                    ctxs[i]->last_error = "SCF did not reach scf_tol within max_scf iterations";
        return s;
    } catch (const Error& e) {
        for (int i = 1; i < n; ++i) ctxs[i]->last_error = e.msg;
        return sdft::fail(ctxs[0], e);
    }
}

sdft_status sdft_reset(sdft_ctx* c) { SDFT_TRY(c, { sdft::reset_state(c); SDFT_CUDA(cudaStreamSynchronize(c->stream)); }) }

static sdft_status copy_out(sdft_ctx* c, const std::vector<double>& v, double* host, size_t n) {
    SDFT_TRY(c, {
        SDFT_REQUIRE(host != nullptr, SDFT_ERR_INVALID_ARG, "null output");
        SDFT_REQUIRE(!v.empty(), SDFT_ERR_INVALID_ARG, "no result available (run sdft_scf first)");
        SDFT_REQUIRE(n >= v.size(), SDFT_ERR_INVALID_ARG, "output buffer too short");
        std::memcpy(host, v.data(), sizeof(double) * v.size());
    })
}

sdft_status sdft_get_eigenvalues(sdft_ctx* c, double* host, size_t n) { return copy_out(c, c ? c->eig_host : std::vector<double>(), host, n); }
sdft_status sdft_get_occupations(sdft_ctx* c, double* host, size_t n) { return copy_out(c, c ? c->occ_host : std::vector<double>(), host, n); }
sdft_status sdft_get_forces(sdft_ctx* c, double* host, size_t n) { return copy_out(c, c ? c->forces : std::vector<double>(), host, n); }

static sdft_status copy_field(sdft_ctx* c, const double* src, size_t count, double* dst, size_t n, int on_device) {
    SDFT_TRY(c, {
        SDFT_REQUIRE(dst != nullptr, SDFT_ERR_INVALID_ARG, "null output");
        SDFT_REQUIRE(n >= count, SDFT_ERR_INVALID_ARG, "output buffer too short");
        SDFT_CUDA(cudaMemcpyAsync(dst, src, sizeof(double) * count,
                                  on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
        SDFT_CUDA(cudaStreamSynchronize(c->stream));
    })
}

sdft_status sdft_get_density(sdft_ctx* c, double* dst, size_t n, int on_device) {
    if (!c) return SDFT_ERR_INVALID_ARG;
    return copy_field(c, c->rho_out, (size_t)c->opt.nspin * c->ng, dst, n, on_device);
}
sdft_status sdft_get_pseudocharge(sdft_ctx* c, double* dst, size_t n, int on_device) {
    if (!c) return SDFT_ERR_INVALID_ARG;
    return copy_field(c, c->b, (size_t)c->ng, dst, n, on_device);
}
sdft_status sdft_get_sad_density(sdft_ctx* c, double* dst, size_t n, int on_device) {
    if (!c) return SDFT_ERR_INVALID_ARG;
    return copy_field(c, c->rho_sad, (size_t)c->ng, dst, n, on_device);
}

sdft_status sdft_set_density(sdft_ctx* c, const double* src, size_t n, int on_device) {
    SDFT_TRY(c, {
        const size_t need = (size_t)c->opt.nspin * c->ng;
        SDFT_REQUIRE(src != nullptr && n == need, SDFT_ERR_INVALID_ARG, "density size must be nspin*ngrid");
        if (!on_device) SDFT_REQUIRE(sdft::finite_all(src, n), SDFT_ERR_NONFINITE, "density contains NaN/Inf");
        SDFT_CUDA(cudaMemcpyAsync(c->rho_user, src, sizeof(double) * n,
                                  on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream));
        SDFT_CUDA(cudaMemcpyAsync(c->rho_in, c->rho_user, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->stream));
        c->user_density = true;
        SDFT_CUDA(cudaStreamSynchronize(c->stream));
    })
}

sdft_status sdft_move_atoms(sdft_ctx* c, const double* pos, int guess, double* coef) {
    SDFT_TRY(c, {
        SDFT_REQUIRE(pos != nullptr && (guess == 0 || guess == 1), SDFT_ERR_INVALID_ARG, "arguments");
        SDFT_REQUIRE(sdft::finite_all(pos, 3 * (size_t)c->natom), SDFT_ERR_NONFINITE, "positions contain NaN/Inf");
        sdft::move_atoms(c, pos, guess);
        if (coef) {
            coef[0] = guess ? c->last_alfe[0] : 0.0;
            coef[1] = guess ? c->last_alfe[1] : 0.0;
        }
        SDFT_CUDA(cudaStreamSynchronize(c->stream));
    })
}

sdft_status sdft_get_eig_stats(const sdft_ctx* c, int* refined_accepted, int* refined_rejected) {
    if (!c) return SDFT_ERR_INVALID_ARG;
    if (refined_accepted) *refined_accepted = c->reig_accepted;
    if (refined_rejected) *refined_rejected = c->reig_fallbacks;
    return SDFT_OK;
}

sdft_status sdft_get_input_density(sdft_ctx* c, double* dst, size_t n, int on_device) {
    SDFT_TRY(c, {
        const size_t need = (size_t)c->opt.nspin * c->ng;
        SDFT_REQUIRE(dst != nullptr && n >= need, SDFT_ERR_INVALID_ARG, "buffer shorter than nspin*ngrid");
        SDFT_CUDA(cudaMemcpyAsync(dst, c->rho_in, sizeof(double) * need,
                                  on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
        SDFT_CUDA(cudaStreamSynchronize(c->stream));
    })
}

sdft_status sdft_get_scf_log(sdft_ctx* c, sdft_iter_record* host, size_t cap, size_t* count) {
    SDFT_TRY(c, {
        if (count) *count = c->log.size();
        if (host) std::memcpy(host, c->log.data(), sizeof(sdft_iter_record) * std::min(cap, c->log.size()));
    })
}

static sdft::Problem& problem_of(sdft_ctx* c, int spin, int kpt) {
    SDFT_REQUIRE(spin >= 0 && spin < c->opt.nspin && kpt >= 0 && kpt < c->opt.nkpt, SDFT_ERR_INVALID_ARG,
                 "spin / k-point index out of range");
    return c->probs[spin * c->opt.nkpt + kpt];
}

sdft_status sdft_set_orbitals(sdft_ctx* c, int spin, int kpt, const void* dev, size_t bytes) {
    SDFT_TRY(c, {
        sdft::Problem& P = problem_of(c, spin, kpt);
        const size_t need = sdft::block_elems_bytes(c, c->opt.precision, P.cplx, c->opt.nstates);
        SDFT_REQUIRE(dev != nullptr && bytes == need, SDFT_ERR_INVALID_ARG, "orbital block size mismatch");
        SDFT_CUDA(cudaMemcpyAsync(P.X, dev, bytes, cudaMemcpyDeviceToDevice, c->stream));
        SDFT_CUDA(cudaStreamSynchronize(c->stream));
    })
}

sdft_status sdft_get_orbitals(sdft_ctx* c, int spin, int kpt, void* dev, size_t bytes) {
    SDFT_TRY(c, {
        sdft::Problem& P = problem_of(c, spin, kpt);
        const size_t need = sdft::block_elems_bytes(c, c->opt.precision, P.cplx, c->opt.nstates);
        SDFT_REQUIRE(dev != nullptr && bytes == need, SDFT_ERR_INVALID_ARG, "orbital block size mismatch");
        SDFT_CUDA(cudaMemcpyAsync(dev, P.X, bytes, cudaMemcpyDeviceToDevice, c->stream));
        SDFT_CUDA(cudaStreamSynchronize(c->stream));
    })
}

sdft_status sdft_set_veff(sdft_ctx* c, int spin, const double* v, int on_device) {
    SDFT_TRY(c, {
        SDFT_REQUIRE(spin >= 0 && spin < c->opt.nspin && v, SDFT_ERR_INVALID_ARG, "spin / pointer");
        if (!on_device) SDFT_REQUIRE(sdft::finite_all(v, (size_t)c->ng), SDFT_ERR_NONFINITE, "V_eff contains NaN/Inf");
        double* dst = c->veff + (long long)spin * c->ng;
        SDFT_CUDA(cudaMemcpyAsync(dst, v, sizeof(double) * c->ng,
                                  on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream));
        sdft::veff_to_float(c, spin);
        SDFT_CUDA(cudaStreamSynchronize(c->stream));
    })
}

static void check_block_args(sdft_ctx* c, int spin, int kpt, int precision, int ncol) {
    SDFT_REQUIRE(spin >= 0 && spin < c->opt.nspin && kpt >= 0 && kpt < c->opt.nkpt, SDFT_ERR_INVALID_ARG,
                 "spin / k-point index out of range");
    SDFT_REQUIRE(precision == SDFT_FP64 || precision == SDFT_MIXED, SDFT_ERR_INVALID_ARG, "precision");
    SDFT_REQUIRE(ncol >= 1 && ncol <= c->nfilt, SDFT_ERR_INVALID_ARG, "ncol must be in [1, nstates + nbuffer]");
    SDFT_REQUIRE(precision == SDFT_FP64 || c->kb[kpt].cplx || ncol % 2 == 0, SDFT_ERR_INVALID_ARG,
                 "SDFT_MIXED real blocks need an even column count");
}

sdft_status sdft_apply_h(sdft_ctx* c, int spin, int kpt, int precision, const void* x, void* y, int ncol) {
    SDFT_TRY(c, {
        check_block_args(c, spin, kpt, precision, ncol);
        SDFT_REQUIRE(x && y && x != y, SDFT_ERR_INVALID_ARG, "x, y must be distinct device blocks");
        sdft::apply_h(c, kpt, precision, x, y, ncol, c->veff + (long long)spin * c->ng,
                      c->veff32 + (long long)spin * c->ng);
        SDFT_CUDA(cudaStreamSynchronize(c->stream));
        sdft::check_stencil_flag(c);
    })
}

sdft_status sdft_chebyshev_filter(sdft_ctx* c, int spin, int kpt, int precision, const void* x, void* y, int ncol,
                                  int degree, double a, double b, double a0) {
    SDFT_TRY(c, {
        check_block_args(c, spin, kpt, precision, ncol);
        SDFT_REQUIRE(x && y && x != y, SDFT_ERR_INVALID_ARG, "x, y must be distinct device blocks");
        sdft::chebyshev_filter(c, kpt, precision, x, y, ncol, degree, a, b, a0, c->veff + (long long)spin * c->ng,
                               c->veff32 + (long long)spin * c->ng);
        SDFT_CUDA(cudaStreamSynchronize(c->stream));
        sdft::check_stencil_flag(c);
    })
}

sdft_status sdft_rayleigh_ritz(sdft_ctx* c, int spin, int kpt, int precision, const void* y, void* x, double* eig,
                               int ncol) {
    SDFT_TRY(c, {
        check_block_args(c, spin, kpt, precision, ncol);
        SDFT_REQUIRE(x && y && eig && x != y, SDFT_ERR_INVALID_ARG, "pointers");
        sdft::rayleigh_ritz(c, kpt, precision, y, x, eig, ncol, c->veff + (long long)spin * c->ng,
                            c->veff32 + (long long)spin * c->ng);
        SDFT_CUDA(cudaStreamSynchronize(c->stream));
    })
}

sdft_status sdft_subspace_matrices(sdft_ctx* c, int kpt, int precision, const void* y, const void* hy, void* m,
                                   void* hs, int ncol) {
    SDFT_TRY(c, {
        check_block_args(c, 0, kpt, precision, ncol);
        SDFT_REQUIRE(y && hy && m && hs, SDFT_ERR_INVALID_ARG, "pointers");
        sdft::subspace_gram(c, precision, c->kb[kpt].cplx, y, hy, (double*)m, (double*)hs, ncol);
        SDFT_CUDA(cudaStreamSynchronize(c->stream));
    })
}

sdft_status sdft_rotate(sdft_ctx* c, int kpt, int precision, const void* y, const void* q, void* x, int ncol) {
    SDFT_TRY(c, {
        check_block_args(c, 0, kpt, precision, ncol);
        SDFT_REQUIRE(y && q && x && x != y, SDFT_ERR_INVALID_ARG, "pointers");
        sdft::rotate_block(c, precision, c->kb[kpt].cplx, y, (const double*)q, x, ncol);
        SDFT_CUDA(cudaStreamSynchronize(c->stream));
    })
}

sdft_status sdft_poisson(sdft_ctx* c, const double* f, double* phi, double tol, int max_iter, int* iters) {
    SDFT_TRY(c, {
        SDFT_REQUIRE(f && phi && tol > 0 && max_iter >= 1, SDFT_ERR_INVALID_ARG, "arguments");
        const int it = c->opt.precision == SDFT_MIXED ? sdft::poisson_mixed(c, f, phi, tol, max_iter)
                                                      : sdft::poisson_aar(c, f, phi, tol, max_iter);
        SDFT_CUDA(cudaStreamSynchronize(c->stream));
        if (iters) *iters = it < 0 ? -it : it;
        if (it < 0) throw Error{SDFT_ERR_NOT_CONVERGED, "Poisson AAR did not reach the tolerance"};
    })
}

sdft_status sdft_kerker(sdft_ctx* c, const double* f, double* out, int nchan, double k0, double tol, int max_iter) {
    SDFT_TRY(c, {
        SDFT_REQUIRE(f && out && f != out && nchan >= 1 && std::isfinite(k0) && k0 > 0 && tol > 0 && max_iter >= 1,
                     SDFT_ERR_INVALID_ARG, "arguments");
        for (int ch = 0; ch < nchan; ++ch) {
            const int it = sdft::kerker_apply(c, f + (long long)ch * c->ng, out + (long long)ch * c->ng, k0, tol,
                                              max_iter);
            if (it < 0) throw Error{SDFT_ERR_NOT_CONVERGED, "Kerker screened-Poisson solve did not reach tol"};
        }
        SDFT_CUDA(cudaStreamSynchronize(c->stream));
    })
}

sdft_status sdft_mix_step(sdft_ctx* c, const double* x_in, const double* x_out, double* x_next) {
    SDFT_TRY(c, {
        SDFT_REQUIRE(x_in && x_out && x_next && x_next != x_in && x_next != x_out, SDFT_ERR_INVALID_ARG, "arguments");
        const size_t bytes = sizeof(double) * (size_t)c->opt.nspin * (size_t)c->ng;
        SDFT_CUDA(cudaMemcpyAsync(c->rho_in, x_in, bytes, cudaMemcpyDeviceToDevice, c->stream));
        SDFT_CUDA(cudaMemcpyAsync(c->rho_out, x_out, bytes, cudaMemcpyDeviceToDevice, c->stream));
        sdft::pulay_update(c);
        SDFT_CUDA(cudaMemcpyAsync(x_next, c->rho_in, bytes, cudaMemcpyDeviceToDevice, c->stream));
        SDFT_CUDA(cudaStreamSynchronize(c->stream));
    })
}

sdft_status sdft_lda(sdft_ctx* c, int nspin, const double* rho, double* exc, double* vxc, size_t n) {
    SDFT_TRY(c, {
        SDFT_REQUIRE((nspin == 1 || nspin == 2) && rho && exc && vxc, SDFT_ERR_INVALID_ARG, "arguments");
        sdft::lda_device(c, nspin, rho, exc, vxc, n);
        SDFT_CUDA(cudaStreamSynchronize(c->stream));
    })
}

sdft_status sdft_fermi(sdft_ctx* c, const double* eig, double* occ, double* mu, double* ts) {
    SDFT_TRY(c, {
        SDFT_REQUIRE(eig && occ, SDFT_ERR_INVALID_ARG, "pointers");
        sdft::fermi_device(c, eig, occ, c->scal + 8);
        double h[3];
        SDFT_CUDA(cudaMemcpyAsync(h, c->scal + 8, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
        SDFT_CUDA(cudaStreamSynchronize(c->stream));
        if (mu) *mu = h[0];
        if (ts) *ts = h[1];
    })
}

sdft_status sdft_lanczos_bounds(sdft_ctx* c, int spin, int kpt, int steps, double* lower, double* upper) {
    SDFT_TRY(c, {
        SDFT_REQUIRE(spin >= 0 && spin < c->opt.nspin && kpt >= 0 && kpt < c->opt.nkpt && steps >= 2 && lower && upper,
                     SDFT_ERR_INVALID_ARG, "arguments");
        sdft::lanczos(c, spin, kpt, steps, lower, upper);
    })
}

sdft_status sdft_subspace_matrices_noalloc(int precision, int is_complex, const void* y, const void* hy,
                                           int64_t ngrid, int ncol, double* m, double* hs, void* cuda_stream) {
    try {
        sdft::g_create_error.clear();
        SDFT_REQUIRE(precision == SDFT_FP64 || precision == SDFT_MIXED, SDFT_ERR_INVALID_ARG, "precision");
        SDFT_REQUIRE(y && hy && m && hs, SDFT_ERR_INVALID_ARG, "null pointer");
        SDFT_REQUIRE(ngrid >= 1 && ncol >= 1, SDFT_ERR_INVALID_ARG, "ngrid and ncol must be >= 1");
        SDFT_REQUIRE(precision == SDFT_FP64 || is_complex || ncol % 2 == 0, SDFT_ERR_INVALID_ARG,
                     "SDFT_MIXED real blocks need an even column count");
        sdft::subspace_gram_noalloc(precision, is_complex != 0, y, hy, (long long)ngrid, ncol, m, hs,
                                    (cudaStream_t)cuda_stream);
        return SDFT_OK;
    } catch (const Error& e) {
        sdft::g_create_error = e.msg;
        return e.code;
    }
}

#define SDFT_TRY_NOCTX(...)               \
    try {                                 \
        sdft::g_create_error.clear();     \
        __VA_ARGS__;                      \
        return SDFT_OK;                   \
    } catch (const Error& e) {            \
        sdft::g_create_error = e.msg;     \
        return e.code;                    \
    }

sdft_status sdft_mlp_dataset(sdft_ctx* c, uint16_t* feat, float* target) {
    SDFT_TRY(c, {
        SDFT_REQUIRE(feat != nullptr, SDFT_ERR_INVALID_ARG, "null feature pointer");
        sdft::mlp_dataset(c, feat, target);
    })
}

sdft_status sdft_mlp_loss_grad(const uint16_t* feat, const float* target, int64_t npts, int64_t batch,
                               int64_t start, const float* params, float* grad, double* loss, void* st) {
    SDFT_TRY_NOCTX({
        SDFT_REQUIRE(feat && target && params && grad && loss, SDFT_ERR_INVALID_ARG, "null pointer");
        SDFT_REQUIRE(npts >= 1 && batch >= 1 && batch <= npts && start >= 0, SDFT_ERR_INVALID_ARG,
                     "need 1 <= batch <= npts and start >= 0");
        sdft::mlp_loss_grad(feat, target, npts, batch, start, params, grad, loss, (cudaStream_t)st);
    })
}

sdft_status sdft_mlp_adam(float* params, const float* grad, float* m, float* v, int step, double lr, void* st) {
    SDFT_TRY_NOCTX({
        SDFT_REQUIRE(params && grad && m && v, SDFT_ERR_INVALID_ARG, "null pointer");
        SDFT_REQUIRE(step >= 1 && lr > 0, SDFT_ERR_INVALID_ARG, "need step >= 1 and lr > 0");
        sdft::mlp_adam(params, grad, m, v, step, lr, (cudaStream_t)st);
    })
}

sdft_status sdft_mlp_train(const uint16_t* feat, const float* target, int64_t npts, int64_t batch, float* params,
                           float* grad, float* m, float* v, int first_step, int nsteps, double lr, double* loss,
                           void* st) {
    SDFT_TRY_NOCTX({
        SDFT_REQUIRE(feat && target && params && grad && m && v && loss, SDFT_ERR_INVALID_ARG, "null pointer");
        SDFT_REQUIRE(npts >= 1 && batch >= 1 && batch <= npts, SDFT_ERR_INVALID_ARG, "need 1 <= batch <= npts");
        SDFT_REQUIRE(first_step >= 1 && nsteps >= 0 && lr > 0, SDFT_ERR_INVALID_ARG,
                     "need first_step >= 1, nsteps >= 0, lr > 0");
        if (nsteps > 0)
            sdft::mlp_train(feat, target, npts, batch, params, grad, m, v, first_step, nsteps, lr, loss,
                            (cudaStream_t)st);
    })
}

sdft_status sdft_mlp_forward(const uint16_t* feat, int64_t npts, const float* params, float* y, void* st) {
    SDFT_TRY_NOCTX({
        SDFT_REQUIRE(feat && params && y, SDFT_ERR_INVALID_ARG, "null pointer");
        SDFT_REQUIRE(npts >= 0, SDFT_ERR_INVALID_ARG, "npts < 0");
        if (npts > 0) sdft::mlp_forward(feat, npts, params, y, (cudaStream_t)st);
    })
}

sdft_status sdft_mlp_predict(sdft_ctx* c, const float* params) {
    SDFT_TRY(c, {
        SDFT_REQUIRE(params != nullptr, SDFT_ERR_INVALID_ARG, "null parameter pointer");
        sdft::mlp_guess(c, params);
    })
}

sdft_status sdft_set_timing(sdft_ctx* c, int on) {
    SDFT_TRY(c, {
        sdft::resolve_timing(c);
        c->timing = on != 0;
    })
}

sdft_status sdft_get_kernel_stats(sdft_ctx* c, int family, sdft_kernel_stats* out) {
    SDFT_TRY(c, {
        SDFT_REQUIRE(family >= 0 && family < SDFT_K_COUNT && out, SDFT_ERR_INVALID_ARG, "family / pointer");
        sdft::resolve_timing(c);
        *out = c->kstat[family];
    })
}

sdft_status sdft_reset_kernel_stats(sdft_ctx* c) {
    SDFT_TRY(c, {
        sdft::resolve_timing(c);
        for (int k = 0; k < SDFT_K_COUNT; ++k) c->kstat[k] = sdft_kernel_stats{};
    })
}

sdft_status sdft_chebyshev_filter_multi(sdft_ctx* const* ctxs, int n, const void* const* x, void* const* y,
                                        int degree, const double* a, const double* b, const double* a0) {
    if (!ctxs || n < 1 || !ctxs[0]) return SDFT_ERR_INVALID_ARG;
    sdft_ctx* c0 = ctxs[0];
    SDFT_TRY(c0, {
        SDFT_REQUIRE(n <= 64 && x && y && a && b && a0, SDFT_ERR_INVALID_ARG, "need 1..64 cells and all arrays");
        std::vector<sdft_ctx*> cs(n);
        std::vector<const void*> xs(n);
        std::vector<void*> ys(n);
        for (int i = 0; i < n; ++i) {
            sdft_ctx* c = ctxs[i];
            SDFT_REQUIRE(c != nullptr && x[i] && y[i] && x[i] != y[i], SDFT_ERR_INVALID_ARG, "null context or block");
            SDFT_REQUIRE(c->stream == c0->stream, SDFT_ERR_INVALID_ARG, "all contexts must share one stream");
            SDFT_REQUIRE(c->opt.precision == SDFT_MIXED && !c->kb[0].cplx, SDFT_ERR_INVALID_ARG,
                         "multi-cell filter takes SDFT_MIXED Gamma-point contexts");
            cs[i] = c;
            xs[i] = x[i];
            ys[i] = y[i];
        }
        sdft::chebyshev_filter_multi(cs, xs, ys, degree, a, b, a0);
        SDFT_CUDA(cudaStreamSynchronize(c0->stream));
    })
}

sdft_status sdft_subspace_eig(sdft_ctx* c, int is_complex, double* m, double* hs, double* eig, int ncol) {
    SDFT_TRY(c, {
        SDFT_REQUIRE(m && hs && eig, SDFT_ERR_INVALID_ARG, "null pointer");
        SDFT_REQUIRE(ncol >= 1 && ncol <= c->nfilt, SDFT_ERR_INVALID_ARG,
                     "ncol must be in [1, nstates + nbuffer] (solver workspace is sized for it)");
        bool any_cplx = false;
        for (const auto& P : c->probs) any_cplx = any_cplx || P.cplx;
        SDFT_REQUIRE(!is_complex || any_cplx, SDFT_ERR_INVALID_ARG,
                     "complex eigensolve needs a context with a complex (k != 0) problem");
        sdft::generalized_eig(c, is_complex != 0, m, hs, eig, ncol);
    })
}

sdft_status sdft_get_stencil_variant(const sdft_ctx* c, int is_complex, int* index, char* name, size_t cap) {
    if (!c || !index) return SDFT_ERR_INVALID_ARG;
    const int k = is_complex ? 1 : 0;
    *index = c->stencil_last[k];
    if (name && cap > 0) {
        const char* s = c->stencil_last_name[k] ? c->stencil_last_name[k] : "";
        std::strncpy(name, s, cap - 1);
        name[cap - 1] = 0;
    }
    return SDFT_OK;
}

sdft_status sdft_launch_count(const sdft_ctx* c, uint64_t* count) {
    if (!c || !count) return SDFT_ERR_INVALID_ARG;
    *count = c->launches;
    return SDFT_OK;
}

}  // extern "C"
