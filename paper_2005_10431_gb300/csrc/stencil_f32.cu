// Instantiations of the fused stencil / Chebyshev-step kernels (see stencil_impl.cuh)
// for FP32 blocks (two lanes per element: an orbital pair, or re/im of a Bloch orbital).
#include "stencil_impl.cuh"

#include <array>
#include <vector>

namespace sdft {
namespace {
// variants timed by the autotuner.  Column tiles: (TX, TY, queue prefetch PF, min blocks per SM,
// cp.async stages D).  Row tiles: (TY rows of full x extent, PF, min blocks per SM, D).
template <int TY, int MAXT, int D>
bool row_ok(const sdft_ctx* c, int ncolE) { return row_variant_ok<TY, MAXT, D>(c, ncolE); }

// row variants: (CPLX, TY, PF, max threads, min blocks per SM, D)
const StepVariant<float2> kReal[] = {
    {&launch_variant<float2, false, 32, 8, 2, 2, 4>, nullptr, "col32x8"},
    {&launch_variant<float2, false, 32, 8, 3, 2, 3>, nullptr, "col32x8pf3"},
    {&launch_variant<float2, false, 32, 16, 2, 1, 3>, nullptr, "col32x16"},
    {&launch_variant<float2, false, 32, 4, 2, 4, 4>, nullptr, "col32x4"},
    {&launch_variant<float2, false, 32, 8, 2, 3, 3>, nullptr, "col32x8occ3"},
    {&launch_variant<float2, false, 32, 8, 2, 4, 3>, nullptr, "col32x8occ4"},
    {&launch_variant<float2, false, 32, 4, 2, 6, 3>, nullptr, "col32x4occ6"},
    {&launch_row_variant<false, 4, 1, 256, 2, 3>, &row_ok<4, 256, 3>, "row4", &launch_row_group<false, 4, 1, 256, 2, 3>},
    {&launch_row_variant<false, 8, 1, 512, 1, 3>, &row_ok<8, 512, 3>, "row8", &launch_row_group<false, 8, 1, 512, 1, 3>},
    {&launch_row_variant<false, 5, 2, 320, 1, 3>, &row_ok<5, 320, 3>, "row5", &launch_row_group<false, 5, 2, 320, 1, 3>},
    {&launch_row_variant<false, 6, 2, 384, 1, 3>, &row_ok<6, 384, 3>, "row6", &launch_row_group<false, 6, 2, 384, 1, 3>},
    // TMA-fed slab tiles (stencil_tma.cu): (n1, TY rows, NP pairs, RY rows per thread, KB slots, stages,
    // min blocks per SM)
    {&launch_slab_variant<80, 8, 2, 1, 2, 3, 1>, &slab_variant_ok<80, 8, 2, 2, 3>, "slab80"},
    {&launch_slab_variant<80, 8, 1, 1, 2, 4, 1>, &slab_variant_ok<80, 8, 1, 2, 4>, "slab80np1"},
    {&launch_slab_variant<120, 8, 1, 1, 2, 4, 1>, &slab_variant_ok<120, 8, 1, 2, 4>, "slab120"},
    {&launch_slab_variant<40, 8, 2, 1, 2, 4, 1>, &slab_variant_ok<40, 8, 2, 2, 4>, "slab40"},
    {&launch_slab_variant<80, 8, 1, 2, 2, 4, 1>, &slab_variant_ok<80, 8, 1, 2, 4>, "slab80ry2"},
};
const StepVariant<float2> kCplx[] = {
    {&launch_variant<float2, true, 32, 8, 2, 2, 4>, nullptr, "col32x8"},
    {&launch_variant<float2, true, 32, 8, 3, 2, 3>, nullptr, "col32x8pf3"},
    {&launch_row_variant<true, 4, 1, 256, 2, 3>, &row_ok<4, 256, 3>, "row4", &launch_row_group<true, 4, 1, 256, 2, 3>},
    {&launch_row_variant<true, 8, 1, 256, 2, 3>, &row_ok<8, 256, 3>, "row8", &launch_row_group<true, 8, 1, 256, 2, 3>},
    {&launch_row_variant<true, 10, 1, 256, 2, 3>, &row_ok<10, 256, 3>, "row10", &launch_row_group<true, 10, 1, 256, 2, 3>},
};
constexpr int kNReal = sizeof(kReal) / sizeof(kReal[0]);
constexpr int kNCplx = sizeof(kCplx) / sizeof(kCplx[0]);
}  // namespace

template <>
void launch_kb_project<float2>(sdft_ctx* c, int kpt, const float2* Y, float2* C, int ncolE) {
    launch_project_impl<float2>(c, kpt, Y, C, ncolE);
}

template <>
void launch_cheb_step<float2>(sdft_ctx* c, int kpt, const float2* Y, const float2* Yprev, float2* Ynext, int ncolE,
                              const float* V, const float2* kbC, double alpha, double beta, double shift,
                              bool with_kinetic) {
    const bool cplx = c->kb[kpt].cplx;
    const StepVariant<float2>* table = cplx ? kCplx : kReal;
    const int nvar = cplx ? kNCplx : kNReal;
    int& choice = c->stencil_choice[cplx ? 1 : 0];
    int pick = choice;
    if (pick < 0) {
        // when the caller wants the output's KB coefficients too, the variants are timed with them (fused
        // or by the separate pass, into the caller's target buffer, which the real launch then rewrites)
        float2* kb_next = c->kb_next;
        c->kb_next = nullptr;
        bool fused = true;
        pick = autotune_stencil<float2>(c, table, nvar, kpt, Y, Yprev, Ynext, ncolE, V, kbC, alpha, beta, shift,
                                        kb_next, kb_next ? &launch_kb_project<float2> : nullptr, &fused);
        c->kb_next = kb_next;
        if (pick >= 0) {   // small calls are not timed and do not fix the choice
            choice = pick;
            if (kb_next) c->stencil_fuse = fused;
        } else {
            pick = 0;
        }
    }
    if (!c->stencil_fuse) c->kb_next = nullptr;   // the separate projection pass was timed faster
    c->kb_next_done = false;
    // the chosen variant may not fit this call (another column count): fall back to the column tile
    const int v = (table[pick].ok == nullptr || table[pick].ok(c, ncolE)) ? pick : 0;
    c->stencil_last[cplx ? 1 : 0] = v;
    c->stencil_last_name[cplx ? 1 : 0] = table[v].name;
    table[v].fn(c, kpt, Y, Yprev, Ynext, ncolE, V, kbC, alpha, beta, shift, with_kinetic, true);
}

// scalar FP32, Laplacian-only: the correction solves of the mixed-precision Poisson solver
template <>
void launch_cheb_step<float>(sdft_ctx* c, int kpt, const float* Y, const float* Yprev, float* Ynext, int ncolE,
                             const float* V, const float* kbC, double alpha, double beta, double shift,
                             bool with_kinetic) {
    launch_variant<float, false, 32, 8, 2, 2, 3>(c, kpt, Y, Yprev, Ynext, ncolE, V, kbC, alpha, beta, shift,
                                                 with_kinetic, true);
}


// grouped FP32 launches: the row variant used is the autotuned one when it is a row tile that
// fits, else the first row tile that fits; -1 if none does (callers then loop over problems)
int group_variant_f32(sdft_ctx* c, bool cplx, int ncolE) {
    const StepVariant<float2>* table = cplx ? kCplx : kReal;
    const int nvar = cplx ? kNCplx : kNReal;
    const int ch = c->stencil_choice[cplx ? 1 : 0];
    if (ch >= 0 && table[ch].group && table[ch].ok(c, ncolE)) return ch;
    for (int v = 0; v < nvar; ++v)
        if (table[v].group && table[v].ok(c, ncolE)) return v;
    return -1;
}

// time every fitting row variant on one grouped launch (tab: a table whose Ynext may be
// overwritten) and return the fastest
int autotune_group_f32(sdft_ctx* c, bool cplx, const RowProblem* grp, int nprob, int ncolE, bool haskb) {
    const StepVariant<float2>* table = cplx ? kCplx : kReal;
    const int nvar = cplx ? kNCplx : kNReal;
    if (const char* env = getenv("SDFT_STENCIL_VARIANT")) {
        const int v = atoi(env);
        if (v >= 0 && v < nvar && table[v].group && table[v].ok(c, ncolE)) return v;
    }
    cudaEvent_t a, b;
    SDFT_CUDA(cudaEventCreate(&a));
    SDFT_CUDA(cudaEventCreate(&b));
    int best = -1;
    float best_ms = 1e30f;
    for (int v = 0; v < nvar; ++v) {
        if (!table[v].group || !table[v].ok(c, ncolE)) continue;
        table[v].group(c, 0, grp, nprob, ncolE, false, haskb);   // warm-up
        SDFT_CUDA(cudaEventRecord(a, c->stream));
        for (int r = 0; r < 2; ++r) table[v].group(c, 0, grp, nprob, ncolE, false, haskb);
        SDFT_CUDA(cudaEventRecord(b, c->stream));
        SDFT_CUDA(cudaEventSynchronize(b));
        float ms = 0.f;
        SDFT_CUDA(cudaEventElapsedTime(&ms, a, b));
        if (ms < best_ms) {
            best_ms = ms;
            best = v;
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return best;
}

void launch_group_step_f32(sdft_ctx* c, bool cplx, int variant, const RowProblem* grp, int nprob, int ncolE,
                           bool prev, bool haskb) {
    const StepVariant<float2>* table = cplx ? kCplx : kReal;
    c->stencil_last[cplx ? 1 : 0] = variant;
    c->stencil_last_name[cplx ? 1 : 0] = table[variant].name;
    table[variant].group(c, 0, grp, nprob, ncolE, prev, haskb);
}

// One column-tile launch over several cells (each its own context, grid and block); probs[i].A
// carries cell i's recurrence step.  All contexts share the stream of the first one.
void launch_multi_step_f32(const std::vector<sdft_ctx*>& ctxs, std::vector<MultiProblem>& probs, bool prev) {
    constexpr int TX = 32, TY = 8, PF = 2, MINB = 2, D = 4;
    const int n = (int)probs.size();
    SDFT_REQUIRE(n >= 1 && n <= MULTI_MAX, SDFT_ERR_INVALID_ARG, "multi-cell launch takes 1..64 cells");
    sdft_ctx* c0 = ctxs[0];
    long long total = 0;
    int max_natom = 1;
    double bytes = 0;
    for (int i = 0; i < n; ++i) {
        MultiProblem& P = probs[i];
        const sdft_ctx* c = ctxs[i];
        P.tiles_x = (c->n[0] + TX - 1) / TX;
        P.tiles_y = (c->n[1] + TY - 1) / TY;
        P.cta_begin = (int)total;
        total += (long long)P.tiles_x * P.tiles_y * (c->nfilt / 2) * P.A.nzc;
        P.cta_end = (int)total;
        max_natom = std::max(max_natom, c->natom);
        bytes += (double)(c->nfilt / 2) * (double)c->ng * sizeof(float2) * (prev ? 3.0 : 2.0);
    }
    SDFT_REQUIRE(total < (1LL << 31), SDFT_ERR_INVALID_ARG, "multi-cell launch too large");
    SDFT_CUDA(cudaMemcpyToSymbolAsync(c_multi, probs.data(), sizeof(MultiProblem) * n, 0, cudaMemcpyHostToDevice,
                                      c0->stream));
    const size_t dsm = sizeof(Stage<float2, float, float, TX, TY, 3>) * D + sizeof(float2) * (size_t)max_natom;
    ScopedTimer timer(c0, SDFT_K_STENCIL, bytes);
    auto launch = [&](auto kfn) {
        if (dsm > 48 * 1024)
            SDFT_CUDA(cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dsm));
        kfn<<<(unsigned)total, dim3(TX, TY), dsm, c0->stream>>>(n);
    };
    if (prev) launch(cheb_multi_kernel<TX, TY, PF, MINB, D, true>);
    else launch(cheb_multi_kernel<TX, TY, PF, MINB, D, false>);
    SDFT_CUDA(cudaGetLastError());
    count_launch(c0);
}

// z chunks of one cell inside a multi-cell launch: at least 16 planes per chunk, enough CTAs overall
int multi_nzc(const sdft_ctx* c, long long ctas_other) {
    const long long want = 8LL * 152;
    const long long base = (long long)((c->n[0] + 31) / 32) * ((c->n[1] + 7) / 8) * (c->nfilt / 2);
    int nzc = 1;
    while (ctas_other + base * nzc < want && c->n[2] / (nzc + 1) >= 16) ++nzc;
    return nzc;
}

StepArgs<float> multi_args(sdft_ctx* c, double alpha, double beta, double shift, int nzc) {
    const int zchunk = (c->n[2] + nzc - 1) / nzc;
    return make_args<float>(c, 0, alpha, beta, shift, zchunk, (c->n[2] + zchunk - 1) / zchunk);
}

void chebyshev_filter_multi(const std::vector<sdft_ctx*>& ctxs, const std::vector<const void*>& X,
                            const std::vector<void*>& Y, int m, const double* a, const double* b, const double* a0) {
    const int n = (int)ctxs.size();
    SDFT_REQUIRE(m >= 1, SDFT_ERR_INVALID_ARG, "degree must be >= 1");
    // per cell: the recurrence scalars and a ring of its own block buffers (T1, T2, Y)
    std::vector<double> e(n), cc(n), sigma1(n), sigma(n);
    std::vector<std::array<float2*, 3>> ring(n);
    long long ctas = 0;
    std::vector<int> nzc(n);
    for (int i = 0; i < n; ++i) {
        sdft_ctx* c = ctxs[i];
        SDFT_REQUIRE(b[i] > a[i] && a[i] > a0[i], SDFT_ERR_INVALID_ARG, "filter bounds must satisfy a0 < a < b");
        e[i] = 0.5 * (b[i] - a[i]);
        cc[i] = 0.5 * (b[i] + a[i]);
        sigma1[i] = sigma[i] = e[i] / (a0[i] - cc[i]);
        float2* t[2];
        int got = 0;
        for (int k = 0; k < 4 && got < 2; ++k)
            if (c->blk[k] != X[i] && c->blk[k] != Y[i]) t[got++] = (float2*)c->blk[k];
        SDFT_REQUIRE(got == 2, SDFT_ERR_INVALID_ARG, "no free block buffers for the filter");
        ring[i] = {t[0], t[1], (float2*)Y[i]};
        nzc[i] = multi_nzc(c, ctas);
        ctas += (long long)((c->n[0] + 31) / 32) * ((c->n[1] + 7) / 8) * (c->nfilt / 2) * nzc[i];
    }
    auto slot = [&](int i, int k) -> float2* { return ring[i][(((2 - (m - k)) % 3) + 3) % 3]; };
    // KB projections of every (step, cell): one table, uploaded once, one grouped launch per step
    sdft_ctx* c0 = ctxs[0];
    std::vector<KBProblem> ktab;
    std::vector<int> kcell;
    int max_natom = 0, max_ncolE = 0;
    for (int i = 0; i < n; ++i) {
        const KBTables& kb = ctxs[i]->kb[0];
        if (kb.S == 0 || kb.natom == 0) continue;
        kcell.push_back(i);
        max_natom = std::max(max_natom, kb.natom);
        max_ncolE = std::max(max_ncolE, ctxs[i]->nfilt / 2);
    }
    const int nk = (int)kcell.size();
    if (nk > 0) {
        ktab.reserve((size_t)m * nk);
        for (int k = 1; k <= m; ++k)
            for (int i : kcell) {
                sdft_ctx* c = ctxs[i];
                const KBTables& kb = c->kb[0];
                const float2* cur = k == 1 ? (const float2*)X[i] : slot(i, k - 1);
                ktab.push_back(KBProblem{cur, c->C32, kb.cnt, kb.idx, kb.val32, kb.gamma, kb.cap, kb.natom,
                                         c->nfilt / 2, c->ng});
            }
        if (c0->m_ktab_cap < (int)ktab.size()) {
            c0->m_ktab = (KBProblem*)ctx_alloc(c0, sizeof(KBProblem) * ktab.size());
            c0->m_ktab_cap = (int)ktab.size();
        }
        // pageable source: the copy is staged before the call returns, so ktab may go out of scope
        SDFT_CUDA(cudaMemcpyAsync(c0->m_ktab, ktab.data(), sizeof(KBProblem) * ktab.size(), cudaMemcpyHostToDevice,
                                  c0->stream));
    }
    std::vector<MultiProblem> probs(n);
    for (int k = 1; k <= m; ++k) {
        if (nk > 0) launch_multi_project_f32(c0, c0->m_ktab + (size_t)(k - 1) * nk, nk, max_natom, max_ncolE);
        for (int i = 0; i < n; ++i) {
            sdft_ctx* c = ctxs[i];
            const float2* cur = k == 1 ? (const float2*)X[i] : slot(i, k - 1);
            const float2* prv = k == 1 ? nullptr : (k == 2 ? (const float2*)X[i] : slot(i, k - 2));
            const bool kb = c->kb[0].S > 0;
            double alpha, beta = 0.0;
            if (k == 1) {
                alpha = sigma1[i] / e[i];
            } else {
                const double s2 = 1.0 / (2.0 / sigma1[i] - sigma[i]);
                alpha = 2.0 * s2 / e[i];
                beta = sigma[i] * s2;
                sigma[i] = s2;
            }
            MultiProblem& P = probs[i];
            P.A = multi_args(c, alpha, beta, cc[i], nzc[i]);
            P.Y = cur;
            P.Yprev = prv;
            P.Ynext = slot(i, k);
            P.V = c->veff32;
            P.C = (const float2*)c->C32;
            P.patom = c->kb[0].patom;
            P.pval = c->kb[0].pval32;
            P.nslot = kb ? c->kb[0].S : 0;
        }
        launch_multi_step_f32(ctxs, probs, k > 1);
    }
}

void launch_group_project_f32(sdft_ctx* c, bool cplx, const KBProblem* grp, int nprob, int ncolE) {
    launch_project_group_impl<float2>(c, grp, nprob, ncolE, cplx);
}

void launch_multi_project_f32(sdft_ctx* c, const KBProblem* grp, int nprob, int max_natom, int max_ncolE) {
    launch_project_multi_impl<float2>(c, grp, nprob, max_natom, max_ncolE);
}

}  // namespace sdft
