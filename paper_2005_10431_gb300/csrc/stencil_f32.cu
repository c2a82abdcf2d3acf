// Instantiations of the fused stencil / Chebyshev-step kernels (see stencil_impl.cuh)
// for FP32 blocks (two lanes per element: an orbital pair, or re/im of a Bloch orbital).
#include "stencil_impl.cuh"

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
void launch_cheb_step<float2>(sdft_ctx* c, int kpt, const float2* Y, const float2* Yprev, float2* Ynext, int ncolE,
                              const float* V, const float2* kbC, double alpha, double beta, double shift,
                              bool with_kinetic) {
    const bool cplx = c->kb[kpt].cplx;
    const StepVariant<float2>* table = cplx ? kCplx : kReal;
    const int nvar = cplx ? kNCplx : kNReal;
    int& choice = c->stencil_choice[cplx ? 1 : 0];
    int pick = choice;
    if (pick < 0) {
        pick = autotune_stencil<float2>(c, table, nvar, kpt, Y, Yprev, Ynext, ncolE, V, kbC, alpha, beta, shift);
        if (pick >= 0) choice = pick;   // small calls are not timed and do not fix the choice
        else pick = 0;
    }
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

template <>
void launch_kb_project<float2>(sdft_ctx* c, int kpt, const float2* Y, float2* C, int ncolE) {
    launch_project_impl<float2>(c, kpt, Y, C, ncolE);
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

void launch_group_project_f32(sdft_ctx* c, bool cplx, const KBProblem* grp, int nprob, int ncolE) {
    launch_project_group_impl<float2>(c, grp, nprob, ncolE, cplx);
}

}  // namespace sdft
