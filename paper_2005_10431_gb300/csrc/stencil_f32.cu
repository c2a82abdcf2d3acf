// Instantiations of the fused stencil / Chebyshev-step kernels (see stencil_impl.cuh)
// for FP32 blocks (two lanes per element: an orbital pair, or re/im of a Bloch orbital).
#include "stencil_impl.cuh"

namespace sdft {
namespace {
// tile variants (TX x TY threads, prefetch planes, min blocks per SM) timed by the autotuner
// (TX, TY, queue prefetch PF, min blocks per SM, cp.async stages D)
const StepLauncher<float2> kReal[] = {
    &launch_variant<float2, false, 32, 8, 2, 2, 4>, &launch_variant<float2, false, 32, 8, 3, 2, 3>,
    &launch_variant<float2, false, 32, 16, 2, 1, 3>, &launch_variant<float2, false, 32, 4, 2, 4, 4>};
const StepLauncher<float2> kCplx[] = {&launch_variant<float2, true, 32, 8, 2, 2, 4>,
                                      &launch_variant<float2, true, 32, 8, 3, 2, 3>};
}  // namespace

template <>
void launch_cheb_step<float2>(sdft_ctx* c, int kpt, const float2* Y, const float2* Yprev, float2* Ynext, int ncolE,
                              const float* V, const float2* kbC, double alpha, double beta, double shift,
                              bool with_kinetic) {
    const bool cplx = c->kb[kpt].cplx;
    const StepLauncher<float2>* table = cplx ? kCplx : kReal;
    const int nvar = cplx ? 2 : 4;
    int& choice = c->stencil_choice[cplx ? 1 : 0];
    if (choice < 0)
        choice = autotune_stencil<float2>(c, table, nvar, kpt, Y, Yprev, Ynext, ncolE, V, kbC, alpha, beta, shift);
    table[choice](c, kpt, Y, Yprev, Ynext, ncolE, V, kbC, alpha, beta, shift, with_kinetic, true);
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

}  // namespace sdft
