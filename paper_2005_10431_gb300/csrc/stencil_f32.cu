// Instantiations of the fused stencil / Chebyshev-step kernels (see stencil_impl.cuh)
// for one element type per translation unit, so the variants compile in parallel.
#include "stencil_impl.cuh"

namespace sdft {

template <>
void launch_cheb_step<float2>(sdft_ctx* c, int kpt, const float2* Y, const float2* Yprev, float2* Ynext, int ncolE,
                              const float* V, const float2* kbC, double alpha, double beta, double shift,
                              bool with_kinetic) {
    if (c->kb[kpt].cplx)
        launch_variant<float2, true, 32, 8, 2>(c, kpt, Y, Yprev, Ynext, ncolE, V, kbC, alpha, beta, shift, with_kinetic);
    else
        launch_variant<float2, false, 32, 8, 2>(c, kpt, Y, Yprev, Ynext, ncolE, V, kbC, alpha, beta, shift, with_kinetic);
}

template <>
void launch_kb_project<float2>(sdft_ctx* c, int kpt, const float2* Y, float2* C, int ncolE) {
    launch_project_impl<float2>(c, kpt, Y, C, ncolE);
}

}  // namespace sdft
