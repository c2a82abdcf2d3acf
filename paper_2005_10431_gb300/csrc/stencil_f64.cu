// Instantiations of the fused stencil / Chebyshev-step kernels (see stencil_impl.cuh)
// for one element type per translation unit, so the variants compile in parallel.
#include "stencil_impl.cuh"

namespace sdft {

template <>
void launch_cheb_step<double>(sdft_ctx* c, int kpt, const double* Y, const double* Yprev, double* Ynext, int ncolE,
                              const double* V, const double* kbC, double alpha, double beta, double shift,
                              bool with_kinetic) {
    launch_variant<double, false, 32, 8, 2, 1, 3>(c, kpt, Y, Yprev, Ynext, ncolE, V, kbC, alpha, beta, shift, with_kinetic,
                                              true);
}

template <>
void launch_kb_project<double>(sdft_ctx* c, int kpt, const double* Y, double* C, int ncolE) {
    launch_project_impl<double>(c, kpt, Y, C, ncolE);
}

}  // namespace sdft
