// Instantiations of the fused stencil / Chebyshev-step kernels (see stencil_impl.cuh)
// for one element type per translation unit, so the variants compile in parallel.
#include "stencil_impl.cuh"

namespace sdft {

template <>
void launch_cheb_step<double2>(sdft_ctx* c, int kpt, const double2* Y, const double2* Yprev, double2* Ynext, int ncolE,
                               const double* V, const double2* kbC, double alpha, double beta, double shift,
                               bool with_kinetic) {
    launch_variant<double2, true, 32, 8, 2, 1, 3>(c, kpt, Y, Yprev, Ynext, ncolE, V, kbC, alpha, beta, shift, with_kinetic,
                                              true);
}

template <>
void launch_kb_project<double2>(sdft_ctx* c, int kpt, const double2* Y, double2* C, int ncolE) {
    launch_project_impl<double2>(c, kpt, Y, C, ncolE);
}

}  // namespace sdft
