// Instantiations of the fused stencil / Chebyshev-step kernels (see stencil_impl.cuh)
// for one element type per translation unit, so the variants compile in parallel.
#include "stencil_impl.cuh"

#include <algorithm>

namespace sdft {

namespace {
// Isolated systems (Dirichlet): the same fused step with zero values beyond the grid, one thread per
// (point, column) with direct loads (the cells of this mode are small, molecules in a box).
__global__ void __launch_bounds__(256)
cheb_step_dirichlet_kernel(const double* __restrict__ Y, const double* __restrict__ Yprev, double* __restrict__ Ynext,
                           const double* __restrict__ V, const double* __restrict__ C, const int* __restrict__ patom,
                           const double* __restrict__ pval, int nslot, int natom, int ncol,
                           const __grid_constant__ StepArgs<double> A) {
    const long long ng = A.ng;
    const int n1 = A.n1, n2 = A.n2, n3 = A.n3;
    const long long plane = (long long)n1 * n2;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)ncol * ng;
         e += (long long)gridDim.x * blockDim.x) {
        const int col = (int)(e / ng);
        const long long g = e - (long long)col * ng;
        const int k = (int)(g / plane);
        const int rem = (int)(g - k * plane);
        const int j = rem / n1, i = rem - j * n1;
        const double* y = Y + (long long)col * ng;
        const double yc = y[g];
        double ax = 0.0, ay = 0.0, az = 0.0;
#pragma unroll
        for (int r = 1; r <= FD_RADIUS; ++r) {
            ax += A.cx[r] * ((i + r < n1 ? y[g + r] : 0.0) + (i - r >= 0 ? y[g - r] : 0.0));
            ay += A.cy[r] * ((j + r < n2 ? y[g + r * n1] : 0.0) + (j - r >= 0 ? y[g - r * n1] : 0.0));
            az += A.cz[r] * ((k + r < n3 ? y[g + r * plane] : 0.0) + (k - r >= 0 ? y[g - r * plane] : 0.0));
        }
        double acc = A.c0 * yc + ax + ay + az;
        if (V) acc += V[g] * yc;
        if (C)
            for (int s = 0; s < nslot; ++s) {
                const int a = patom[(long long)s * ng + g];
                if (a >= 0) acc += pval[(long long)s * ng + g] * C[(long long)col * natom + a];
            }
        double out = A.alpha * (acc - A.shift * yc);
        if (Yprev) out -= A.beta * Yprev[(long long)col * ng + g];
        Ynext[(long long)col * ng + g] = out;
    }
}
}  // namespace

template <>
void launch_cheb_step<double>(sdft_ctx* c, int kpt, const double* Y, const double* Yprev, double* Ynext, int ncolE,
                              const double* V, const double* kbC, double alpha, double beta, double shift,
                              bool with_kinetic) {
    if (c->opt.boundary == SDFT_BC_DIRICHLET) {
        SDFT_REQUIRE(with_kinetic, SDFT_ERR_INVALID_ARG, "stencil step without kinetic term is not built");
        const KBTables& kb = c->kb[kpt];
        StepArgs<double> A = make_args<double>(c, kpt, alpha, beta, shift, c->n[2], 1);
        const long long total = (long long)ncolE * c->ng;
        const unsigned nb = (unsigned)std::min<long long>((total + 255) / 256, 152LL * 32);
        ScopedTimer timer(c, SDFT_K_STENCIL64, (double)ncolE * (double)c->ng * sizeof(double) * (Yprev ? 3.0 : 2.0));
        cheb_step_dirichlet_kernel<<<nb, 256, 0, c->stream>>>(Y, Yprev, Ynext, V, kb.S > 0 ? kbC : nullptr, kb.patom,
                                                             kb.pval64, kb.S, c->natom, ncolE, A);
        SDFT_CUDA(cudaGetLastError());
        count_launch(c);
        return;
    }
    launch_variant<double, false, 32, 8, 2, 1, 3>(c, kpt, Y, Yprev, Ynext, ncolE, V, kbC, alpha, beta, shift, with_kinetic,
                                              true);
}

template <>
void launch_kb_project<double>(sdft_ctx* c, int kpt, const double* Y, double* C, int ncolE) {
    launch_project_impl<double>(c, kpt, Y, C, ncolE);
}

}  // namespace sdft
