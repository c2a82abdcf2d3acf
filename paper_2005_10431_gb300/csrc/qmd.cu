// Moving atoms between SCF runs and the extrapolated starting point of the next SCF (paper Sec. 2.1:
// in quantum molecular dynamics the density guess of later MD steps is extrapolated from earlier
// steps; the cited scheme is D. Alfe, Comput. Phys. Commun. 118 (1999) 31).
//
// After every SCF the context keeps, for its last three runs, the positions R_i and the density
// correction Delta_i = rho_out - rho_SAD(R_i) (spin-split as the SAD guess is).  For new positions R
// the coefficients (alpha, beta) fit the new displacement by the two previous ones,
//     R - R_0 ~ alpha (R_0 - R_1) + beta (R_1 - R_2)        (least squares, minimum-image differences),
// and the same combination moves the density correction:
//     rho = rho_SAD(R) + Delta_0 + alpha (Delta_0 - Delta_1) + beta (Delta_1 - Delta_2),
// clamped at zero and renormalised to N_e.  The orbitals and filter bounds of the last SCF are kept
// as the starting subspace (the upper bound is refreshed by Lanczos for the moved atoms).
#include "internal.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>

namespace sdft {
namespace {

__global__ void sad_split_kernel(const double* __restrict__ sad, int nspin, double moment, double* __restrict__ out,
                                 long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        if (nspin == 1) {
            out[i] = sad[i];
        } else {
            out[i] = 0.5 * sad[i] * (1.0 + moment);
            out[n + i] = 0.5 * sad[i] * (1.0 - moment);
        }
    }
}

__global__ void diff_kernel(const double* __restrict__ a, const double* b, double* out, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = a[i] - b[i];
}

__global__ void fill_kernel(double* __restrict__ out, double v, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = v;
}

// out = base + sum_k coef[k] * D_k (k < count), then max(out, 0); n = nspin * ng
__global__ void extrapolate_kernel(const double* __restrict__ base, const double* __restrict__ d0,
                                   const double* __restrict__ d1, const double* __restrict__ d2, double c0, double c1,
                                   double c2, double* __restrict__ out, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        double v = base[i];
        if (d0) v += c0 * d0[i];
        if (d1) v += c1 * d1[i];
        if (d2) v += c2 * d2[i];
        out[i] = v > 0.0 ? v : 0.0;
    }
}

inline unsigned nbk(long long n) { return (unsigned)std::min<long long>((n + 255) / 256, 152LL * 16); }

double min_image(double d, double L) { return d - L * std::nearbyint(d / L); }

}  // namespace

// Alfe coefficients from the newest-first history of positions (count <= 3 entries)
void alfe_coefficients(const sdft_ctx* c, const double* R, const std::vector<const double*>& hist, double* alpha,
                       double* beta) {
    *alpha = 0.0;
    *beta = 0.0;
    const int na3 = 3 * c->natom;
    if (hist.size() < 2) return;
    std::vector<double> dn(na3), d1(na3), d2(na3);
    for (int i = 0; i < na3; ++i) {
        const double L = c->L[i % 3];
        dn[i] = min_image(R[i] - hist[0][i], L);
        d1[i] = min_image(hist[0][i] - hist[1][i], L);
        d2[i] = hist.size() >= 3 ? min_image(hist[1][i] - hist[2][i], L) : 0.0;
    }
    double a11 = 0, a12 = 0, a22 = 0, b1 = 0, b2 = 0;
    for (int i = 0; i < na3; ++i) {
        a11 += d1[i] * d1[i];
        a12 += d1[i] * d2[i];
        a22 += d2[i] * d2[i];
        b1 += dn[i] * d1[i];
        b2 += dn[i] * d2[i];
    }
    if (a11 <= 0.0) return;
    const double det = a11 * a22 - a12 * a12;
    if (hist.size() >= 3 && det > 1e-12 * a11 * a22) {
        *alpha = (b1 * a22 - b2 * a12) / det;
        *beta = (a11 * b2 - a12 * b1) / det;
    } else {
        *alpha = b1 / a11;   // two past runs, or collinear displacements: one term
    }
}

// record rho_out - rho_SAD(R) and R of the SCF that just finished (ring of three)
void push_scf_history(sdft_ctx* c) {
    const long long nv = (long long)c->opt.nspin * c->ng;
    if (!c->hist_drho) c->hist_drho = (double*)ctx_alloc(c, sizeof(double) * 3 * (size_t)nv);
    double* slot = c->hist_drho + (long long)c->hist_head * nv;
    sad_split_kernel<<<nbk(c->ng), 256, 0, c->stream>>>(c->rho_sad, c->opt.nspin, c->opt.initial_moment, slot, c->ng);
    diff_kernel<<<nbk(nv), 256, 0, c->stream>>>(c->rho_out, slot, slot, nv);
    SDFT_CUDA(cudaGetLastError());
    count_launch(c, 2);
    c->hist_pos[c->hist_head] = c->pos;
    c->hist_head = (c->hist_head + 1) % 3;
    c->hist_count = std::min(c->hist_count + 1, 3);
}

void move_atoms(sdft_ctx* c, const double* pos, int guess) {
    const int na3 = 3 * c->natom;
    c->pos.assign(pos, pos + na3);
    // geometry-dependent fields: pseudocharge and SAD density, KB tables, overlap energies
    build_pseudocharge_and_sad(c);
    for (size_t k = 0; k < c->kb.size(); ++k) {
        release_kb_tables(c, (int)k);
        build_kb_tables(c, (int)k);
    }
    host_energy_constants(c);
    c->mix_k = 0;
    c->mix_count = 0;
    c->mix_head = 0;
    c->log.clear();
    if (guess == 0 || c->hist_count == 0) {
        c->user_density = false;
        c->warm_start = false;
        reset_state(c);
        return;
    }
    // newest-first history
    std::vector<const double*> hp;
    std::vector<const double*> hd;
    const long long nv = (long long)c->opt.nspin * c->ng;
    for (int i = 0; i < c->hist_count; ++i) {
        const int slot = ((c->hist_head - 1 - i) % 3 + 3) % 3;
        hp.push_back(c->hist_pos[slot].data());
        hd.push_back(c->hist_drho + (long long)slot * nv);
    }
    double alpha = 0.0, beta = 0.0;
    alfe_coefficients(c, pos, hp, &alpha, &beta);
    c->last_alfe[0] = alpha;
    c->last_alfe[1] = beta;
    // rho = rho_SAD(R) + (1 + alpha) D0 + (beta - alpha) D1 - beta D2, clamped, renormalised
    double* base = c->work64;
    sad_split_kernel<<<nbk(c->ng), 256, 0, c->stream>>>(c->rho_sad, c->opt.nspin, c->opt.initial_moment, base, c->ng);
    extrapolate_kernel<<<nbk(nv), 256, 0, c->stream>>>(base, hd[0], hd.size() > 1 ? hd[1] : nullptr,
                                                       hd.size() > 2 ? hd[2] : nullptr, 1.0 + alpha, beta - alpha,
                                                       -beta, c->rho_user, nv);
    SDFT_CUDA(cudaGetLastError());
    count_launch(c, 2);
    {   // renormalise to N_e: dV * sum over spins and points = N_e
        double* ones = c->work64 + 2 * c->ng;
        fill_kernel<<<nbk(nv), 256, 0, c->stream>>>(ones, 1.0, nv);
        count_launch(c);
        const double* a[1] = {c->rho_user};
        const double* b[1] = {ones};
        double s = 0.0;
        dots_host(c, 1, a, b, nv, &s);
        SDFT_REQUIRE(std::isfinite(s) && s > 0.0, SDFT_ERR_NONFINITE, "extrapolated density has no electrons");
        axpby_dev(c, c->rho_user, c->rho_user, 0.0, c->nelec / (c->dV * s), nv);
    }
    SDFT_CUDA(cudaMemcpyAsync(c->rho_in, c->rho_user, sizeof(double) * nv, cudaMemcpyDeviceToDevice, c->stream));
    c->user_density = true;
    c->warm_start = true;
    // the kept orbitals start the filter; refresh the spectrum's upper bound for the moved atoms
    for (Problem& P : c->probs) {
        if (!P.have_bounds) continue;
        double lo, up;
        lanczos(c, P.spin, P.kpt, c->opt.lanczos_steps, &lo, &up);
        P.upper = std::max(P.upper, up);
    }
    SDFT_CUDA(cudaStreamSynchronize(c->stream));
}

}  // namespace sdft
