// Learned initial density for the SCF (the paper starts from a superposition of atomic densities,
// Sec. 2.1, and lists machine learning as future work, Sec. 4): a 32 -> 64 -> 64 -> 1 SiLU network
// on atom-centred radial descriptors predicts rho* - rho_SAD at every grid point.
//
//   G_j(x) = sum_a sum_T exp(-(r - mu_j)^2 / (2 eta^2)) f_c(r), r = |x - R_a - T| <= 6.5 bohr,
//   f_c(r) = (cos(pi r / 6.5) + 1)/2, mu_j = 6 j/31, eta = 6/31.
//
// Features are stored in BF16; the forward and backward passes use BF16-rounded weights with
// FP32 activations and accumulation; Adam keeps FP32 master weights and moments.
// Training kernel: persistent CTAs, 64-point tiles; activations of a tile live in shared memory
// and the CTA's gradient is accumulated in shared memory, then added to the global gradient once.
#include "internal.cuh"

#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>

namespace sdft {
namespace {

constexpr int NF = 32, NH = 64;
constexpr int OW1 = 0, OB1 = OW1 + NH * NF, OW2 = OB1 + NH, OB2 = OW2 + NH * NH, OW3 = OB2 + NH, OB3 = OW3 + NH;
constexpr int NP = OB3 + 1;   // 6337 parameters
constexpr int TP = 64;        // points per tile
constexpr double RC = 6.5;

__device__ __forceinline__ float silu(float z) { return z / (1.f + __expf(-z)); }
__device__ __forceinline__ float dsilu(float z) {
    const float s = 1.f / (1.f + __expf(-z));
    return s * (1.f + z * (1.f - s));
}
__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

__global__ void descriptor_kernel(const double* __restrict__ pos, int natom, int n1, int n2, int n3, double h1,
                                  double h2, double h3, double L1, double L2, double L3,
                                  __nv_bfloat16* __restrict__ feat) {
    const long long ng = (long long)n1 * n2 * n3;
    const double eta = 6.0 / 31.0;
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < ng; g += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(g % n1), j = (int)((g / n1) % n2), k = (int)(g / ((long long)n1 * n2));
        const double X[3] = {i * h1, j * h2, k * h3};
        const double L[3] = {L1, L2, L3};
        float G[NF];
#pragma unroll
        for (int q = 0; q < NF; ++q) G[q] = 0.f;
        for (int a = 0; a < natom; ++a) {
            int tlo[3], thi[3];
            for (int d = 0; d < 3; ++d) {
                tlo[d] = (int)ceil((X[d] - pos[3 * a + d] - RC) / L[d]);
                thi[d] = (int)floor((X[d] - pos[3 * a + d] + RC) / L[d]);
            }
            for (int t2 = tlo[2]; t2 <= thi[2]; ++t2)
                for (int t1 = tlo[1]; t1 <= thi[1]; ++t1)
                    for (int t0 = tlo[0]; t0 <= thi[0]; ++t0) {
                        const double dx = X[0] - pos[3 * a] - t0 * L1, dy = X[1] - pos[3 * a + 1] - t1 * L2,
                                     dz = X[2] - pos[3 * a + 2] - t2 * L3;
                        const double r = sqrt(dx * dx + dy * dy + dz * dz);
                        if (r > RC) continue;
                        const float fc = (float)(0.5 * (cos(M_PI * r / RC) + 1.0));
                        const float rf = (float)r, inv2e2 = (float)(1.0 / (2.0 * eta * eta));
#pragma unroll
                        for (int q = 0; q < NF; ++q) {
                            const float u = rf - (float)(6.0 * q / 31.0);
                            G[q] = fmaf(expf(-u * u * inv2e2), fc, G[q]);
                        }
                    }
        }
#pragma unroll
        for (int q = 0; q < NF; ++q) feat[g * NF + q] = __float2bfloat16_rn(G[q]);
    }
}

struct MlpSmem {
    float W1T[NF][NH];   // W1 transposed (bf16-rounded)
    float b1[NH];
    float W2T[NH][NH];   // W2T[g][h] = W2[h][g] (forward: thread h reads a row of W2T)
    float W2N[NH][NH];   // W2 itself (backward: thread g reads a row of W2)
    float b2[NH];
    float w3[NH];
    float b3;
    float X[TP][NF];
    float Z1[TP][NH];
    float H1[TP][NH];
    float Z2[TP][NH];
    float dy[TP];
};

// TRAIN: accumulate d(mean loss)/d(params) into grad (global, FP32) and the loss sum into loss.
// !TRAIN: y = network output.
// TRAIN visits the batch points perm((start + i) mod npts), i < nb, perm(j) = j * mult mod npts
// (mult coprime to npts); inference visits points 0 .. nb-1 in order.
template <bool TRAIN>
__global__ void __launch_bounds__(256) mlp_tile_kernel(const __nv_bfloat16* __restrict__ feat,
                                                       const float* __restrict__ target, long long npts,
                                                       long long nb, long long start, long long mult,
                                                       const float* __restrict__ params, float* __restrict__ y_out,
                                                       float* __restrict__ grad, double* __restrict__ loss,
                                                       double inv_n) {
    extern __shared__ __align__(16) unsigned char smraw[];
    MlpSmem& S = *reinterpret_cast<MlpSmem*>(smraw);
    float* gacc = reinterpret_cast<float*>(smraw + sizeof(MlpSmem));   // [NP] (TRAIN only)
    const int tid = threadIdx.x;
    for (int q = tid; q < NH * NF; q += blockDim.x) {
        const int h = q / NF, f = q - h * NF;
        S.W1T[f][h] = bf16r(params[OW1 + q]);
    }
    for (int q = tid; q < NH * NH; q += blockDim.x) {
        const int h = q / NH, g = q - h * NH;
        const float w = bf16r(params[OW2 + q]);
        S.W2T[g][h] = w;
        S.W2N[h][g] = w;
    }
    for (int q = tid; q < NH; q += blockDim.x) {
        S.b1[q] = bf16r(params[OB1 + q]);
        S.b2[q] = bf16r(params[OB2 + q]);
        S.w3[q] = bf16r(params[OW3 + q]);
    }
    if (tid == 0) S.b3 = bf16r(params[OB3]);
    if (TRAIN)
        for (int q = tid; q < NP; q += blockDim.x) gacc[q] = 0.f;
    double lsum = 0.0;
    __syncthreads();
    __shared__ long long pidx[TP];
    const long long ntile = (nb + TP - 1) / TP;
    const int h = tid & (NH - 1);   // neuron of this thread
    const int pg = tid >> 6;        // point group: points pg*16 .. pg*16+15
    for (long long tile = blockIdx.x; tile < ntile; tile += gridDim.x) {
        const long long p0 = tile * TP;
        const int np = (int)(nb - p0 < TP ? nb - p0 : TP);
        if (tid < TP) {
            long long gi = p0 + tid;
            if (TRAIN && tid < np) gi = (((start + gi) % npts) * mult) % npts;
            pidx[tid] = gi;
        }
        __syncthreads();
        for (int q = tid; q < TP * NF; q += blockDim.x) {
            const int p = q / NF;
            S.X[p][q - p * NF] = p < np ? __bfloat162float(feat[pidx[p] * NF + (q - p * NF)]) : 0.f;
        }
        __syncthreads();
        // layer 1: Z1 = X W1^T + b1
        {
            float acc[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) acc[i] = S.b1[h];
            for (int f = 0; f < NF; ++f) {
                const float w = S.W1T[f][h];
#pragma unroll
                for (int i = 0; i < 16; ++i) acc[i] = fmaf(S.X[pg * 16 + i][f], w, acc[i]);
            }
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                S.Z1[pg * 16 + i][h] = acc[i];
                S.H1[pg * 16 + i][h] = silu(acc[i]);
            }
        }
        __syncthreads();
        // layer 2: Z2 = H1 W2^T + b2
        {
            float acc[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) acc[i] = S.b2[h];
            for (int g = 0; g < NH; ++g) {
                const float w = S.W2T[g][h];
#pragma unroll
                for (int i = 0; i < 16; ++i) acc[i] = fmaf(S.H1[pg * 16 + i][g], w, acc[i]);
            }
#pragma unroll
            for (int i = 0; i < 16; ++i) S.Z2[pg * 16 + i][h] = acc[i];
        }
        __syncthreads();
        // output: y = silu(Z2) . w3 + b3 ; 4 threads per point (16 neurons each)
        {
            const int p = tid >> 2, part = tid & 3;
            float s = 0.f;
            for (int g = part * 16; g < part * 16 + 16; ++g) s = fmaf(silu(S.Z2[p][g]), S.w3[g], s);
            s += __shfl_xor_sync(0xffffffffu, s, 1);
            s += __shfl_xor_sync(0xffffffffu, s, 2);
            if (part == 0) {
                const float y = s + S.b3;
                if (!TRAIN) {
                    if (p < np) y_out[p0 + p] = y;
                } else {
                    const float e = p < np ? y - target[pidx[p]] : 0.f;
                    lsum += (double)e * e;
                    S.dy[p] = (float)(2.0 * inv_n) * e;
                }
            }
        }
        __syncthreads();
        if (TRAIN) {
            // d w3[h] = sum_p dy_p silu(Z2[p][h]);  d b3 = sum_p dy_p   (thread h < 64)
            if (tid < NH) {
                float s = 0.f;
                for (int p = 0; p < TP; ++p) s = fmaf(S.dy[p], silu(S.Z2[p][tid]), s);
                gacc[OW3 + tid] += s;
            } else if (tid == NH) {
                float s = 0.f;
                for (int p = 0; p < TP; ++p) s += S.dy[p];
                gacc[OB3] += s;
            }
            __syncthreads();
            // dZ2 = dy w3 silu'(Z2)  (in place)
            for (int q = tid; q < TP * NH; q += blockDim.x) {
                const int p = q / NH, g = q - p * NH;
                S.Z2[p][g] = S.dy[p] * S.w3[g] * dsilu(S.Z2[p][g]);
            }
            __syncthreads();
            // d W2[h][g] = sum_p dZ2[p][h] H1[p][g]; d b2[h] = sum_p dZ2[p][h]
            for (int q = tid; q < NH * NH; q += blockDim.x) {
                const int hh = q / NH, g = q - hh * NH;
                float s = 0.f;
                for (int p = 0; p < TP; ++p) s = fmaf(S.Z2[p][hh], S.H1[p][g], s);
                gacc[OW2 + q] += s;
            }
            if (tid < NH) {
                float s = 0.f;
                for (int p = 0; p < TP; ++p) s += S.Z2[p][tid];
                gacc[OB2 + tid] += s;
            }
            __syncthreads();
            // dZ1[p][g] = (sum_h dZ2[p][h] W2[h][g]) silu'(Z1[p][g])  (stored over H1)
            {
                float acc[16];
#pragma unroll
                for (int i = 0; i < 16; ++i) acc[i] = 0.f;
                const int g = h;
                for (int hh = 0; hh < NH; ++hh) {
                    const float w = S.W2N[hh][g];
#pragma unroll
                    for (int i = 0; i < 16; ++i) acc[i] = fmaf(S.Z2[pg * 16 + i][hh], w, acc[i]);
                }
                __syncthreads();
#pragma unroll
                for (int i = 0; i < 16; ++i) S.H1[pg * 16 + i][g] = acc[i] * dsilu(S.Z1[pg * 16 + i][g]);
            }
            __syncthreads();
            // d W1[h][f] = sum_p dZ1[p][h] X[p][f]; d b1[h] = sum_p dZ1[p][h]
            for (int q = tid; q < NH * NF; q += blockDim.x) {
                const int hh = q / NF, f = q - hh * NF;
                float s = 0.f;
                for (int p = 0; p < TP; ++p) s = fmaf(S.H1[p][hh], S.X[p][f], s);
                gacc[OW1 + q] += s;
            }
            if (tid < NH) {
                float s = 0.f;
                for (int p = 0; p < TP; ++p) s += S.H1[p][tid];
                gacc[OB1 + tid] += s;
            }
        }
        __syncthreads();
    }
    if (TRAIN) {
        for (int q = tid; q < NP; q += blockDim.x) atomicAdd(&grad[q], gacc[q]);
        for (int off = 16; off > 0; off >>= 1) lsum += __shfl_down_sync(0xffffffffu, lsum, off);
        if ((tid & 31) == 0) atomicAdd(loss, lsum * inv_n);
    }
}

__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, int n, float lr, float b1, float b2, float eps, float c1, float c2) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

__global__ void guess_kernel(const double* __restrict__ sad, const float* __restrict__ y, double* __restrict__ out,
                             long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = fmax(sad[i] + (double)y[i], 0.0);
}

__global__ void scale_kernel(double* __restrict__ x, const double* __restrict__ s, double nelec_over_dv, long long n) {
    const double f = nelec_over_dv / s[0];
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        x[i] *= f;
}

__global__ void sum_kernel(const double* __restrict__ x, long long n, double* __restrict__ out) {
    __shared__ double sh[32];
    double s = 0.0;
    for (long long i = threadIdx.x; i < n; i += blockDim.x) s += x[i];
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
        out[0] = t;
    }
}

__global__ void split_kernel(const double* __restrict__ rho, int nspin, double moment, double* __restrict__ out,
                             long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        if (nspin == 1) {
            out[i] = rho[i];
        } else {
            out[i] = 0.5 * rho[i] * (1.0 + moment);
            out[n + i] = 0.5 * rho[i] * (1.0 - moment);
        }
    }
}

__global__ void target_kernel(const double* __restrict__ rho, int nspin, const double* __restrict__ sad,
                              float* __restrict__ t, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        double r = rho[i];
        if (nspin == 2) r += rho[n + i];
        t[i] = (float)(r - sad[i]);
    }
}

size_t tile_smem(bool train) { return sizeof(MlpSmem) + (train ? sizeof(float) * NP : 0); }

int tile_grid(cudaStream_t) {
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    return std::max(1, nsm);
}

}  // namespace

int mlp_nparam() { return NP; }

// features of every grid point of the context's cell; target (optional) = rho_out - rho_SAD of the
// last SCF, summed over spins
void mlp_dataset(sdft_ctx* c, void* feat, float* target) {
    double* dpos = reinterpret_cast<double*>(c->work64);   // positions staged in grid scratch
    SDFT_CUDA(cudaMemcpyAsync(dpos, c->pos.data(), sizeof(double) * 3 * c->natom, cudaMemcpyHostToDevice, c->stream));
    descriptor_kernel<<<(unsigned)std::min<long long>((c->ng + 255) / 256, 152LL * 16), 256, 0, c->stream>>>(
        dpos, c->natom, c->n[0], c->n[1], c->n[2], c->h[0], c->h[1], c->h[2], c->L[0], c->L[1], c->L[2],
        reinterpret_cast<__nv_bfloat16*>(feat));
    SDFT_CUDA(cudaGetLastError());
    count_launch(c);
    if (target) {
        target_kernel<<<(unsigned)std::min<long long>((c->ng + 255) / 256, 152LL * 16), 256, 0, c->stream>>>(
            c->rho_out, c->opt.nspin, c->rho_sad, target, c->ng);
        SDFT_CUDA(cudaGetLastError());
        count_launch(c);
    }
    SDFT_CUDA(cudaStreamSynchronize(c->stream));
}

long long perm_mult(long long npts) { return npts % 1000003LL == 0 ? 999983LL : 1000003LL; }

// grad (FP32 [NP]) is overwritten; the batch's mean squared error is added to *loss (device)
void mlp_loss_grad(const void* feat, const float* target, long long npts, long long batch, long long start,
                   const float* params, float* grad, double* loss, cudaStream_t st) {
    SDFT_CUDA(cudaMemsetAsync(grad, 0, sizeof(float) * NP, st));
    const size_t sm = tile_smem(true);
    SDFT_CUDA(cudaFuncSetAttribute(mlp_tile_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    const long long ntile = (batch + TP - 1) / TP;
    const int grid = (int)std::min<long long>(ntile, tile_grid(st));
    mlp_tile_kernel<true><<<grid, 256, sm, st>>>(reinterpret_cast<const __nv_bfloat16*>(feat), target, npts, batch,
                                                  start % npts, perm_mult(npts), params, nullptr, grad, loss,
                                                  1.0 / (double)batch);
    SDFT_CUDA(cudaGetLastError());
}

void mlp_forward(const void* feat, long long npts, const float* params, float* y, cudaStream_t st) {
    const size_t sm = tile_smem(false);
    SDFT_CUDA(cudaFuncSetAttribute(mlp_tile_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    const long long ntile = (npts + TP - 1) / TP;
    const int grid = (int)std::min<long long>(ntile, 4LL * tile_grid(st));
    mlp_tile_kernel<false><<<grid, 256, sm, st>>>(reinterpret_cast<const __nv_bfloat16*>(feat), nullptr, npts, npts,
                                                   0, 1, params, y, nullptr, nullptr, 1.0);
    SDFT_CUDA(cudaGetLastError());
}

void mlp_adam(float* p, const float* g, float* m, float* v, int step, double lr, cudaStream_t st) {
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
    adam_kernel<<<(NP + 255) / 256, 256, 0, st>>>(p, g, m, v, NP, (float)lr, b1, b2, 1e-8f, c1, c2);
    SDFT_CUDA(cudaGetLastError());
}

// nsteps of mini-batch Adam; step s (counted from first_step) uses the batch starting at
// (s - 1) * batch; loss_dev[s - first_step] receives that batch's loss before the update
void mlp_train(const void* feat, const float* target, long long npts, long long batch, float* params, float* grad,
               float* m, float* v, int first_step, int nsteps, double lr, double* loss_dev, cudaStream_t st) {
    SDFT_CUDA(cudaMemsetAsync(loss_dev, 0, sizeof(double) * nsteps, st));
    for (int k = 0; k < nsteps; ++k) {
        const int step = first_step + k;
        const long long start = (long long)((((unsigned long long)(step - 1)) * (unsigned long long)batch) %
                                            (unsigned long long)npts);
        mlp_loss_grad(feat, target, npts, batch, start, params, grad, loss_dev + k, st);
        mlp_adam(params, grad, m, v, step, lr, st);
    }
}

// rho_guess = max(rho_SAD + y, 0) renormalised to N_e, split into spins, stored as the user guess
void mlp_guess(sdft_ctx* c, const float* params) {
    const long long ng = c->ng;
    if (!c->mlp_scratch) c->mlp_scratch = ctx_alloc(c, (size_t)ng * (NF * 2 + sizeof(float)));
    void* feat = c->mlp_scratch;                                              // [ng][32] bf16
    float* y = reinterpret_cast<float*>(static_cast<char*>(c->mlp_scratch) + (size_t)ng * NF * 2);
    mlp_dataset(c, feat, nullptr);
    mlp_forward(feat, ng, params, y, c->stream);
    double* g = c->work64 + 8 * ng;
    guess_kernel<<<(unsigned)std::min<long long>((ng + 255) / 256, 152LL * 16), 256, 0, c->stream>>>(c->rho_sad, y, g,
                                                                                                    ng);
    sum_kernel<<<1, 1024, 0, c->stream>>>(g, ng, c->scal + 32);
    scale_kernel<<<(unsigned)std::min<long long>((ng + 255) / 256, 152LL * 16), 256, 0, c->stream>>>(
        g, c->scal + 32, c->nelec / c->dV, ng);
    SDFT_CUDA(cudaGetLastError());
    count_launch(c, 4);
    // spin split as for the SAD guess; the guess becomes the user density of the next SCF
    split_kernel<<<(unsigned)std::min<long long>((ng + 255) / 256, 152LL * 16), 256, 0, c->stream>>>(
        g, c->opt.nspin, c->opt.initial_moment, c->rho_user, ng);
    SDFT_CUDA(cudaGetLastError());
    count_launch(c);
    SDFT_CUDA(cudaMemcpyAsync(c->rho_in, c->rho_user, sizeof(double) * c->opt.nspin * ng, cudaMemcpyDeviceToDevice,
                              c->stream));
    c->user_density = true;
    SDFT_CUDA(cudaStreamSynchronize(c->stream));
}

}  // namespace sdft
