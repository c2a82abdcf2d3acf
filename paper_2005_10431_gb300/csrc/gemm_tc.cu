// Subspace Gram matrices of Rayleigh-Ritz on the 5th-generation tensor cores (paper Sec. 2.1
// CheFSI; Sec. 4 names the subspace work as the step that dominates at scale):
//   M = Y^T Y,  Hs = Y^T (H Y)   for FP32 orbital blocks (paired layout), ncol up to ~1000,
// as BF16x3 split products  a*b ~ hi(a)hi(b) + hi(a)lo(b) + lo(a)hi(b),  hi = bf16(a),
// lo = bf16(a - hi), accumulated in FP32 in tensor memory (TMEM).
//
// One CTA = one 128 x 128 tile pair (i, j >= i) of the output and one split of the grid (the
// contraction index, up to ~1.7 M points).  All 256 threads stream FP32 Y / HY from HBM, split
// every value into bf16 hi and lo and store them into K-major, 128-byte-swizzled shared-memory
// tiles (two stages); thread 0 issues tcgen05.mma (M=128, N=128, K=16) for both products and
// tracks completion with tcgen05.commit on an mbarrier.  The epilogue reads the two FP32
// accumulators with tcgen05.ld and writes per-split partial tiles that a second kernel sums in
// FP64.  Every mbarrier wait is bounded: on timeout the kernel sets an error flag and returns.
#include "internal.cuh"

#include <cuda_bf16.h>

#include <algorithm>
#include <cstdlib>
#include <vector>

namespace sdft {
namespace {

constexpr int TC_M = 128;          // rows of a tile (orbitals i)
constexpr int TC_N = 128;          // columns of a tile (orbitals j)
constexpr int TC_K = 64;           // grid points per stage (one 128-byte swizzle row of bf16)
constexpr int TILE_BYTES = TC_M * TC_K * 2;  // one bf16 operand tile: 16 KB
constexpr int NSTAGE = 2;
// per stage: A hi/lo, B hi/lo (Y_j), C hi/lo (HY_j)
constexpr int STAGE_BYTES = 6 * TILE_BYTES;
constexpr long long WAIT_LIMIT = 1LL << 26;  // try_wait polls before giving up

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(su32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    for (long long i = 0; i < WAIT_LIMIT; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// ---- tcgen05 wrappers ------------------------------------------------------------------
__device__ __forceinline__ void tmem_alloc(uint32_t* dst_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(dst_smem)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar))
                 : "memory");
}
__device__ __forceinline__ void fence_after_sync() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_before_sync() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// 32 lanes x 32 bit, 8 consecutive columns per thread
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float* v) {
    uint32_t r[8];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

// Shared-memory matrix descriptor, K-major tile with 128-byte swizzle: 8-row groups of 1024 B
// (stride byte offset 1024), descriptor version 1, layout type SWIZZLE_128B (2).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)(1) << 16;                 // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)((1024 >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;                   // descriptor version
    d |= (uint64_t)2 << 61;                   // SWIZZLE_128B
    return d;
}
// Instruction descriptor, kind::f16: FP32 accumulator, BF16 A and B, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// byte offset of element (r, k) of a [rows x 64] bf16 K-major SW128 tile
__device__ __forceinline__ uint32_t sw128_off(int r, int k) {
    return (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((((k >> 3) ^ (r & 7)) & 7) << 4) + (k & 7) * 2);
}

__device__ __forceinline__ void split_bf16(float x, __nv_bfloat16& hi, __nv_bfloat16& lo) {
    hi = __float2bfloat16_rn(x);
    lo = __float2bfloat16_rn(x - __bfloat162float(hi));
}

// Gram operand tiles [128 orbitals x 64 points] of the paired FP32 layout: the global loads of a
// tile's items go to registers first (all tiles of a stage are requested before any is converted,
// and the next stage is requested while the current one's MMAs run), then the values are split
// into bf16 hi/lo and stored.  Items: 2 per thread (256 threads, 64 orbital pairs x 8 chunks).
constexpr int TC_ITEMS = (TC_M / 2) * (TC_K / 8) / 256;

struct TileRegs {
    float4 v[TC_ITEMS][4];   // 8 float2 (orbital pair, 8 consecutive points) per item
};

__device__ __forceinline__ void load_tile(const float* __restrict__ Y, long long ng, int ncol, int row0,
                                          long long g0, long long g1, TileRegs& R) {
#pragma unroll
    for (int it = 0; it < TC_ITEMS; ++it) {
        const int item = threadIdx.x + it * 256;
        const int pr = item / (TC_K / 8);
        const int ch = item - pr * (TC_K / 8);
        const int orb = row0 + 2 * pr;
        const long long gs = g0 + ch * 8;
        const float2* src = reinterpret_cast<const float2*>(Y) + ((long long)(orb >> 1) * ng + gs);
        // 16-byte loads need an even ngrid (gs is a multiple of 8, the column offset (orb/2) ngrid)
        const bool vec = (ng & 1) == 0;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (orb < ncol) {
                if (vec && gs + 2 * q + 1 < g1) {
                    v = __ldg(reinterpret_cast<const float4*>(src + 2 * q));
                } else {
                    float2 w0 = make_float2(0.f, 0.f), w1 = make_float2(0.f, 0.f);
                    if (gs + 2 * q < g1) w0 = __ldg(src + 2 * q);
                    if (gs + 2 * q + 1 < g1) w1 = __ldg(src + 2 * q + 1);
                    v = make_float4(w0.x, w0.y, w1.x, w1.y);
                }
            }
            R.v[it][q] = v;
        }
    }
}

__device__ __forceinline__ void store_tile(const TileRegs& R, unsigned char* hi_tile, unsigned char* lo_tile) {
#pragma unroll
    for (int it = 0; it < TC_ITEMS; ++it) {
        const int item = threadIdx.x + it * 256;
        const int pr = item / (TC_K / 8);
        const int ch = item - pr * (TC_K / 8);
        const int r0 = 2 * pr;
        __align__(16) __nv_bfloat16 h0[8], l0[8], h1[8], l1[8];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float4 v = R.v[it][q];
            split_bf16(v.x, h0[2 * q], l0[2 * q]);
            split_bf16(v.y, h1[2 * q], l1[2 * q]);
            split_bf16(v.z, h0[2 * q + 1], l0[2 * q + 1]);
            split_bf16(v.w, h1[2 * q + 1], l1[2 * q + 1]);
        }
        *reinterpret_cast<uint4*>(hi_tile + sw128_off(r0, ch * 8)) = *reinterpret_cast<uint4*>(h0);
        *reinterpret_cast<uint4*>(lo_tile + sw128_off(r0, ch * 8)) = *reinterpret_cast<uint4*>(l0);
        *reinterpret_cast<uint4*>(hi_tile + sw128_off(r0 + 1, ch * 8)) = *reinterpret_cast<uint4*>(h1);
        *reinterpret_cast<uint4*>(lo_tile + sw128_off(r0 + 1, ch * 8)) = *reinterpret_cast<uint4*>(l1);
    }
}

struct TilePair {
    int ti, tj;
};

// grid: (tile pairs, splits); 256 threads; dynamic smem NSTAGE * STAGE_BYTES + 2 KB
__global__ void __launch_bounds__(256, 1)
gram_tc_kernel(const float* __restrict__ Y, const float* __restrict__ HY, int ncol, long long ng, long long chunk,
               const TilePair* __restrict__ pairs, float* __restrict__ part, int* __restrict__ err) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // align by offsetting the array itself (not through an integer cast): accesses stay shared-memory ones
    unsigned char* smem = smem_raw + ((1024u - ((unsigned)__cvta_generic_to_shared(smem_raw) & 1023u)) & 1023u);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + NSTAGE * STAGE_BYTES);   // one per stage
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + NSTAGE);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const TilePair tp = pairs[blockIdx.x];
    const int row_i = tp.ti * TC_M, row_j = tp.tj * TC_N;
    const long long g0 = blockIdx.y * chunk;
    const long long g1 = min(ng, g0 + chunk);
    const int ntile = (int)((g1 - g0 + TC_K - 1) / TC_K);

    if (threadIdx.x == 0) {
        for (int s = 0; s < NSTAGE; ++s) mbar_init(&bars[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tmem_alloc(tmem_slot, 256);   // columns [0,128): M tile, [128,256): Hs tile
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = *tmem_slot;
    // one MMA computes both accumulators: A (Y_i) against the stacked 256-row operand [Y_j; HY_j]
    constexpr uint32_t idesc = idesc_bf16(TC_M, 2 * TC_N);
    bool ok = true;

    TileRegs ra, rb, rc;   // the next stage's operands, requested one stage ahead
    auto load_stage = [&](int t) {
        const long long gt = g0 + (long long)t * TC_K;
        load_tile(Y, ng, ncol, row_i, gt, g1, ra);
        load_tile(Y, ng, ncol, row_j, gt, g1, rb);
        load_tile(HY, ng, ncol, row_j, gt, g1, rc);
    };
    if (ntile > 0) load_stage(0);
    for (int t = 0; t < ntile; ++t) {
        const int s = t % NSTAGE;
        unsigned char* st = smem + s * STAGE_BYTES;
        // stage: A hi, A lo, then [B hi; C hi] and [B lo; C lo] as 256-row K-major operands
        unsigned char *a_hi = st, *a_lo = st + TILE_BYTES, *b_hi = st + 2 * TILE_BYTES, *c_hi = st + 3 * TILE_BYTES;
        unsigned char *b_lo = st + 4 * TILE_BYTES, *c_lo = st + 5 * TILE_BYTES;
        // the MMAs that read this stage two tiles ago must be complete before it is refilled
        if (t >= NSTAGE) {
            // the outcome is made block-uniform, so that every thread takes the same path through the
            // barriers below (a thread that timed out must not leave while others wait for it)
            const bool waited = mbar_wait(&bars[s], (uint32_t)(((t - NSTAGE) / NSTAGE) & 1));
            if (!__syncthreads_and(waited)) {
                ok = false;
                break;
            }
        }
        store_tile(ra, a_hi, a_lo);
        store_tile(rb, b_hi, b_lo);
        store_tile(rc, c_hi, c_lo);
        fence_proxy_async_smem();
        __syncthreads();
        if (threadIdx.x == 0) {
            fence_after_sync();
            const uint32_t ah = su32(a_hi), al = su32(a_lo);
            const uint32_t bch = su32(b_hi), bcl = su32(b_lo);   // [B; C] hi and lo, 256 rows each
#pragma unroll
            for (int kk = 0; kk < TC_K / 16; ++kk) {
                const uint32_t ko = kk * 32;  // 16 bf16 = 32 bytes along the swizzled row
                const uint32_t acc0 = (t > 0 || kk > 0) ? 1u : 0u;
                // [M | Hs] += Ahi [B;C]hi^T + Ahi [B;C]lo^T + Alo [B;C]hi^T   (TMEM columns 0..255)
                mma_bf16(tmem, sw128_desc(ah + ko), sw128_desc(bch + ko), idesc, acc0);
                mma_bf16(tmem, sw128_desc(ah + ko), sw128_desc(bcl + ko), idesc, 1u);
                mma_bf16(tmem, sw128_desc(al + ko), sw128_desc(bch + ko), idesc, 1u);
            }
            mma_commit(&bars[s]);
        }
        if (t + 1 < ntile) load_stage(t + 1);   // in flight while this stage's MMAs run
    }
    // drain: wait for the last commit of every stage that was used
    if (ok) {
        for (int t = std::max(0, ntile - NSTAGE); t < ntile; ++t) {
            const int s = t % NSTAGE;
            if (!mbar_wait(&bars[s], (uint32_t)((t / NSTAGE) & 1))) ok = false;
        }
    }
    fence_after_sync();
    ok = __syncthreads_and(ok) != 0;   // block-uniform: the error path below is taken by all threads or none
    if (!ok) {
        if (threadIdx.x == 0) atomicExch(err, 1);
        // bounded second wait for MMAs still in flight before the tensor memory is released
        for (int s = 0; s < NSTAGE; ++s)
            for (int par = 0; par < 2; ++par) mbar_wait(&bars[s], par);
        __syncthreads();
        if (warp == 0) tmem_dealloc(tmem, 256);
        return;
    }
    // epilogue: warps 0-3 read rows 32w..32w+31 of both accumulators (TMEM lanes = rows)
    const long long nn = (long long)ncol * ncol;
    float* pm = part + (long long)blockIdx.y * 2 * nn;
    float* ph = pm + nn;
    if (warp < 4 && ntile > 0) {
        const int row = 32 * warp + lane;
        const int gi = row_i + row;
        for (int c0 = 0; c0 < TC_N; c0 += 8) {
            float vm[8], vh[8];
            const uint32_t lane_base = (uint32_t)(32 * warp) << 16;
            tmem_ld8(tmem + lane_base + c0, vm);
            tmem_ld8(tmem + lane_base + 128 + c0, vh);
            if (gi < ncol) {
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const int gj = row_j + c0 + e;
                    if (gj < ncol && gj >= gi) {
                        pm[(long long)gi + (long long)gj * ncol] = vm[e];
                        ph[(long long)gi + (long long)gj * ncol] = vh[e];
                    }
                }
            }
        }
    }
    fence_before_sync();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, 256);
}

// sum FP32 partials over splits in FP64 (upper triangle) and mirror
__global__ void gram_tc_reduce_kernel(const float* __restrict__ part, int nsplit, int ncol, double* __restrict__ M,
                                      double* __restrict__ Hs) {
    const long long nn = (long long)ncol * ncol;
    for (long long o = blockIdx.x * (long long)blockDim.x + threadIdx.x; o < nn; o += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(o % ncol), j = (int)(o / ncol);
        if (j < i) continue;
        double m = 0.0, h = 0.0;
        for (int s = 0; s < nsplit; ++s) {
            m += (double)part[(long long)s * 2 * nn + o];
            h += (double)part[(long long)s * 2 * nn + nn + o];
        }
        const long long ot = (long long)j + (long long)i * ncol;
        M[o] = m;
        M[ot] = m;
        Hs[o] = h;
        Hs[ot] = h;
    }
}

// ---------------------------------------------------------------------------------------
// Rotation X = Y Q on the tensor cores (BF16x3, FP32 accumulation):
//   D[128 grid points][128 orbitals j] = sum_k Y[g][k] Q[k][j]  (A = Y tile, B[j][k] = Q[k][j]).
// The producer transposes the paired-layout Y tile into a K-major (orbital-contiguous) swizzled
// tile; Q (FP64, column-major) is K-major as stored.  grid = (grid-point tiles, j tiles).
// ---------------------------------------------------------------------------------------
constexpr int ROT_STAGE_BYTES = 4 * TILE_BYTES;   // A hi/lo, B hi/lo

// A tile: rows = grid points g0.. (128), k = orbitals k0..k0+63 of the paired layout (a work item
// = one grid point x 16 consecutive orbitals); B tile: rows = output orbitals j0.. (128),
// k = input orbitals: B[j][k] = Q[k + j n].  Both are staged inside the kernel's main loop.
__global__ void __launch_bounds__(256, 1)
rotate_tc_kernel(const float* __restrict__ Y, const float* __restrict__ Q32, float* __restrict__ X, int ncol,
                 long long ng, int* __restrict__ err) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // align by offsetting the array itself (not through an integer cast): accesses stay shared-memory ones
    unsigned char* smem = smem_raw + ((1024u - ((unsigned)__cvta_generic_to_shared(smem_raw) & 1023u)) & 1023u);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + NSTAGE * ROT_STAGE_BYTES);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + NSTAGE);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long g0 = (long long)blockIdx.x * TC_M;
    const int j0 = blockIdx.y * TC_N;
    const int nk = (ncol + TC_K - 1) / TC_K;
    if (threadIdx.x == 0) {
        for (int s = 0; s < NSTAGE; ++s) mbar_init(&bars[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tmem_alloc(tmem_slot, 128);
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = *tmem_slot;
    constexpr uint32_t idesc = idesc_bf16(TC_M, TC_N);
    bool ok = true;
    // operands of the next stage, requested one stage ahead (in flight while the MMAs run)
    constexpr int NA = TC_M * (TC_K / 16) / 256, NB = TC_N * (TC_K / 8) / 256;
    float2 va[NA][8];
    float vb[NB][8];
    auto load_stage = [&](int t) {
        const int k0 = t * TC_K;
#pragma unroll
        for (int it = 0; it < NA; ++it) {
            const int item = threadIdx.x + it * 256;
            const int r = item % TC_M, q = item / TC_M;
            const long long g = g0 + r;
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int k = k0 + 16 * q + 2 * e;
                va[it][e] = (g < ng && k < ncol)
                                ? __ldg(reinterpret_cast<const float2*>(Y) + ((long long)(k >> 1) * ng + g))
                                : make_float2(0.f, 0.f);
            }
        }
#pragma unroll
        for (int it = 0; it < NB; ++it) {
            const int item = threadIdx.x + it * 256;
            const int r = item / (TC_K / 8), ch = item - r * (TC_K / 8);
            const int j = j0 + r;
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int k = k0 + ch * 8 + e;
                vb[it][e] = (j < ncol && k < ncol) ? __ldg(Q32 + (long long)k + (long long)j * ncol) : 0.f;
            }
        }
    };
    if (nk > 0) load_stage(0);
    for (int t = 0; t < nk; ++t) {
        const int s = t % NSTAGE;
        unsigned char* st = smem + s * ROT_STAGE_BYTES;
        unsigned char *a_hi = st, *a_lo = st + TILE_BYTES, *b_hi = st + 2 * TILE_BYTES, *b_lo = st + 3 * TILE_BYTES;
        if (t >= NSTAGE) {
            // the outcome is made block-uniform, so that every thread takes the same path through the
            // barriers below (a thread that timed out must not leave while others wait for it)
            const bool waited = mbar_wait(&bars[s], (uint32_t)(((t - NSTAGE) / NSTAGE) & 1));
            if (!__syncthreads_and(waited)) {
                ok = false;
                break;
            }
        }
        {
#pragma unroll
            for (int it = 0; it < NA; ++it) {
                const int item = threadIdx.x + it * 256;
                const int r = item % TC_M, q = item / TC_M;
                __align__(16) __nv_bfloat16 h[16], l[16];
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    split_bf16(va[it][e].x, h[2 * e], l[2 * e]);
                    split_bf16(va[it][e].y, h[2 * e + 1], l[2 * e + 1]);
                }
                *reinterpret_cast<uint4*>(a_hi + sw128_off(r, 16 * q)) = *reinterpret_cast<uint4*>(h);
                *reinterpret_cast<uint4*>(a_hi + sw128_off(r, 16 * q + 8)) = *reinterpret_cast<uint4*>(h + 8);
                *reinterpret_cast<uint4*>(a_lo + sw128_off(r, 16 * q)) = *reinterpret_cast<uint4*>(l);
                *reinterpret_cast<uint4*>(a_lo + sw128_off(r, 16 * q + 8)) = *reinterpret_cast<uint4*>(l + 8);
            }
#pragma unroll
            for (int it = 0; it < NB; ++it) {
                const int item = threadIdx.x + it * 256;
                const int r = item / (TC_K / 8), ch = item - r * (TC_K / 8);
                __align__(16) __nv_bfloat16 h[8], l[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) split_bf16(vb[it][e], h[e], l[e]);
                *reinterpret_cast<uint4*>(b_hi + sw128_off(r, ch * 8)) = *reinterpret_cast<uint4*>(h);
                *reinterpret_cast<uint4*>(b_lo + sw128_off(r, ch * 8)) = *reinterpret_cast<uint4*>(l);
            }
        }
        fence_proxy_async_smem();
        __syncthreads();
        if (threadIdx.x == 0) {
            fence_after_sync();
            const uint32_t ah = su32(a_hi), al = su32(a_lo), bh = su32(b_hi), bl = su32(b_lo);
#pragma unroll
            for (int kk = 0; kk < TC_K / 16; ++kk) {
                const uint32_t ko = kk * 32;
                mma_bf16(tmem, sw128_desc(ah + ko), sw128_desc(bh + ko), idesc, (t > 0 || kk > 0) ? 1u : 0u);
                mma_bf16(tmem, sw128_desc(ah + ko), sw128_desc(bl + ko), idesc, 1u);
                mma_bf16(tmem, sw128_desc(al + ko), sw128_desc(bh + ko), idesc, 1u);
            }
            mma_commit(&bars[s]);
        }
        if (t + 1 < nk) load_stage(t + 1);
    }
    if (ok) {
        for (int t = std::max(0, nk - NSTAGE); t < nk; ++t) {
            const int s = t % NSTAGE;
            if (!mbar_wait(&bars[s], (uint32_t)((t / NSTAGE) & 1))) ok = false;
        }
    }
    fence_after_sync();
    ok = __syncthreads_and(ok) != 0;   // block-uniform: the error path below is taken by all threads or none
    if (!ok) {
        if (threadIdx.x == 0) atomicExch(err, 1);
        for (int s = 0; s < NSTAGE; ++s)
            for (int par = 0; par < 2; ++par) mbar_wait(&bars[s], par);
        __syncthreads();
        if (warp == 0) tmem_dealloc(tmem, 128);
        return;
    }
    // epilogue: row = grid point, 8 orbitals per tcgen05.ld; store pairs into the paired layout
    if (warp < 4) {
        const long long g = g0 + 32 * warp + lane;
        const uint32_t lane_base = (uint32_t)(32 * warp) << 16;
        for (int c0 = 0; c0 < TC_N; c0 += 8) {
            float v[8];
            tmem_ld8(tmem + lane_base + c0, v);
            if (g < ng) {
#pragma unroll
                for (int e = 0; e < 8; e += 2) {
                    const int j = j0 + c0 + e;
                    if (j < ncol)
                        reinterpret_cast<float2*>(X)[(long long)(j >> 1) * ng + g] = make_float2(v[e], v[e + 1]);
                }
            }
        }
    }
    fence_before_sync();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, 128);
}

}  // namespace



// X = Y Q for FP32 paired blocks; Q32 is Q in FP32, column-major ncol x ncol
void rotate_tc(sdft_ctx* c, const void* Y, const float* Q32, void* X, int ncol) {
    int* derr = reinterpret_cast<int*>(c->scal + 5);
    SDFT_CUDA(cudaMemsetAsync(derr, 0, sizeof(int), c->stream));
    const size_t dsm = NSTAGE * ROT_STAGE_BYTES + 1024 + 256;
    SDFT_CUDA(cudaFuncSetAttribute(rotate_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dsm));
    dim3 grid((unsigned)((c->ng + TC_M - 1) / TC_M), (ncol + TC_N - 1) / TC_N);
    ScopedTimer timer(c, SDFT_K_ROTATE, 0.0, 2.0 * (double)c->ng * ncol * ncol);
    rotate_tc_kernel<<<grid, 256, dsm, c->stream>>>((const float*)Y, Q32, (float*)X, ncol, c->ng, derr);
    SDFT_CUDA(cudaGetLastError());
    count_launch(c);
    int herr = 0;
    SDFT_CUDA(cudaMemcpyAsync(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    SDFT_CUDA(cudaStreamSynchronize(c->stream));
    if (herr) throw Error{SDFT_ERR_DEVICE_TIMEOUT, "tensor-core rotation: an mbarrier wait timed out"};
}

namespace {
}  // namespace

static bool tc_block_ok(int precision, bool cplx, int ncol) {
    return precision == SDFT_MIXED && !cplx && ncol >= 32 && ncol % 2 == 0 && getenv("SDFT_NO_TCGEN05") == nullptr;
}
// the Gram's tile-pair table holds at most 64 pairs (10 tiles of 128 columns); wider blocks use the
// CUDA-core Gram
bool gram_tc_supported(int precision, bool cplx, int ncol) {
    const int tiles = (ncol + TC_M - 1) / TC_M;
    return tc_block_ok(precision, cplx, ncol) && tiles * (tiles + 1) / 2 <= 64;
}
bool rotate_tc_supported(int precision, bool cplx, int ncol) { return tc_block_ok(precision, cplx, ncol); }

void subspace_gram_tc(sdft_ctx* c, const void* Y, const void* HY, double* M, double* Hs, int ncol) {
    const int tiles = (ncol + TC_M - 1) / TC_M;
    std::vector<TilePair> hp;
    for (int i = 0; i < tiles; ++i)
        for (int j = i; j < tiles; ++j) hp.push_back(TilePair{i, j});
    const int npair = (int)hp.size();
    const long long nn = (long long)ncol * ncol;
    // splits: about two CTAs per SM in total, bounded by the partial buffer (FP32, 2 nn per split)
    long long nsplit = std::max<long long>(1, (2LL * 152) / npair);
    nsplit = std::min<long long>(nsplit, (long long)(c->part_elems * 2 / (2 * nn)));
    nsplit = std::max<long long>(1, std::min<long long>(nsplit, (c->ng + TC_K - 1) / TC_K));
    long long chunk = (c->ng + nsplit - 1) / nsplit;
    chunk = (chunk + TC_K - 1) / TC_K * TC_K;
    nsplit = (c->ng + chunk - 1) / chunk;
    SDFT_REQUIRE((size_t)(nsplit * 2 * nn) <= c->part_elems * 2, SDFT_ERR_INVALID_ARG, "gram_tc: partials");
    TilePair* dpairs = reinterpret_cast<TilePair*>(c->scal + 512);   // <= 64 pairs fit in [512, 1024)
    SDFT_REQUIRE(npair <= 64, SDFT_ERR_INVALID_ARG, "gram_tc: too many tiles");
    SDFT_CUDA(cudaMemcpyAsync(dpairs, hp.data(), sizeof(TilePair) * npair, cudaMemcpyHostToDevice, c->stream));
    int* derr = reinterpret_cast<int*>(c->scal + 4);
    SDFT_CUDA(cudaMemsetAsync(derr, 0, sizeof(int), c->stream));
    const size_t dsm = NSTAGE * STAGE_BYTES + 1024 + 256;
    SDFT_CUDA(cudaFuncSetAttribute(gram_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dsm));
    ScopedTimer timer(c, SDFT_K_GRAM, 0.0, 2.0 * (double)c->ng * ncol * ncol);
    float* part = reinterpret_cast<float*>(c->part);
    gram_tc_kernel<<<dim3(npair, (unsigned)nsplit), 256, dsm, c->stream>>>(
        (const float*)Y, (const float*)HY, ncol, c->ng, chunk, dpairs, part, derr);
    SDFT_CUDA(cudaGetLastError());
    gram_tc_reduce_kernel<<<(unsigned)std::min<long long>((nn + 255) / 256, 2048), 256, 0, c->stream>>>(
        part, (int)nsplit, ncol, M, Hs);
    SDFT_CUDA(cudaGetLastError());
    count_launch(c, 2);
    int herr = 0;
    SDFT_CUDA(cudaMemcpyAsync(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    SDFT_CUDA(cudaStreamSynchronize(c->stream));
    if (herr) throw Error{SDFT_ERR_DEVICE_TIMEOUT, "tensor-core Gram: an mbarrier wait timed out"};
}

}  // namespace sdft
