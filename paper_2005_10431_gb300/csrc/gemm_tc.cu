// Rayleigh-Ritz GEMMs on the 5th-generation tensor cores (paper Sec. 2.1 CheFSI; Sec. 4 names the
// subspace work as the step that dominates at scale), for FP32 orbital blocks in the paired layout
// (float2 per grid point holding orbitals 2p and 2p + 1):
//   Gram      M = Y^T Y,  Hs = Y^T (H Y)      (contraction over grid points)
//   rotation  X = Y Q                         (contraction over orbitals)
// as BF16x3 split products  a*b ~ hi(a)hi(b) + hi(a)lo(b) + lo(a)hi(b),  hi = bf16(a),
// lo = bf16(a - hi), accumulated in FP32 in tensor memory (TMEM).
//
// GB300 design (warp-specialised, mbarrier pipelines, no CTA-wide barrier in the main loops):
//   warp 0      TMA producer: 2-D tensor copies of the raw FP32 tiles straight from the paired
//               layout (the float2 pair is one 8-byte element) into shared-memory stages;
//   converters  split every raw value into bf16 hi / lo and write K-major, 128-byte-swizzled
//               operand rows [32 hi | 32 lo]; afterwards they drain TMEM and run the epilogue;
//   warp 1      one thread issues tcgen05.mma for the three split products per 16-wide K step and
//               frees each stage with tcgen05.commit on its mbarrier.
// One 128-byte row holds 32 hi and 32 lo values of one operand row, so the hi and lo operands of a
// K step are the same shared-memory descriptor advanced by 64 bytes along the swizzled row.  Raw
// tiles are read and converted rows written without bank conflicts.  Every wait is bounded in time
// (global timer): on timeout the kernel raises a shared abort flag that ends every role's loop,
// waits (bounded) for its own copies and MMAs in flight, releases its tensor memory and reports.
//
// The rotation converts each Y value once per block of output orbitals and runs at about half of
// the tensor pipe.  The Gram is bound by shared-memory bandwidth: per 32-point stage the copies
// write 48 KB, the converters read and write 48 KB each and the MMAs read 72 KB (the split products
// read A_hi and B_hi twice), about 1700 cycles of shared-memory traffic against about 1000 of MMA.
// Measured alternatives that did not beat it at full size (1.7 M points x 520 states): a deeper
// ring, more converter warps, an L2 prefetch of later stages (50 % slower), and a separate split
// pass into bf16 planes feeding a converter-free Gram (45 % of the pipe on a 110 k-point slice,
// but 2.7x DRAM re-reads at full size plus the pass itself).
#include "internal.cuh"

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdlib>
#include <vector>

namespace sdft {

// tiled tensor-map encoding (defined with the stencil's tensor maps)
void tma_encode_tiled(CUtensorMap* m, CUtensorMapDataType t, int rank, const void* base, const cuuint64_t* dims,
                      const cuuint64_t* strides_bytes, const cuuint32_t* box, CUtensorMapSwizzle sw);

namespace {

constexpr int TC_M = 128;         // accumulator rows = TMEM lanes
constexpr int KS = 32;            // contraction elements per pipeline stage
constexpr int ROWB = 128;         // bytes of one converted operand row: 32 hi + 32 lo bf16
constexpr int NRAW = 2;           // raw FP32 stages (TMA destination)
constexpr int NCONV = 2;          // converted bf16 stages (MMA operands)
constexpr int NCV = 8;            // rotation: converter / epilogue warps
constexpr int NTHREADS = 32 * (2 + NCV);
constexpr int G_NCV = 12;         // Gram: converter warps (the first 8 also drain and write the result)
constexpr int G_NDRAIN = 8;
constexpr int G_NTHREADS = 32 * (2 + G_NCV);
constexpr unsigned long long WAIT_NS = 2000000000ull;   // a wait gives up after 2 s (global timer)
constexpr uint32_t SUSPEND_NS = 10000000u;   // try_wait suspend-time hint: the thread sleeps until the
                                             // phase completes (or this limit), instead of spinning

// Gram stage: raw = 3 tiles (Y_i, Y_j, HY_j) x 2 copies of [64 pairs x 16 points x 8 B] (48 KB),
// converted in place to A (128 rows) + B (up to 256 rows: Y_j then HY_j), also 48 KB
constexpr int G_RAW_TILE = 2 * 64 * 128;                 // 16 KB
constexpr int G_STAGE = 3 * G_RAW_TILE;                 // 48 KB
constexpr int G_CONV_A = TC_M * ROWB;                   // 16 KB
constexpr int G_NST = 4;                                // stages in the ring
constexpr int G_SMEM = G_NST * G_STAGE;
// rotation stage sizes: raw = [16 pairs x 128 points x 8 B]; converted A = 128 rows; B = nj rows
constexpr int R_RAW_STAGE = 16 * TC_M * 8;              // 16 KB
constexpr int R_CONV_A = TC_M * ROWB;                   // 16 KB
constexpr int R_MAX_NJ = 256;

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(su32(bar)), "r"(parity), "r"(SUSPEND_NS)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// wait bounded in time that also gives up once another role has raised the abort flag
__device__ __forceinline__ bool mbar_wait_or_abort(uint64_t* bar, uint32_t parity, volatile int* abort_flag) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    while (true) {
        if (mbar_try_wait(bar, parity)) return true;
        if (*abort_flag) return false;
        if (global_ns() - t0 > WAIT_NS) {
            *abort_flag = 1;
            return false;
        }
    }
}
// bounded wait without the abort check (draining work already in flight)
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    while (global_ns() - t0 <= WAIT_NS)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
// the same wait for a whole warp: lane 0 polls, the outcome is broadcast (warp-uniform)
// (then every lane observes the completed phase itself, which gives each lane the acquire; the
// phase cannot move on before this warp arrives on its partner barrier, so that wait succeeds at once)
__device__ __forceinline__ bool warp_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag) {
    int ok = 0;
    if ((threadIdx.x & 31) == 0) ok = mbar_wait_or_abort(bar, parity, abort_flag) ? 1 : 0;
    ok = __shfl_sync(0xffffffffu, ok, 0);
    if (ok) mbar_wait(bar, parity);
    return ok != 0;
}

// barrier among the `nthreads` threads that use named barrier `id`, returning the AND of `v` over them
__device__ __forceinline__ bool named_bar_and(int id, int nthreads, bool v) {
    uint32_t r;
    asm volatile(
        "{\n .reg .pred p, q;\n setp.ne.u32 q, %1, 0;\n bar.red.and.pred p, %2, %3, q;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(r)
        : "r"((uint32_t)v), "r"(id), "r"(nthreads)
        : "memory");
    return r != 0;
}
__device__ __forceinline__ void tma2(void* dst, const CUtensorMap* m, int c0, int c1, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];" ::"r"(su32(dst)),
        "l"(m), "r"(c0), "r"(c1), "r"(su32(bar))
        : "memory");
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

// byte offset of 16-byte chunk `chunk` (0..7) of row r in a 128-byte-swizzled tile
__device__ __forceinline__ uint32_t swz(int r, int chunk) { return (uint32_t)(r * ROWB + (((chunk ^ r) & 7) << 4)); }

__device__ __forceinline__ float4 lds128(uint32_t a) {
    float4 v;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(a));
    return v;
}
__device__ __forceinline__ float2 lds64(uint32_t a) {
    float2 v;
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(a));
    return v;
}
__device__ __forceinline__ void sts128(uint32_t a, const uint32_t* v) {
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(a), "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3])
                 : "memory");
}

// hi = bf16_rn(x), lo = bf16_rn(x - hi) for two values; first value in the low half of each word
__device__ __forceinline__ void split2(float a, float b, uint32_t& hi, uint32_t& lo) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    const float2 hf = __bfloat1622float2(h);
    const __nv_bfloat162 l = __floats2bfloat162_rn(a - hf.x, b - hf.y);
    hi = *reinterpret_cast<const uint32_t*>(&h);
    lo = *reinterpret_cast<const uint32_t*>(&l);
}

// three split products of one 32-wide stage: for each 16-wide K step, hi*hi, hi*lo, lo*hi
__device__ __forceinline__ void issue_split_mmas(uint32_t tmem, uint32_t a, uint32_t b, uint32_t idesc, bool first) {
#pragma unroll
    for (int kk = 0; kk < 2; ++kk) {
        const uint32_t ko = kk * 32;   // 16 bf16 = 32 bytes along the swizzled row
        mma_bf16(tmem, sw128_desc(a + ko), sw128_desc(b + ko), idesc, (first && kk == 0) ? 0u : 1u);
        mma_bf16(tmem, sw128_desc(a + ko), sw128_desc(b + 64 + ko), idesc, 1u);
        mma_bf16(tmem, sw128_desc(a + 64 + ko), sw128_desc(b + ko), idesc, 1u);
    }
}

struct TilePair {
    int ti, tj;
};

// rows of column tile j that the Gram stores: 128, or the ragged last tile rounded up to 16
__host__ __device__ inline int tile_width(int ncol, int tj) {
    const int w = min(TC_M, ncol - tj * TC_M);
    return (w + 15) / 16 * 16;
}

// ---------------------------------------------------------------------------------------
// Gram.  CTA = one tile pair (i, j >= i) x one split of the grid points.  Per stage of 32 points:
// raw Y_i, Y_j, HY_j (each two 16-point copies of 64 pairs, 128-byte swizzle); converted A = Y_i
// (128 rows), B = [Y_j (w rows); HY_j (w rows)], one MMA of N = 2w per split product and K step,
// accumulators [M_ij | Hs_ij] in TMEM columns [0, 2w).
//
// The tensor cores add into the FP32 accumulator without rounding to nearest, so an accumulation
// chain over tens of thousands of points drifts (6e-4 relative on the diagonal of M at 86 400
// points).  The chain is therefore cut into blocks of GBLK stages (256 points): after each block
// the epilogue warps add the accumulator (TMEM columns [0, 256)) into a running FP32 sum kept in
// TMEM columns [256, 512) with CUDA-core, round-to-nearest adds, and release it; the next block's
// first MMA overwrites it.  A block is drained after the converters have prepared the next stage,
// so the tensor cores wait only for the drain itself.
// ---------------------------------------------------------------------------------------
constexpr int GBLK = 8;

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const float* v) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32};" ::"r"(taddr),
        "f"(v[0]), "f"(v[1]), "f"(v[2]), "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7]), "f"(v[8]), "f"(v[9]),
        "f"(v[10]), "f"(v[11]), "f"(v[12]), "f"(v[13]), "f"(v[14]), "f"(v[15]), "f"(v[16]), "f"(v[17]), "f"(v[18]),
        "f"(v[19]), "f"(v[20]), "f"(v[21]), "f"(v[22]), "f"(v[23]), "f"(v[24]), "f"(v[25]), "f"(v[26]), "f"(v[27]),
        "f"(v[28]), "f"(v[29]), "f"(v[30]), "f"(v[31])
        : "memory");
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

__global__ void __launch_bounds__(G_NTHREADS, 1)
gram_tc_kernel(const __grid_constant__ CUtensorMap tmY, const __grid_constant__ CUtensorMap tmHY, int ncol,
               long long ng, long long chunk, const TilePair* __restrict__ pairs, float* __restrict__ part,
               int* __restrict__ err) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // align by offsetting the array itself (not through an integer cast): accesses stay shared-memory ones
    unsigned char* smem = smem_raw + ((1024u - ((unsigned)__cvta_generic_to_shared(smem_raw) & 1023u)) & 1023u);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + G_SMEM);   // copies of stage s landed
    uint64_t* conv_full = full + G_NST;         // stage s converted (one arrival per converter warp)
    uint64_t* empty = conv_full + G_NST;        // the MMAs reading stage s completed
    uint64_t* acc_full = empty + G_NST;         // block k of the accumulation chain complete (phase k)
    uint64_t* acc_empty = acc_full + 1;         // block k drained (phase k)
    uint64_t* fin_bar = acc_empty + 1;          // all MMAs complete (abort path only)
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(fin_bar + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const TilePair tp = pairs[blockIdx.x];
    const int row_i = tp.ti * TC_M, row_j = tp.tj * TC_M;
    const int wj = tile_width(ncol, tp.tj);
    const long long g0 = blockIdx.y * chunk;
    const long long g1 = min(ng, g0 + chunk);
    const int ntile = (int)((g1 - g0 + KS - 1) / KS);
    const int nblk = (ntile + GBLK - 1) / GBLK;

    if (threadIdx.x == 0) {
        for (int s = 0; s < G_NST; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&conv_full[s], G_NCV);
            mbar_init(&empty[s], 1);
        }
        mbar_init(acc_full, 1);
        mbar_init(acc_empty, G_NDRAIN);
        mbar_init(fin_bar, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // columns [0, w): block accumulator of M, [w, 2w): of Hs; [256, 384) and [384, 512): running sums
    if (warp == 0) tmem_alloc(tmem_slot, 512);
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        // ---- TMA producer: G_NST stages in flight (an L2 prefetch further ahead measured slower) ----
        if (lane == 0) {
            int issued = 0;
            for (int t = 0; t < ntile; ++t) {
                const int s = t % G_NST;
                if (t >= G_NST && !mbar_wait_or_abort(&empty[s], (uint32_t)(((t - G_NST) / G_NST) & 1), abort_flag))
                    break;
                unsigned char* st = smem + s * G_STAGE;
                mbar_expect_tx(&full[s], G_STAGE);
                const int gx = (int)(g0 + (long long)t * KS);
#pragma unroll
                for (int b = 0; b < 2; ++b) {
                    tma2(st + b * (G_RAW_TILE / 2), &tmY, gx + 16 * b, row_i / 2, &full[s]);
                    tma2(st + G_RAW_TILE + b * (G_RAW_TILE / 2), &tmY, gx + 16 * b, row_j / 2, &full[s]);
                    tma2(st + 2 * G_RAW_TILE + b * (G_RAW_TILE / 2), &tmHY, gx + 16 * b, row_j / 2, &full[s]);
                }
                issued = t + 1;
            }
            // the copies still in flight must land before the CTA may leave
            if (*abort_flag)
                for (int t = std::max(0, issued - G_NST); t < issued; ++t) mbar_wait(&full[t % G_NST], (t / G_NST) & 1);
        }
    } else if (warp == 1) {
        // ---- MMA issuer ----
        if (lane == 0) {
            const uint32_t idesc = idesc_bf16(TC_M, 2 * wj);
            for (int t = 0; t < ntile; ++t) {
                const int s = t % G_NST, k = t / GBLK;
                const bool first = (t % GBLK) == 0;
                // a new block overwrites the accumulator: the previous block must have been drained
                if (first && k > 0 && !mbar_wait_or_abort(acc_empty, (uint32_t)((k - 1) & 1), abort_flag)) break;
                if (!mbar_wait_or_abort(&conv_full[s], (uint32_t)((t / G_NST) & 1), abort_flag)) break;
                fence_after_sync();
                unsigned char* st = smem + s * G_STAGE;
                issue_split_mmas(tmem, su32(st), su32(st + G_CONV_A), idesc, first);
                mma_commit(&empty[s]);
                if ((t % GBLK) == GBLK - 1 || t == ntile - 1)
                    mma_commit(acc_full);   // completes once every MMA of the block has completed
            }
            if (*abort_flag) {
                // every MMA issued so far must complete before the tensor memory is released
                mma_commit(fin_bar);
                mbar_wait(fin_bar, 0);
            }
        }
    } else {
        // ---- converters (in place: every converter warp reads its raw values into registers, a
        // named barrier among the converter warps, then the split rows are written over the raw
        // tiles), then the drains of the accumulation blocks and the epilogue (converter warps 0-7).
        // Work item = (tile T, block of 8 pairs); converter warp cw takes items cw and cw + 12. ----
        const int cw = warp - 2;
        const int pl = (lane & 3) + 4 * (lane >> 4);              // pair within the item's 8
        const int cq = ((lane >> 2) & 1) + 2 * ((lane >> 3) & 1);  // 8-point chunk of the stage
        // per item: raw tile, pair row, and the stage-relative shared-memory offsets (fixed for the
        // whole kernel): 4 16-byte raw reads, 4 16-byte writes (rows r0, r0 + 1; hi chunk, lo chunk)
        uint32_t ld_off[2][4], st_off[2][4];
        bool item_on[2];
#pragma unroll
        for (int it = 0; it < 2; ++it) {
            const int wi = cw + G_NCV * it;                        // 0..23
            const int T = wi >> 3, p = 8 * (wi & 7) + pl;
#pragma unroll
            for (int q = 0; q < 4; ++q)
                ld_off[it][q] = (uint32_t)(T * G_RAW_TILE + (cq >> 1) * (G_RAW_TILE / 2) + p * ROWB +
                                           (((((cq & 1) * 4 + q) ^ p) & 7) << 4));
            const int r0 = (T == 2 ? wj : 0) + 2 * p;
            const uint32_t base = T == 0 ? 0u : (uint32_t)G_CONV_A;
            st_off[it][0] = base + swz(r0, cq);
            st_off[it][1] = base + swz(r0, 4 + cq);
            st_off[it][2] = base + swz(r0 + 1, cq);
            st_off[it][3] = base + swz(r0 + 1, 4 + cq);
            item_on[it] = T == 0 || 2 * p < wj;                    // rows beyond a narrow B tile are unused
        }
        const bool drainer = cw < G_NDRAIN;
        const int quarter = warp & 3, half = (cw >> 2) & 1;       // TMEM lanes 32 quarter.., M or Hs columns
        const uint32_t lanes = (uint32_t)(32 * quarter) << 16;
        const uint32_t acc_addr = tmem + lanes + (uint32_t)(half * wj);
        const uint32_t sum_addr = tmem + lanes + 256u + (uint32_t)(half * TC_M);
        int drained = 0;
        auto drain = [&](int k) -> bool {
            if (!warp_wait(acc_full, (uint32_t)(k & 1), abort_flag)) return false;
            fence_after_sync();
            for (int q = 0; q < TC_M / 32; ++q) {
                if (32 * q < wj) {   // (a 32-column read past w only reads the other block's columns)
                    float v[32];
                    tmem_ld32(acc_addr + 32 * q, v);
                    if (k > 0) {
                        float u[32];
                        tmem_ld32(sum_addr + 32 * q, u);
#pragma unroll
                        for (int e = 0; e < 32; ++e) v[e] += u[e];
                    }
                    tmem_st32(sum_addr + 32 * q, v);
                }
            }
            fence_before_sync();
            __syncwarp();
            if (lane == 0) mbar_arrive(acc_empty);
            return true;
        };
        bool ok = true;
        for (int t = 0; t < ntile; ++t) {
            const int s = t % G_NST;
            const uint32_t st = su32(smem + s * G_STAGE);
            bool mine = ok && warp_wait(&full[s], (uint32_t)((t / G_NST) & 1), abort_flag);
            float4 r[2][4];
            if (mine) {
#pragma unroll
                for (int it = 0; it < 2; ++it)
#pragma unroll
                    for (int q = 0; q < 4; ++q) r[it][q] = lds128(st + ld_off[it][q]);
            }
            // every converter warp reaches this barrier once per stage; the outcome is the same for all
            ok = named_bar_and(1, G_NCV * 32, mine);
            if (!ok) break;
#pragma unroll
            for (int it = 0; it < 2; ++it) {
                if (!item_on[it]) continue;
                uint32_t h0[4], l0[4], h1[4], l1[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {   // r = (2p, 2p+1) at two consecutive points
                    split2(r[it][q].x, r[it][q].z, h0[q], l0[q]);
                    split2(r[it][q].y, r[it][q].w, h1[q], l1[q]);
                }
                sts128(st + st_off[it][0], h0);
                sts128(st + st_off[it][1], l0);
                sts128(st + st_off[it][2], h1);
                sts128(st + st_off[it][3], l1);
            }
            fence_proxy_async_smem();   // generic-proxy writes -> visible to the tensor cores
            __syncwarp();
            if (lane == 0) mbar_arrive(&conv_full[s]);
            // the block that ended with the previous stage, now that this stage is ready for the MMA
            if (drainer && t >= 1 && ((t - 1) % GBLK) == GBLK - 1) {
                ok = drain(drained);
                ++drained;
            }
        }
        // the last block, then the epilogue: rows of M (converter warps 0-3) or Hs (4-7)
        if (drainer) {
            if (ok && drained < nblk && drain(drained)) ++drained;
            if (drained == nblk && nblk > 0 && !*abort_flag) {
                fence_after_sync();
                const int gi = row_i + 32 * quarter + lane;
                const long long nn = (long long)ncol * ncol;
                float* dstp = part + (long long)blockIdx.y * 2 * nn + (half ? nn : 0);
                for (int q = 0; q < TC_M / 32; ++q) {
                    if (32 * q < wj) {
                        float v[32];
                        tmem_ld32(sum_addr + 32 * q, v);
                        if (gi < ncol) {
#pragma unroll
                            for (int e = 0; e < 32; ++e) {
                                const int gj = row_j + 32 * q + e;
                                if (32 * q + e < wj && gj < ncol && gj >= gi)
                                    dstp[(long long)gi + (long long)gj * ncol] = v[e];
                            }
                        }
                    }
                }
            }
        }
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    if (threadIdx.x == 0 && *abort_flag) atomicExch(err, 1);
    if (warp == 0) tmem_dealloc(tmem, 512);
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
// Rotation X = Y Q:  D[128 grid points][nj orbitals j] = sum_k Y[g][k] Q[k][j].
// A = Y tile, K-major over orbitals: raw copies [16 pairs x 128 points] are transposed by the
// converters into rows g = [32 orbitals hi | 32 lo].  B[j][k] = Q[k][j] comes pre-split from
// qsplit_kernel as rows j = [32 hi | 32 lo] per stage and is copied by TMA straight into the
// operand stage.  CTA = one tile of 128 grid points x one block of nj <= 256 output orbitals.
// ---------------------------------------------------------------------------------------
__global__ void qsplit_kernel(const double* __restrict__ Q, int ncol, int nk, __nv_bfloat16* __restrict__ Qs) {
    // Qs[j][t * 64 + h * 32 + kk] = (h ? lo : hi)(Q[(t * 32 + kk) + j * ncol])   (0 beyond ncol)
    const long long total = (long long)ncol * nk * 32;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
        const int kk = (int)(e & 31);
        const long long r = e >> 5;
        const int t = (int)(r % nk);
        const int j = (int)(r / nk);
        const int k = t * 32 + kk;
        const float x = k < ncol ? (float)Q[(long long)k + (long long)j * ncol] : 0.f;
        const __nv_bfloat16 hi = __float2bfloat16_rn(x);
        const __nv_bfloat16 lo = __float2bfloat16_rn(x - __bfloat162float(hi));
        __nv_bfloat16* row = Qs + (long long)j * nk * 64 + t * 64;
        row[kk] = hi;
        row[32 + kk] = lo;
    }
}

__global__ void __launch_bounds__(NTHREADS, 2)
rotate_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmQ,
                 float* __restrict__ X, int ncol, long long ng, int nk, int nj, int nsj, uint32_t tmem_cols,
                 int* __restrict__ err) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = smem_raw + ((1024u - ((unsigned)__cvta_generic_to_shared(smem_raw) & 1023u)) & 1023u);
    const int conv_stage = R_CONV_A + nj * ROWB;
    unsigned char* raw = smem;
    unsigned char* conv = smem + NRAW * R_RAW_STAGE;
    uint64_t* raw_full = reinterpret_cast<uint64_t*>(conv + NCONV * conv_stage);
    uint64_t* raw_empty = raw_full + NRAW;
    uint64_t* conv_full = raw_empty + NRAW;
    uint64_t* conv_empty = conv_full + NCONV;
    uint64_t* b_full = conv_empty + NCONV;
    uint64_t* acc_full = b_full + NCONV;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acc_full + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long g0 = (long long)(blockIdx.x / nsj) * TC_M;
    const int j0 = (blockIdx.x % nsj) * nj;

    if (threadIdx.x == 0) {
        for (int s = 0; s < NRAW; ++s) {
            mbar_init(&raw_full[s], 1);
            mbar_init(&raw_empty[s], NCV);
        }
        for (int s = 0; s < NCONV; ++s) {
            mbar_init(&conv_full[s], NCV);
            mbar_init(&conv_empty[s], 1);
            mbar_init(&b_full[s], 1);
        }
        mbar_init(acc_full, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tmem_alloc(tmem_slot, tmem_cols);   // a power of two >= max(32, nj)
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        // ---- TMA producer: raw Y copies run up to NRAW stages ahead, Q copies NCONV ahead ----
        if (lane == 0) {
            int issued_a = 0, issued_b = 0;
            for (int t = 0; t < nk; ++t) {
                const int s = t % NRAW, c = t % NCONV;
                if (t >= NRAW && !mbar_wait_or_abort(&raw_empty[s], (uint32_t)(((t - NRAW) / NRAW) & 1), abort_flag))
                    break;
                mbar_expect_tx(&raw_full[s], R_RAW_STAGE);
                tma2(raw + s * R_RAW_STAGE, &tmA, (int)g0, t * 16, &raw_full[s]);
                issued_a = t + 1;
                if (t >= NCONV &&
                    !mbar_wait_or_abort(&conv_empty[c], (uint32_t)(((t - NCONV) / NCONV) & 1), abort_flag))
                    break;
                mbar_expect_tx(&b_full[c], (uint32_t)(nj * ROWB));
                tma2(conv + c * conv_stage + R_CONV_A, &tmQ, t * 64, j0, &b_full[c]);
                issued_b = t + 1;
            }
            if (*abort_flag) {
                for (int t = std::max(0, issued_a - NRAW); t < issued_a; ++t) mbar_wait(&raw_full[t % NRAW], (t / NRAW) & 1);
                for (int t = std::max(0, issued_b - NCONV); t < issued_b; ++t)
                    mbar_wait(&b_full[t % NCONV], (t / NCONV) & 1);
            }
        }
    } else if (warp == 1) {
        // ---- MMA issuer: N = nj as one MMA (nj <= 256, multiple of 16) ----
        if (lane == 0) {
            const uint32_t idesc = idesc_bf16(TC_M, nj);
            for (int t = 0; t < nk; ++t) {
                const int c = t % NCONV;
                if (!mbar_wait_or_abort(&conv_full[c], (uint32_t)((t / NCONV) & 1), abort_flag)) break;
                if (!mbar_wait_or_abort(&b_full[c], (uint32_t)((t / NCONV) & 1), abort_flag)) break;
                fence_after_sync();
                unsigned char* st = conv + c * conv_stage;
                issue_split_mmas(tmem, su32(st), su32(st + R_CONV_A), idesc, t == 0);
                mma_commit(&conv_empty[c]);
            }
            mma_commit(acc_full);
            if (*abort_flag) mbar_wait(acc_full, 0);
        }
    } else {
        // ---- converters: item = (grid point g, group u of 8 orbitals = 4 pairs) ----
        const int cw = warp - 2;
        for (int t = 0; t < nk; ++t) {
            const int s = t % NRAW, c = t % NCONV;
            if (!warp_wait(&raw_full[s], (uint32_t)((t / NRAW) & 1), abort_flag)) break;
            if (t >= NCONV && !warp_wait(&conv_empty[c], (uint32_t)(((t - NCONV) / NCONV) & 1), abort_flag)) break;
            const uint32_t rst = su32(raw + s * R_RAW_STAGE);
            const uint32_t ca = su32(conv + c * conv_stage);
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int item = cw * 32 + lane + 256 * i;
                const int g = item & (TC_M - 1), u = item >> 7;
                uint32_t h[4], l[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const float2 w = lds64(rst + (uint32_t)(((4 * u + e) * TC_M + g) * 8));   // orbitals 8u+2e, +1
                    split2(w.x, w.y, h[e], l[e]);
                }
                sts128(ca + swz(g, u), h);
                sts128(ca + swz(g, 4 + u), l);
            }
            fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(&raw_empty[s]);
                mbar_arrive(&conv_full[c]);
            }
        }
        // ---- epilogue: lanes = grid points, columns = orbitals; converter warps 0-3 the first
        // half of the columns, 4-7 the second ----
        const bool done = warp_wait(acc_full, 0, abort_flag) && !*abort_flag;
        if (done) {
            fence_after_sync();
            const int quarter = warp & 3, half = cw >> 2;
            const long long g = g0 + 32 * quarter + lane;
            const uint32_t lane_base = (uint32_t)(32 * quarter) << 16;
            const int ch = nj / 2;   // a multiple of 8
            for (int c0 = half * ch; c0 < (half + 1) * ch; c0 += 8) {
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
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    if (threadIdx.x == 0 && *abort_flag) atomicExch(err, 1);
    if (warp == 0) tmem_dealloc(tmem, tmem_cols);
}

// 2-D map of an FP32 paired block: 8-byte elements (one orbital pair at one point), [pairs][ng]
void paired_map(CUtensorMap* m, const void* base, long long ng, int npairs, int box_points, int box_pairs,
                CUtensorMapSwizzle sw) {
    const cuuint64_t dims[2] = {(cuuint64_t)ng, (cuuint64_t)npairs};
    const cuuint64_t st[1] = {(cuuint64_t)ng * 8};
    const cuuint32_t box[2] = {(cuuint32_t)box_points, (cuuint32_t)box_pairs};
    tma_encode_tiled(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, base, dims, st, box, sw);
}

}  // namespace

static bool tc_block_ok(const sdft_ctx* c, int precision, bool cplx, int ncol) {
    // TMA copies of the paired layout need a pair row stride (8 ngrid bytes) that is a multiple of 16
    return precision == SDFT_MIXED && !cplx && ncol >= 32 && ncol % 2 == 0 && (c->ng % 2) == 0 && !c->gemm_fp32 &&
           getenv("SDFT_NO_TCGEN05") == nullptr;
}
// the Gram's tile-pair table holds at most 64 pairs (10 tiles of 128 columns); wider blocks use the
// CUDA-core Gram
bool gram_tc_supported(const sdft_ctx* c, int precision, bool cplx, int ncol) {
    const int tiles = (ncol + TC_M - 1) / TC_M;
    return tc_block_ok(c, precision, cplx, ncol) && tiles * (tiles + 1) / 2 <= 64;
}
bool rotate_tc_supported(const sdft_ctx* c, int precision, bool cplx, int ncol) {
    return tc_block_ok(c, precision, cplx, ncol);
}

size_t qsplit_bytes(int ncol) { return (size_t)ncol * (size_t)((ncol + KS - 1) / KS) * 64 * 2; }

// X = Y Q for FP32 paired blocks; Q is FP64, column-major ncol x ncol
void rotate_tc(sdft_ctx* c, const void* Y, const double* Q, void* X, int ncol) {
    const int nk = (ncol + KS - 1) / KS;
    __nv_bfloat16* Qs = reinterpret_cast<__nv_bfloat16*>(c->Qsplit);
    SDFT_REQUIRE(Qs != nullptr && qsplit_bytes(ncol) <= c->qsplit_bytes, SDFT_ERR_INVALID_ARG,
                 "tensor-core rotation: split-Q buffer too small");
    int* derr = reinterpret_cast<int*>(c->scal + 5);
    SDFT_CUDA(cudaMemsetAsync(derr, 0, sizeof(int), c->stream));
    const long long nq = (long long)ncol * nk * 32;
    qsplit_kernel<<<(unsigned)std::min<long long>((nq + 255) / 256, 152LL * 8), 256, 0, c->stream>>>(Q, ncol, nk, Qs);
    SDFT_CUDA(cudaGetLastError());
    // output-orbital blocks of at most 256 columns, equal widths rounded up to 16
    const int nsj = (ncol + R_MAX_NJ - 1) / R_MAX_NJ;
    const int nj = ((ncol + nsj - 1) / nsj + 15) / 16 * 16;
    CUtensorMap mA, mQ;
    paired_map(&mA, Y, c->ng, ncol / 2, TC_M, 16, CU_TENSOR_MAP_SWIZZLE_NONE);
    {
        const cuuint64_t dims[2] = {(cuuint64_t)nk * 64, (cuuint64_t)ncol};
        const cuuint64_t st[1] = {(cuuint64_t)nk * 64 * 2};
        const cuuint32_t box[2] = {64, (cuuint32_t)nj};
        tma_encode_tiled(&mQ, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, Qs, dims, st, box, CU_TENSOR_MAP_SWIZZLE_128B);
    }
    const size_t dsm = (size_t)NRAW * R_RAW_STAGE + (size_t)NCONV * (R_CONV_A + nj * ROWB) + 1024 + 256;
    SDFT_CUDA(cudaFuncSetAttribute(rotate_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dsm));
    const long long ntile = (c->ng + TC_M - 1) / TC_M;
    uint32_t tcols = 32;
    while (tcols < (uint32_t)nj) tcols *= 2;
    ScopedTimer timer(c, SDFT_K_ROTATE, 0.0, 2.0 * (double)c->ng * ncol * ncol);
    rotate_tc_kernel<<<(unsigned)(ntile * nsj), NTHREADS, dsm, c->stream>>>(mA, mQ, (float*)X, ncol, c->ng, nk, nj,
                                                                          nsj, tcols, derr);
    SDFT_CUDA(cudaGetLastError());
    count_launch(c, 2);
    int herr = 0;
    SDFT_CUDA(cudaMemcpyAsync(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    SDFT_CUDA(cudaStreamSynchronize(c->stream));
    if (herr) throw Error{SDFT_ERR_DEVICE_TIMEOUT, "tensor-core rotation: an mbarrier wait timed out"};
}

void subspace_gram_tc(sdft_ctx* c, const void* Y, const void* HY, double* M, double* Hs, int ncol) {
    const int tiles = (ncol + TC_M - 1) / TC_M;
    std::vector<TilePair> hp;
    for (int i = 0; i < tiles; ++i)
        for (int j = i; j < tiles; ++j) hp.push_back(TilePair{i, j});
    const int npair = (int)hp.size();
    SDFT_REQUIRE(npair <= 64, SDFT_ERR_INVALID_ARG, "gram_tc: too many tiles");
    const long long nn = (long long)ncol * ncol;
    // splits: about two CTAs per SM in total, bounded by the partial buffer (FP32, 2 nn per split)
    long long nsplit = std::max<long long>(1, (2LL * 152) / npair);
    nsplit = std::min<long long>(nsplit, (long long)(c->part_elems * 2 / (2 * nn)));
    nsplit = std::max<long long>(1, std::min<long long>(nsplit, (c->ng + KS - 1) / KS));
    long long chunk = (c->ng + nsplit - 1) / nsplit;
    chunk = (chunk + KS - 1) / KS * KS;
    nsplit = (c->ng + chunk - 1) / chunk;
    SDFT_REQUIRE((size_t)(nsplit * 2 * nn) <= c->part_elems * 2, SDFT_ERR_INVALID_ARG, "gram_tc: partials");
    TilePair* dpairs = reinterpret_cast<TilePair*>(c->scal + 512);   // <= 64 pairs fit in [512, 1024)
    SDFT_CUDA(cudaMemcpyAsync(dpairs, hp.data(), sizeof(TilePair) * npair, cudaMemcpyHostToDevice, c->stream));
    int* derr = reinterpret_cast<int*>(c->scal + 4);
    SDFT_CUDA(cudaMemsetAsync(derr, 0, sizeof(int), c->stream));
    CUtensorMap mY, mHY;
    paired_map(&mY, Y, c->ng, ncol / 2, 16, 64, CU_TENSOR_MAP_SWIZZLE_128B);
    paired_map(&mHY, HY, c->ng, ncol / 2, 16, 64, CU_TENSOR_MAP_SWIZZLE_128B);
    const size_t dsm = (size_t)G_SMEM + 1024 + 256;
    SDFT_CUDA(cudaFuncSetAttribute(gram_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dsm));
    // algorithmic flops: two full ngrid x ncol x ncol products (M and Hs), 2 flops per multiply-add
    ScopedTimer timer(c, SDFT_K_GRAM, 0.0, 4.0 * (double)c->ng * ncol * ncol);
    float* part = reinterpret_cast<float*>(c->part);
    gram_tc_kernel<<<dim3(npair, (unsigned)nsplit), G_NTHREADS, dsm, c->stream>>>(mY, mHY, ncol, c->ng, chunk, dpairs,
                                                                                part, derr);
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
