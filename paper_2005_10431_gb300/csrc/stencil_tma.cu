// Fused H Y + Chebyshev step for FP32 real blocks (paired layout), TMA-fed slab tile.
//
//   Ynext = alpha * (H Y - shift * Y) - beta * Yprev,
//   H Y   = -1/2 L_h Y + V .* Y + sum_a beta_a (gamma_a beta_a^T Y)
// (paper Sec. 2.1: matrix-free H application with the finite-difference stencil and the outer
// product form of the nonlocal operator; three-term recurrence of the scaled Chebyshev filter).
//
// GB300 design.  A CTA owns a slab of TY whole x-rows (n1 points each) of NP consecutive orbital
// pairs and marches along z.  One producer warp feeds a D-stage shared-memory ring with TMA tensor
// copies: per plane the TY rows and the 6 + 6 y-halo rows of every pair (one 4-D box when the slab
// does not touch the periodic y boundary, two boxes per pair when it does), the Yprev rows, the
// V_eff rows, the per-point KB slot tables (atom, value) and, by one bulk copy, the KB
// coefficients gamma_a beta_a^T Y of the plane's NP pairs (a few KB, read from L2).  Compute warps wait on the stage's
// mbarrier, so there is no CTA-wide barrier per plane; each compute thread owns two adjacent
// x-points of one row for all NP pairs.  x-neighbours come from the staged row with the periodic
// wrap folded into six per-thread column offsets (n1 even: a 16-byte pair of points never
// straddles the wrap), y-neighbours from the staged halo rows, z-neighbours from a register queue
// of 16-byte vectors; the stage of plane z also carries the rows of plane z + 6, the queue's next
// entry, so no global load sits on the compute path.  V_eff and the KB tables are staged once per
// plane and shared by the NP pairs.  With every stage the producer also prefetches a later plane's
// rows into L2, so the copies mostly hit L2.  Every mbarrier wait is bounded: on timeout the thread records an
// error flag and leaves its loop; the CTA then drains the copies it issued before exiting.
#include "internal.cuh"

#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>
#include <mutex>

namespace sdft {

int* stencil_error_flag(sdft_ctx* c) { return reinterpret_cast<int*>(c->scal + 1600); }

void check_stencil_flag(sdft_ctx* c) {
    int h = 0;
    SDFT_CUDA(cudaMemcpyAsync(&h, stencil_error_flag(c), sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    SDFT_CUDA(cudaStreamSynchronize(c->stream));
    if (h) {
        SDFT_CUDA(cudaMemsetAsync(stencil_error_flag(c), 0, sizeof(int), c->stream));
        throw Error{SDFT_ERR_DEVICE_TIMEOUT, "slab stencil: an mbarrier wait timed out"};
    }
}

namespace {

constexpr int R = FD_RADIUS;
constexpr long long SLAB_WAIT_LIMIT = 1LL << 24;   // try_wait polls before a wait gives up

struct SlabArgs {
    float cx[R + 1], cy[R + 1], cz[R + 1];
    float c0, alpha, beta, shift;
    int n2, n3, ncolE, natom, nslab;
    int sstride;         // bytes per stage: the static regions plus the KB coefficient window
    long long ng;
    int total;           // (pair group, plane) units of one slab: ngroups * n3
    int per_cta;         // units per CTA
};
constexpr int PFD = 10;  // planes between a stage's copies and the L2 prefetch issued with them

// ---- PTX wrappers ----------------------------------------------------------------------
__device__ __forceinline__ uint32_t s32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mb_init(uint64_t* b, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(s32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mb_expect_tx(uint64_t* b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(s32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mb_arrive(uint64_t* b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(s32(b)) : "memory");
}
__device__ __forceinline__ bool mb_try_wait(uint64_t* b, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(s32(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool mb_wait(uint64_t* b, uint32_t parity) {
    for (long long i = 0; i < SLAB_WAIT_LIMIT; ++i)
        if (mb_try_wait(b, parity)) return true;
    return false;
}
__device__ __forceinline__ void tma3(void* dst, const CUtensorMap* m, int c0, int c1, int c2, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(s32(dst)),
        "l"(m), "r"(c0), "r"(c1), "r"(c2), "r"(s32(bar))
        : "memory");
}
__device__ __forceinline__ void tma4(void* dst, const CUtensorMap* m, int c0, int c1, int c2, int c3, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
        "%5}], [%6];" ::"r"(s32(dst)),
        "l"(m), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(s32(bar))
        : "memory");
}

// global float2 reduction (vector red, sm_90 and later)
__device__ __forceinline__ void red_add2(float2* p, float2 v) {
    asm volatile("red.global.add.v2.f32 [%0], {%1, %2};" ::"l"(p), "f"(v.x), "f"(v.y) : "memory");
}

// untiled bulk copy global -> shared: both addresses 16-byte aligned, bytes a multiple of 16
__device__ __forceinline__ void bulk_copy(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(s32(dst)),
        "l"(src), "r"(bytes), "r"(s32(bar))
        : "memory");
}

__device__ __forceinline__ void prefetch3(const CUtensorMap* m, int c0, int c1, int c2) {
    asm volatile("cp.async.bulk.prefetch.tensor.3d.L2.global.tile [%0, {%1, %2, %3}];" ::"l"(m), "r"(c0), "r"(c1),
                 "r"(c2)
                 : "memory");
}
__device__ __forceinline__ void prefetch4(const CUtensorMap* m, int c0, int c1, int c2, int c3) {
    asm volatile("cp.async.bulk.prefetch.tensor.4d.L2.global.tile [%0, {%1, %2, %3, %4}];" ::"l"(m), "r"(c0), "r"(c1),
                 "r"(c2), "r"(c3)
                 : "memory");
}

// ---- shared-memory loads by 32-bit shared address ---------------------------------------
// explicit vector loads: a 16-byte read must stay one 128-bit access (two 8-byte reads of every
// other word would put threads t and t+8 of a half-warp on the same banks)
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
__device__ __forceinline__ int2 lds64i(uint32_t a) {
    int2 v;
    asm volatile("ld.shared.v2.s32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "r"(a));
    return v;
}

// ---- packed FP32 pair arithmetic (Blackwell f32x2) --------------------------------------
__device__ __forceinline__ unsigned long long pk(float2 a) {
    return (unsigned long long)__float_as_uint(a.x) | ((unsigned long long)__float_as_uint(a.y) << 32);
}
__device__ __forceinline__ float2 upk(unsigned long long u) {
    return make_float2(__uint_as_float((unsigned)(u & 0xffffffffu)), __uint_as_float((unsigned)(u >> 32)));
}
__device__ __forceinline__ float2 fma2(float s, float2 a, float2 acc) {   // acc + s * a
    unsigned long long r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(pk(make_float2(s, s))), "l"(pk(a)), "l"(pk(acc)));
    return upk(r);
}
__device__ __forceinline__ float2 fma2v(float2 s, float2 a, float2 acc) {   // acc + s .* a
    unsigned long long r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(pk(s)), "l"(pk(a)), "l"(pk(acc)));
    return upk(r);
}
__device__ __forceinline__ float2 add2(float2 a, float2 b) {
    unsigned long long r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(pk(a)), "l"(pk(b)));
    return upk(r);
}
__device__ __forceinline__ float2 lo2(float4 v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(float4 v) { return make_float2(v.z, v.w); }

// shared-memory layout of one stage (bytes), all regions 128-byte aligned for the TMA writes
template <int N1, int TY, int NP, int S>
struct SlabLayout {
    static constexpr int ROWS = TY + 2 * R;
    static constexpr int TILE_PAIR = ROWS * N1;                   // float2 per pair
    static constexpr int TILE = NP * TILE_PAIR * 8;               // bytes
    static constexpr int PREV = NP * TY * N1 * 8;
    static constexpr int VB = TY * N1 * 4;
    static constexpr int KA = S * TY * N1 * 4;
    static constexpr int QROWS = NP * TY * N1 * 8;                // interior rows of plane z + R (z-queue)
    static constexpr int OFF_Q = TILE;
    static constexpr int OFF_PREV = OFF_Q + QROWS;
    static constexpr int OFF_V = OFF_PREV + PREV;
    static constexpr int OFF_KA = OFF_V + VB;
    static constexpr int OFF_KV = OFF_KA + KA;
    static constexpr int STAGE = OFF_KV + KA;
    static_assert(TILE % 128 == 0 && QROWS % 128 == 0 && PREV % 128 == 0 && VB % 128 == 0 && KA % 128 == 0, "TMA regions must be 128-B aligned");
};

// KB coefficient window of a stage: the NP * natom float2 of the plane's pair group, copied from a
// 16-byte aligned start one float2 early when col0 * natom is odd, rounded up to 16 bytes
constexpr int slab_kc_bytes(int NP, int natom) { return ((NP * natom + 2) * 8 + 127) / 128 * 128; }

template <int N1, int TY, int NP, int S, int D>
constexpr size_t slab_smem_bytes(int natom) {
    return (size_t)(SlabLayout<N1, TY, NP, S>::STAGE + slab_kc_bytes(NP, natom)) * D + 16 * (size_t)(2 * D) + 128;
}

// Persistent schedule: CTA b works on slab b mod nslab (TY rows) and on the contiguous run
// [k W, (k+1) W) of that slab's (pair group, plane) units, k = b / nslab, units ordered group-major
// with planes z = 0..n3-1 within a group (group = NP consecutive pairs), W = ceil(units / CTAs per
// slab): every SM gets the same number of planes whatever the group count, and CTAs of neighbouring
// slabs move through the same planes together.  A run restarts the z-queue (2R planes of warm-up
// loads) at each group it enters.  block: TY * N1/2 compute threads + one producer warp.
// register cap: each of the SM's four schedulers owns a quarter of the 64 K registers and the warps of
// the CTA ((TY / RY) * N1/2 + 32 threads) are spread over them, MINB CTAs per SM
template <int N1, int TY, int RY, int MINB>
constexpr int slab_maxreg() {
    constexpr int warps = ((TY / RY) * (N1 / 2) + 32 + 31) / 32;
    constexpr int per_sched = (warps + 3) / 4 * MINB;
    constexpr int r = 16384 / per_sched / 32 / 8 * 8;
    return r > 255 ? 255 : r;
}

// PROJ (with KB, RY = 1): the step also accumulates the KB coefficients of its output,
// Cn[col][a] += sum_points beta_a(point) Ynext[point][col] (Cn zeroed before, scaled by gamma_a after,
// by the host), which the next step would otherwise compute by a separate pass over Ynext.  Each thread keeps, per KB slot,
// the atom that slot held on the previous plane and a running sum for it (the slot's atom changes
// only where the z-line of the thread's two points enters or leaves a projector sphere) and adds the
// sum into Cn with one vector reduction when the atom changes and at the end of a pair group; the
// second point of a slot whose atom differs from the first point's is added at once.
template <int N1, int TY, int NP, int RY, int S, int D, int MINB, bool PREV, bool KB, bool PROJ>
__global__ void __maxnreg__((slab_maxreg<N1, TY, RY, MINB>()))
cheb_slab_kernel(const float2* __restrict__ Y, float2* __restrict__ Ynext, const float2* __restrict__ C,
                 float2* __restrict__ Cn,
                 const __grid_constant__ CUtensorMap tmYfull, const __grid_constant__ CUtensorMap tmY6,
                 const __grid_constant__ CUtensorMap tmYmid, const __grid_constant__ CUtensorMap tmP,
                 const __grid_constant__ CUtensorMap tmV, const __grid_constant__ CUtensorMap tmKA,
                 const __grid_constant__ CUtensorMap tmKV, const __grid_constant__ CUtensorMap tmQ,
                 const __grid_constant__ SlabArgs A, int* __restrict__ err) {
    using L = SlabLayout<N1, TY, NP, S>;
    constexpr int HX = N1 / 2;
    constexpr int NCOMP = (TY / RY) * HX;    // compute threads: RY rows x 2 points x NP pairs each
    constexpr int NCW = NCOMP / 32;          // compute warps
    constexpr int QN = 2 * R + 1;            // register queue length (plane z + R arrives with stage z)
    static_assert(TY % RY == 0, "RY must divide TY");
    static_assert(!PROJ || (KB && RY == 1), "the fused projection needs the KB term and one row per thread");
    static_assert(NCOMP % 32 == 0, "compute threads must fill whole warps");
    extern __shared__ __align__(128) unsigned char smem_raw[];
    // align by offsetting the array itself (not through an integer cast), so that the compiler keeps
    // treating every access as a shared-memory access (LDS/STS rather than generic loads and stores)
    unsigned char* smem = smem_raw + ((128u - ((unsigned)__cvta_generic_to_shared(smem_raw) & 127u)) & 127u);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + (size_t)A.sstride * D);
    uint64_t* empty = full + D;

    const int tid = threadIdx.x;
    const int n3 = A.n3;
    const int slab = blockIdx.x % A.nslab;
    const int fbeg = (blockIdx.x / A.nslab) * A.per_cta;
    const int fend = min(A.total, fbeg + A.per_cta);
    if (fbeg >= fend) return;                // whole CTA, before any barrier
    const int plane = N1 * A.n2;
    const unsigned ngu = (unsigned)A.ng;

    if (tid == NCOMP) {
        for (int s = 0; s < D; ++s) {
            mb_init(&full[s], 1);
            mb_init(&empty[s], NCW);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    bool ok = true;
    int issued = 0;   // planes whose copies the producer lane has issued
    if (tid >= NCOMP) {
        // ---------------- producer warp: one lane issues every copy ----------------
        if (tid == NCOMP) {
            constexpr uint32_t sbytes = L::TILE + L::QROWS + (PREV ? L::PREV : 0) + L::VB + (KB ? 2 * L::KA : 0);
            int j = 0;
            for (int f = fbeg; f < fend && ok;) {
                const int grp = f / n3, z0 = f - grp * n3;
                const int z1 = min(n3, z0 + (fend - f));
                const int y0 = slab * TY, col0 = grp * NP;
                const bool wrap = (y0 < R) || (y0 + TY + R > A.n2);
                // KB coefficients of the group: float2 elements [e0 - o, e0 - o + kcn) of C, e0 = col0 * natom
                // (the host pads C by two pair columns and two elements past the block, so the window of the
                // last group stays inside its allocation)
                const long long e0 = (long long)col0 * A.natom;
                const int o = (int)(e0 & 1);
                const uint32_t kcn = (uint32_t)((o + NP * A.natom + 1) & ~1);
                const uint32_t bytes = sbytes + (KB ? kcn * 8u : 0u);
                for (int z = z0; z < z1; ++z, ++j) {
                    const int s = j % D;
                    if (j >= D && !mb_wait(&empty[s], ((j / D) - 1) & 1)) {
                        ok = false;
                        break;
                    }
                    unsigned char* st = smem + (size_t)s * A.sstride;
                    mb_expect_tx(&full[s], bytes);
                    if (KB) bulk_copy(st + L::STAGE, C + (e0 - o), kcn * 8u, &full[s]);
                    if (!wrap) {
                        tma4(st, &tmYfull, 0, y0 - R, z, col0, &full[s]);
                    } else {
#pragma unroll
                        for (int p = 0; p < NP; ++p) {
                            unsigned char* t = st + (size_t)p * L::TILE_PAIR * 8;
                            if (y0 < R) {   // y0 == 0: halo rows n2-6..n2-1 on top, then rows 0..TY+5
                                tma4(t, &tmY6, 0, A.n2 - R, z, col0 + p, &full[s]);
                                tma4(t + R * N1 * 8, &tmYmid, 0, 0, z, col0 + p, &full[s]);
                            } else {        // y0 + TY == n2: rows y0-6..n2-1, then halo rows 0..5
                                tma4(t, &tmYmid, 0, y0 - R, z, col0 + p, &full[s]);
                                tma4(t + (TY + R) * N1 * 8, &tmY6, 0, 0, z, col0 + p, &full[s]);
                            }
                        }
                    }
                    tma4(st + L::OFF_Q, &tmQ, 0, y0, z + R < n3 ? z + R : z + R - n3, col0, &full[s]);
                    if (PREV) tma4(st + L::OFF_PREV, &tmP, 0, y0, z, col0, &full[s]);
                    tma3(st + L::OFF_V, &tmV, 0, y0, z, &full[s]);
                    if (KB) {
                        tma4(st + L::OFF_KA, &tmKA, 0, y0, z, 0, &full[s]);
                        tma4(st + L::OFF_KV, &tmKV, 0, y0, z, 0, &full[s]);
                    }
                    issued = j + 1;
                    // L2 prefetch of a later plane of this piece: its first touch from HBM (the Y rows
                    // that the z-queue loads, Yprev, V, KB tables) then overlaps the current planes
                    const int zp = z + PFD;
                    if (zp < z1) {
                        prefetch4(&tmYfull, 0, y0 - R, zp, col0);
                        if (PREV) prefetch4(&tmP, 0, y0, zp, col0);
                        prefetch3(&tmV, 0, y0, zp);
                        if (KB) {
                            prefetch4(&tmKA, 0, y0, zp, 0);
                            prefetch4(&tmKV, 0, y0, zp, 0);
                        }
                    }
                }
                f += z1 - z0;
            }
            if (!ok) atomicExch(err, 1);
        }
    } else {
        // ---------------- compute warps ----------------
        const int ty0 = (tid / HX) * RY, tx = tid - (tid / HX) * HX;
        const int gx = 2 * tx;
        // wrapped x-columns (float2 units within a row) of the neighbour pairs x-6.., x+2.. of this pair
        int xc[6];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            int l = gx - 6 + 2 * k, r = gx + 2 + 2 * k;
            xc[k] = (l < 0 ? l + N1 : l) * 8;            // byte offsets within a row
            xc[3 + k] = (r >= N1 ? r - N1 : r) * 8;
        }
        const uint32_t smem_s = s32(smem);
        int j = 0;
        for (int f = fbeg; f < fend && ok;) {
            const int grp = f / n3, z0 = f - grp * n3;
            const int z1 = min(n3, z0 + (fend - f));
            const int col0 = grp * NP;
            const unsigned gxy = (unsigned)((slab * TY + ty0) * N1 + gx);   // first of the thread's RY rows
            const uint32_t kco = (uint32_t)(L::STAGE + 8 * (int)(((long long)col0 * A.natom) & 1));
            const int nvalid = min(NP, A.ncolE - col0);   // pairs of this group that exist
            const float2* Yg = Y + (size_t)col0 * ngu;
            float2* Zg = Ynext + (size_t)col0 * ngu;
            // fused projection state of this group: per slot the atom being summed and its sums
            int pcur[PROJ ? S : 1];
            float2 pacc[PROJ ? S : 1][NP];
            auto pflush = [&](int k) {
                if (PROJ && pcur[k] >= 0) {
#pragma unroll
                    for (int p = 0; p < NP; ++p) {
                        if (p < nvalid) red_add2(Cn + (size_t)(col0 + p) * A.natom + pcur[k], pacc[k][p]);
                        pacc[k][p] = make_float2(0.f, 0.f);
                    }
                }
            };
            if (PROJ) {
#pragma unroll
                for (int k = 0; k < S; ++k) {
                    pcur[k] = -1;
#pragma unroll
                    for (int p = 0; p < NP; ++p) pacc[k][p] = make_float2(0.f, 0.f);
                }
            }
            float4 q[NP][RY][QN];
            {   // planes z0 - R .. z0 + R - 1 of the queue; each stage then brings plane z + R
                int wz = z0 - R < 0 ? z0 - R + n3 : z0 - R;
#pragma unroll
                for (int s2 = 0; s2 < 2 * R; ++s2) {
#pragma unroll
                    for (int p = 0; p < NP; ++p)
#pragma unroll
                        for (int rr = 0; rr < RY; ++rr)
                            q[p][rr][s2] = p < nvalid ? *reinterpret_cast<const float4*>(
                                                            Yg + p * ngu + (unsigned)(wz * plane) + gxy + rr * N1)
                                                      : make_float4(0.f, 0.f, 0.f, 0.f);
                    if (++wz == n3) wz = 0;
                }
            }
            for (int zb = z0; zb < z1 && ok; zb += QN) {
#pragma unroll
                for (int ph = 0; ph < QN; ++ph) {
                    const int z = zb + ph;
                    if (z < z1 && ok) {
                        const int s = j % D;
                        // a warp-uniform outcome keeps the __syncwarp below convergent
                        if (!__all_sync(0xffffffffu, mb_wait(&full[s], (j / D) & 1))) {
                            ok = false;
                            if ((tid & 31) == 0) atomicExch(err, 2);
                            break;
                        }
                        const uint32_t st = smem_s + (uint32_t)(s * A.sstride);
#pragma unroll
                        for (int p = 0; p < NP; ++p)   // plane z + R of the queue (zero rows past ncolE)
#pragma unroll
                            for (int rr = 0; rr < RY; ++rr)
                                q[p][rr][(ph + 2 * R) % QN] =
                                    lds128(st + L::OFF_Q + (uint32_t)(((p * TY + ty0 + rr) * N1 + gx) * 8));
                        const unsigned g = (unsigned)(z * plane) + gxy;
#pragma unroll
                        for (int rr = 0; rr < RY; ++rr) {
                            const int ty = ty0 + rr;
                            const float2 vv = lds64(st + L::OFF_V + (uint32_t)((ty * N1 + gx) * 4));
                            // KB term of both points and all NP pairs: the slot tables are read once per
                            // plane; the coefficient of pair p and atom a sits at [p][a] of the stage's
                            // window, and an unused slot (atom -1, or a slot past the table: atom 0,
                            // value 0) contributes exactly zero
                            float2 kb0[NP], kb1[NP];
#pragma unroll
                            for (int p = 0; p < NP; ++p) kb0[p] = kb1[p] = make_float2(0.f, 0.f);
                            // fused projection: weights of the two points in each slot's running sum, and the
                            // slots whose second point belongs to another atom (added at once)
                            float pw0[PROJ ? S : 1], pw1[PROJ ? S : 1];
                            unsigned pstray = 0u;
                            if (KB) {
                                const uint32_t Cg = st + kco;
#pragma unroll
                                for (int k = 0; k < S; ++k) {
                                    const int2 ka = lds64i(st + L::OFF_KA + (uint32_t)(((k * TY + ty) * N1 + gx) * 4));
                                    const float2 kv = lds64(st + L::OFF_KV + (uint32_t)(((k * TY + ty) * N1 + gx) * 4));
                                    const bool v0 = (unsigned)ka.x < (unsigned)A.natom;
                                    const bool v1 = (unsigned)ka.y < (unsigned)A.natom;
                                    if (PROJ) {
                                        const int a0 = (v0 && kv.x != 0.f) ? ka.x : -1;
                                        const int a1 = (v1 && kv.y != 0.f) ? ka.y : -1;
                                        const int t = a0 >= 0 ? a0 : a1;
                                        if (t != pcur[k]) {
                                            pflush(k);
                                            pcur[k] = t;
                                        }
                                        pw0[k] = a0 >= 0 ? kv.x : 0.f;
                                        pw1[k] = (a1 >= 0 && a1 == t) ? kv.y : 0.f;
                                        if (a1 >= 0 && a1 != t) pstray |= 1u << k;
                                    }
                                    const uint32_t c0p = Cg + (v0 ? (uint32_t)ka.x * 8u : 0u);
                                    const uint32_t c1p = Cg + (v1 ? (uint32_t)ka.y * 8u : 0u);
#pragma unroll
                                    for (int p = 0; p < NP; ++p) {
                                        const float2 z2 = make_float2(0.f, 0.f);
                                        const float2 g0 = lds64(c0p + (uint32_t)(p * A.natom * 8));
                                        const float2 g1 = lds64(c1p + (uint32_t)(p * A.natom * 8));
                                        kb0[p] = fma2(kv.x, v0 ? g0 : z2, kb0[p]);
                                        kb1[p] = fma2(kv.y, v1 ? g1 : z2, kb1[p]);
                                    }
                                }
                            }
#pragma unroll
                            for (int p = 0; p < NP; ++p) {
                                const uint32_t T = st + (uint32_t)((p * L::TILE_PAIR + (R + ty) * N1) * 8);
                                const float4 cen = q[p][rr][(ph + R) % QN];
                                const float2 c0v = lo2(cen), c1v = hi2(cen);
                                float2 a0 = fma2(A.c0, c0v, kb0[p]);
                                float2 a1 = fma2(A.c0, c1v, kb1[p]);
                                float2 b0 = make_float2(0.f, 0.f), b1 = b0, d0 = b0, d1 = b0;
                                {   // x: points x-6 .. x+7 of the pair from six 16-byte reads
                                    const float4 L0 = lds128(T + xc[0]);
                                    const float4 L1 = lds128(T + xc[1]);
                                    const float4 L2 = lds128(T + xc[2]);
                                    const float4 R0 = lds128(T + xc[3]);
                                    const float4 R1 = lds128(T + xc[4]);
                                    const float4 R2 = lds128(T + xc[5]);
                                    a0 = fma2(A.cx[1], add2(hi2(L2), c1v), a0);
                                    a0 = fma2(A.cx[2], add2(lo2(L2), lo2(R0)), a0);
                                    a0 = fma2(A.cx[3], add2(hi2(L1), hi2(R0)), a0);
                                    a0 = fma2(A.cx[4], add2(lo2(L1), lo2(R1)), a0);
                                    a0 = fma2(A.cx[5], add2(hi2(L0), hi2(R1)), a0);
                                    a0 = fma2(A.cx[6], add2(lo2(L0), lo2(R2)), a0);
                                    a1 = fma2(A.cx[1], add2(c0v, lo2(R0)), a1);
                                    a1 = fma2(A.cx[2], add2(hi2(L2), hi2(R0)), a1);
                                    a1 = fma2(A.cx[3], add2(lo2(L2), lo2(R1)), a1);
                                    a1 = fma2(A.cx[4], add2(hi2(L1), hi2(R1)), a1);
                                    a1 = fma2(A.cx[5], add2(lo2(L1), lo2(R2)), a1);
                                    a1 = fma2(A.cx[6], add2(hi2(L0), hi2(R2)), a1);
                                }
                                // y: rows of this thread's own RY rows come from the registers of the queue
                                const uint32_t Tc = T + (uint32_t)(gx * 8);
#pragma unroll
                                for (int r = 1; r <= R; ++r) {
                                    float4 up, dn;
                                    if (rr - r >= 0) up = q[p][rr - r >= 0 ? rr - r : 0][(ph + R) % QN];
                                    else up = lds128(Tc - (uint32_t)(r * N1 * 8));
                                    if (rr + r < RY) dn = q[p][rr + r < RY ? rr + r : 0][(ph + R) % QN];
                                    else dn = lds128(Tc + (uint32_t)(r * N1 * 8));
                                    const float4 zu = q[p][rr][(ph + R + r) % QN], zd = q[p][rr][(ph + R - r + QN) % QN];
                                    b0 = fma2(A.cy[r], add2(lo2(up), lo2(dn)), b0);
                                    b1 = fma2(A.cy[r], add2(hi2(up), hi2(dn)), b1);
                                    d0 = fma2(A.cz[r], add2(lo2(zu), lo2(zd)), d0);
                                    d1 = fma2(A.cz[r], add2(hi2(zu), hi2(zd)), d1);
                                }
                                a0 = add2(a0, add2(b0, d0));
                                a1 = add2(a1, add2(b1, d1));
                                a0 = fma2(vv.x, c0v, a0);
                                a1 = fma2(vv.y, c1v, a1);
                                float2 o0 = fma2(A.alpha, fma2(-A.shift, c0v, a0), make_float2(0.f, 0.f));
                                float2 o1 = fma2(A.alpha, fma2(-A.shift, c1v, a1), make_float2(0.f, 0.f));
                                if (PREV) {
                                    const float4 pv = lds128(st + L::OFF_PREV + (uint32_t)(((p * TY + ty) * N1 + gx) * 8));
                                    o0 = fma2(-A.beta, lo2(pv), o0);
                                    o1 = fma2(-A.beta, hi2(pv), o1);
                                }
                                if (p < nvalid)
                                    *reinterpret_cast<float4*>(Zg + p * ngu + g + rr * N1) =
                                        make_float4(o0.x, o0.y, o1.x, o1.y);
                                if (PROJ) {
#pragma unroll
                                    for (int k = 0; k < S; ++k) {
                                        pacc[k][p] = fma2(pw0[k], o0, pacc[k][p]);
                                        pacc[k][p] = fma2(pw1[k], o1, pacc[k][p]);
                                        if ((pstray >> k) & 1u) {   // rare: reread the slot of the second point
                                            const int a1 = lds64i(st + L::OFF_KA + (uint32_t)(((k * TY + ty) * N1 + gx) * 4)).y;
                                            const float w1 = lds64(st + L::OFF_KV + (uint32_t)(((k * TY + ty) * N1 + gx) * 4)).y;
                                            if (p < nvalid)
                                                red_add2(Cn + (size_t)(col0 + p) * A.natom + a1,
                                                         make_float2(w1 * o1.x, w1 * o1.y));
                                        }
                                    }
                                }
                            }
                        }
                        // this warp has read the stage: release it to the producer
                        __syncwarp();
                        if ((tid & 31) == 0) mb_arrive(&empty[s]);
                        ++j;
                    }
                }
            }
            if (PROJ && ok) {
#pragma unroll
                for (int k = 0; k < S; ++k) pflush(k);
            }
            f += z1 - z0;
        }
    }
    // every thread reaches this barrier; then drain the copies the producer issued so that no TMA
    // write is in flight when the CTA's shared memory is released
    __syncthreads();
    if (tid == NCOMP) {
        for (int j = max(0, issued - D); j < issued; ++j) {
            const int s = j % D;
            if (!mb_wait(&full[s], (j / D) & 1)) break;
        }
    }
}

// C[col][a] *= gamma_a over ne = ncol * natom coefficients (the fused projection's last factor)
__global__ void kb_gamma_scale_kernel(float2* __restrict__ C, const double* __restrict__ gamma, int natom,
                                      long long ne) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < ne; i += (long long)gridDim.x * blockDim.x) {
        const float g = (float)gamma[i % natom];
        C[i] = make_float2(g * C[i].x, g * C[i].y);
    }
}

// ---- host side: tensor maps ----------------------------------------------------------
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        cudaGetLastError();
    });
    SDFT_REQUIRE(fn != nullptr, SDFT_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
    return fn;
}

void encode(CUtensorMap* m, CUtensorMapDataType t, int rank, const void* base, const cuuint64_t* dims,
            const cuuint64_t* strides_bytes, const cuuint32_t* box) {
    cuuint32_t es[5] = {1, 1, 1, 1, 1};
    const CUresult r = encode_fn()(m, t, (cuuint32_t)rank, const_cast<void*>(base), dims, strides_bytes, box, es,
                                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                   CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    SDFT_REQUIRE(r == CUDA_SUCCESS, SDFT_ERR_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
}

// 4-D map of an FP32 paired block [ncolE][n3][n2][n1] (float2 elements) with box (n1, rows, 1, pairs)
void block_map(CUtensorMap* m, const sdft_ctx* c, const float2* base, int ncolE, int rows, int pairs) {
    const cuuint64_t dims[4] = {(cuuint64_t)c->n[0], (cuuint64_t)c->n[1], (cuuint64_t)c->n[2], (cuuint64_t)ncolE};
    const cuuint64_t st[3] = {(cuuint64_t)c->n[0] * 8, (cuuint64_t)c->n[0] * c->n[1] * 8, (cuuint64_t)c->ng * 8};
    const cuuint32_t box[4] = {(cuuint32_t)c->n[0], (cuuint32_t)rows, 1, (cuuint32_t)pairs};
    encode(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 4, base, dims, st, box);
}

}  // namespace

// tiled tensor map with a chosen swizzle (the tensor-core GEMMs' copies)
void tma_encode_tiled(CUtensorMap* m, CUtensorMapDataType t, int rank, const void* base, const cuuint64_t* dims,
                      const cuuint64_t* strides_bytes, const cuuint32_t* box, CUtensorMapSwizzle sw) {
    cuuint32_t es[5] = {1, 1, 1, 1, 1};
    const CUresult r = encode_fn()(m, t, (cuuint32_t)rank, const_cast<void*>(base), dims, strides_bytes, box, es,
                                   CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    SDFT_REQUIRE(r == CUDA_SUCCESS, SDFT_ERR_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
}

int sm_count() {
    static int nsm = 0;
    if (nsm == 0) {
        int dev = 0;
        SDFT_CUDA(cudaGetDevice(&dev));
        SDFT_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    }
    return nsm;
}

// the persistent schedule of a slab launch (see launch_slab_variant): CTAs per slab, units per CTA
struct SlabSchedule {
    int nper, per_cta;
};
SlabSchedule slab_schedule(const sdft_ctx* c, int ncolE, int NP, int TY, int MINB) {
    const int nslab = c->n[1] / TY, ngrp = (ncolE + NP - 1) / NP;
    const int total = ngrp * c->n[2];
    SlabSchedule s;
    s.nper = std::max(1, std::min(sm_count() * MINB / nslab, total));
    s.per_cta = (total + s.nper - 1) / s.nper;
    return s;
}

// row of the variant table: usable when the grid's n1 is the template's, TY divides n2 with at
// least two slabs, the block is real FP32, the KB table has at most S slots per point, and the
// D stages with their KB coefficient windows fit in shared memory (every slab variant is
// instantiated with one CTA per SM)
template <int N1, int TY, int NP, int S, int D>
bool slab_variant_ok(const sdft_ctx* c, int ncolE) {
    if (c->n[0] != N1 || c->n[1] % TY || c->n[1] < 2 * TY || TY < R || ncolE <= 0) return false;
    for (const KBTables& kb : c->kb)
        if (kb.cplx || kb.S > S) return false;
    return slab_smem_bytes<N1, TY, NP, S, D>(c->natom) <= 227 * 1024;
}

template <int N1, int TY, int NP, int RY, int S, int D, int MINB>
void launch_slab_variant(sdft_ctx* c, int kpt, const float2* Y, const float2* Yprev, float2* Ynext, int ncolE,
                         const float* V, const float2* kbC, double alpha, double beta, double shift, bool kin,
                         bool timed) {
    SDFT_REQUIRE(kin && V != nullptr, SDFT_ERR_INVALID_ARG, "slab stencil variant needs V and the kinetic term");
    SDFT_REQUIRE((slab_variant_ok<N1, TY, NP, S, D>(c, ncolE)), SDFT_ERR_INVALID_ARG, "slab stencil variant does not fit");
    const KBTables& kb = c->kb[kpt];
    const bool prev = Yprev != nullptr, haskb = kbC != nullptr && kb.S > 0;
    const int nslab = c->n[1] / TY, ngrp = (ncolE + NP - 1) / NP;
    SDFT_REQUIRE((long long)nslab * ngrp * c->n[2] < (1LL << 30) && (long long)ncolE * c->ng < (1LL << 31),
                 SDFT_ERR_INVALID_ARG, "slab stencil: block too large for 32-bit offsets");
    // every slab gets the same number of CTAs, which take equal runs of its (pair group, plane) units in
    // the same order: CTAs of neighbouring slabs then work on the same planes of the same pairs at the
    // same time, so the y-halo rows one slab reads are the interior rows its neighbour has just pulled
    // into L2 (a few SMs may stay idle so that the counts are equal)
    const int total = ngrp * c->n[2];
    const SlabSchedule sch = slab_schedule(c, ncolE, NP, TY, MINB);
    const int nper = sch.nper, per_cta = sch.per_cta;
    const int nblk = nper * nslab;
    const size_t dsm = slab_smem_bytes<N1, TY, NP, S, D>(c->natom);
    // the coefficient window of the last group reads at most (ncolE + NP - 1) * natom + 1 float2 of C
    SDFT_REQUIRE(!haskb || ((kbC == reinterpret_cast<const float2*>(c->C32) ||
                             kbC == reinterpret_cast<const float2*>(c->C32b)) &&
                            ((uintptr_t)kbC & 15) == 0 && (long long)(ncolE + NP - 1) * c->natom + 1 <= c->c32_elems),
                 SDFT_ERR_INVALID_ARG, "slab stencil: KB coefficient buffer misaligned or too short");
    SlabArgs A;
    for (int r = 0; r <= R; ++r) {
        A.cx[r] = (float)c->coef.cx[r];
        A.cy[r] = (float)c->coef.cy[r];
        A.cz[r] = (float)c->coef.cz[r];
    }
    A.c0 = (float)c->coef.c0;
    A.alpha = (float)alpha;
    A.beta = (float)beta;
    A.shift = (float)shift;
    A.n2 = c->n[1];
    A.n3 = c->n[2];
    A.ncolE = ncolE;
    A.nslab = nslab;
    A.sstride = SlabLayout<N1, TY, NP, S>::STAGE + slab_kc_bytes(NP, c->natom);
    A.total = total;
    A.per_cta = per_cta;
    A.natom = c->natom;
    A.ng = c->ng;
    // tensor maps (FP64 element type: each float2 is moved as one 8-byte element)
    CUtensorMap mfull, m6, mmid, mp, mv, mka, mkv;
    block_map(&mfull, c, Y, ncolE, TY + 2 * R, NP);
    block_map(&m6, c, Y, ncolE, R, 1);
    block_map(&mmid, c, Y, ncolE, TY + R, 1);
    block_map(&mp, c, prev ? Yprev : Y, ncolE, TY, NP);
    CUtensorMap mq;
    block_map(&mq, c, Y, ncolE, TY, NP);
    {
        const cuuint64_t dims[3] = {(cuuint64_t)c->n[0], (cuuint64_t)c->n[1], (cuuint64_t)c->n[2]};
        const cuuint64_t st[2] = {(cuuint64_t)c->n[0] * 4, (cuuint64_t)c->n[0] * c->n[1] * 4};
        const cuuint32_t box[3] = {(cuuint32_t)N1, (cuuint32_t)TY, 1};
        encode(&mv, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, V, dims, st, box);
    }
    if (haskb) {
        const cuuint64_t dims[4] = {(cuuint64_t)c->n[0], (cuuint64_t)c->n[1], (cuuint64_t)c->n[2], (cuuint64_t)S};
        const cuuint64_t st[3] = {(cuuint64_t)c->n[0] * 4, (cuuint64_t)c->n[0] * c->n[1] * 4, (cuuint64_t)c->ng * 4};
        const cuuint32_t box[4] = {(cuuint32_t)N1, (cuuint32_t)TY, 1, (cuuint32_t)S};
        // slots kb.S .. S-1 do not exist in the table: reading them would leave its allocation, so the
        // map's slot extent is kb.S and TMA fills the missing slots with zeros (atom 0, value 0)
        const cuuint64_t dims_k[4] = {dims[0], dims[1], dims[2], (cuuint64_t)kb.S};
        encode(&mka, CU_TENSOR_MAP_DATA_TYPE_INT32, 4, kb.patom, dims_k, st, box);
        encode(&mkv, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, kb.pval32, dims_k, st, box);
    } else {
        mka = mv;
        mkv = mv;
    }
    dim3 grid((unsigned)nblk);
    dim3 block((TY / RY) * (N1 / 2) + 32);
    int* err = stencil_error_flag(c);
    ScopedTimer timer(timed ? c : nullptr, SDFT_K_STENCIL,
                      (double)ncolE * (double)c->ng * sizeof(float2) * (prev ? 3.0 : 2.0));
#define SDFT_SLAB(P, K, J)                                                                                       \
    do {                                                                                                         \
        auto kfn = cheb_slab_kernel<N1, TY, NP, RY, S, D, MINB, P, K, J>;                                         \
        SDFT_CUDA(cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dsm));             \
        kfn<<<grid, block, dsm, c->stream>>>(Y, Ynext, kbC, Cn, mfull, m6, mmid, mp, mv, mka, mkv, mq, A, err);    \
    } while (0)
    // fused projection of the output's KB coefficients into the buffer the caller offered
    float2* Cn = (haskb && RY == 1) ? c->kb_next : nullptr;
    if (Cn != nullptr) {
        SDFT_REQUIRE(Cn != kbC && (Cn == reinterpret_cast<float2*>(c->C32) || Cn == reinterpret_cast<float2*>(c->C32b)),
                     SDFT_ERR_INVALID_ARG, "slab stencil: fused projection target is not a KB coefficient buffer");
        SDFT_CUDA(cudaMemsetAsync(Cn, 0, sizeof(float2) * (size_t)ncolE * c->natom, c->stream));
    }
    if constexpr (RY == 1) {
        if (prev && Cn) SDFT_SLAB(true, true, true);
        else if (!prev && Cn) SDFT_SLAB(false, true, true);
        else if (prev && haskb) SDFT_SLAB(true, true, false);
        else if (!prev && haskb) SDFT_SLAB(false, true, false);
        else if (prev && !haskb) SDFT_SLAB(true, false, false);
        else SDFT_SLAB(false, false, false);
    } else {
        if (prev && haskb) SDFT_SLAB(true, true, false);
        else if (!prev && haskb) SDFT_SLAB(false, true, false);
        else if (prev && !haskb) SDFT_SLAB(true, false, false);
        else SDFT_SLAB(false, false, false);
    }
#undef SDFT_SLAB
    SDFT_CUDA(cudaGetLastError());
    count_launch(c);
    if (Cn != nullptr) {
        // Cn[col][a] *= gamma_a
        const long long ne = (long long)ncolE * c->natom;
        kb_gamma_scale_kernel<<<(unsigned)std::min<long long>((ne + 255) / 256, 1024), 256, 0, c->stream>>>(
            Cn, kb.gamma, c->natom, ne);
        SDFT_CUDA(cudaGetLastError());
        count_launch(c);
        c->kb_next_done = true;
    }
}

// instantiations used by the FP32 variant table (stencil_f32.cu)
#define SDFT_SLAB_OK(N1, TY, NP, S, D) template bool slab_variant_ok<N1, TY, NP, S, D>(const sdft_ctx*, int);
SDFT_SLAB_OK(80, 8, 2, 2, 3)
SDFT_SLAB_OK(80, 8, 1, 2, 4)
SDFT_SLAB_OK(120, 8, 1, 2, 4)
SDFT_SLAB_OK(40, 8, 2, 2, 4)
#undef SDFT_SLAB_OK
#define SDFT_SLAB_INST(N1, TY, NP, RY, S, D, MINB)                                                                 \
    template void launch_slab_variant<N1, TY, NP, RY, S, D, MINB>(sdft_ctx*, int, const float2*, const float2*,   \
                                                                 float2*, int, const float*, const float2*, double, \
                                                                 double, double, bool, bool);
SDFT_SLAB_INST(80, 8, 2, 1, 2, 3, 1)
SDFT_SLAB_INST(80, 8, 1, 1, 2, 4, 1)
SDFT_SLAB_INST(80, 8, 1, 2, 2, 4, 1)
SDFT_SLAB_INST(120, 8, 1, 1, 2, 4, 1)
SDFT_SLAB_INST(40, 8, 2, 1, 2, 4, 1)
#undef SDFT_SLAB_INST

}  // namespace sdft
