// Matrix-free Hamiltonian application fused with the Chebyshev three-term recurrence
// (paper Sec. 2.1: "Hamiltonian-matrix/vector products are performed in matrix-free fashion,
// using the finite-difference stencil for the Laplacian and the outer product nature of the
// nonlocal pseudopotential operator"; filter of Zhou et al. 2006 / Zhou & Saad 2007).
//
//   Ynext = alpha * (H Y - shift * Y) - beta * Yprev,
//   H Y   = -1/2 L_h Y + V .* Y + sum_a beta_a (gamma_a beta_a^H Y)
//
// Kernel design (GB300): one CTA owns a TX x TY column tile of the grid and marches along z
// for one element-column.  The 13 z-neighbours of each thread's point live in a register
// queue (plus PF planes of prefetch), so every Y value enters the SM once from its own
// column; only the x/y halo of the current plane goes through shared memory (double-buffered,
// one __syncthreads per plane).  Periodic/Bloch wrap is done with index arithmetic on the
// loads (TMA's zero fill cannot express a periodic halo).  FP32 blocks carry two lanes per
// element (two orbitals, or re/im) and use Blackwell's packed f32x2 FMA.
#pragma once
#include <type_traits>
#include "internal.cuh"

namespace sdft {
namespace {

// ---- element arithmetic ---------------------------------------------------------------
__device__ __forceinline__ unsigned long long f2u(float2 a) {
    return (unsigned long long)__float_as_uint(a.x) | ((unsigned long long)__float_as_uint(a.y) << 32);
}
__device__ __forceinline__ float2 u2f(unsigned long long u) {
    return make_float2(__uint_as_float((unsigned)(u & 0xffffffffu)), __uint_as_float((unsigned)(u >> 32)));
}
// acc + s * a   (scalar s broadcast to both lanes)
__device__ __forceinline__ float2 efma(float s, float2 a, float2 acc) {
    unsigned long long r;
    unsigned long long ss = f2u(make_float2(s, s));
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(ss), "l"(f2u(a)), "l"(f2u(acc)));
    return u2f(r);
}
__device__ __forceinline__ float2 eadd(float2 a, float2 b) {
    unsigned long long r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2u(a)), "l"(f2u(b)));
    return u2f(r);
}
__device__ __forceinline__ double efma(double s, double a, double acc) { return fma(s, a, acc); }
__device__ __forceinline__ float efma(float s, float a, float acc) { return fmaf(s, a, acc); }
__device__ __forceinline__ float eadd(float a, float b) { return a + b; }
__device__ __forceinline__ double eadd(double a, double b) { return a + b; }
__device__ __forceinline__ double2 efma(double s, double2 a, double2 acc) {
    return make_double2(fma(s, a.x, acc.x), fma(s, a.y, acc.y));
}
__device__ __forceinline__ double2 eadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }

template <typename E> __device__ __forceinline__ E ezero();
template <> __device__ __forceinline__ float2 ezero<float2>() { return make_float2(0.f, 0.f); }
template <> __device__ __forceinline__ double ezero<double>() { return 0.0; }
template <> __device__ __forceinline__ float ezero<float>() { return 0.f; }
template <> __device__ __forceinline__ double2 ezero<double2>() { return make_double2(0.0, 0.0); }

// complex multiply (for CPLX element types): a * b
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cmul_conj(float2 a, float2 b) {  // conj(a) * b
    return make_float2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ double2 cmul_conj(double2 a, double2 b) {
    return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}

template <typename S>
struct StepArgs {
    S cx[FD_RADIUS + 1], cy[FD_RADIUS + 1], cz[FD_RADIUS + 1];
    S c0, alpha, beta, shift;
    S phr[3], phi[3];           // Bloch phase exp(2 pi i kappa_d) per axis
    int n1, n2, n3, zchunk, nzc, natom;
    long long ng;
};

__device__ __forceinline__ int wrapi(int x, int n, int& t) {
    // x in any range -> [0, n), t = floor(x / n)
    int q = x / n;
    int r = x - q * n;
    if (r < 0) { r += n; --q; }
    t = q;
    return r;
}

template <typename E, typename S>
__device__ __forceinline__ E apply_phase(E v, int t, S pr, S pi) {
    return v;
}
template <>
__device__ __forceinline__ float2 apply_phase<float2, float>(float2 v, int t, float pr, float pi) {
    // v * (pr + i pi)^t, t small
    float2 w = v;
    if (t > 0) {
        for (int k = 0; k < t; ++k) w = cmul(w, make_float2(pr, pi));
    } else {
        for (int k = 0; k < -t; ++k) w = cmul(w, make_float2(pr, -pi));
    }
    return w;
}
template <>
__device__ __forceinline__ double2 apply_phase<double2, double>(double2 v, int t, double pr, double pi) {
    double2 w = v;
    if (t > 0) {
        for (int k = 0; k < t; ++k) w = cmul(w, make_double2(pr, pi));
    } else {
        for (int k = 0; k < -t; ++k) w = cmul(w, make_double2(pr, -pi));
    }
    return w;
}

// Column of a load: flat xy offset of the wrapped (x, y) and its Bloch phase (complex blocks).
template <typename E>
struct ColRef {
    long long base;
    E ph;
};

template <typename E> __device__ __forceinline__ E eone();
template <> __device__ __forceinline__ float2 eone<float2>() { return make_float2(1.f, 0.f); }
template <> __device__ __forceinline__ double eone<double>() { return 1.0; }
template <> __device__ __forceinline__ float eone<float>() { return 1.f; }
template <> __device__ __forceinline__ double2 eone<double2>() { return make_double2(1.0, 0.0); }

template <typename E, typename S, bool CPLX>
__device__ __forceinline__ ColRef<E> make_col(int x, int y, const StepArgs<S>& A) {
    int tx, ty;
    int wx = wrapi(x, A.n1, tx), wy = wrapi(y, A.n2, ty);
    ColRef<E> r;
    r.base = (long long)wy * A.n1 + wx;
    r.ph = eone<E>();
    if constexpr (CPLX) {
        if (tx) r.ph = apply_phase<E, S>(r.ph, tx, A.phr[0], A.phi[0]);
        if (ty) r.ph = apply_phase<E, S>(r.ph, ty, A.phr[1], A.phi[1]);
    }
    return r;
}

// load the element of column `cr` at unwrapped plane z (Bloch phases for complex blocks)
template <typename E, typename S, bool CPLX>
__device__ __forceinline__ E load_col(const E* __restrict__ Yc, const ColRef<E>& cr, int z,
                                      const StepArgs<S>& A) {
    int tz;
    const int wz = wrapi(z, A.n3, tz);
    E v = Yc[(long long)wz * A.n1 * A.n2 + cr.base];
    if constexpr (CPLX) {
        if constexpr (Elem<E>::lanes == 2 && !std::is_same<E, double>::value) {
            v = cmul(v, cr.ph);
            if (tz) v = apply_phase<E, S>(v, tz, A.phr[2], A.phi[2]);
        }
    }
    return v;
}

// Wrapped plane index advanced one plane at a time (no division in the loop): wz = z mod n3,
// tz = floor(z / n3) (Bloch wrap count), off = wz * n1 * n2.
struct ZTrack {
    int wz, tz;
    long long off;
};
__device__ __forceinline__ void ztrack_init(ZTrack& t, int z, int n3, long long plane) {
    t.wz = wrapi(z, n3, t.tz);
    t.off = (long long)t.wz * plane;
}
__device__ __forceinline__ void ztrack_next(ZTrack& t, int n3, long long plane) {
    if (++t.wz == n3) {
        t.wz = 0;
        ++t.tz;
        t.off = 0;
    } else {
        t.off += plane;
    }
}

template <typename E, typename S, bool CPLX>
__device__ __forceinline__ E load_at(const E* __restrict__ Yc, long long idx, const E& colph, int tz,
                                     const StepArgs<S>& A) {
    E v = Yc[idx];
    if constexpr (CPLX) {
        v = cmul(v, colph);
        if (tz) v = apply_phase<E, S>(v, tz, A.phr[2], A.phi[2]);
    }
    return v;
}

// ---- asynchronous global -> shared copies (cp.async, LDGSTS) ---------------------------
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
template <int BYTES>
__device__ __forceinline__ void cp_async(void* smem_dst, const void* gsrc) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(smem_u32(smem_dst)), "l"(gsrc), "n"(BYTES));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

// Shared-memory stage of one z-plane: the x/y halo tile (interior filled from the register
// queue), and the per-point operands Yprev, V and the KB slots of the TX x TY columns.
template <typename E, typename S, typename KV, int TX, int TY, int SP>
struct Stage {
    E tile[TY + 2 * FD_RADIUS][TX + 2 * FD_RADIUS];
    E prev[TY][TX];
    S v[TY][TX];
    int kat[SP][TY][TX];
    KV kval[SP][TY][TX];
};

// One CTA: TX x TY grid columns, planes [z0, z1), one element-column (orbital pair / Bloch
// orbital).  z-neighbours: register queue, loaded PF planes ahead.  x/y halo and per-point
// operands: D-stage cp.async ring, issued D-1 planes ahead, one __syncthreads per plane.
// Body of the column tile for block (bx, by, bz) = (x tile, y tile, column * nzc + z chunk).
template <typename E, bool CPLX, int TX, int TY, int PF, int D, bool PREV, bool KB, bool VLOC, bool KIN>
__device__ __forceinline__ void
cheb_step_body(const E* __restrict__ Y, const E* __restrict__ Yprev, E* __restrict__ Ynext,
               const typename Elem<E>::S* __restrict__ V, const E* __restrict__ C,
               const int* __restrict__ patom, const void* __restrict__ pval, const int nslot,
               const StepArgs<typename Elem<E>::S>& A, const int bx, const int by, const int bz) {
    using S = typename Elem<E>::S;
    using KV = typename std::conditional<CPLX, E, S>::type;   // KB value type at a grid point
    constexpr int R = FD_RADIUS;
    constexpr int QN = 2 * R + 1 + PF;      // register queue length
    constexpr int NT = TX * TY;
    constexpr int NHALO = 2 * R * (TX + TY);
    constexpr int HPT = (NHALO + NT - 1) / NT;  // halo elements per thread
    constexpr int SP = 3;                   // KB slots staged per point (more are read directly)
    using St = Stage<E, S, KV, TX, TY, SP>;
    extern __shared__ __align__(16) unsigned char dyn_smem[];
    St* stage = reinterpret_cast<St*>(dyn_smem);
    E* Cs = reinterpret_cast<E*>(dyn_smem + sizeof(St) * D);  // KB coefficients of this column [natom]

    const int tx = threadIdx.x, ty = threadIdx.y;
    const int tid = ty * TX + tx;
    const int x0 = bx * TX, y0 = by * TY;
    const int col = bz / A.nzc;
    const int zc = bz - col * A.nzc;
    const int z0 = zc * A.zchunk;
    const int z1 = min(A.n3, z0 + A.zchunk);
    const int gx = x0 + tx, gy = y0 + ty;
    const bool valid = gx < A.n1 && gy < A.n2;
    const long long plane = (long long)A.n1 * A.n2;
    const E* __restrict__ Yc = Y + (long long)col * A.ng;
    const E* __restrict__ Pc = Yprev + (long long)col * A.ng;
    const KV* __restrict__ pv = reinterpret_cast<const KV*>(pval);
    if (KB)
        for (int i = tid; i < A.natom; i += NT) Cs[i] = C[(long long)col * A.natom + i];

    // halo slots owned by this thread: local (ly, lx) in the tile
    int hly[HPT], hlx[HPT];
    ColRef<E> hcol[HPT];
#pragma unroll
    for (int k = 0; k < HPT; ++k) {
        int i = tid + k * NT;
        if (i < 2 * R * TY) {               // x halo: rows 0..TY-1, 6 columns left and right
            int row = i / (2 * R), j = i - row * (2 * R);
            hly[k] = R + row;
            hlx[k] = j < R ? j : TX + j;
        } else if (i < NHALO) {             // y halo: 6 rows above and below, TX columns
            int j = i - 2 * R * TY;
            int row = j / TX, cc = j - row * TX;
            hly[k] = row < R ? row : TY + row;
            hlx[k] = R + cc;
        } else {
            hly[k] = -1;
            hlx[k] = 0;
        }
        hcol[k] = make_col<E, S, CPLX>(x0 - R + hlx[k], y0 - R + max(hly[k], 0), A);
    }
    const ColRef<E> mycol = make_col<E, S, CPLX>(gx, gy, A);
    const long long gxy = (long long)gy * A.n1 + gx;

    // issue the cp.async copies of plane z (always inside [0, n3): no z wrap) into stage st
    auto issue = [&](int z, int st) {
        if (z < z1) {
            St& S_ = stage[st];
            const long long off = (long long)z * plane;
#pragma unroll
            for (int k = 0; k < HPT; ++k)
                if (hly[k] >= 0) cp_async<sizeof(E)>(&S_.tile[hly[k]][hlx[k]], Yc + off + hcol[k].base);
            if (valid) {
                const long long g = off + gxy;
                if (PREV) cp_async<sizeof(E)>(&S_.prev[ty][tx], Pc + g);
                if (VLOC) cp_async<sizeof(S)>(&S_.v[ty][tx], V + g);
                if (KB) {
#pragma unroll
                    for (int s2 = 0; s2 < SP; ++s2)
                        if (s2 < nslot) {
                            cp_async<4>(&S_.kat[s2][ty][tx], patom + s2 * A.ng + g);
                            cp_async<sizeof(KV)>(&S_.kval[s2][ty][tx], pv + s2 * A.ng + g);
                        }
                }
            }
        }
        cp_async_commit();  // one group per plane, possibly empty, keeps the group count uniform
    };

    E q[QN];
    ZTrack zq;   // plane z + R + PF, the next queue load
    {
        ZTrack t;
        ztrack_init(t, z0 - R, A.n3, plane);
#pragma unroll
        for (int s2 = 0; s2 < 2 * R + PF; ++s2) {
            q[s2] = load_at<E, S, CPLX>(Yc, t.off + mycol.base, mycol.ph, t.tz, A);
            ztrack_next(t, A.n3, plane);
        }
        zq = t;
    }
#pragma unroll
    for (int d = 0; d < D - 1; ++d) issue(z0 + d, d);

    for (int zb = z0; zb < z1; zb += QN) {
#pragma unroll
        for (int ph = 0; ph < QN; ++ph) {
            const int z = zb + ph;
            if (z < z1) {
                const int st = (z - z0) % D;
                St& S_ = stage[st];
                const E center = q[(ph + R) % QN];
                // plane z: own copies complete, interior from the queue, Bloch phases on the halo
                cp_async_wait<D - 2>();
                S_.tile[R + ty][R + tx] = center;
                if constexpr (CPLX) {
#pragma unroll
                    for (int k = 0; k < HPT; ++k)
                        if (hly[k] >= 0) S_.tile[hly[k]][hlx[k]] = cmul(S_.tile[hly[k]][hlx[k]], hcol[k].ph);
                }
                // next queue plane (register prefetch PF planes ahead)
                q[(ph + 2 * R + PF) % QN] = load_at<E, S, CPLX>(Yc, zq.off + mycol.base, mycol.ph, zq.tz, A);
                ztrack_next(zq, A.n3, plane);
                __syncthreads();
                // every thread finished plane z-1: its stage takes plane z+D-1
                issue(z + D - 1, (z - z0 + D - 1) % D);
                if (valid) {
                    const long long g = (long long)z * plane + gxy;
                    E acc = ezero<E>();
                    if (KIN) {
                        // three independent chains (z, x, y) instead of one 19-deep FMA chain
                        E az = efma(A.c0, center, ezero<E>()), ax = ezero<E>(), ay = ezero<E>();
#pragma unroll
                        for (int r = 1; r <= R; ++r) {
                            az = efma(A.cz[r], eadd(q[(ph + R + r) % QN], q[(ph + R - r + QN) % QN]), az);
                            ax = efma(A.cx[r], eadd(S_.tile[R + ty][R + tx + r], S_.tile[R + ty][R + tx - r]), ax);
                            ay = efma(A.cy[r], eadd(S_.tile[R + ty + r][R + tx], S_.tile[R + ty - r][R + tx]), ay);
                        }
                        acc = eadd(az, eadd(ax, ay));
                    }
                    if (VLOC) acc = efma(S_.v[ty][tx], center, acc);
                    if (KB) {
                        // sum_s beta_s(g) * C[atom_s]: slots are padded with atom -1
#pragma unroll
                        for (int s2 = 0; s2 < SP; ++s2) {
                            if (s2 < nslot) {
                                const int a2 = S_.kat[s2][ty][tx];
                                if (a2 >= 0) {
                                    if constexpr (CPLX) acc = eadd(acc, cmul(S_.kval[s2][ty][tx], Cs[a2]));
                                    else acc = efma(S_.kval[s2][ty][tx], Cs[a2], acc);
                                }
                            }
                        }
                        for (int s2 = SP; s2 < nslot; ++s2) {
                            const int a2 = __ldg(patom + s2 * A.ng + g);
                            if (a2 >= 0) {
                                if constexpr (CPLX) acc = eadd(acc, cmul(pv[s2 * A.ng + g], Cs[a2]));
                                else acc = efma(pv[s2 * A.ng + g], Cs[a2], acc);
                            }
                        }
                    }
                    // out = alpha * (acc - shift * center) - beta * prev
                    E t = efma(-A.shift, center, acc);
                    E out = ezero<E>();
                    out = efma(A.alpha, t, out);
                    if (PREV) out = efma(-A.beta, S_.prev[ty][tx], out);
                    Ynext[(long long)col * A.ng + g] = out;
                }
            }
        }
    }
    cp_async_wait<0>();
}

template <typename E, bool CPLX, int TX, int TY, int PF, int MINB, int D, bool PREV, bool KB, bool VLOC, bool KIN>
__global__ void __launch_bounds__(TX * TY, MINB)
cheb_step_kernel(const E* __restrict__ Y, const E* __restrict__ Yprev, E* __restrict__ Ynext,
                 const typename Elem<E>::S* __restrict__ V, const E* __restrict__ C,
                 const int* __restrict__ patom, const void* __restrict__ pval, const int nslot, const int ncolE,
                 const __grid_constant__ StepArgs<typename Elem<E>::S> A) {
    // A is referenced in place (grid constant): no copy of the argument block
    cheb_step_body<E, CPLX, TX, TY, PF, D, PREV, KB, VLOC, KIN>(Y, Yprev, Ynext, V, C, patom, pval, nslot, A,
                                                                 blockIdx.x, blockIdx.y, blockIdx.z);
}

// ---- several grids in one launch (independent cells of uneven size, FP32 real blocks) -----
}  // namespace
struct MultiProblem {                 // one cell's block in a multi-grid launch of the column tile
    StepArgs<float> A;                // grid, coefficients, recurrence step, z chunking
    const float2* Y;
    const float2* Yprev;
    float2* Ynext;
    const float* V;
    const float2* C;
    const int* patom;
    const void* pval;
    int nslot, tiles_x, tiles_y, cta_begin, cta_end;
};
namespace {
__constant__ MultiProblem c_multi[MULTI_MAX];

// grid: the CTAs of every problem, problem p owning [cta_begin, cta_end) (tiles_x * tiles_y * ncolE * nzc)
template <int TX, int TY, int PF, int MINB, int D, bool PREV>
__global__ void __launch_bounds__(TX * TY, MINB) cheb_multi_kernel(const int nprob) {
    const int b = blockIdx.x;
    int p = 0;
    while (p + 1 < nprob && b >= c_multi[p].cta_end) ++p;
    const MultiProblem& P = c_multi[p];
    const int local = b - P.cta_begin;
    const int bx = local % P.tiles_x;
    const int rest = local / P.tiles_x;
    const int by = rest % P.tiles_y;
    const int bz = rest / P.tiles_y;
    cheb_step_body<float2, false, TX, TY, PF, D, PREV, true, true, true>(P.Y, P.Yprev, P.Ynext, P.V, P.C, P.patom,
                                                                          P.pval, P.nslot, P.A, bx, by, bz);
}

// ---- row-tile variant (FP32 blocks, n1 even) --------------------------------------------
// A CTA owns TY whole x-rows (n1 points, two consecutive points per thread, one 16-byte vector)
// and marches along z for one element-column.  Because the tile spans the full x extent, the x
// halo is the row's own periodic wrap: the threads at both row ends copy their points into
// 6-point pads on the far side of the shared-memory row (with the Bloch phase for complex
// blocks), so no x-halo is read from memory.  The 12 y-halo rows (with their pads) are
// staged by cp.async 16-byte copies in a D-stage ring; z-neighbours come from a register queue
// of 16-byte vectors.  Per-point operands (V, KB slots, Yprev) are read straight from L2.
constexpr int ROW_HALO_UNITS_PER_THREAD = 4;
constexpr int ROW_X0 = FD_RADIUS;   // shared-row entry of x = 0 (after the 6-point left pad)
// shared row stride (float2): left pad, n1 points, right pad; even, so 16-byte reads stay aligned
// (a 128-byte aligned layout measured slower: its extra padding cost one resident CTA per SM)
__host__ __device__ inline int row_stride(int n1) { return n1 + 2 * FD_RADIUS; }


template <bool CPLX, int TY, int PF, int MAXT, int MINB, int D, bool PREV, bool KB, bool VLOC>
__global__ void __launch_bounds__(MAXT, MINB)
cheb_row_kernel(const float2* __restrict__ Y_, const float2* __restrict__ Yprev_, float2* __restrict__ Ynext_,
                const float* __restrict__ V_, const float2* __restrict__ C_, const int* __restrict__ patom_,
                const void* __restrict__ pval_, const int nslot_, const StepArgs<float> A, const int ncolE,
                const RowProblem* __restrict__ grp) {
    // one problem, or (grp != null) problem blockIdx.z / (ncolE nzc) of a grouped launch
    const float2* __restrict__ Y = Y_;
    const float2* __restrict__ Yprev = Yprev_;
    float2* __restrict__ Ynext = Ynext_;
    const float* __restrict__ V = V_;
    const float2* __restrict__ C = C_;
    const int* __restrict__ patom = patom_;
    const void* __restrict__ pval = pval_;
    int nslot = nslot_;
    float alpha = A.alpha, beta = A.beta, shift = A.shift;
    float phr[3] = {A.phr[0], A.phr[1], A.phr[2]}, phi[3] = {A.phi[0], A.phi[1], A.phi[2]};
    int zlin = blockIdx.z;
    if (grp) {
        const int prob = blockIdx.z / (ncolE * A.nzc);
        zlin -= prob * ncolE * A.nzc;
        const RowProblem& P = grp[prob];
        Y = P.Y;
        Yprev = P.Yprev;
        Ynext = P.Ynext;
        V = P.V;
        C = P.C;
        patom = P.patom;
        pval = P.pval;
        nslot = P.nslot;
        alpha = P.alpha;
        beta = P.beta;
        shift = P.shift;
        for (int d = 0; d < 3; ++d) {
            phr[d] = P.phr[d];
            phi[d] = P.phi[d];
        }
    }
    using KV = typename std::conditional<CPLX, float2, float>::type;
    constexpr int R = FD_RADIUS;
    constexpr int QN = 2 * R + 1 + PF;
    constexpr int K = ROW_HALO_UNITS_PER_THREAD;
    const int HX = blockDim.x;                 // n1 / 2
    const int n1 = A.n1;
    // shared row: point x at entry ROW_X0 + x, left pad (x = -6..-1) just below, right pad
    // (x = n1..n1+5) just above
    const int RS = row_stride(n1);
    const int SE = (TY + 2 * R) * RS;          // one stage (float2)
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int NT = HX * TY, tid = ty * HX + tx;
    constexpr int SP = 3;                      // KB slots staged per point (more are read directly)
    using KV2 = typename std::conditional<CPLX, float4, float2>::type;   // KB values of two points
    extern __shared__ __align__(16) unsigned char dyn_smem[];
    float2* tiles = reinterpret_cast<float2*>(dyn_smem);
    // per-stage operands of the thread's two points: Yprev, V, KB slots (atom, value)
    unsigned char* opbase = dyn_smem + sizeof(float2) * (size_t)D * SE;
    const int opstride = (NT * (16 + 8 + SP * 8 + SP * (int)sizeof(KV2)) + 15) & ~15;   // 16-byte aligned stages
    float2* Cs = reinterpret_cast<float2*>(opbase + (size_t)D * opstride);
    auto op_prev = [&](int st) { return reinterpret_cast<float4*>(opbase + st * opstride) + tid; };
    auto op_v = [&](int st) { return reinterpret_cast<float2*>(opbase + st * opstride + NT * 16) + tid; };
    auto op_kat = [&](int st, int k) {
        return reinterpret_cast<int2*>(opbase + st * opstride + NT * 24) + k * NT + tid;
    };
    auto op_kval = [&](int st, int k) {
        return reinterpret_cast<KV2*>(opbase + st * opstride + NT * (24 + SP * 8)) + k * NT + tid;
    };
    const int y0 = blockIdx.x * TY;
    const int col = zlin / A.nzc;
    const int zc = zlin - col * A.nzc;
    const int z0 = zc * A.zchunk;
    const int z1 = min(A.n3, z0 + A.zchunk);
    const long long plane = (long long)n1 * A.n2;
    const float2* __restrict__ Yc = Y + (long long)col * A.ng;
    const int gy = y0 + ty, gx = 2 * tx;
    const long long gxy = (long long)gy * n1 + gx;
    if (KB)
        for (int i = tid; i < A.natom; i += NT) Cs[i] = C[(long long)col * A.natom + i];

    // y-halo units (two points each): 12 rows x (HX interior + 3 left-pad + 3 right-pad)
    // hdst: shared entry; complex blocks keep the unit's wrap code (tx+1) | (ty+1) << 2 in bits 24..27
    int hdst[K], hsrc[K];
    const int upr = HX + 6;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int u = tid + k * NT;
        hdst[k] = -1;
        hsrc[k] = 0;
        if (u < 2 * R * upr) {
            const int hr = u / upr, j = u - hr * upr;
            const int trow = hr < R ? hr : TY + hr;          // tile row
            int tyw;
            const int wy = wrapi(y0 - R + trow, A.n2, tyw);
            int x, entry, txw = 0;
            if (j < HX) { x = 2 * j; entry = ROW_X0 + 2 * j; }
            else if (j < HX + 3) { x = n1 - R + 2 * (j - HX); entry = ROW_X0 - R + 2 * (j - HX); txw = -1; }
            else { x = 2 * (j - HX - 3); entry = ROW_X0 + n1 + 2 * (j - HX - 3); txw = 1; }
            hdst[k] = trow * RS + entry;
            hsrc[k] = wy * n1 + x;
            if constexpr (CPLX) hdst[k] |= ((txw + 1) | ((tyw + 1) << 2)) << 24;
        }
    }
    constexpr int HMASK = CPLX ? 0xFFFFFF : -1;
    float2 phxp = make_float2(1.f, 0.f), phxm = make_float2(1.f, 0.f);   // x wrap +1 / -1
    if constexpr (CPLX) {
        phxp = make_float2(phr[0], phi[0]);
        phxm = make_float2(phr[0], -phi[0]);
    }

    const float2* __restrict__ Pc = Yprev + (long long)col * A.ng;
    auto issue = [&](int z, int st) {
        if (z < z1) {
            float2* T = tiles + st * SE;
            const long long off = (long long)z * plane;
            const float2* src = Yc + off;
#pragma unroll
            for (int k = 0; k < K; ++k)
                if (hdst[k] >= 0) cp_async<16>(T + (hdst[k] & HMASK), src + hsrc[k]);
            const long long g = off + gxy;
            if (PREV) cp_async<16>(op_prev(st), Pc + g);
            if (VLOC) cp_async<8>(op_v(st), V + g);
            if (KB) {
#pragma unroll
                for (int k = 0; k < SP; ++k)
                    if (k < nslot) {
                        cp_async<8>(op_kat(st, k), patom + k * A.ng + g);
                        cp_async<sizeof(KV2)>(op_kval(st, k), reinterpret_cast<const KV*>(pval) + k * A.ng + g);
                    }
            }
        }
        cp_async_commit();
    };
    auto ld4 = [](const float2* p) { return *reinterpret_cast<const float4*>(p); };
    auto cm = [](float4 v, float2 ph) {
        const float2 a = cmul(make_float2(v.x, v.y), ph), b = cmul(make_float2(v.z, v.w), ph);
        return make_float4(a.x, a.y, b.x, b.y);
    };

    float4 q[QN];
    ZTrack zq;
    {
        ZTrack t;
        ztrack_init(t, z0 - R, A.n3, plane);
#pragma unroll
        for (int s2 = 0; s2 < 2 * R + PF; ++s2) {
            float4 v = ld4(Yc + t.off + gxy);
            if constexpr (CPLX)
                if (t.tz) v = cm(v, apply_phase<float2, float>(make_float2(1.f, 0.f), t.tz, phr[2], phi[2]));
            q[s2] = v;
            ztrack_next(t, A.n3, plane);
        }
        zq = t;
    }
#pragma unroll
    for (int d = 0; d < D - 1; ++d) issue(z0 + d, d);

    const int own = (R + ty) * RS + ROW_X0 + gx;   // this thread's first point in a stage
    for (int zb = z0; zb < z1; zb += QN) {
#pragma unroll
        for (int ph = 0; ph < QN; ++ph) {
            const int z = zb + ph;
            if (z < z1) {
                float2* T = tiles + ((z - z0) % D) * SE;
                const float4 cen = q[(ph + R) % QN];
                cp_async_wait<D - 2>();
                *reinterpret_cast<float4*>(T + own) = cen;
                if (tx < 3) *reinterpret_cast<float4*>(T + own + n1) = CPLX ? cm(cen, phxp) : cen;
                if (tx >= HX - 3) *reinterpret_cast<float4*>(T + own - n1) = CPLX ? cm(cen, phxm) : cen;
                if constexpr (CPLX) {
#pragma unroll
                    for (int k = 0; k < K; ++k) {
                        const int code = hdst[k] >> 24;
                        if (hdst[k] >= 0 && code != 5) {   // 5: no wrap in x or y
                            const int txw = (code & 3) - 1, tyw = (code >> 2) - 1;
                            float2 ph = txw > 0 ? phxp : (txw < 0 ? phxm : make_float2(1.f, 0.f));
                            if (tyw) ph = cmul(ph, make_float2(phr[1], tyw > 0 ? phi[1] : -phi[1]));
                            float4* p = reinterpret_cast<float4*>(T + (hdst[k] & HMASK));
                            *p = cm(*p, ph);
                        }
                    }
                }
                {
                    float4 v = ld4(Yc + zq.off + gxy);
                    if constexpr (CPLX)
                        if (zq.tz)
                            v = cm(v, apply_phase<float2, float>(make_float2(1.f, 0.f), zq.tz, phr[2], phi[2]));
                    q[(ph + 2 * R + PF) % QN] = v;
                    ztrack_next(zq, A.n3, plane);
                }
                __syncthreads();
                issue(z + D - 1, (z - z0 + D - 1) % D);

                const float2 c0 = make_float2(cen.x, cen.y), c1 = make_float2(cen.z, cen.w);
                // per point three independent accumulation chains (x, y, z) instead of one
                float2 a0 = efma(A.c0, c0, ezero<float2>()), a1 = efma(A.c0, c1, ezero<float2>());
                float2 b0 = ezero<float2>(), b1 = ezero<float2>(), d0 = ezero<float2>(), d1 = ezero<float2>();
                {   // x: six 16-byte reads cover x-6 .. x+7 of the pair
                    const float4 L0 = ld4(T + own - 6), L1 = ld4(T + own - 4), L2 = ld4(T + own - 2);
                    const float4 R0 = ld4(T + own + 2), R1 = ld4(T + own + 4), R2 = ld4(T + own + 6);
#define LO(v) make_float2(v.x, v.y)
#define HI(v) make_float2(v.z, v.w)
                    a0 = efma(A.cx[1], eadd(HI(L2), c1), a0);
                    a0 = efma(A.cx[2], eadd(LO(L2), LO(R0)), a0);
                    a0 = efma(A.cx[3], eadd(HI(L1), HI(R0)), a0);
                    a0 = efma(A.cx[4], eadd(LO(L1), LO(R1)), a0);
                    a0 = efma(A.cx[5], eadd(HI(L0), HI(R1)), a0);
                    a0 = efma(A.cx[6], eadd(LO(L0), LO(R2)), a0);
                    a1 = efma(A.cx[1], eadd(c0, LO(R0)), a1);
                    a1 = efma(A.cx[2], eadd(HI(L2), HI(R0)), a1);
                    a1 = efma(A.cx[3], eadd(LO(L2), LO(R1)), a1);
                    a1 = efma(A.cx[4], eadd(HI(L1), HI(R1)), a1);
                    a1 = efma(A.cx[5], eadd(LO(L1), LO(R2)), a1);
                    a1 = efma(A.cx[6], eadd(HI(L0), HI(R2)), a1);
                }
#pragma unroll
                for (int r = 1; r <= R; ++r) {
                    const float4 up = ld4(T + own - r * RS), dn = ld4(T + own + r * RS);
                    const float4 zu = q[(ph + R + r) % QN], zd = q[(ph + R - r + QN) % QN];
                    b0 = efma(A.cy[r], eadd(LO(up), LO(dn)), b0);
                    b1 = efma(A.cy[r], eadd(HI(up), HI(dn)), b1);
                    d0 = efma(A.cz[r], eadd(LO(zu), LO(zd)), d0);
                    d1 = efma(A.cz[r], eadd(HI(zu), HI(zd)), d1);
                }
                a0 = eadd(a0, eadd(b0, d0));
                a1 = eadd(a1, eadd(b1, d1));
                const long long g = (long long)z * plane + gxy;
                const int st = (z - z0) % D;
                if (VLOC) {
                    const float2 v = *op_v(st);
                    a0 = efma(v.x, c0, a0);
                    a1 = efma(v.y, c1, a1);
                }
                if (KB) {
                    auto kb_add = [&](int2 at, KV2 kv) {
                        if constexpr (CPLX) {
                            if (at.x >= 0) a0 = eadd(a0, cmul(LO(kv), Cs[at.x]));
                            if (at.y >= 0) a1 = eadd(a1, cmul(HI(kv), Cs[at.y]));
                        } else {
                            if (at.x >= 0) a0 = efma(kv.x, Cs[at.x], a0);
                            if (at.y >= 0) a1 = efma(kv.y, Cs[at.y], a1);
                        }
                    };
#pragma unroll
                    for (int k = 0; k < SP; ++k)
                        if (k < nslot) kb_add(*op_kat(st, k), *op_kval(st, k));
                    for (int k = SP; k < nslot; ++k) {   // slots beyond the staged ones: straight from L2
                        const int2 at = __ldg(reinterpret_cast<const int2*>(patom + k * A.ng + g));
                        if (at.x < 0 && at.y < 0) break;   // unused slots (-1) sit at the end
                        kb_add(at, __ldg(reinterpret_cast<const KV2*>(reinterpret_cast<const KV*>(pval) + k * A.ng + g)));
                    }
                }
                // out = alpha (acc - shift center) - beta prev
                float2 o0 = efma(alpha, efma(-shift, c0, a0), ezero<float2>());
                float2 o1 = efma(alpha, efma(-shift, c1, a1), ezero<float2>());
                if (PREV) {
                    const float4 pv = *op_prev(st);
                    o0 = efma(-beta, LO(pv), o0);
                    o1 = efma(-beta, HI(pv), o1);
                }
                *reinterpret_cast<float4*>(Ynext + (long long)col * A.ng + g) = make_float4(o0.x, o0.y, o1.x, o1.y);
#undef LO
#undef HI
            }
        }
    }
    cp_async_wait<0>();
}

// KB projection: C[col][a] = gamma_a * sum_j conj(beta_a(j)) Y[idx_j, col], NC columns per CTA
template <typename E, bool CPLX, int NC>
__global__ void __launch_bounds__(256, 3)
kb_project_kernel(const E* __restrict__ Y_, E* __restrict__ C_, const int* __restrict__ cnt_,
                  const int* __restrict__ idx_, const void* __restrict__ val_,
                  const double* __restrict__ gamma_, int cap_, int natom, int ncolE, long long ng,
                  const KBProblem* __restrict__ grp) {
    using S = typename Elem<E>::S;
    // one problem, or (grp != null) problem blockIdx.z of a grouped launch
    const E* __restrict__ Y = Y_;
    E* __restrict__ C = C_;
    const int* __restrict__ cnt = cnt_;
    const int* __restrict__ idx = idx_;
    const void* __restrict__ val = val_;
    const double* __restrict__ gamma = gamma_;
    int cap = cap_;
    if (grp) {
        const KBProblem& P = grp[blockIdx.z];
        Y = reinterpret_cast<const E*>(P.Y);
        C = reinterpret_cast<E*>(P.C);
        cnt = P.cnt;
        idx = P.idx;
        val = P.val;
        gamma = P.gamma;
        cap = P.cap;
        natom = P.natom;
        ncolE = P.ncolE;
        ng = P.ng;
    }
    const int a = blockIdx.x;
    const int c0 = blockIdx.y * NC;
    if (a >= natom || c0 >= ncolE) return;   // grouped launch sized for the largest problem
    const int m = cnt[a];
    E acc[NC];
#pragma unroll
    for (int k = 0; k < NC; ++k) acc[k] = ezero<E>();
    // two projector points per pass (2 NC independent gathers in flight per thread); the points of
    // one thread are summed in the same order as one at a time
    auto add_point = [&](long long e, int g) {
#pragma unroll
        for (int k = 0; k < NC; ++k) {
            if (c0 + k < ncolE) {
                E y = Y[(long long)(c0 + k) * ng + g];
                if constexpr (CPLX) {
                    E b = reinterpret_cast<const E*>(val)[e];
                    acc[k] = eadd(acc[k], cmul_conj(b, y));
                } else {
                    S b = reinterpret_cast<const S*>(val)[e];
                    acc[k] = efma(b, y, acc[k]);
                }
            }
        }
    };
    int j = threadIdx.x;
    for (; j + (int)blockDim.x < m; j += 2 * blockDim.x) {
        const long long e0 = (long long)a * cap + j, e1 = e0 + blockDim.x;
        const int g0 = idx[e0], g1 = idx[e1];
        E y0[NC], y1[NC];
#pragma unroll
        for (int k = 0; k < NC; ++k) {
            const bool in = c0 + k < ncolE;
            y0[k] = in ? Y[(long long)(c0 + k) * ng + g0] : ezero<E>();
            y1[k] = in ? Y[(long long)(c0 + k) * ng + g1] : ezero<E>();
        }
#pragma unroll
        for (int k = 0; k < NC; ++k) {
            if constexpr (CPLX) {
                const E b0 = reinterpret_cast<const E*>(val)[e0], b1 = reinterpret_cast<const E*>(val)[e1];
                acc[k] = eadd(acc[k], cmul_conj(b0, y0[k]));
                acc[k] = eadd(acc[k], cmul_conj(b1, y1[k]));
            } else {
                const S b0 = reinterpret_cast<const S*>(val)[e0], b1 = reinterpret_cast<const S*>(val)[e1];
                acc[k] = efma(b0, y0[k], acc[k]);
                acc[k] = efma(b1, y1[k], acc[k]);
            }
        }
    }
    if (j < m) add_point((long long)a * cap + j, idx[(long long)a * cap + j]);
    // block reduction (warp shuffles, then smem across warps)
    __shared__ E red[NC][8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NC; ++k) {
        E v = acc[k];
        for (int off = 16; off > 0; off >>= 1) {
            if constexpr (sizeof(E) == 8 && Elem<E>::lanes == 1) {
                v += __shfl_down_sync(0xffffffffu, v, off);
            } else {
                E o;
                o.x = __shfl_down_sync(0xffffffffu, v.x, off);
                o.y = __shfl_down_sync(0xffffffffu, v.y, off);
                v = eadd(v, o);
            }
        }
        if (lane == 0) red[k][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x < NC && c0 + (int)threadIdx.x < ncolE) {
        const int k = threadIdx.x;
        E v = red[k][0];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) v = eadd(v, red[k][w]);
        const S gm = (S)gamma[a];
        E out = efma(gm, v, ezero<E>());
        C[(long long)(c0 + k) * natom + a] = out;
    }
}

inline bool haskb_dsm(const void* kbC, const KBTables& kb) { return kbC != nullptr && kb.S > 0; }

template <typename S>
StepArgs<S> make_args(sdft_ctx* c, int kpt, double alpha, double beta, double shift, int zchunk, int nzc) {
    StepArgs<S> A;
    for (int r = 0; r <= FD_RADIUS; ++r) {
        A.cx[r] = (S)c->coef.cx[r];
        A.cy[r] = (S)c->coef.cy[r];
        A.cz[r] = (S)c->coef.cz[r];
    }
    A.c0 = (S)c->coef.c0;
    A.alpha = (S)alpha;
    A.beta = (S)beta;
    A.shift = (S)shift;
    for (int d = 0; d < 3; ++d) {
        double kd = c->kpts.empty() ? 0.0 : c->kpts[3 * kpt + d];
        A.phr[d] = (S)cos(2.0 * M_PI * kd);
        A.phi[d] = (S)sin(2.0 * M_PI * kd);
    }
    A.n1 = c->n[0];
    A.n2 = c->n[1];
    A.n3 = c->n[2];
    A.zchunk = zchunk;
    A.nzc = nzc;
    A.natom = c->natom;
    A.ng = c->ng;
    return A;
}

template <typename E, bool CPLX, int TX, int TY, int PF, int MINB, int D>
void launch_variant(sdft_ctx* c, int kpt, const E* Y, const E* Yprev, E* Ynext, int ncolE,
                    const typename Elem<E>::S* V, const E* kbC, double alpha, double beta, double shift,
                    bool kin, bool timed) {
    using S = typename Elem<E>::S;
    const int tiles = ((c->n[0] + TX - 1) / TX) * ((c->n[1] + TY - 1) / TY);
    // enough CTAs to fill 152 SMs several times over; each z chunk >= 16 planes
    long long want = 8LL * 152;
    int nzc = 1;
    const int ngrp = ncolE;
    while ((long long)tiles * ngrp * nzc < want && c->n[2] / (nzc + 1) >= 16) ++nzc;
    const int zchunk = (c->n[2] + nzc - 1) / nzc;
    nzc = (c->n[2] + zchunk - 1) / zchunk;
    StepArgs<S> A = make_args<S>(c, kpt, alpha, beta, shift, zchunk, nzc);
    dim3 grid((c->n[0] + TX - 1) / TX, (c->n[1] + TY - 1) / TY, (unsigned)(ngrp * nzc));
    dim3 block(TX, TY);
    const KBTables& kb = c->kb[kpt];
    const void* pval = std::is_same<S, float>::value ? (const void*)kb.pval32 : (const void*)kb.pval64;
    using KV = typename std::conditional<CPLX, E, S>::type;
    const size_t dsm = sizeof(Stage<E, S, KV, TX, TY, 3>) * D +
                       (haskb_dsm(kbC, kb) ? sizeof(E) * (size_t)std::max(1, c->natom) : 0);
    const bool prev = Yprev != nullptr, hasv = V != nullptr, haskb = kbC != nullptr && kb.S > 0;
    ScopedTimer timer(timed ? c : nullptr, sizeof(S) == 8 ? SDFT_K_STENCIL64 : SDFT_K_STENCIL,
                      (double)ncolE * (double)c->ng * sizeof(E) * (prev ? 3.0 : 2.0));
#define SDFT_STEP(P, K, VV, KN)                                                                      \
    do {                                                                                             \
        auto kfn = cheb_step_kernel<E, CPLX, TX, TY, PF, MINB, D, P, K, VV, KN>;                      \
        if (dsm > 48 * 1024)                                                                         \
            SDFT_CUDA(cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dsm)); \
        kfn<<<grid, block, dsm, c->stream>>>(Y, Yprev, Ynext, V, kbC, kb.patom, pval, kb.S, ncolE, A); \
    } while (0)
    SDFT_REQUIRE(kin, SDFT_ERR_INVALID_ARG, "stencil step without kinetic term is not built");
    if (hasv) {
        if (prev && haskb) SDFT_STEP(true, true, true, true);
        else if (!prev && haskb) SDFT_STEP(false, true, true, true);
        else if (prev && !haskb) SDFT_STEP(true, false, true, true);
        else SDFT_STEP(false, false, true, true);
    } else {
        // Laplacian-only form used by the Poisson solver (real, single vector, FP64 or FP32)
        SDFT_REQUIRE(prev && !haskb, SDFT_ERR_INVALID_ARG, "stencil variant without V_eff needs Yprev and no KB");
        if constexpr (std::is_same<E, double>::value || std::is_same<E, float>::value)
            SDFT_STEP(true, false, false, true);
        else SDFT_REQUIRE(false, SDFT_ERR_INVALID_ARG, "Laplacian-only stencil is real only");
    }
#undef SDFT_STEP
    SDFT_CUDA(cudaGetLastError());
    count_launch(c);
}

// dynamic shared memory of the row tile: D stages of the halo'd rows and of the per-point operands,
// then the KB coefficients of the column (the complex layout is the larger, used for the fit check)
template <bool CPLX>
size_t row_smem_bytes(const sdft_ctx* c, int TY, int D, int NT) {
    const size_t kv2 = CPLX ? 16 : 8;
    return sizeof(float2) * (size_t)D * (TY + 2 * FD_RADIUS) * row_stride(c->n[0]) +
           (size_t)D * ((NT * (16 + 8 + 3 * 8 + 3 * kv2) + 15) & ~(size_t)15) +
           sizeof(float2) * (size_t)std::max(1, c->natom);
}

// row-tile variant: usable when n1 is even, TY divides n2, the CTA has at most 512 threads and
// the y halo fits ROW_HALO_UNITS_PER_THREAD 16-byte copies per thread
template <int TY, int MAXT, int D>
bool row_variant_ok(const sdft_ctx* c, int ncolE) {
    const int n1 = c->n[0], n2 = c->n[1];
    if (n1 % 2 || n2 % TY || n1 < 2 * FD_RADIUS) return false;
    const int HX = n1 / 2, NT = HX * TY;
    if (NT > MAXT || NT < 64) return false;
    if (2 * FD_RADIUS * (HX + 6) > ROW_HALO_UNITS_PER_THREAD * NT) return false;
    return row_smem_bytes<true>(c, TY, D, NT) <= 200 * 1024 && ncolE > 0;
}

// one launch of the row tile for one problem (grp null) or for nprob problems of a group (grp:
// device table of RowProblem; kpt then only selects the shared grid quantities)
template <bool CPLX, int TY, int PF, int MAXT, int MINB, int D>
void launch_row_impl(sdft_ctx* c, int kpt, const float2* Y, const float2* Yprev, float2* Ynext, int ncolE,
                     const float* V, const float2* kbC, double alpha, double beta, double shift, bool timed,
                     int nprob, const RowProblem* grp, bool prev, bool haskb) {
    SDFT_REQUIRE((row_variant_ok<TY, MAXT, D>(c, ncolE)), SDFT_ERR_INVALID_ARG, "row stencil variant does not fit");
    const int n1 = c->n[0];
    const int ytiles = c->n[1] / TY;
    long long want = 6LL * 152;
    int nzc = 1;
    while ((long long)ytiles * ncolE * nprob * nzc < want && c->n[2] / (nzc + 1) >= 24) ++nzc;
    const int zchunk = (c->n[2] + nzc - 1) / nzc;
    nzc = (c->n[2] + zchunk - 1) / zchunk;
    StepArgs<float> A = make_args<float>(c, kpt, alpha, beta, shift, zchunk, nzc);
    SDFT_REQUIRE((long long)ncolE * nprob * nzc < 65536, SDFT_ERR_INVALID_ARG, "too many columns for one launch");
    dim3 grid(ytiles, 1, (unsigned)(ncolE * nprob * nzc));
    dim3 block(n1 / 2, TY);
    const KBTables& kb = c->kb[kpt];
    const size_t dsm = row_smem_bytes<CPLX>(c, TY, D, (n1 / 2) * TY);
    ScopedTimer timer(timed ? c : nullptr, SDFT_K_STENCIL,
                      (double)nprob * ncolE * (double)c->ng * sizeof(float2) * (prev ? 3.0 : 2.0));
#define SDFT_ROW(P, KK)                                                                               \
    do {                                                                                              \
        auto kfn = cheb_row_kernel<CPLX, TY, PF, MAXT, MINB, D, P, KK, true>;                          \
        SDFT_CUDA(cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dsm));  \
        kfn<<<grid, block, dsm, c->stream>>>(Y, Yprev, Ynext, V, kbC, kb.patom, kb.pval32, kb.S, A, ncolE, grp); \
    } while (0)
    if (prev && haskb) SDFT_ROW(true, true);
    else if (!prev && haskb) SDFT_ROW(false, true);
    else if (prev && !haskb) SDFT_ROW(true, false);
    else SDFT_ROW(false, false);
#undef SDFT_ROW
    SDFT_CUDA(cudaGetLastError());
    count_launch(c);
}

template <bool CPLX, int TY, int PF, int MAXT, int MINB, int D>
void launch_row_variant(sdft_ctx* c, int kpt, const float2* Y, const float2* Yprev, float2* Ynext, int ncolE,
                        const float* V, const float2* kbC, double alpha, double beta, double shift, bool kin,
                        bool timed) {
    SDFT_REQUIRE(kin && V != nullptr, SDFT_ERR_INVALID_ARG, "row stencil variant needs V and the kinetic term");
    const bool prev = Yprev != nullptr, haskb = kbC != nullptr && c->kb[kpt].S > 0;
    launch_row_impl<CPLX, TY, PF, MAXT, MINB, D>(c, kpt, Y, Yprev, Ynext, ncolE, V, kbC, alpha, beta, shift, timed,
                                                 1, nullptr, prev, haskb);
}

template <bool CPLX, int TY, int PF, int MAXT, int MINB, int D>
void launch_row_group(sdft_ctx* c, int kpt, const RowProblem* grp, int nprob, int ncolE, bool prev, bool haskb) {
    launch_row_impl<CPLX, TY, PF, MAXT, MINB, D>(c, kpt, nullptr, nullptr, nullptr, ncolE, nullptr, nullptr, 1.0,
                                                 0.0, 0.0, true, nprob, grp, prev, haskb);
}
using GroupLauncher = void (*)(sdft_ctx*, int, const RowProblem*, int, int, bool, bool);

template <typename E>
using StepLauncher = void (*)(sdft_ctx*, int, const E*, const E*, E*, int, const typename Elem<E>::S*, const E*,
                              double, double, double, bool, bool);
template <typename E>
struct StepVariant {
    StepLauncher<E> fn;
    bool (*ok)(const sdft_ctx*, int);   // null: always usable
    const char* name;
    GroupLauncher group = nullptr;      // grouped launch over problems (row tiles only)
};

// Stencil tile autotuner: time every compiled variant on the real operands (Ynext is rewritten by
// the chosen variant afterwards) and keep the fastest for this context.  SDFT_STENCIL_VARIANT=k
// forces variant k.  Small problems use variant 0 without timing.
template <typename E>
// proj (not null): the caller also needs the KB coefficients of the step's output, so each variant is
// timed with them: followed by the separate projection pass `project` into proj, and, where the
// variant offers a fused projection (it then sets c->kb_next_done), also with that; *fused tells
// which of the two the fastest variant used
int autotune_stencil(sdft_ctx* c, const StepVariant<E>* table, int nvar, int kpt, const E* Y, const E* Yprev,
                     E* Ynext, int ncolE, const typename Elem<E>::S* V, const E* kbC, double alpha, double beta,
                     double shift, E* proj = nullptr,
                     void (*project)(sdft_ctx*, int, const E*, E*, int) = nullptr, bool* fused = nullptr) {
    auto usable = [&](int v) { return table[v].ok == nullptr || table[v].ok(c, ncolE); };
    if (const char* env = getenv("SDFT_STENCIL_VARIANT")) {
        const int v = atoi(env);
        if (v >= 0 && v < nvar && usable(v)) return v;
    }
    if (nvar == 1 || (double)c->ng * ncolE < 4e6 || V == nullptr) return -1;   // not tuned: caller uses 0
    cudaEvent_t a, b;
    SDFT_CUDA(cudaEventCreate(&a));
    SDFT_CUDA(cudaEventCreate(&b));
    int best = 0;
    float best_ms = 1e30f;
    // one step (and the output's projection when asked for); returns whether it was fused
    auto run = [&](int v, bool fuse) {
        if (proj != nullptr) {
            c->kb_next = fuse ? reinterpret_cast<decltype(c->kb_next)>(proj) : nullptr;
            c->kb_next_done = false;
        }
        table[v].fn(c, kpt, Y, Yprev, Ynext, ncolE, V, kbC, alpha, beta, shift, true, false);
        bool done = false;
        if (proj != nullptr) {
            done = c->kb_next_done;
            if (!done) project(c, kpt, Ynext, proj, ncolE);
            c->kb_next = nullptr;
            c->kb_next_done = false;
        }
        return done;
    };
    bool best_fused = false;
    for (int v = 0; v < nvar; ++v) {
        if (!usable(v)) continue;
        for (int fuse = 0; fuse < (proj != nullptr ? 2 : 1); ++fuse) {
            const bool f = run(v, fuse != 0);   // warm-up
            if (fuse && !f) break;              // no fused projection in this variant
            SDFT_CUDA(cudaEventRecord(a, c->stream));
            for (int r = 0; r < 3; ++r) run(v, fuse != 0);
            SDFT_CUDA(cudaEventRecord(b, c->stream));
            SDFT_CUDA(cudaEventSynchronize(b));
            float ms = 0.f;
            SDFT_CUDA(cudaEventElapsedTime(&ms, a, b));
            if (ms < best_ms) {
                best_ms = ms;
                best = v;
                best_fused = fuse != 0;
            }
        }
    }
    if (fused) *fused = best_fused;
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return best;
}

}  // namespace

template <typename E>
void launch_project_group_impl(sdft_ctx* c, const KBProblem* grp, int nprob, int ncolE, bool cplx) {
    const int natom = c->natom;
    if (natom == 0 || ncolE == 0 || nprob == 0) return;
    constexpr int NC = 8;
    dim3 grid(natom, (ncolE + NC - 1) / NC, nprob);
    ScopedTimer timer(c, SDFT_K_KB_PROJECT);
    if (cplx) {
        if constexpr (!std::is_same<E, double>::value)
            kb_project_kernel<E, true, NC><<<grid, 256, 0, c->stream>>>(nullptr, nullptr, nullptr, nullptr, nullptr,
                                                                       nullptr, 0, natom, ncolE, c->ng, grp);
    } else {
        kb_project_kernel<E, false, NC><<<grid, 256, 0, c->stream>>>(nullptr, nullptr, nullptr, nullptr, nullptr,
                                                                    nullptr, 0, natom, ncolE, c->ng, grp);
    }
    SDFT_CUDA(cudaGetLastError());
    count_launch(c);
}

// one launch over problems of different sizes (cells of a multi-cell filter): grid sized for the
// largest, blocks past a problem's atoms or columns return at once
template <typename E>
void launch_project_multi_impl(sdft_ctx* c, const KBProblem* grp, int nprob, int max_natom, int max_ncolE) {
    if (max_natom == 0 || max_ncolE == 0 || nprob == 0) return;
    constexpr int NC = 8;
    dim3 grid(max_natom, (max_ncolE + NC - 1) / NC, nprob);
    ScopedTimer timer(c, SDFT_K_KB_PROJECT);
    kb_project_kernel<E, false, NC><<<grid, 256, 0, c->stream>>>(nullptr, nullptr, nullptr, nullptr, nullptr, nullptr,
                                                                0, 0, 0, 0, grp);
    SDFT_CUDA(cudaGetLastError());
    count_launch(c);
}

template <typename E>
void launch_project_impl(sdft_ctx* c, int kpt, const E* Y, E* C, int ncolE) {
    const KBTables& kb = c->kb[kpt];
    if (kb.natom == 0 || ncolE == 0) return;
    constexpr int NC = 8;
    dim3 grid(kb.natom, (ncolE + NC - 1) / NC);
    ScopedTimer timer(c, SDFT_K_KB_PROJECT);
    using S = typename Elem<E>::S;
    const void* val = std::is_same<S, float>::value ? (const void*)kb.val32 : (const void*)kb.val64;
    if (kb.cplx) {
        if constexpr (!std::is_same<E, double>::value)
            kb_project_kernel<E, true, NC><<<grid, 256, 0, c->stream>>>(Y, C, kb.cnt, kb.idx, val, kb.gamma,
                                                                       kb.cap, kb.natom, ncolE, c->ng, nullptr);
    } else {
        kb_project_kernel<E, false, NC><<<grid, 256, 0, c->stream>>>(Y, C, kb.cnt, kb.idx, val, kb.gamma, kb.cap,
                                                                    kb.natom, ncolE, c->ng, nullptr);
    }
    SDFT_CUDA(cudaGetLastError());
    count_launch(c);
}

}  // namespace sdft
