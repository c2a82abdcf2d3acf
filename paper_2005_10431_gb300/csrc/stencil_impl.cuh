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
template <typename E, bool CPLX, int TX, int TY, int PF, int MINB, int D, bool PREV, bool KB, bool VLOC, bool KIN>
__global__ void __launch_bounds__(TX * TY, MINB)
cheb_step_kernel(const E* __restrict__ Y, const E* __restrict__ Yprev, E* __restrict__ Ynext,
                 const typename Elem<E>::S* __restrict__ V, const E* __restrict__ C,
                 const int* __restrict__ patom, const void* __restrict__ pval, const int nslot, const int ncolE,
                 const StepArgs<typename Elem<E>::S> A) {
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
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int col = blockIdx.z / A.nzc;
    const int zc = blockIdx.z - col * A.nzc;
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
                        acc = efma(A.c0, center, acc);
#pragma unroll
                        for (int r = 1; r <= R; ++r) {
                            acc = efma(A.cz[r], eadd(q[(ph + R + r) % QN], q[(ph + R - r + QN) % QN]), acc);
                            acc = efma(A.cx[r], eadd(S_.tile[R + ty][R + tx + r], S_.tile[R + ty][R + tx - r]), acc);
                            acc = efma(A.cy[r], eadd(S_.tile[R + ty + r][R + tx], S_.tile[R + ty - r][R + tx]), acc);
                        }
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

// KB projection: C[col][a] = gamma_a * sum_j conj(beta_a(j)) Y[idx_j, col], NC columns per CTA
template <typename E, bool CPLX, int NC>
__global__ void __launch_bounds__(256)
kb_project_kernel(const E* __restrict__ Y, E* __restrict__ C, const int* __restrict__ cnt,
                  const int* __restrict__ idx, const void* __restrict__ val,
                  const double* __restrict__ gamma, int cap, int natom, int ncolE, long long ng) {
    using S = typename Elem<E>::S;
    const int a = blockIdx.x;
    const int c0 = blockIdx.y * NC;
    const int m = cnt[a];
    E acc[NC];
#pragma unroll
    for (int k = 0; k < NC; ++k) acc[k] = ezero<E>();
    for (int j = threadIdx.x; j < m; j += blockDim.x) {
        const long long e = (long long)a * cap + j;
        const int g = idx[e];
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
    }
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
    ScopedTimer timer(timed ? c : nullptr, SDFT_K_STENCIL,
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

template <typename E>
using StepLauncher = void (*)(sdft_ctx*, int, const E*, const E*, E*, int, const typename Elem<E>::S*, const E*,
                              double, double, double, bool, bool);

// Stencil tile autotuner: time every compiled variant on the real operands (Ynext is rewritten by
// the chosen variant afterwards) and keep the fastest for this context.  SDFT_STENCIL_VARIANT=k
// forces variant k.  Small problems use variant 0 without timing.
template <typename E>
int autotune_stencil(sdft_ctx* c, const StepLauncher<E>* table, int nvar, int kpt, const E* Y, const E* Yprev,
                     E* Ynext, int ncolE, const typename Elem<E>::S* V, const E* kbC, double alpha, double beta,
                     double shift) {
    if (const char* env = getenv("SDFT_STENCIL_VARIANT")) {
        const int v = atoi(env);
        if (v >= 0 && v < nvar) return v;
    }
    if (nvar == 1 || (double)c->ng * ncolE < 4e6) return 0;
    cudaEvent_t a, b;
    SDFT_CUDA(cudaEventCreate(&a));
    SDFT_CUDA(cudaEventCreate(&b));
    int best = 0;
    float best_ms = 1e30f;
    for (int v = 0; v < nvar; ++v) {
        table[v](c, kpt, Y, Yprev, Ynext, ncolE, V, kbC, alpha, beta, shift, true, false);  // warm-up
        SDFT_CUDA(cudaEventRecord(a, c->stream));
        for (int r = 0; r < 3; ++r) table[v](c, kpt, Y, Yprev, Ynext, ncolE, V, kbC, alpha, beta, shift, true, false);
        SDFT_CUDA(cudaEventRecord(b, c->stream));
        SDFT_CUDA(cudaEventSynchronize(b));
        float ms = 0.f;
        SDFT_CUDA(cudaEventElapsedTime(&ms, a, b));
        if (ms < best_ms) {
            best_ms = ms;
            best = v;
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return best;
}


}  // namespace

template <typename E>
void launch_project_impl(sdft_ctx* c, int kpt, const E* Y, E* C, int ncolE) {
    const KBTables& kb = c->kb[kpt];
    if (kb.natom == 0 || ncolE == 0) return;
    constexpr int NC = 4;
    dim3 grid(kb.natom, (ncolE + NC - 1) / NC);
    ScopedTimer timer(c, SDFT_K_KB_PROJECT);
    using S = typename Elem<E>::S;
    const void* val = std::is_same<S, float>::value ? (const void*)kb.val32 : (const void*)kb.val64;
    if (kb.cplx) {
        if constexpr (!std::is_same<E, double>::value)
            kb_project_kernel<E, true, NC><<<grid, 256, 0, c->stream>>>(Y, C, kb.cnt, kb.idx, val, kb.gamma,
                                                                       kb.cap, kb.natom, ncolE, c->ng);
    } else {
        kb_project_kernel<E, false, NC><<<grid, 256, 0, c->stream>>>(Y, C, kb.cnt, kb.idx, val, kb.gamma, kb.cap,
                                                                    kb.natom, ncolE, c->ng);
    }
    SDFT_CUDA(cudaGetLastError());
    count_launch(c);
}

}  // namespace sdft
