// Device building blocks of the TMOP partial-assembly kernels (sm_103a).
//
// One CTA processes EPB elements; each element is owned by TPE = MX*MX
// threads (MX = max(p+1, nq1d)) laid out as a (tx, ty) square.  The 1D
// tables B1D/G1D (paper Sec. 3.1, eq. B_G_1D) and the element's nodal block
// live in shared memory.  Jacobians at the quadrature points are obtained by
// sum factorisation (Sec. 3.2): one 1D contraction per direction, each
// O(p^{d+1}); the transposed contractions return quadrature data to the
// nodes (Sec. 3.3 and 3.4).  In 3D a thread owning (q1, q2) walks the q3
// column, so the last contraction of each direction stays in registers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "dfloat.cuh"

namespace tmop {

// Iteration index of a MINRES launch: k >= 0 as given, k < 0 the device
// counter stored right after the stop iteration (MinresState::k: stop[1]), so
// that an iteration's launches are the same in every iteration (CUDA graph
// replay).
__device__ __forceinline__ int iter_of(const int *stop, int k) { return k >= 0 ? k : stop[1]; }

enum { MET_2 = 2, MET_7 = 7, MET_9 = 9, MET_55 = 55, MET_302 = 302, MET_303 = 303,
       MET_303_55 = 30355 };

// Metric ids defined for dimension d, and those whose 3D form uses I2 = |cof T|^2.
__host__ __device__ inline bool metric_valid(int m, int d)
{
    if (m == MET_2) return d == 2;
    if (m == MET_302 || m == MET_303 || m == MET_303_55) return d == 3;
    return m == MET_55 || m == MET_7 || m == MET_9;
}
__host__ __device__ inline bool metric_uses_I2(int m, int d)
{
    return d == 3 && (m == MET_302 || m == MET_7 || m == MET_9);
}
enum { TGT_IDENTITY = 0, TGT_SIZE = 1, TGT_DISCRETE = 2 };

template <int D_, int P_, int Q_>
struct Cfg {
    static constexpr int D = D_, P = P_, NI = P_ + 1, NQ = Q_;
    static constexpr int MX = NI > NQ ? NI : NQ;
    static constexpr int NP = D == 3 ? NI * NI * NI : NI * NI;
    static constexpr int NQD = D == 3 ? NQ * NQ * NQ : NQ * NQ;
    static constexpr int DD = D * D;
    static constexpr int NS = DD * (DD + 1) / 2;            // packed symmetric H
    // Stored d2mu/dT2 of one element: entries s of the packed upper triangle
    // at the NQD points, in element blocks of HST values (PAIRS: rounded up to
    // a multiple of 4 for aligned pair loads).
    // PAIRS (3D, an element's n_q x n_q columns in one warp: the collocated
    // action kernels, which load two entries at once): NS/2 planes of entry
    // pairs, entries 2g and 2g+1 of a point side by side, then for odd NS the
    // plane of the last entry.  Otherwise one plane per entry, [s][q], for the
    // kernels that read one entry at a time across consecutive points.
    static constexpr bool PAIRS = D == 3 && NQ * NQ <= 32;
    static constexpr int NPR = NS / 2;
    static constexpr int HST = PAIRS ? (NS * NQD + 3) & ~3 : NS * NQD;
    static __host__ __device__ constexpr int hoff(int s, int q)
    {
        return !PAIRS ? s * NQD + q
                      : (s < 2 * NPR ? ((s >> 1) * NQD + q) * 2 + (s & 1) : 2 * NPR * NQD + q);
    }
    static constexpr int TPE = MX * MX;                      // threads per element
    // elements per CTA: ~128 threads in 3D, ~256 in 2D.  In 3D, when an
    // element fits in a warp, whole elements per warp (4 warps per CTA), so
    // that the warp-synchronous action kernel can use the same tiles.
    static constexpr int EPW = TPE <= 32 ? 32 / TPE : 0;
    static constexpr int EPB_ = (D == 3 && EPW > 0) ? 4 * EPW : (D == 3 ? 128 : 256) / TPE;
    static constexpr int EPB = EPB_ < 1 ? 1 : EPB_;
    static constexpr int NT = ((EPB * TPE + 31) / 32) * 32;  // CTA size, whole warps
    // per-element shared scratch (in elements of the compute type)
    static constexpr int SU = NP > NQD ? NP : NQD;
    static constexpr int S1 = D == 3 ? 2 * NI * NI * NQ : 2 * NI * NQ;
    static constexpr int S2 = D == 3 ? 3 * NI * NQ * NQ : 0;
};

// Kernel parameters shared by every element kernel.
struct ElemParams {
    const int32_t *__restrict__ map;   // E x NP
    int64_t E, Nx;
    const double *__restrict__ tab;    // B[NQ*NI], G[NQ*NI], w1d[NQ]
    const float *__restrict__ tabf;    // same, FP32
    const df *__restrict__ tabw;       // same, double-float
    int metric, target;
    double h0;
    const double *__restrict__ eta = nullptr;   // nodal field of the discrete target (Nx)
    double *__restrict__ detq = nullptr;        // k_energy: det A at every point (E x NQD) when set
};

// ---- batched launches: one grid over the element tiles of many meshes ----
// Per-mesh device data of a batch (owned by the batch object).
struct BMesh {
    ElemParams P;                       // map, sizes, tables, metric, target, h0
    const int32_t *csr_ptr, *csr_idx;   // transposed element map
    const uint8_t *fixed;               // d*Nx or nullptr
    void *ptr[24];                      // role -> buffer (see enum Role)
    int64_t ndof;
    int ntile_e;                        // element tiles (CTAs) of this mesh
    int nchunk;                         // vector tiles of this mesh
};
enum Role {
    ROLE_NONE = -1, ROLE_X = 0, ROLE_XT, ROLE_G, ROLE_DX, ROLE_H, ROLE_EV64, ROLE_EVR, ROLE_DIAG,
    ROLE_MINV, ROLE_PART, ROLE_VPART, ROLE_X0, ROLE_KV0 = 12   // ROLE_KV0 .. ROLE_KV0 + 7
};
// Launch-level batch arguments; tiles == nullptr means a single-mesh launch.
struct BatchArgs {
    const int2 *tiles;          // (mesh, tile) of every CTA
    const BMesh *meshes;
    int in, aux, out;           // roles of the kernel's pointer arguments
    const int *stop;            // per-mesh stop_iter words (stride stop_stride ints)
    int stop_stride;
};

// Resolve the CTA's mesh: overwrite P and the pointer arguments, return the tile.
__device__ __forceinline__ int64_t resolve_tile(ElemParams &P, const BatchArgs &B, const void *&in,
                                                const void *&aux, void *&out, const int *&stop)
{
    if (!B.tiles) return blockIdx.x;
    const int2 t = B.tiles[blockIdx.x];
    const BMesh &m = B.meshes[t.x];
    P = m.P;
    if (B.in >= 0) in = m.ptr[B.in];
    if (B.aux >= 0) aux = m.ptr[B.aux];
    if (B.out >= 0) out = m.ptr[B.out];
    if (B.stop) stop = B.stop + (int64_t)t.x * B.stop_stride;
    return t.y;
}

// Shared-memory layout of one CTA: tables, then EPB element slots, then maps.
template <class C, class R>
struct Layout {
    static constexpr int TAB = 2 * C::NQ * C::NI + C::NQ;                  // B, G, w
    static constexpr int TAB_PAD = (TAB + 1) & ~1;
    static constexpr int SLOT_BASE = C::SU + C::S1 + C::S2 + C::DD * C::NQD;
    static constexpr int SLOT = (SLOT_BASE + C::D * C::NQD + 1) & ~1;      // + physical coords
    static constexpr size_t bytes = sizeof(R) * (size_t)(TAB_PAD + C::EPB * SLOT) +
                                    sizeof(int) * (size_t)(C::EPB * C::NP);
};

// -------------------------------------------------------------------------
// Sum-factorised contractions.  All threads of the CTA call these (they
// contain __syncthreads); threads outside an element's active square idle.
// Index conventions: nodes u[(i3*NI + i2)*NI + i1], quadrature points
// f[(q3*NQ + q2)*NQ + q1]; B[q*NI + i].
// -------------------------------------------------------------------------

// 3D: node values u -> reference gradient components a0 = d/dxbar1,
// a1 = d/dxbar2, a2 = d/dxbar3 and (optionally) values xv at the points.
template <class C, class R>
__device__ __forceinline__ void fwd3(const R *__restrict__ B, const R *__restrict__ G,
                                     const R *u, R *s1, R *s2, R *a0, R *a1, R *a2, R *xv,
                                     int tx, int ty, bool act)
{
    constexpr int NI = C::NI, NQ = C::NQ;
    constexpr int O1 = NI * NI * NQ, O2 = NI * NQ * NQ;
    if (act && tx < NQ && ty < NI) {          // contract i1 -> q1
#pragma unroll
        for (int i3 = 0; i3 < NI; ++i3) {
            R b = 0, g = 0;
#pragma unroll
            for (int i1 = 0; i1 < NI; ++i1) {
                const R v = u[(i3 * NI + ty) * NI + i1];
                b += B[tx * NI + i1] * v;
                g += G[tx * NI + i1] * v;
            }
            s1[(i3 * NI + ty) * NQ + tx] = b;
            s1[O1 + (i3 * NI + ty) * NQ + tx] = g;
        }
    }
    __syncthreads();
    if (act && tx < NQ && ty < NQ) {          // contract i2 -> q2
#pragma unroll
        for (int i3 = 0; i3 < NI; ++i3) {
            R bb = 0, bg = 0, gb = 0;
#pragma unroll
            for (int i2 = 0; i2 < NI; ++i2) {
                const R sb = s1[(i3 * NI + i2) * NQ + tx];
                const R sg = s1[O1 + (i3 * NI + i2) * NQ + tx];
                const R Bq = B[ty * NI + i2], Gq = G[ty * NI + i2];
                bb += Bq * sb;
                bg += Gq * sb;
                gb += Bq * sg;
            }
            s2[(i3 * NQ + ty) * NQ + tx] = gb;
            s2[O2 + (i3 * NQ + ty) * NQ + tx] = bg;
            s2[2 * O2 + (i3 * NQ + ty) * NQ + tx] = bb;
        }
    }
    __syncthreads();
    if (act && tx < NQ && ty < NQ) {          // contract i3 -> q3 (column in registers)
        R c0[NI], c1[NI], c2[NI];
#pragma unroll
        for (int i3 = 0; i3 < NI; ++i3) {
            c0[i3] = s2[(i3 * NQ + ty) * NQ + tx];
            c1[i3] = s2[O2 + (i3 * NQ + ty) * NQ + tx];
            c2[i3] = s2[2 * O2 + (i3 * NQ + ty) * NQ + tx];
        }
#pragma unroll
        for (int q3 = 0; q3 < NQ; ++q3) {
            R r0 = 0, r1 = 0, r2 = 0, rx = 0;
#pragma unroll
            for (int i3 = 0; i3 < NI; ++i3) {
                const R Bq = B[q3 * NI + i3], Gq = G[q3 * NI + i3];
                r0 += Bq * c0[i3];
                r1 += Bq * c1[i3];
                r2 += Gq * c2[i3];
                rx += Bq * c2[i3];
            }
            const int q = (q3 * NQ + ty) * NQ + tx;
            a0[q] = r0;
            a1[q] = r1;
            a2[q] = r2;
            if (xv) xv[q] = rx;
        }
    }
    __syncthreads();
}

// 3D transpose: out_i = sum_q [y0 d1w_i + y1 d2w_i + y2 d3w_i](q).
template <class C, class R>
__device__ __forceinline__ void bwd3(const R *__restrict__ B, const R *__restrict__ G,
                                     const R *y0, const R *y1, const R *y2, R *s1, R *s2,
                                     R *out, int tx, int ty, bool act)
{
    constexpr int NI = C::NI, NQ = C::NQ;
    constexpr int O1 = NI * NI * NQ, O2 = NI * NQ * NQ;
    if (act && tx < NQ && ty < NQ) {          // q3 -> i3
        R c0[NQ], c1[NQ], c2[NQ];
#pragma unroll
        for (int q3 = 0; q3 < NQ; ++q3) {
            const int q = (q3 * NQ + ty) * NQ + tx;
            c0[q3] = y0[q];
            c1[q3] = y1[q];
            c2[q3] = y2[q];
        }
#pragma unroll
        for (int i3 = 0; i3 < NI; ++i3) {
            R z0 = 0, z1 = 0, z2 = 0;
#pragma unroll
            for (int q3 = 0; q3 < NQ; ++q3) {
                const R Bq = B[q3 * NI + i3], Gq = G[q3 * NI + i3];
                z0 += Bq * c0[q3];
                z1 += Bq * c1[q3];
                z2 += Gq * c2[q3];
            }
            s2[(i3 * NQ + ty) * NQ + tx] = z0;
            s2[O2 + (i3 * NQ + ty) * NQ + tx] = z1;
            s2[2 * O2 + (i3 * NQ + ty) * NQ + tx] = z2;
        }
    }
    __syncthreads();
    if (act && tx < NQ && ty < NI) {          // q2 -> i2
#pragma unroll
        for (int i3 = 0; i3 < NI; ++i3) {
            R a = 0, b = 0;
#pragma unroll
            for (int q2 = 0; q2 < NQ; ++q2) {
                const R Bq = B[q2 * NI + ty], Gq = G[q2 * NI + ty];
                a += Bq * s2[(i3 * NQ + q2) * NQ + tx];
                b += Gq * s2[O2 + (i3 * NQ + q2) * NQ + tx] + Bq * s2[2 * O2 + (i3 * NQ + q2) * NQ + tx];
            }
            s1[(i3 * NI + ty) * NQ + tx] = a;
            s1[O1 + (i3 * NI + ty) * NQ + tx] = b;
        }
    }
    __syncthreads();
    if (act && tx < NI && ty < NI) {          // q1 -> i1
#pragma unroll
        for (int i3 = 0; i3 < NI; ++i3) {
            R o = 0;
#pragma unroll
            for (int q1 = 0; q1 < NQ; ++q1)
                o += G[q1 * NI + tx] * s1[(i3 * NI + ty) * NQ + q1] +
                     B[q1 * NI + tx] * s1[O1 + (i3 * NI + ty) * NQ + q1];
            out[(i3 * NI + ty) * NI + tx] = o;
        }
    }
    __syncthreads();
}

// 3D transpose with arbitrary per-direction tables (diagonal assembly):
// out_i += sum_q f(q) T1(q1,i1) T2(q2,i2) T3(q3,i3).
template <class C, class R>
__device__ __forceinline__ void bwd3_tab(const R *__restrict__ T1, const R *__restrict__ T2,
                                         const R *__restrict__ T3, const R *f, R *s1, R *s2,
                                         R *out, int tx, int ty, bool act)
{
    constexpr int NI = C::NI, NQ = C::NQ;
    if (act && tx < NQ && ty < NQ) {
        R c[NQ];
#pragma unroll
        for (int q3 = 0; q3 < NQ; ++q3) c[q3] = f[(q3 * NQ + ty) * NQ + tx];
#pragma unroll
        for (int i3 = 0; i3 < NI; ++i3) {
            R z = 0;
#pragma unroll
            for (int q3 = 0; q3 < NQ; ++q3) z += T3[q3 * NI + i3] * c[q3];
            s2[(i3 * NQ + ty) * NQ + tx] = z;
        }
    }
    __syncthreads();
    if (act && tx < NQ && ty < NI) {
#pragma unroll
        for (int i3 = 0; i3 < NI; ++i3) {
            R a = 0;
#pragma unroll
            for (int q2 = 0; q2 < NQ; ++q2) a += T2[q2 * NI + ty] * s2[(i3 * NQ + q2) * NQ + tx];
            s1[(i3 * NI + ty) * NQ + tx] = a;
        }
    }
    __syncthreads();
    if (act && tx < NI && ty < NI) {
#pragma unroll
        for (int i3 = 0; i3 < NI; ++i3) {
            R o = 0;
#pragma unroll
            for (int q1 = 0; q1 < NQ; ++q1) o += T1[q1 * NI + tx] * s1[(i3 * NI + ty) * NQ + q1];
            out[(i3 * NI + ty) * NI + tx] += o;
        }
    }
    __syncthreads();
}

// 2D: node values u[i2*NI + i1] -> a0 = d/dxbar1, a1 = d/dxbar2, values xv.
template <class C, class R>
__device__ __forceinline__ void fwd2(const R *__restrict__ B, const R *__restrict__ G,
                                     const R *u, R *s1, R *a0, R *a1, R *xv, int tx, int ty,
                                     bool act)
{
    constexpr int NI = C::NI, NQ = C::NQ, O1 = NI * NQ;
    if (act && tx < NQ && ty < NI) {
        R b = 0, g = 0;
#pragma unroll
        for (int i1 = 0; i1 < NI; ++i1) {
            const R v = u[ty * NI + i1];
            b += B[tx * NI + i1] * v;
            g += G[tx * NI + i1] * v;
        }
        s1[ty * NQ + tx] = b;
        s1[O1 + ty * NQ + tx] = g;
    }
    __syncthreads();
    if (act && tx < NQ && ty < NQ) {
        R r0 = 0, r1 = 0, rx = 0;
#pragma unroll
        for (int i2 = 0; i2 < NI; ++i2) {
            const R Bq = B[ty * NI + i2], Gq = G[ty * NI + i2];
            const R sb = s1[i2 * NQ + tx], sg = s1[O1 + i2 * NQ + tx];
            r0 += Bq * sg;
            r1 += Gq * sb;
            rx += Bq * sb;
        }
        const int q = ty * NQ + tx;
        a0[q] = r0;
        a1[q] = r1;
        if (xv) xv[q] = rx;
    }
    __syncthreads();
}

template <class C, class R>
__device__ __forceinline__ void bwd2(const R *__restrict__ B, const R *__restrict__ G,
                                     const R *y0, const R *y1, R *s1, R *out, int tx, int ty,
                                     bool act)
{
    constexpr int NI = C::NI, NQ = C::NQ, O1 = NI * NQ;
    if (act && tx < NQ && ty < NI) {
        R a = 0, b = 0;
#pragma unroll
        for (int q2 = 0; q2 < NQ; ++q2) {
            a += B[q2 * NI + ty] * y0[q2 * NQ + tx];
            b += G[q2 * NI + ty] * y1[q2 * NQ + tx];
        }
        s1[ty * NQ + tx] = a;
        s1[O1 + ty * NQ + tx] = b;
    }
    __syncthreads();
    if (act && tx < NI && ty < NI) {
        R o = 0;
#pragma unroll
        for (int q1 = 0; q1 < NQ; ++q1)
            o += G[q1 * NI + tx] * s1[ty * NQ + q1] + B[q1 * NI + tx] * s1[O1 + ty * NQ + q1];
        out[ty * NI + tx] = o;
    }
    __syncthreads();
}

template <class C, class R>
__device__ __forceinline__ void bwd2_tab(const R *__restrict__ T1, const R *__restrict__ T2,
                                         const R *f, R *s1, R *out, int tx, int ty, bool act)
{
    constexpr int NI = C::NI, NQ = C::NQ;
    if (act && tx < NQ && ty < NI) {
        R a = 0;
#pragma unroll
        for (int q2 = 0; q2 < NQ; ++q2) a += T2[q2 * NI + ty] * f[q2 * NQ + tx];
        s1[ty * NQ + tx] = a;
    }
    __syncthreads();
    if (act && tx < NI && ty < NI) {
        R o = 0;
#pragma unroll
        for (int q1 = 0; q1 < NQ; ++q1) o += T1[q1 * NI + tx] * s1[ty * NQ + q1];
        out[ty * NI + tx] += o;
    }
    __syncthreads();
}

// -------------------------------------------------------------------------
// Quality metrics at one point (paper Sec. 2.2, Sec. 4.1), FP64.
//
// mu is a function of the invariants I1 = |T|^2, tau = det T and (3D)
// I2 = |cof T|^2 (|T^-1|^2 = I2 / tau^2).  With g1 = 2T, gt = cof T and
// g2 = 2 (I1 T - T T^T T):
//   dmu/dT       = f1 g1 + ft gt + f2 g2
//   d2mu/dT2     = f1 2Id + ft d2tau + f2 d2I2 + sum_uv f_uv g_u (x) g_v.
// -------------------------------------------------------------------------
// Packed index of (r, s), r <= s, in a row-major upper triangle of size DD.
template <int DD>
__host__ __device__ constexpr int pidx(int r, int s)
{
    return r * DD - r * (r - 1) / 2 + (s - r);
}

struct Inv {
    double f1, ft, f2;               // first derivatives of mu w.r.t. (I1, tau, I2)
    double f11, f1t, ftt, f12, f2t;  // second derivatives (f22 = 0 for all metrics)
};

template <int D>
__device__ __forceinline__ void cofactor(const double *T, double *Cf)
{
    if (D == 2) {
        Cf[0] = T[3]; Cf[1] = -T[2]; Cf[2] = -T[1]; Cf[3] = T[0];
    } else {
        Cf[0] = T[4] * T[8] - T[5] * T[7];
        Cf[1] = T[5] * T[6] - T[3] * T[8];
        Cf[2] = T[3] * T[7] - T[4] * T[6];
        Cf[3] = T[2] * T[7] - T[1] * T[8];
        Cf[4] = T[0] * T[8] - T[2] * T[6];
        Cf[5] = T[1] * T[6] - T[0] * T[7];
        Cf[6] = T[1] * T[5] - T[2] * T[4];
        Cf[7] = T[2] * T[3] - T[0] * T[5];
        Cf[8] = T[0] * T[4] - T[1] * T[3];
    }
}

// tau^(-1/3) for tau > 0: a float estimate refined by two Newton steps on
// f(y) = y^-3 - tau, y <- y (4 - tau y^3) / 3 (quadratic convergence, ~1e-7
// -> ~1e-14 -> rounding); about 15 FP64 operations where cbrt and two
// divisions took ~45.  Outside the float range: the library cbrt.
__device__ __forceinline__ double rcbrt_newton(double t)
{
    if (!(t > 1e-30 && t < 1e30)) return 1.0 / cbrt(t);
    double y = (double)rcbrtf((float)t);
#pragma unroll
    for (int i = 0; i < 2; ++i) y = y * (4.0 - t * (y * y * y)) * (1.0 / 3.0);
    return y;
}

// mu and the scalar derivatives for metric id at invariants (I1, tau, I2).
// mu_7 = |T - T^-t|^2 = I1 - 2D + |T^-1|^2 (the cross term <T, T^-t> is
// tr(T^-1 T) = D), with |T^-1|^2 = I2 / tau^2 in 3D and I1 / tau^2 in 2D;
// mu_9 = tau mu_7.
template <int D>
__device__ __forceinline__ double metric_scalars(int id, double I1, double tau, double I2, Inv &v)
{
    v.f1 = v.ft = v.f2 = v.f11 = v.f1t = v.ftt = v.f12 = v.f2t = 0.0;
    double mu = 0.0;
    if (id == MET_303 || id == MET_303_55) {
        const double y = rcbrt_newton(tau);           // tau^(-1/3)
        const double c = y * y;                      // tau^(-2/3)
        const double it = c * y;                     // 1 / tau
        // constant factors as products (a division by a literal is a full FP64 division)
        constexpr double k3 = 1.0 / 3.0, k9 = -2.0 / 9.0, k27 = 10.0 / 27.0;
        mu = I1 * c * k3 - 1.0;
        v.f1 = c * k3;
        v.f1t = k9 * c * it;
        v.ft = v.f1t * I1;
        v.ftt = k27 * I1 * c * it * it;
        if (id == MET_303_55) {
            mu += (tau - 1.0) * (tau - 1.0);
            v.ft += 2.0 * (tau - 1.0);
            v.ftt += 2.0;
        }
        return mu;
    }
    const double it = 1.0 / tau;
    if (id == MET_2) {
        mu = 0.5 * I1 * it - 1.0;
        v.f1 = 0.5 * it;
        v.ft = -0.5 * I1 * it * it;
        v.f1t = -0.5 * it * it;
        v.ftt = I1 * it * it * it;
    } else if (id == MET_302) {
        constexpr double k9 = 1.0 / 9.0;
        const double it2 = it * it, s9 = it2 * k9;
        mu = I1 * I2 * s9 - 1.0;
        v.f1 = I2 * s9;
        v.f2 = I1 * s9;
        v.ft = -2.0 * I1 * I2 * s9 * it;
        v.f12 = s9;
        v.f1t = -2.0 * I2 * s9 * it;
        v.f2t = -2.0 * I1 * s9 * it;
        v.ftt = 6.0 * I1 * I2 * s9 * it2;
    } else if (id == MET_7 || id == MET_9) {
        const double it2 = it * it;
        const double J = (D == 3 ? I2 : I1) * it2;            // |T^-1|^2
        if (id == MET_7) {
            mu = I1 + J - 2.0 * D;
            if (D == 3) {
                v.f1 = 1.0;
                v.f2 = it2;
                v.ft = -2.0 * J * it;
                v.f2t = -2.0 * it2 * it;
                v.ftt = 6.0 * J * it2;
            } else {
                v.f1 = 1.0 + it2;
                v.ft = -2.0 * J * it;
                v.f1t = -2.0 * it2 * it;
                v.ftt = 6.0 * J * it2;
            }
        } else {
            mu = tau * (I1 + J - 2.0 * D);
            if (D == 3) {
                v.f1 = tau;
                v.f2 = it;
                v.ft = I1 - J - 6.0;
                v.f1t = 1.0;
                v.f2t = -it2;
                v.ftt = 2.0 * J * it;
            } else {
                v.f1 = tau + it;
                v.ft = I1 - J - 4.0;
                v.f1t = 1.0 - it2;
                v.ftt = 2.0 * J * it;
            }
        }
    } else if (id == MET_55) {
        mu = (tau - 1.0) * (tau - 1.0);
        v.ft = 2.0 * (tau - 1.0);
        v.ftt = 2.0;
    }
    return mu;
}

template <int D>
__device__ __forceinline__ void invariants(const double *T, double &I1, double &tau, double &I2,
                                           double *Cf);

// mu alone, in FP64 from the FP64 image of T.  The energy is the line-search
// quantity: near a zero-energy optimum mu = O(rounding), and an error in I1
// or tau enters mu at first order (unlike an error in T, which enters at
// second order where dmu/dT = 0), so there I1, tau and I2 are formed in FP64
// even when T came from double-float contractions (the double-float floor of
// F, ~4e-15 S_F, stopped Newton short of |dF|/|dF0| = 1e-10).
template <int D>
__device__ __forceinline__ double metric_mu_fp64(int id, const double *T)
{
    double Cf[D * D], I1, tau, I2;
    invariants<D>(T, I1, tau, I2, Cf);
    Inv v;
    return metric_scalars<D>(id, I1, tau, I2, v);
}

template <int D>
__device__ __forceinline__ void invariants(const double *T, double &I1, double &tau, double &I2,
                                           double *Cf)
{
    constexpr int DD = D * D;
    I1 = 0.0;
#pragma unroll
    for (int i = 0; i < DD; ++i) I1 += T[i] * T[i];
    cofactor<D>(T, Cf);
    tau = 0.0;
#pragma unroll
    for (int b = 0; b < D; ++b) tau += T[b] * Cf[b];
    I2 = 0.0;
    if (D == 3) {
#pragma unroll
        for (int i = 0; i < DD; ++i) I2 += Cf[i] * Cf[i];
    }
}

// cof T in double-float (same entry order as cofactor()).
template <int D>
__device__ __forceinline__ void cofactor_dw(const df *T, df *Cf)
{
    if (D == 2) {
        Cf[0] = T[3]; Cf[1] = -T[2]; Cf[2] = -T[1]; Cf[3] = T[0];
    } else {
        Cf[0] = dw_fms(T[4], T[8], T[5], T[7]);
        Cf[1] = dw_fms(T[5], T[6], T[3], T[8]);
        Cf[2] = dw_fms(T[3], T[7], T[4], T[6]);
        Cf[3] = dw_fms(T[2], T[7], T[1], T[8]);
        Cf[4] = dw_fms(T[0], T[8], T[2], T[6]);
        Cf[5] = dw_fms(T[1], T[6], T[0], T[7]);
        Cf[6] = dw_fms(T[1], T[5], T[2], T[4]);
        Cf[7] = dw_fms(T[2], T[3], T[0], T[5]);
        Cf[8] = dw_fms(T[0], T[4], T[1], T[3]);
    }
}

// Pointwise algebra on the FP32 pipes for the metrics of (I1, tau): B300
// issues FP64 ~60x slower than FP32, and the per-point FP64 algebra bounded
// the energy, gradient and set-up kernels.  T = A / w from the double-float
// Jacobian (unit: w = 1, no scaling), cof T, I1 = |T|^2 and tau = det T in
// double-float; I1 and tau are returned in double for the metric's scalar
// derivatives, which stay FP64.
template <int D, int NQD>
__device__ __forceinline__ void point_T_dw(const df *sA, int q, double iws, bool unit, df *T, df *Cf,
                                           double &I1, double &tau, df *I1w = nullptr,
                                           df *tauw = nullptr)
{
    const df s = from_db<df>(iws);
#pragma unroll
    for (int r = 0; r < D * D; ++r) T[r] = unit ? sA[r * NQD + q] : to_df(sA[r * NQD + q] * s);
    cofactor_dw<D>(T, Cf);
    df a(0.0f, 0.0f), t(0.0f, 0.0f);
#pragma unroll
    for (int r = 0; r < D * D; ++r) acc_add(a, T[r] * T[r]);
#pragma unroll
    for (int b = 0; b < D; ++b) acc_add(t, T[b] * Cf[b]);
    a = norm(a);
    t = norm(t);
    if (I1w) *I1w = a;
    if (tauw) *tauw = t;
    I1 = to_db(a);
    tau = to_db(t);
}

// mu_303 (+ mu_55) and its scalar derivatives in double-float, for the
// kernels whose remaining FP64 work was these scalars: tau^(-1/3) by a float
// estimate and two Newton steps y <- y + y (1 - tau y^3) / 3 in double-float,
// then c = y^2 = tau^(-2/3), 1/tau = c y, mu = I1 c / 3 - 1,
// f1 = c / 3, f1t = -2 c / (9 tau), ft = f1t I1, ftt = 10 I1 c / (27 tau^2)
// (plus (tau - 1)^2, 2 (tau - 1), 2 for the size term).
struct InvW {
    df f1, ft, f1t, ftt;
};
__device__ __forceinline__ df dw_sub(const df &a, const df &b) { return add_norm(a.h, -b.h, a.l - b.l); }
__device__ __forceinline__ df dw_mul(const df &a, const df &b) { return to_df(a * b); }
__device__ __forceinline__ df metric303_dw(const df &I1, const df &tau, bool size_term, InvW &v)
{
    const df one(1.0f, 0.0f);
    df y(rcbrtf(tau.h), 0.0f);
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const df ty3 = dw_mul(tau, dw_mul(dw_mul(y, y), y));
        const df r = dw_sub(one, ty3);
        y = y + dw_mul(y, dw_mul(r, from_db<df>(1.0 / 3.0)));
    }
    const df c = dw_mul(y, y), it = dw_mul(c, y);
    const df k3 = from_db<df>(1.0 / 3.0), k9 = from_db<df>(-2.0 / 9.0), k27 = from_db<df>(10.0 / 27.0);
    df mu = dw_sub(dw_mul(dw_mul(I1, c), k3), one);
    v.f1 = dw_mul(c, k3);
    v.f1t = dw_mul(k9, dw_mul(c, it));
    v.ft = dw_mul(v.f1t, I1);
    v.ftt = dw_mul(dw_mul(k27, dw_mul(I1, c)), dw_mul(it, it));
    if (size_term) {
        const df tm = dw_sub(tau, one);
        mu = mu + dw_mul(tm, tm);
        v.ft = v.ft + df(2.0f * tm.h, 2.0f * tm.l);
        v.ftt = v.ftt + df(2.0f, 0.0f);
    }
    return mu;
}

// 3D, double-float: I2 = |cof T|^2, T^T T, T T^T and g2 = dI2/dT = 2 (I1 T - T T^T T).
__device__ __forceinline__ double i2_dw(const df *T, const df *Cf, const df &I1, df *g2, df *TtT,
                                        df *TTt)
{
    df s(0.0f, 0.0f);
#pragma unroll
    for (int r = 0; r < 9; ++r) acc_add(s, Cf[r] * Cf[r]);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            df a(0.0f, 0.0f), b(0.0f, 0.0f);
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                acc_add(a, T[k * 3 + i] * T[k * 3 + j]);
                acc_add(b, T[i * 3 + k] * T[j * 3 + k]);
            }
            TtT[i * 3 + j] = norm(a);
            TTt[i * 3 + j] = norm(b);
        }
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            df a(0.0f, 0.0f);
            acc_add(a, I1 * T[i * 3 + j]);
#pragma unroll
            for (int k = 0; k < 3; ++k) acc_add(a, -(T[i * 3 + k] * TtT[k * 3 + j]));
            const df n = norm(a);
            g2[i * 3 + j] = df(2.0f * n.h, 2.0f * n.l);
        }
    return to_db(norm(s));
}

// g2 = dI2/dT = 2 (I1 T - T T^T T) (3D only).
__device__ __forceinline__ void dI2_3(const double *T, double I1, double *g2, double *TtT,
                                      double *TTt)
{
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            double s = 0, u = 0;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                s += T[k * 3 + i] * T[k * 3 + j];
                u += T[i * 3 + k] * T[j * 3 + k];
            }
            TtT[i * 3 + j] = s;
            TTt[i * 3 + j] = u;
        }
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            double s = 0;
#pragma unroll
            for (int k = 0; k < 3; ++k) s += T[i * 3 + k] * TtT[k * 3 + j];
            g2[i * 3 + j] = 2.0 * (I1 * T[i * 3 + j] - s);
        }
}

// sign of the permutation (a, c, 3-a-c) for distinct a != c in {0,1,2}
__device__ __forceinline__ double eps3(int a, int c)
{
    const int m = 3 - a - c;
    return ((a == 0 && c == 1 && m == 2) || (a == 1 && c == 2 && m == 0) || (a == 2 && c == 0 && m == 1))
               ? 1.0 : -1.0;
}

// Entry (r, s) = ((a,b), (c,e)) of d2mu/dT2.
template <int D>
__device__ __forceinline__ double metric_K_entry(int r, int s, const double *T, const double *Cf,
                                                 const double *g2, const double *TtT,
                                                 const double *TTt, double I1, const Inv &v)
{
    const int a = r / D, b = r % D, c = s / D, e = s % D;
    const double g1r = 2.0 * T[r], g1s = 2.0 * T[s];
    double k = v.f11 * g1r * g1s + v.f1t * (g1r * Cf[s] + Cf[r] * g1s) + v.ftt * Cf[r] * Cf[s];
    if (r == s) k += 2.0 * v.f1;
    // d2 tau / dT_ab dT_ce
    double d2t = 0.0;
    if (D == 2) {
        if (a != c && b != e) d2t = (a == 0 ? 1.0 : -1.0) * (b == 0 ? 1.0 : -1.0);
    } else {
        if (a != c && b != e) d2t = eps3(a, c) * eps3(b, e) * T[(3 - a - c) * 3 + (3 - b - e)];
    }
    k += v.ft * d2t;
    if (D == 3 && (v.f2 != 0.0 || v.f12 != 0.0 || v.f2t != 0.0)) {
        k += v.f12 * (g1r * g2[s] + g2[r] * g1s) + v.f2t * (g2[r] * Cf[s] + Cf[r] * g2[s]);
        double d2 = 4.0 * T[r] * T[s];
        if (r == s) d2 += 2.0 * I1;
        if (a == c) d2 -= 2.0 * TtT[e * 3 + b];
        d2 -= 2.0 * T[a * 3 + e] * T[c * 3 + b];
        if (b == e) d2 -= 2.0 * TTt[a * 3 + c];
        k += v.f2 * d2;
    }
    return k;
}

// Size field of the size target and the target scale w (W = w I).
template <int D>
__device__ __forceinline__ double target_scale(int target, double h0, const double *xq)
{
    if (target != TGT_SIZE) return 1.0;
    const double twopi = 6.283185307179586476925286766559;
    double s = 0.5;
#pragma unroll
    for (int k = 0; k < D; ++k) s *= sin(twopi * xq[k]);
    s += 1.0;
    return h0 * (D == 3 ? cbrt(s) : sqrt(s));
}

// Target scale of the discrete target, w = h0 eta_q^(1/D); NaN when
// eta_q <= 0 (no target: the callers treat the point as inverted).
template <int D>
__device__ __forceinline__ double discrete_scale(double h0, double eta_q)
{
    if (!(eta_q > 0.0)) return __longlong_as_double(0x7ff8000000000000LL);
    return h0 * (D == 3 ? cbrt(eta_q) : sqrt(eta_q));
}

// Table of the compute type R.
template <class R> __device__ __forceinline__ const R *table_of(const ElemParams &P);
template <> __device__ __forceinline__ const double *table_of<double>(const ElemParams &P) { return P.tab; }
template <> __device__ __forceinline__ const float *table_of<float>(const ElemParams &P) { return P.tabf; }
template <> __device__ __forceinline__ const df *table_of<df>(const ElemParams &P) { return P.tabw; }

// Normalised product in the compute type.
__device__ __forceinline__ double prod(double a, double b) { return a * b; }
__device__ __forceinline__ float prod(float a, float b) { return a * b; }
__device__ __forceinline__ df prod(const df &a, const df &b) { return to_df(a * b); }


}  // namespace tmop
