// 3D Hessian action with a collocated derivative, one element per group of
// lanes of one warp (sm_103a).
//
// y = G^T B^T (H : B G v) (paper Sec. 3.4, eq. vm_pa_hess).  The reference
// gradient of a nodal field is taken in two steps: its values at the Gauss
// points by three B contractions (B_qi = l_i(chi_q)), then the collocated
// derivative D_qk = m_k'(chi_q) of the Lagrange polynomials m_k through the
// points along each direction.  G = D B holds exactly (a polynomial of degree
// p < n_q is reproduced by its values at the points), so dA is the same
// quantity as in Sec. 3.2; with n_q = p+1 the forward pass costs 6 n^4 instead
// of 8 n^4 multiply-adds per component, and the transposed pass the same.
//
// Thread mapping: the n_q x n_q lanes of an element own the (q1, q2) columns
// and walk q3, so every contraction along q3 (B and D) reads its operands from
// registers and its table entries from the kernel parameter space
// (compile-time indices), while the contractions along q1 and q2 go through two
// small per-element shared buffers.  An element never spans two warps: the
// stages synchronise with __syncwarp, and the CTA-wide barrier is used once,
// for the tables.  Accumulators start from their first product (no add to
// zero) and intermediate values are left unnormalised: a double-float value
// with a low word of a few ulp(h) is a valid operand of the error-free
// products.
//
// Variants (chosen per configuration by the autotuner, autotune.cu):
//   SC = false  the q3 column of dA / Y stays in registers (9 n_q values);
//   SC = true   it lives in shared memory (fewer registers, more resident
//               warps); ROLL keeps one copy of the point body (less code);
//   WPB         warps per CTA (2, 4 or 8); a warp finds its own element tile,
//               so a CTA may span two tiles of a batched launch;
//   MINB        minimum resident CTAs per SM asked of the register allocator;
//   AL          (shared-memory columns) the columns are blocked per warp and
//               the two contraction buffers live in column rows that are dead
//               at the time: rows 6-8 (component 2) during the forward pass,
//               rows 0-2 (component 0) during the transposed pass, which
//               frees 2 x BUF values per element of shared memory for more
//               resident CTAs;
//   GA          the input values of all three components are gathered into
//               registers before the forward pass (one exposed gather latency
//               per element instead of three).
#pragma once

#include <type_traits>

#include "elem_kernels.cuh"

namespace tmop {

// 1D tables of the collocated action, passed by value in the kernel
// parameter space: B[q * NI + i] and D[q * NQ + k].
template <class R, int NI, int NQ>
struct ColTab {
    R B[NQ * NI];
    R D[NQ * NQ];
};

template <class C, int WPB_ = 4>
struct Apply3cShape {
    static constexpr int TPE = C::NQ * C::NQ;                 // one lane per (q1, q2) column
    static_assert(TPE <= 32, "an element must fit in one warp");
    static constexpr int EPW = 32 / TPE;                       // elements per warp
    static constexpr int WPB = WPB_;                           // warps per CTA
    static constexpr int EPB = EPW * WPB;                      // elements per CTA
    static constexpr int NT = 32 * WPB;
    static constexpr int BUF = C::NQ * C::NQ * C::NQ;          // >= NP, NQ NI^2, NQ^2 NI
    static constexpr int NPL = (C::NP + TPE - 1) / TPE;        // map entries per lane
    static constexpr int TABN = C::NQ * C::NI + C::NQ * C::NQ;
    // Stride of the two buffers of consecutive elements of a warp, in values of
    // R: every stage reads or writes one n_q x n_q plane per element, at the
    // same plane offset for all lanes, so elements whose planes start
    // span = TPE * sizeof(R) / 4 banks apart use disjoint banks when
    // EPW * span <= 32 (no two-way conflict between the elements of a warp).
    template <class R>
    static constexpr int es_padded()
    {
        constexpr int w = (int)(sizeof(R) / 4);
        constexpr int span = TPE * w;
        if (span >= 32 || EPW == 1) return 2 * BUF;
        int es = 2 * BUF;
        while ((es * w) % 32 != span % 32) ++es;
        return es;
    }
    // AL: the buffers of a warp's elements lie in three column rows of the
    // warp (3 * NQ * 32 values); padded stride where that still fits
    template <class R>
    static constexpr int es(bool al)
    {
        return (!al || 2 * BUF + (EPW - 1) * es_padded<R>() <= 3 * C::NQ * 32) ? es_padded<R>()
                                                                              : 2 * BUF;
    }
    static_assert(2 * EPW * BUF <= 3 * C::NQ * 32, "aliased buffers");
    template <class R>
    static constexpr size_t bytes(bool sc, bool al = false)
    {
        return sizeof(R) * (size_t)(((TABN + 1) & ~1) + (al ? 0 : EPB * es<R>(false)) +
                                    (sc ? 9 * C::NQ * NT : 0));
    }
};

// First term of an accumulation (no add to zero); the df product stays unnormalised.
__device__ __forceinline__ df mul1(const df &a, const df &b)
{
    const dprod p = a * b;
    return df(p.p, p.e);
}
__device__ __forceinline__ float mul1(float a, float b) { return a * b; }
__device__ __forceinline__ double mul1(double a, double b) { return a * b; }

// Streaming loads of the stored data (read once per action).
__device__ __forceinline__ df ld_stream(const df *p)
{
    const float2 v = __ldcs(reinterpret_cast<const float2 *>(p));
    return df(v.x, v.y);
}
__device__ __forceinline__ float ld_stream(const float *p) { return __ldcs(p); }
__device__ __forceinline__ double ld_stream(const double *p) { return __ldcs(p); }
// Two consecutive stored values (an entry pair of the stored layout; p is
// aligned to their combined size).
__device__ __forceinline__ void ld_stream2(const df *p, df &a, df &b)
{
    const float4 v = __ldcs(reinterpret_cast<const float4 *>(p));
    a = df(v.x, v.y);
    b = df(v.z, v.w);
}
__device__ __forceinline__ void ld_stream2(const float *p, float &a, float &b)
{
    const float2 v = __ldcs(reinterpret_cast<const float2 *>(p));
    a = v.x;
    b = v.y;
}
__device__ __forceinline__ void ld_stream2(const double *p, double &a, double &b)
{
    const double2 v = __ldcs(reinterpret_cast<const double2 *>(p));
    a = v.x;
    b = v.y;
}

// Conversions of the gathered input and of the element-vector output (the
// FP64-unit conversions measured faster here than the bit-level ones).
template <class RC> __device__ __forceinline__ RC cvt_in(double v) { return RC(v); }
template <class RC> __device__ __forceinline__ RC cvt_in(float v) { return RC(v); }
__device__ __forceinline__ double cvt_out(const df &v) { return (double)v; }
__device__ __forceinline__ double cvt_out(double v) { return v; }
__device__ __forceinline__ float cvt_out(float v) { return v; }

// f(integral_constant<int, 0>), ..., f(integral_constant<int, N-1>), in order
// (a loop whose index is a constant expression in the body).
template <int N, class F>
__device__ __forceinline__ void static_for(F &&f)
{
    if constexpr (N > 0) {
        static_for<N - 1>(f);
        f(std::integral_constant<int, N - 1>{});
    }
}

// Row and column of the k-th entry of the packed upper triangle of a 9 x 9
// symmetric matrix (the inverse of pidx<9>).
__host__ __device__ constexpr int prow9(int k)
{
    int r = 0;
    while (k >= 9 - r) {
        k -= 9 - r;
        ++r;
    }
    return r;
}
__host__ __device__ constexpr int pcol9(int k) { return prow9(k) + (k - pidx<9>(prow9(k), prow9(k))); }

// PFN (rolled shared-memory columns): prefetch the next point's stored values
// into L2 while the current point is multiplied.  PIPE (shared-memory
// columns): the thread's stored values, in order (point, packed entry), are
// taken in chunks of 9 held in two register buffers, the loads of chunk j+1
// issued before the multiply-adds of chunk j; the same arithmetic in the same
// order as the plain point loop.
template <class C, class RV, class RC, int WPB, bool SC, bool ROLL, int MINB, bool PFN = false,
          bool PIPE = false, bool AL = false, bool GA = false>
__global__ void __launch_bounds__(Apply3cShape<C, WPB>::NT, MINB)
k_apply3c(ElemParams P, const RV *__restrict__ v, const RC *__restrict__ H, RV *__restrict__ ev,
          const int *__restrict__ stop_iter, int k, BatchArgs BA, int64_t ntiles,
          const ColTab<RC, C::NI, C::NQ> T)
{
    static_assert(C::D == 3, "3D kernel");
    using S = Apply3cShape<C, WPB>;
    static_assert(C::EPB == 4 * S::EPW, "element tiles of the other kernels hold four warps");
    constexpr int NI = C::NI, NQ = C::NQ, NP = C::NP, NQD = C::NQD, NS = C::NS, BUF = S::BUF;

    extern __shared__ __align__(16) unsigned char smem[];
    RC *Bs = reinterpret_cast<RC *>(smem);                  // B[q * NI + i]
    RC *Ds = Bs + NQ * NI;                                  // D[q * NQ + k]
    // copy the tables from the parameter space, compile-time indices only (a
    // thread-indexed copy would make the compiler place the tables in local memory)
    if (threadIdx.x == 0) {
#pragma unroll
        for (int i = 0; i < NQ * NI; ++i) Bs[i] = T.B[i];
#pragma unroll
        for (int i = 0; i < NQ * NQ; ++i) Ds[i] = T.D[i];
    }
    __syncthreads();                                        // the only CTA-wide barrier

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int slot = lane / S::TPE;
    const bool act = slot < S::EPW;
    const int t = lane - slot * S::TPE;
    const int el = warp * S::EPW + (act ? slot : 0);        // element slot in the CTA
    const int tx = t % NQ, ty = t / NQ;
    // the warp's element tile: g = global element slot, tiles of C::EPB elements
    const int64_t g = (int64_t)blockIdx.x * S::EPB + warp * S::EPW;
    int64_t e0 = g;                                         // first element of the warp
    const int *stop = stop_iter;
    if (BA.tiles) {
        const int64_t ti = g / C::EPB;
        if (ti >= ntiles) return;                           // past the last tile of the batch
        const int2 tt = BA.tiles[ti];
        const BMesh &mb = BA.meshes[tt.x];
        P = mb.P;
        if (BA.in >= 0) v = static_cast<const RV *>(mb.ptr[BA.in]);
        if (BA.aux >= 0) H = static_cast<const RC *>(mb.ptr[BA.aux]);
        if (BA.out >= 0) ev = static_cast<RV *>(mb.ptr[BA.out]);
        if (BA.stop) stop = BA.stop + (int64_t)tt.x * BA.stop_stride;
        e0 = (int64_t)tt.y * C::EPB + g % C::EPB;
    }
    if (stop && *stop < iter_of(stop, k)) return;          // MINRES already stopped

    static_assert(!AL || SC, "aliased buffers need shared-memory columns");
    // SC: the dA / Y columns of every thread, [(r * NQ + q3) * NT + thread],
    // or with AL blocked per warp, [warp][(r * NQ + q3) * 32 + lane]
    constexpr int CST = AL ? 32 : S::NT;                    // stride of a column row
    RC *cs = Bs + ((S::TABN + 1) & ~1) + (AL ? warp * 9 * NQ * 32 : S::EPB * S::template es<RC>(false));
    const int ci = AL ? lane : threadIdx.x;                 // the thread's column
    // AL: the buffers of the forward pass in rows 6-8 (component 2), of the
    // transposed pass in rows 0-2 (component 0)
    constexpr int ES = S::template es<RC>(AL);              // buffer stride per element
    RC *b0 = AL ? cs + 6 * NQ * 32 + (act ? slot : 0) * ES
                : Bs + ((S::TABN + 1) & ~1) + el * ES;
    RC *b1 = b0 + BUF;
    const int64_t e = e0 + (act ? slot : 0);
    const bool valid = act && e < P.E;
    int m[S::NPL];
#pragma unroll
    for (int j = 0; j < S::NPL; ++j) {
        const int i = t + j * S::TPE;
        m[j] = (valid && i < NP) ? P.map[e * NP + i] : 0;
    }
    RV gv[GA ? 3 : 1][S::NPL];
    if (GA) {
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int j = 0; j < S::NPL; ++j) {
                const int i = t + j * S::TPE;
                gv[GA ? c : 0][j] = (valid && i < NP) ? v[c * P.Nx + m[j]] : RV(0);
            }
    }

    RC col[SC ? 1 : 9][NQ];                                 // dA_{cb} then Y_{cb} at (tx, ty, q3)
#define COLW(r, q3) (SC ? cs[((r) * NQ + (q3)) * CST + ci] : col[SC ? 0 : (r)][q3])

    // ---- forward: values at the points, then the collocated derivative
#pragma unroll 1
    for (int c = 0; c < 3; ++c) {
#pragma unroll
        for (int j = 0; j < S::NPL; ++j) {
            const int i = t + j * S::TPE;
            if (valid && i < NP) {
                if constexpr (GA) {
                    RV x = gv[0][j];                        // c is a loop variable: unrolled select
#pragma unroll
                    for (int cc = 1; cc < 3; ++cc)
                        if (cc == c) x = gv[GA ? cc : 0][j];
                    b0[i] = cvt_in<RC>(x);
                } else {
                    b0[i] = cvt_in<RC>(v[c * P.Nx + m[j]]);
                }
            }
        }
        __syncwarp();
        if (valid && ty < NI) {                             // i1 -> q1
            RC Bx[NI];
#pragma unroll
            for (int i = 0; i < NI; ++i) Bx[i] = Bs[tx * NI + i];
#pragma unroll
            for (int i3 = 0; i3 < NI; ++i3) {
                const RC *u = b0 + (i3 * NI + ty) * NI;
                RC a = mul1(Bx[0], u[0]);
#pragma unroll
                for (int i1 = 1; i1 < NI; ++i1) acc_add(a, Bx[i1] * u[i1]);
                b1[(i3 * NI + ty) * NQ + tx] = a;
            }
        }
        __syncwarp();
        RC g0[NQ], g1[NQ], g2[NQ];
        if (valid) {
            RC By[NI], s2[NI], U[NQ];
#pragma unroll
            for (int i = 0; i < NI; ++i) By[i] = Bs[ty * NI + i];
#pragma unroll
            for (int i3 = 0; i3 < NI; ++i3) {               // i2 -> q2
                const RC *w = b1 + i3 * NI * NQ + tx;
                RC a = mul1(By[0], w[0]);
#pragma unroll
                for (int i2 = 1; i2 < NI; ++i2) acc_add(a, By[i2] * w[i2 * NQ]);
                s2[i3] = a;
            }
#pragma unroll
            for (int q3 = 0; q3 < NQ; ++q3) {               // i3 -> q3 (registers)
                RC a = mul1(T.B[q3 * NI], s2[0]);
#pragma unroll
                for (int i3 = 1; i3 < NI; ++i3) acc_add(a, T.B[q3 * NI + i3] * s2[i3]);
                U[q3] = a;
            }
#pragma unroll
            for (int q3 = 0; q3 < NQ; ++q3) b0[(q3 * NQ + ty) * NQ + tx] = U[q3];
#pragma unroll
            for (int q3 = 0; q3 < NQ; ++q3) {               // d/dxbar3 (registers)
                RC a = mul1(T.D[q3 * NQ], U[0]);
#pragma unroll
                for (int kk = 1; kk < NQ; ++kk) acc_add(a, T.D[q3 * NQ + kk] * U[kk]);
                g2[q3] = a;
            }
        }
        __syncwarp();
        if (valid) {
            RC Dx[NQ], Dy[NQ];
#pragma unroll
            for (int kk = 0; kk < NQ; ++kk) {
                Dx[kk] = Ds[tx * NQ + kk];
                Dy[kk] = Ds[ty * NQ + kk];
            }
#pragma unroll
            for (int q3 = 0; q3 < NQ; ++q3) {               // d/dxbar1, d/dxbar2
                const RC *row = b0 + (q3 * NQ + ty) * NQ;
                const RC *cl = b0 + q3 * NQ * NQ + tx;
                RC a = mul1(Dx[0], row[0]);
                RC b = mul1(Dy[0], cl[0]);
#pragma unroll
                for (int kk = 1; kk < NQ; ++kk) {
                    acc_add(a, Dx[kk] * row[kk]);
                    acc_add(b, Dy[kk] * cl[kk * NQ]);
                }
                g0[q3] = a;
                g1[q3] = b;
            }
        }
        if (AL && c == 2) __syncwarp();                     // rows 6-8 held the buffers
        if (valid) {
            if (SC) {
#pragma unroll
                for (int q3 = 0; q3 < NQ; ++q3) {
                    cs[((c * 3 + 0) * NQ + q3) * CST + ci] = g0[q3];
                    cs[((c * 3 + 1) * NQ + q3) * CST + ci] = g1[q3];
                    cs[((c * 3 + 2) * NQ + q3) * CST + ci] = g2[q3];
                }
            } else {
                // c is a loop variable: select the register rows with unrolled tests
#pragma unroll
                for (int cc = 0; cc < 3; ++cc)
                    if (cc == c) {
#pragma unroll
                        for (int q3 = 0; q3 < NQ; ++q3) {
                            COLW(cc * 3 + 0, q3) = g0[q3];
                            COLW(cc * 3 + 1, q3) = g1[q3];
                            COLW(cc * 3 + 2, q3) = g2[q3];
                        }
                    }
            }
        }
        __syncwarp();                                       // b0 is reused by the next gather
    }

    // ---- pointwise: Y = H : dA with the symmetric-packed stored data; the
    // packed entries k = 0..NS-1 of a point in order, row 0 starting every sum
    static_assert(NS == 45 && C::PAIRS, "3D packed data in entry-pair planes");
    const RC *He = H + e * (int64_t)C::HST;
    const int pt = ty * NQ + tx;                            // the thread's point of a q3 plane
    // the terms of packed entry KK (row r <= column s, value h); FP32 / FP64
    // multiply-adds as explicit FMAs, so that every variant rounds alike
    auto mac = [](RC &acc, const RC &a, const RC &b) {
        if constexpr (std::is_same<RC, df>::value) acc_add(acc, a * b);
        else acc = fma(a, b, acc);
    };
    auto term = [&](auto KK, const RC &h, const RC *d, RC *y) {
        constexpr int kk = decltype(KK)::value;
        constexpr int r = prow9(kk), sc = pcol9(kk);
        if constexpr (r == 0) {
            y[sc] = mul1(h, d[0]);
            if constexpr (sc > 0) mac(y[0], h, d[sc]);
        } else {
            mac(y[sc], h, d[r]);
            if constexpr (sc != r) mac(y[r], h, d[sc]);
        }
    };
    // the stored values of point q: entry pair planes from He + 2 q, the last
    // entry's plane from He + q (compile-time offsets from the two bases)
    constexpr int LAST = 2 * C::NPR * NQD;
    static_assert(C::hoff(3, 5) == 2 * 5 + 2 * NQD + 1 && C::hoff(NS - 1, 5) == LAST + 5,
                  "the point loop's offsets are those of the stored layout");
    // L2 prefetch of the stored values of point q (one line per entry pair)
    auto prefetch_point = [&](int q) {
        const RC *Hp = He + 2 * q;
#pragma unroll
        for (int g = 0; g < C::NPR; ++g)
            asm volatile("prefetch.global.L2 [%0];" ::"l"(Hp + 2 * g * NQD));
        asm volatile("prefetch.global.L2 [%0];" ::"l"(He + q + LAST));
    };
    // value of packed entry kk (compile time) at point q
    auto hval = [&](auto KK, int q) -> RC {
        constexpr int kk = decltype(KK)::value;
        if constexpr (kk < 2 * C::NPR)
            return ld_stream(He + 2 * q + (2 * (kk >> 1) * NQD + (kk & 1)));
        else
            return ld_stream(He + q + LAST);
    };
    if (PIPE && SC && valid) {
        constexpr int CH = 9, NCH = 5;                  // 45 = 5 chunks of 9 per point
        constexpr int NJ = NQ * NCH;
        constexpr int UJ = (NQ % 2 == 0) ? 2 * NCH : NJ;   // chunks per unrolled body
        RC hb0[CH], hb1[CH];                            // the two chunk buffers
        static_for<CH>([&](auto T2) { hb0[decltype(T2)::value] = hval(T2, pt); });
#pragma unroll 1
        for (int j0 = 0; j0 < NJ; j0 += UJ) {
            RC d[9], y[9];
            static_for<UJ>([&](auto JJ) {
                constexpr int jj = decltype(JJ)::value;
                constexpr int c = jj % NCH;             // chunk of the point
                constexpr int c1 = (jj + 1) % NCH;
                RC *cur = (jj & 1) ? hb1 : hb0;
                RC *nxt = (jj & 1) ? hb0 : hb1;
                const int q3 = j0 / NCH + jj / NCH;
                if (j0 + jj + 1 < NJ) {                 // loads of the next chunk
                    const int qn = (j0 / NCH + (jj + 1) / NCH) * NQ * NQ + pt;
                    static_for<CH>([&](auto T2) {
                        constexpr int t2 = decltype(T2)::value;
                        nxt[t2] = hval(std::integral_constant<int, c1 * CH + t2>{}, qn);
                    });
                    if (PFN && c == 0 && q3 + 1 < NQ) prefetch_point((q3 + 1) * NQ * NQ + pt);
                }
                if constexpr (c == 0) {
#pragma unroll
                    for (int r = 0; r < 9; ++r) d[r] = COLW(r, q3);
                }
                static_for<CH>([&](auto T2) {
                    constexpr int t2 = decltype(T2)::value;
                    term(std::integral_constant<int, c * CH + t2>{}, cur[t2], d, y);
                });
                if constexpr (c == NCH - 1) {
#pragma unroll
                    for (int r = 0; r < 9; ++r) COLW(r, q3) = y[r];
                }
            });
        }
    } else if (valid) {
        // ROLL (shared-memory columns only): one copy of the point body
#pragma unroll(SC && ROLL ? 1 : NQ)
        for (int q3 = 0; q3 < NQ; ++q3) {
            const int q = q3 * NQ * NQ + pt;
            if (PFN && q3 + 1 < NQ) prefetch_point(q + NQ * NQ);
            RC d[9], y[9];
#pragma unroll
            for (int r = 0; r < 9; ++r) d[r] = COLW(r, q3);
            const RC *Hp = He + 2 * q;
            static_for<C::NPR>([&](auto G) {            // entries 2g, 2g+1: one pair load
                constexpr int g = decltype(G)::value;
                RC h0, h1;
                ld_stream2(Hp + 2 * g * NQD, h0, h1);
                term(std::integral_constant<int, 2 * g>{}, h0, d, y);
                term(std::integral_constant<int, 2 * g + 1>{}, h1, d, y);
            });
            term(std::integral_constant<int, NS - 1>{}, ld_stream(He + q + LAST), d, y);
#pragma unroll
            for (int r = 0; r < 9; ++r) COLW(r, q3) = y[r];
        }
    }

    // ---- transposed: D^T along each direction, then B^T along q3, q2, q1
    if (AL) {
        b0 = cs + (act ? slot : 0) * ES;
        b1 = b0 + BUF;
    }
#pragma unroll 1
    for (int c = 0; c < 3; ++c) {
        RC Y0[NQ], Y1[NQ], Y2[NQ];
        if (SC) {
#pragma unroll
            for (int q3 = 0; q3 < NQ; ++q3) {
                Y0[q3] = cs[((c * 3 + 0) * NQ + q3) * CST + ci];
                Y1[q3] = cs[((c * 3 + 1) * NQ + q3) * CST + ci];
                Y2[q3] = cs[((c * 3 + 2) * NQ + q3) * CST + ci];
            }
            if (AL && c == 0) __syncwarp();                 // rows 0-2 become the buffers
        } else {
#pragma unroll
            for (int cc = 0; cc < 3; ++cc)
                if (cc == c) {
#pragma unroll
                    for (int q3 = 0; q3 < NQ; ++q3) {
                        Y0[q3] = COLW(cc * 3 + 0, q3);
                        Y1[q3] = COLW(cc * 3 + 1, q3);
                        Y2[q3] = COLW(cc * 3 + 2, q3);
                    }
                }
        }
        if (valid) {
#pragma unroll
            for (int q3 = 0; q3 < NQ; ++q3) {
                b0[(q3 * NQ + ty) * NQ + tx] = Y0[q3];
                b1[(q3 * NQ + ty) * NQ + tx] = Y1[q3];
            }
        }
        __syncwarp();
        RC W[NI];
        if (valid) {
            RC DTx[NQ], DTy[NQ], Z[NQ];
#pragma unroll
            for (int kk = 0; kk < NQ; ++kk) {
                DTx[kk] = Ds[kk * NQ + tx];
                DTy[kk] = Ds[kk * NQ + ty];
            }
#pragma unroll
            for (int q3 = 0; q3 < NQ; ++q3) {
                const RC *row = b0 + (q3 * NQ + ty) * NQ;
                const RC *cl = b1 + q3 * NQ * NQ + tx;
                RC a = mul1(T.D[q3], Y2[0]);                // D^T along q3 from registers
#pragma unroll
                for (int kk = 1; kk < NQ; ++kk) acc_add(a, T.D[kk * NQ + q3] * Y2[kk]);
#pragma unroll
                for (int kk = 0; kk < NQ; ++kk) {
                    acc_add(a, DTx[kk] * row[kk]);
                    acc_add(a, DTy[kk] * cl[kk * NQ]);
                }
                Z[q3] = a;
            }
#pragma unroll
            for (int i3 = 0; i3 < NI; ++i3) {               // q3 -> i3 (registers)
                RC a = mul1(T.B[i3], Z[0]);
#pragma unroll
                for (int q3 = 1; q3 < NQ; ++q3) acc_add(a, T.B[q3 * NI + i3] * Z[q3]);
                W[i3] = a;
            }
        }
        __syncwarp();                                       // every lane has read b0 and b1
        if (valid) {
#pragma unroll
            for (int i3 = 0; i3 < NI; ++i3) b0[(i3 * NQ + ty) * NQ + tx] = W[i3];
        }
        __syncwarp();
        if (valid && ty < NI) {                             // q2 -> i2
            RC BTy[NQ];
#pragma unroll
            for (int q = 0; q < NQ; ++q) BTy[q] = Bs[q * NI + ty];
#pragma unroll
            for (int i3 = 0; i3 < NI; ++i3) {
                const RC *w = b0 + i3 * NQ * NQ + tx;
                RC a = mul1(BTy[0], w[0]);
#pragma unroll
                for (int q2 = 1; q2 < NQ; ++q2) acc_add(a, BTy[q2] * w[q2 * NQ]);
                b1[(i3 * NI + ty) * NQ + tx] = a;
            }
        }
        __syncwarp();
        if (valid && tx < NI && ty < NI) {                  // q1 -> i1
            RC BTx[NQ];
#pragma unroll
            for (int q = 0; q < NQ; ++q) BTx[q] = Bs[q * NI + tx];
            RV *o_e = ev + (int64_t)c * P.E * NP + e * NP;
#pragma unroll
            for (int i3 = 0; i3 < NI; ++i3) {
                const RC *w = b1 + (i3 * NI + ty) * NQ;
                RC a = mul1(BTx[0], w[0]);
#pragma unroll
                for (int q1 = 1; q1 < NQ; ++q1) acc_add(a, BTx[q1] * w[q1]);
                ev_store(&o_e[(i3 * NI + ty) * NI + tx], a);
            }
        }
        __syncwarp();                                       // b0, b1 are reused by the next component
    }
#undef COLW
}

}  // namespace tmop
