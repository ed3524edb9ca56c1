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
// and walk q3 in registers, so every contraction along q3 (B and D) reads its
// operands from registers and its table entries from the kernel parameter
// space (compile-time indices), while the contractions along q1 and q2 go
// through three small per-element shared buffers.  An element never spans two
// warps: the stages synchronise with __syncwarp, and the CTA-wide barrier is
// used once, for the tables.  Accumulators start from their first product
// (no add to zero) and intermediate values are left unnormalised: a
// double-float value with a low word of a few ulp(h) is a valid operand of the
// error-free products.
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

template <class C>
struct Apply3cShape {
    static constexpr int TPE = C::NQ * C::NQ;                 // one lane per (q1, q2) column
    static_assert(TPE <= 32, "an element must fit in one warp");
    static constexpr int EPW = 32 / TPE;                       // elements per warp
    static constexpr int WPB = 4;                              // warps per CTA
    static constexpr int EPB = EPW * WPB;
    static constexpr int NT = 32 * WPB;
    static constexpr int BUF = C::NQ * C::NQ * C::NQ;          // >= NP, NQ NI^2, NQ^2 NI
    static constexpr int NPL = (C::NP + TPE - 1) / TPE;        // map entries per lane
    static constexpr int TABN = C::NQ * C::NI + C::NQ * C::NQ;
    template <class R>
    static constexpr size_t bytes(bool ga = false, bool sc = false, bool cp = false)
    {
        return sizeof(R) * (size_t)(((TABN + 1) & ~1) + EPB * (3 * BUF + (ga ? 3 * C::NP : 0)) +
                                    (sc ? 9 * C::NQ * NT : 0) + (cp ? C::NS * NT : 0));
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

// Conversions of the gathered input and of the element-vector output.
template <class RC, bool BITS> __device__ __forceinline__ RC cvt_in(double v);
template <> __device__ __forceinline__ df cvt_in<df, false>(double v) { return df(v); }
template <> __device__ __forceinline__ df cvt_in<df, true>(double v) { return df_bits(v); }
template <> __device__ __forceinline__ double cvt_in<double, false>(double v) { return v; }
template <> __device__ __forceinline__ double cvt_in<double, true>(double v) { return v; }
template <class RC, bool BITS> __device__ __forceinline__ RC cvt_in(float v) { return RC(v); }

template <bool BITS> __device__ __forceinline__ double cvt_out(const df &v)
{
    return BITS ? d_bits(v) : (double)v;
}
template <bool BITS> __device__ __forceinline__ double cvt_out(double v) { return v; }
template <bool BITS> __device__ __forceinline__ float cvt_out(float v) { return v; }

// Bulk prefetch of [p, p + bytes) into L2: the 16-byte aligned interior, in
// chunks of at most 16 KB (cp.async.bulk.prefetch.L2).
__device__ __forceinline__ void prefetch_l2(const void *p, size_t bytes)
{
    const uintptr_t a = ((uintptr_t)p + 15) & ~(uintptr_t)15;
    const uintptr_t b = ((uintptr_t)p + bytes) & ~(uintptr_t)15;
    for (uintptr_t q = a; q < b; q += 16384) {
        const unsigned n = (unsigned)((b - q) < 16384 ? (b - q) : 16384);
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(q), "r"(n) : "memory");
    }
}

// PF: 1 = prefetch the element's stored data into L2 at the start, 2 = before
// the last forward component.  GA: gather the three input components at the
// start (one latency instead of three).
// Asynchronous 8-byte copy global -> shared (cp.async, L1-allocating) and its wait.
__device__ __forceinline__ void cp_async8(void *dst, const void *src)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async4(void *dst, const void *src)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;" ::: "memory");
}
template <class RC> __device__ __forceinline__ void cp_async_val(RC *dst, const RC *src)
{
    if constexpr (sizeof(RC) == 8) cp_async8(dst, src);
    else cp_async4(dst, src);
}

// CP: 1 = copy the first q3 plane of the element's stored data to shared memory
// asynchronously at the start of the second forward component, 2 = at the start
// of the kernel; the pointwise product of that plane reads it from there.
template <class C, class RV, class RC, bool BITS, int MINB, int PF = 0, bool GA = false,
          bool SC = false, int CP = 0, bool ROLL = false>
__global__ void __launch_bounds__(Apply3cShape<C>::NT, MINB)
k_apply3c(ElemParams P, const RV *__restrict__ v, const RC *__restrict__ H, RV *__restrict__ ev,
          const int *__restrict__ stop_iter, int k, BatchArgs BA, const ColTab<RC, C::NI, C::NQ> T)
{
    static_assert(C::D == 3, "3D kernel");
    using S = Apply3cShape<C>;
    static_assert(S::EPB == C::EPB, "the element tiles must match the other kernels'");
    constexpr int NI = C::NI, NQ = C::NQ, NP = C::NP, NQD = C::NQD, NS = C::NS, BUF = S::BUF;
    const void *in = v, *aux = H;
    void *out = ev;
    const int *stop = stop_iter;
    const int64_t tile = resolve_tile(P, BA, in, aux, out, stop);
    v = static_cast<const RV *>(in);
    H = static_cast<const RC *>(aux);
    ev = static_cast<RV *>(out);
    if (stop && *stop < k) return;

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

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int slot = lane / S::TPE;
    const bool act = slot < S::EPW;
    const int t = lane - slot * S::TPE;
    const int el = warp * S::EPW + (act ? slot : 0);
    const int tx = t % NQ, ty = t / NQ;
    constexpr int SLOT = 3 * BUF + (GA ? 3 * NP : 0);
    RC *b0 = Bs + ((S::TABN + 1) & ~1) + el * SLOT;
    RC *b1 = b0 + BUF;
    RC *b2 = b1 + BUF;
    RC *ug = b2 + BUF;                                      // GA: the three gathered components
    // SC: the dA / Y columns of every thread, [(r * NQ + q3) * NT + thread]
    RC *cs = Bs + ((S::TABN + 1) & ~1) + S::EPB * SLOT;
    const int64_t e = tile * S::EPB + el;
    const bool valid = act && e < P.E;
    // CP: plane q3 = 0 of the stored data, [s * NT + thread]
    RC *hp = cs + (SC ? 9 * NQ * S::NT : 0);
    auto stage_plane0 = [&]() {
        if (valid) {
            const RC *He = H + e * (int64_t)(NS * NQD) + (ty * NQ + tx);
#pragma unroll
            for (int s = 0; s < NS; ++s) cp_async_val(hp + s * S::NT + threadIdx.x, He + s * NQD);
        }
    };
    int m[S::NPL];
#pragma unroll
    for (int j = 0; j < S::NPL; ++j) {
        const int i = t + j * S::TPE;
        m[j] = (valid && i < NP) ? P.map[e * NP + i] : 0;
    }
    if (PF == 1 && valid && t == 0) prefetch_l2(H + e * (int64_t)(NS * NQD), sizeof(RC) * NS * NQD);
    if (CP == 2) stage_plane0();
    if (GA) {
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int j = 0; j < S::NPL; ++j) {
                const int i = t + j * S::TPE;
                if (valid && i < NP) ug[c * NP + i] = cvt_in<RC, BITS>(v[c * P.Nx + m[j]]);
            }
    }
    __syncthreads();                                        // tables

    RC col[SC ? 1 : 9][NQ];                                 // dA_{cb} then Y_{cb} at (tx, ty, q3)
#define COLW(r, q3) (SC ? cs[((r) * NQ + (q3)) * S::NT + threadIdx.x] : col[SC ? 0 : (r)][q3])

    // ---- forward: values at the points, then the collocated derivative
#pragma unroll 1
    for (int c = 0; c < 3; ++c) {
        if (PF == 2 && c == 2 && valid && t == 0)
            prefetch_l2(H + e * (int64_t)(NS * NQD), sizeof(RC) * NS * NQD);
        if (CP == 1 && c == 1) stage_plane0();
        if (!GA) {
#pragma unroll
            for (int j = 0; j < S::NPL; ++j) {
                const int i = t + j * S::TPE;
                if (valid && i < NP) b0[i] = cvt_in<RC, BITS>(v[c * P.Nx + m[j]]);
            }
        }
        __syncwarp();
        const RC *ub = GA ? ug + c * NP : b0;
        if (valid && ty < NI) {                             // i1 -> q1
            RC Bx[NI];
#pragma unroll
            for (int i = 0; i < NI; ++i) Bx[i] = Bs[tx * NI + i];
#pragma unroll
            for (int i3 = 0; i3 < NI; ++i3) {
                const RC *u = ub + (i3 * NI + ty) * NI;
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
            if (SC) {
#pragma unroll
                for (int q3 = 0; q3 < NQ; ++q3) {
                    cs[((c * 3 + 0) * NQ + q3) * S::NT + threadIdx.x] = g0[q3];
                    cs[((c * 3 + 1) * NQ + q3) * S::NT + threadIdx.x] = g1[q3];
                    cs[((c * 3 + 2) * NQ + q3) * S::NT + threadIdx.x] = g2[q3];
                }
            } else {
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

    // ---- pointwise: Y = H : dA with the symmetric-packed stored data
    if (CP) cp_async_wait_all();
    if (valid) {
        const RC *He = H + e * (int64_t)(NS * NQD) + (ty * NQ + tx);
        // ROLL (columns in shared memory only): one copy of the point body
#pragma unroll (SC && ROLL ? 1 : NQ)
        for (int q3 = 0; q3 < NQ; ++q3) {
            const RC *Hq = He + q3 * NQ * NQ;
            // the (r, s) stored value of this point: staged plane or global memory
            auto hval = [&](int r, int s) -> RC {
                if (CP && q3 == 0) return hp[pidx<9>(r, s) * S::NT + threadIdx.x];
                return ld_stream(Hq + pidx<9>(r, s) * NQD);
            };
            RC d[9], y[9];
#pragma unroll
            for (int r = 0; r < 9; ++r) d[r] = COLW(r, q3);
#pragma unroll
            for (int s = 0; s < 9; ++s) {                   // row r = 0 starts every sum
                const RC h = hval(0, s);
                y[s] = mul1(h, d[0]);
                if (s > 0) acc_add(y[0], h * d[s]);
            }
#pragma unroll
            for (int r = 1; r < 9; ++r)
#pragma unroll
                for (int s = r; s < 9; ++s) {
                    const RC h = hval(r, s);
                    acc_add(y[s], h * d[r]);
                    if (s != r) acc_add(y[r], h * d[s]);
                }
#pragma unroll
            for (int r = 0; r < 9; ++r) COLW(r, q3) = y[r];
        }
    }

    // ---- transposed: D^T along each direction, then B^T along q3, q2, q1
#pragma unroll 1
    for (int c = 0; c < 3; ++c) {
        RC Y0[NQ], Y1[NQ], Y2[NQ];
        if (SC) {
#pragma unroll
            for (int q3 = 0; q3 < NQ; ++q3) {
                Y0[q3] = cs[((c * 3 + 0) * NQ + q3) * S::NT + threadIdx.x];
                Y1[q3] = cs[((c * 3 + 1) * NQ + q3) * S::NT + threadIdx.x];
                Y2[q3] = cs[((c * 3 + 2) * NQ + q3) * S::NT + threadIdx.x];
            }
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
                b2[(i3 * NQ + ty) * NQ + tx] = a;
            }
        }
        __syncwarp();
        if (valid && ty < NI) {                             // q2 -> i2
            RC BTy[NQ];
#pragma unroll
            for (int q = 0; q < NQ; ++q) BTy[q] = Bs[q * NI + ty];
#pragma unroll
            for (int i3 = 0; i3 < NI; ++i3) {
                const RC *w = b2 + i3 * NQ * NQ + tx;
                RC a = mul1(BTy[0], w[0]);
#pragma unroll
                for (int q2 = 1; q2 < NQ; ++q2) acc_add(a, BTy[q2] * w[q2 * NQ]);
                b0[(i3 * NI + ty) * NQ + tx] = a;
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
                const RC *w = b0 + (i3 * NI + ty) * NQ;
                RC a = mul1(BTx[0], w[0]);
#pragma unroll
                for (int q1 = 1; q1 < NQ; ++q1) acc_add(a, BTx[q1] * w[q1]);
                o_e[(i3 * NI + ty) * NI + tx] = RV(cvt_out<BITS>(a));
            }
        }
        __syncwarp();                                       // b0, b1 are reused by the next component
    }
#undef COLW
}

}  // namespace tmop
