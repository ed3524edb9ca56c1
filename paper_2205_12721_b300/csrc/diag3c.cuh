// 3D Hessian diagonal, one element per group of lanes of one warp (sm_103a).
//
// diag_{a,i} = sum_q sum_{b,e} H_{ab,ae}(q) d_b w_i(chi_q) d_e w_i(chi_q)
// (paper Sec. 3.4): for each component a the six pairs b <= e (twice the
// off-diagonal ones), each a three-stage contraction of the stored entry with
// elementwise products of the 1D tables (B B, B G, G G per direction).  The
// lanes of an element own its (q1, q2) columns: the q3 -> i3 stage reads the
// lane's own stored values (entry-pair layout) and contracts in registers, the
// q2 -> i2 and q1 -> i1 stages go through per-element shared buffers; stages
// synchronise with __syncwarp.  The CTA is one element tile of four warps.
// Used for FP32 stored data; the double-float diagonal keeps the block kernel
// k_diag (measured faster there).
#pragma once

#include "apply3c.cuh"

namespace tmop {

// Elementwise table products T[t][q * NI + i]: t = 0 B B, 1 B G, 2 G G.
template <class R, int NI, int NQ>
struct DiagTab {
    R T[3][NQ * NI];
};

template <class C>
struct Diag3cShape {
    using S = Apply3cShape<C, 4>;
    static constexpr int GB = 6 * C::NI * C::NQ * C::NQ;    // q3 -> i3 results, 6 pairs
    static constexpr int HB = 6 * C::NI * C::NI * C::NQ;    // q2 -> i2 results
    static constexpr int TAB = (3 * C::NQ * C::NI + 1) & ~1;
    template <class R>
    static constexpr size_t bytes() { return sizeof(R) * (size_t)(TAB + S::EPB * (GB + HB)); }
};

template <class C, class RV, class RC, int MINB>
__global__ void __launch_bounds__(128, MINB)
k_diag3c(ElemParams P, const RC *__restrict__ H, RV *__restrict__ ev, BatchArgs BA,
         const DiagTab<RC, C::NI, C::NQ> T)
{
    static_assert(C::D == 3 && C::PAIRS, "3D, entry-pair layout");
    using S = Apply3cShape<C, 4>;
    using L = Diag3cShape<C>;
    static_assert(S::NT == C::NT && S::EPB == C::EPB, "the CTA is one element tile");
    constexpr int NI = C::NI, NQ = C::NQ, NQD = C::NQD;
    const void *in = nullptr, *aux = H;
    void *out = ev;
    const int *stop = nullptr;
    const int64_t tile = resolve_tile(P, BA, in, aux, out, stop);
    H = static_cast<const RC *>(aux);
    ev = static_cast<RV *>(out);

    extern __shared__ __align__(16) unsigned char smem[];
    RC *Ts = reinterpret_cast<RC *>(smem);                  // Ts[t * NQ * NI + q * NI + i]
    if (threadIdx.x == 0) {                                 // compile-time indices only
#pragma unroll
        for (int t = 0; t < 3; ++t)
#pragma unroll
            for (int i = 0; i < NQ * NI; ++i) Ts[t * NQ * NI + i] = T.T[t][i];
    }
    __syncthreads();

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int slot = lane / S::TPE;
    const bool act = slot < S::EPW;
    const int t = lane - slot * S::TPE;
    const int tx = t % NQ, ty = t / NQ;
    const int el = warp * S::EPW + (act ? slot : 0);
    const int64_t e = tile * C::EPB + el;
    const bool valid = act && e < P.E;
    RC *gb = Ts + L::TAB + el * (L::GB + L::HB);            // [p][(i3 * NQ + q2) * NQ + q1]
    RC *hb = gb + L::GB;                                    // [p][(i3 * NI + i2) * NQ + q1]
    const RC *He = H + e * (int64_t)C::HST;
    const int pt = ty * NQ + tx;
    constexpr int PB[6] = {0, 0, 0, 1, 1, 2}, PE[6] = {0, 1, 2, 1, 2, 2};

    static_for<3>([&](auto A) {
        constexpr int a = decltype(A)::value;
        if (valid) {                                        // q3 -> i3 (registers)
            static_for<6>([&](auto PP) {
                constexpr int p = decltype(PP)::value;
                constexpr int kk = pidx<9>(a * 3 + PB[p], a * 3 + PE[p]);
                constexpr int t3 = (PB[p] == 2) + (PE[p] == 2);
                RC h[NQ];
#pragma unroll
                for (int q3 = 0; q3 < NQ; ++q3) {
                    const int q = q3 * NQ * NQ + pt;        // the stored layout's offsets
                    const RC v = kk < 2 * C::NPR ? He[2 * q + (2 * (kk >> 1) * NQD + (kk & 1))]
                                                 : He[q + 2 * C::NPR * NQD];
                    h[q3] = PB[p] == PE[p] ? v : twice(v);
                }
#pragma unroll
                for (int i3 = 0; i3 < NI; ++i3) {
                    RC z = mul1(T.T[t3][i3], h[0]);
#pragma unroll
                    for (int q3 = 1; q3 < NQ; ++q3) acc_add(z, T.T[t3][q3 * NI + i3] * h[q3]);
                    gb[p * NI * NQ * NQ + (i3 * NQ + ty) * NQ + tx] = norm(z);
                }
            });
        }
        __syncwarp();
        if (valid && ty < NI) {                             // q2 -> i2
            static_for<6>([&](auto PP) {
                constexpr int p = decltype(PP)::value;
                const RC *T2 = Ts + ((PB[p] == 1) + (PE[p] == 1)) * NQ * NI;
#pragma unroll
                for (int i3 = 0; i3 < NI; ++i3) {
                    const RC *w = gb + p * NI * NQ * NQ + i3 * NQ * NQ + tx;
                    RC z = mul1(T2[ty], w[0]);
#pragma unroll
                    for (int q2 = 1; q2 < NQ; ++q2) acc_add(z, T2[q2 * NI + ty] * w[q2 * NQ]);
                    hb[p * NI * NI * NQ + (i3 * NI + ty) * NQ + tx] = norm(z);
                }
            });
        }
        __syncwarp();
        if (valid && tx < NI && ty < NI) {                  // q1 -> i1, the pairs summed
#pragma unroll
            for (int i3 = 0; i3 < NI; ++i3) {
                RC o = RC(0.0);
                static_for<6>([&](auto PP) {
                    constexpr int p = decltype(PP)::value;
                    const RC *T1 = Ts + ((PB[p] == 0) + (PE[p] == 0)) * NQ * NI;
                    const RC *w = hb + p * NI * NI * NQ + (i3 * NI + ty) * NQ;
#pragma unroll
                    for (int q1 = 0; q1 < NQ; ++q1) acc_add(o, T1[q1 * NI + tx] * w[q1]);
                    o = norm(o);
                });
                RV &dst = ev[(int64_t)a * P.E * C::NP + e * C::NP + (i3 * NI + ty) * NI + tx];
                if constexpr (std::is_same<RV, float>::value) dst = o;
                else dst = to_db(o);
            }
        }
        __syncwarp();                                       // the buffers are reused by the next component
    });
}

}  // namespace tmop
