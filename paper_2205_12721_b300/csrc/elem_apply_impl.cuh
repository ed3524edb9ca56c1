// Launchers of the Hessian-action kernels (the dominant kernel of the Newton
// step), shared by the per-precision translation units elem_apply_*.cu.
//
// Variant numbers (the autotuner's search space, autotune.cu):
//   0  sum-factorised kernels of apply3.cuh / elem_kernels.cuh (register
//      column, slab column for the 9^3 rule, generic otherwise)
//   1  collocated, register column, 4 warps per CTA     (3D, n_q^2 <= 32)
//   2  collocated, register column, 2 warps per CTA
//   3  collocated, shared-memory column, one copy of the point body, a
//      register budget for 512 (FP32: 768) resident threads, 4 warps per CTA
//   4  as 3, 2 warps per CTA
//   5  as 3, 8 warps per CTA
//   6  collocated, shared-memory column, point body unrolled, compiler's
//      register budget, 4 warps per CTA
//   7  as 5, with an L2 prefetch of the next point's stored values
//   8  as 3, with the same prefetch
//   9  as 7, the stored values taken in register-double-buffered chunks of 9
//  10  as 3, the same chunked stream (no L2 prefetch)
//  11  as 3 with the buffers aliased into dead column rows, a register budget
//      for 20 (FP32: 32) resident warps per SM
//  12  as 11, a register budget for 24 resident warps
//  13  as 12 with 8 warps per CTA and the L2 prefetch
//  14  as 11 with the L2 prefetch
//  15  as 12 with the L2 prefetch
//  16  as 13 without the L2 prefetch
//  17  as 12, the three input components gathered into registers up front
//  18  as 11, the same gather
#pragma once

#include <type_traits>

#include "apply3.cuh"
#include "apply3c.cuh"
#include "elem_launch.cuh"

namespace tmop {

// Tables of the collocated action for one (RC, NI, NQ), built once per process.
template <class RC, int NI, int NQ>
static const ColTab<RC, NI, NQ> &coltab()
{
    static const ColTab<RC, NI, NQ> T = [] {
        ColTab<RC, NI, NQ> t;
        double B[NQ * NI], G[NQ * NI], w[NQ], D[NQ * NQ];
        host_basis_tables(NI, NQ, B, G, w);
        host_colloc_deriv(NQ, D);
        for (int i = 0; i < NQ * NI; ++i) t.B[i] = RC(B[i]);
        for (int i = 0; i < NQ * NQ; ++i) t.D[i] = RC(D[i]);
        return t;
    }();
    return T;
}

// RW: resident warps per SM asked of the register allocator (0: 16 for
// double-float / FP64, 24 for FP32, with rolled shared-memory columns; none
// otherwise).
template <class C, class RV, class RC, int WPB, bool SC, bool ROLL = true, bool PFN = false,
          bool PIPE = false, bool AL = false, int RW = 0, bool GA = false>
static cudaError_t run_apply3c(const ElemParams &P, const RV *v, const RC *H, RV *ev, const int *stop,
                               int k, cudaStream_t s, const BatchArgs &B, int64_t ntiles)
{
    using S = Apply3cShape<C, WPB>;
    constexpr bool F32 = std::is_same<RC, float>::value;
    constexpr int MINB = RW > 0 ? RW / WPB : (SC && ROLL) ? (F32 ? 24 : 16) / WPB : 0;
    const int64_t nb = B.tiles ? (ntiles * C::EPB + S::EPB - 1) / S::EPB
                               : (P.E + S::EPB - 1) / S::EPB;
    if (nb == 0) return cudaSuccess;
    const size_t bytes = S::template bytes<RC>(SC, AL);
    auto kern = k_apply3c<C, RV, RC, WPB, SC, ROLL, MINB, PFN, PIPE, AL, GA>;
    cudaError_t e = prepare(kern, bytes);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)nb, S::NT, bytes, s>>>(P, v, H, ev, stop, k, B, ntiles, coltab<RC, C::NI, C::NQ>());
    count_launch();
    return cudaGetLastError();
}

template <class C, class RV, class RC>
static cudaError_t run_apply_legacy(const ElemParams &P, const RV *v, const RC *H, RV *ev,
                                    const int *stop, int k, cudaStream_t s, const BatchArgs &B,
                                    int64_t ntiles)
{
    const int64_t nb = B.tiles ? ntiles : grid_of<C>(P.E);
    if (nb == 0) return cudaSuccess;
    if constexpr (C::D == 3 && C::NQ <= 4 && std::is_same<RC, float>::value) {
        using L = Apply3Layout<C, RC>;
        cudaError_t e = prepare(k_apply3_occ6<C, RV, RC>, L::bytes);
        if (e != cudaSuccess) return e;
        k_apply3_occ6<C, RV, RC><<<(unsigned)nb, C::NT, L::bytes, s>>>(P, v, H, ev, stop, k, B);
    } else if constexpr (C::D == 3 && C::NQ <= 6) {
        using L = Apply3Layout<C, RC>;
        cudaError_t e = prepare(k_apply3<C, RV, RC>, L::bytes);
        if (e != cudaSuccess) return e;
        k_apply3<C, RV, RC><<<(unsigned)nb, C::NT, L::bytes, s>>>(P, v, H, ev, stop, k, B);
    } else if constexpr (C::D == 3 && !(C::NI == 3 && std::is_same<RC, df>::value)) {
        // many points per direction (9^3): the slab-column kernel.  Measured on
        // the 24^3 Kershaw mesh, ms per action (generic -> slab): FP64 class
        // p=1 1.90 -> 1.05, p=3 3.78 -> 2.59, p=4 4.80 -> 3.36, FP32 p=1..4
        // 0.57/0.54/0.67/0.63 -> 0.31/0.37/0.41/0.58; FP64 class p=2 was
        // slower (2.24 -> 2.48) and keeps the generic kernel.
        using L = Apply3sLayout<C, RC>;
        cudaError_t e = prepare(k_apply3s<C, RV, RC>, L::bytes);
        if (e != cudaSuccess) return e;
        k_apply3s<C, RV, RC><<<(unsigned)nb, C::NT, L::bytes, s>>>(P, v, H, ev, stop, k, B);
    } else {
        using L = Layout<C, RC>;
        cudaError_t e = prepare(k_apply<C, RV, RC>, L::bytes);
        if (e != cudaSuccess) return e;
        k_apply<C, RV, RC><<<(unsigned)nb, C::NT, L::bytes, s>>>(P, v, H, ev, stop, k, B);
    }
    count_launch();
    return cudaGetLastError();
}

template <class C>
constexpr int apply_variant_count()
{
    return (C::D == 3 && C::NQ * C::NQ <= 32) ? 19 : 1;
}

template <class C, class RV, class RC>
static cudaError_t run_apply(const ElemParams &P, const RV *v, const RC *H, RV *ev, const int *stop,
                             int k, cudaStream_t s, const BatchArgs &B, int64_t ntiles, int variant)
{
    if constexpr (apply_variant_count<C>() > 1) {
        constexpr bool F32 = std::is_same<RC, float>::value;
        switch (variant) {
            case 1: return run_apply3c<C, RV, RC, 4, false>(P, v, H, ev, stop, k, s, B, ntiles);
            case 2: return run_apply3c<C, RV, RC, 2, false>(P, v, H, ev, stop, k, s, B, ntiles);
            case 3: return run_apply3c<C, RV, RC, 4, true>(P, v, H, ev, stop, k, s, B, ntiles);
            case 4: return run_apply3c<C, RV, RC, 2, true>(P, v, H, ev, stop, k, s, B, ntiles);
            case 5: return run_apply3c<C, RV, RC, 8, true>(P, v, H, ev, stop, k, s, B, ntiles);
            case 6: return run_apply3c<C, RV, RC, 4, true, false>(P, v, H, ev, stop, k, s, B, ntiles);
            case 7: return run_apply3c<C, RV, RC, 8, true, true, true>(P, v, H, ev, stop, k, s, B, ntiles);
            case 8: return run_apply3c<C, RV, RC, 4, true, true, true>(P, v, H, ev, stop, k, s, B, ntiles);
            case 9: return run_apply3c<C, RV, RC, 8, true, true, true, true>(P, v, H, ev, stop, k, s, B, ntiles);
            case 10: return run_apply3c<C, RV, RC, 4, true, true, false, true>(P, v, H, ev, stop, k, s, B, ntiles);
            case 11: return run_apply3c<C, RV, RC, 4, true, true, false, false, true, F32 ? 32 : 20>(P, v, H, ev, stop, k, s, B, ntiles);
            case 12: return run_apply3c<C, RV, RC, 4, true, true, false, false, true, 24>(P, v, H, ev, stop, k, s, B, ntiles);
            case 13: return run_apply3c<C, RV, RC, 8, true, true, true, false, true, 24>(P, v, H, ev, stop, k, s, B, ntiles);
            case 14: return run_apply3c<C, RV, RC, 4, true, true, true, false, true, F32 ? 32 : 20>(P, v, H, ev, stop, k, s, B, ntiles);
            case 15: return run_apply3c<C, RV, RC, 4, true, true, true, false, true, 24>(P, v, H, ev, stop, k, s, B, ntiles);
            case 16: return run_apply3c<C, RV, RC, 8, true, true, false, false, true, 24>(P, v, H, ev, stop, k, s, B, ntiles);
            case 17: return run_apply3c<C, RV, RC, 4, true, true, false, false, true, 24, true>(P, v, H, ev, stop, k, s, B, ntiles);
            case 18: return run_apply3c<C, RV, RC, 4, true, true, false, false, true, F32 ? 32 : 20, true>(P, v, H, ev, stop, k, s, B, ntiles);
            default: break;
        }
    }
    return run_apply_legacy<C, RV, RC>(P, v, H, ev, stop, k, s, B, ntiles);
}

// Launch over one precision: RV vectors, RC stored data and arithmetic.
template <class RV, class RC>
static cudaError_t launch_apply_typed(int d, int p, int q, const ElemParams &P, const void *v,
                                      const void *H, void *ev, const int *stop, int k,
                                      cudaStream_t s, const BatchArgs *B, int64_t ntiles, int variant)
{
    const BatchArgs b0 = B ? *B : BatchArgs{};
#define CASE(D_, P_, Q_)                                                                          \
    case TMOP_KEY(D_, P_, Q_):                                                                    \
        return run_apply<Cfg<D_, P_, Q_>, RV, RC>(P, static_cast<const RV *>(v),                  \
                                                  static_cast<const RC *>(H), static_cast<RV *>(ev), \
                                                  stop, k, s, b0, ntiles, variant);
    TMOP_SWITCH(d, p, q, CASE)
#undef CASE
}

}  // namespace tmop
