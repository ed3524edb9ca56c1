// Hessian-action kernels (the dominant kernel of the Newton step).
#include <type_traits>

#include <cstdlib>

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

// Action kernel variant: 0 = register-column / slab kernels, 1 = collocated
// warp-synchronous kernel, 2 = the same with bit-level double <-> pair
// conversions.  TMOP_APPLY_VARIANT overrides the default for measurements.
static int apply_variant_default()
{
    static const int v = [] {
        const char *s = std::getenv("TMOP_APPLY_VARIANT");
        return s ? std::atoi(s) : -1;
    }();
    return v;
}

template <class C, class RV, class RC>
static cudaError_t run_apply(const ElemParams &P, const RV *v, const RC *H, RV *ev, const int *stop,
                             int k, cudaStream_t s, const BatchArgs &B, int64_t ntiles)
{
    const int64_t nb = B.tiles ? ntiles : grid_of<C>(P.E);
    if (nb == 0) return cudaSuccess;
    if constexpr (C::D == 3 && C::NQ * C::NQ <= 32) {
        int var = apply_variant_default();
        if (var < 0) var = 1;
        if (var >= 1) {
            using S = Apply3cShape<C>;
            const auto &T = coltab<RC, C::NI, C::NQ>();
            auto go = [&](auto kern, bool ga, bool sc = false, bool cp = false) {
                const size_t bytes = S::template bytes<RC>(ga, sc, cp);
                cudaError_t e = prepare(kern, bytes);
                if (e != cudaSuccess) return e;
                kern<<<(unsigned)nb, S::NT, bytes, s>>>(P, v, H, ev, stop, k, B, T);
                count_launch();
                return cudaGetLastError();
            };
            constexpr bool F32 = std::is_same<RC, float>::value;
            switch (var) {
                case 3: return go(k_apply3c<C, RV, RC, false, F32 ? 6 : 4>, false);
                case 5: return go(k_apply3c<C, RV, RC, false, 0, 1, false>, false);
                case 6: return go(k_apply3c<C, RV, RC, false, 0, 0, true>, true);
                case 7: return go(k_apply3c<C, RV, RC, false, 0, 1, true>, true);
                case 8: return go(k_apply3c<C, RV, RC, false, 0, 2, true>, true);
                case 9: return go(k_apply3c<C, RV, RC, false, 0, 0, false, true>, false, true);
                case 10: return go(k_apply3c<C, RV, RC, false, F32 ? 6 : 4, 0, false, true>, false, true);
                case 11: return go(k_apply3c<C, RV, RC, false, F32 ? 8 : 5, 0, false, true>, false, true);
                case 12: return go(k_apply3c<C, RV, RC, false, 0, 0, false, false, 1>, false, false, true);
                case 13: return go(k_apply3c<C, RV, RC, false, 0, 0, false, false, 2>, false, false, true);
                case 14: return go(k_apply3c<C, RV, RC, false, 0, 0, false, true, 1>, false, true, true);
                case 15: return go(k_apply3c<C, RV, RC, false, 0, 0, false, true, 0, true>, false, true);
                case 16: return go(k_apply3c<C, RV, RC, false, F32 ? 6 : 4, 0, false, true, 0, true>, false, true);
                default: return go(k_apply3c<C, RV, RC, false, 0>, false);
            }
        }
    }
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
static cudaError_t run_apply_any(const ElemParams &P, const void *v, const void *H, void *ev,
                                 int prec, const int *stop, int k, cudaStream_t s,
                                 const BatchArgs &B, int64_t nt)
{
    if (prec == TMOP_FP32)
        return run_apply<C, float, float>(P, static_cast<const float *>(v), static_cast<const float *>(H),
                                          static_cast<float *>(ev), stop, k, s, B, nt);
    if (prec == TMOP_FP64_NATIVE)
        return run_apply<C, double, double>(P, static_cast<const double *>(v),
                                            static_cast<const double *>(H), static_cast<double *>(ev),
                                            stop, k, s, B, nt);
    return run_apply<C, double, df>(P, static_cast<const double *>(v), static_cast<const df *>(H),
                                    static_cast<double *>(ev), stop, k, s, B, nt);
}

cudaError_t launch_apply(int d, int p, int q, const ElemParams &P, const void *v, const void *H,
                         void *ev, int prec, const int *stop_iter, int k, cudaStream_t s,
                         const BatchArgs *B, int64_t ntiles)
{
    const BatchArgs b0 = B ? *B : BatchArgs{};
#define CASE(D_, P_, Q_) \
    case TMOP_KEY(D_, P_, Q_): \
        return run_apply_any<Cfg<D_, P_, Q_>>(P, v, H, ev, prec, stop_iter, k, s, b0, ntiles);
    TMOP_SWITCH(d, p, q, CASE)
#undef CASE
}

}  // namespace tmop
