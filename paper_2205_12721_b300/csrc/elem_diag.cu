// Hessian-diagonal kernels (Jacobi preconditioner).
#include "diag3c.cuh"
#include "elem_launch.cuh"

namespace tmop {

// Table products of the warp-synchronous diagonal for one (RC, NI, NQ), built
// once per process from the FP64 tables.
template <class RC, int NI, int NQ>
static const DiagTab<RC, NI, NQ> &diagtab()
{
    static const DiagTab<RC, NI, NQ> T = [] {
        DiagTab<RC, NI, NQ> t;
        double B[NQ * NI], G[NQ * NI], w[NQ];
        host_basis_tables(NI, NQ, B, G, w);
        for (int i = 0; i < NQ * NI; ++i) {
            t.T[0][i] = RC(B[i] * B[i]);
            t.T[1][i] = RC(B[i] * G[i]);
            t.T[2][i] = RC(G[i] * G[i]);
        }
        return t;
    }();
    return T;
}

template <class C, class RV, class RC>
static cudaError_t run_diag(const ElemParams &P, const RC *H, RV *ev, cudaStream_t s,
                            const BatchArgs &B, int64_t ntiles)
{
    const int64_t nb = B.tiles ? ntiles : grid_of<C>(P.E);
    if (nb == 0) return cudaSuccess;
    if constexpr (C::D == 3 && C::NQ * C::NQ <= 32 && std::is_same<RC, float>::value) {
        // the warp-synchronous kernel for FP32 stored data (48^3 Q3: 0.338 -> 0.244 ms);
        // with double-float data it measured slower than the block kernel (1.11 -> 1.25 ms)
        constexpr size_t bytes = Diag3cShape<C>::template bytes<RC>();
        auto kern = k_diag3c<C, RV, RC, 4>;
        cudaError_t e = prepare(kern, bytes);
        if (e != cudaSuccess) return e;
        kern<<<(unsigned)nb, C::NT, bytes, s>>>(P, H, ev, B, diagtab<RC, C::NI, C::NQ>());
        count_launch();
        return cudaGetLastError();
    }
    using L = Layout<C, RC>;
    cudaError_t e = prepare(k_diag<C, RV, RC>, L::bytes);
    if (e != cudaSuccess) return e;
    k_diag<C, RV, RC><<<(unsigned)nb, C::NT, L::bytes, s>>>(P, H, ev, B);
    count_launch();
    return cudaGetLastError();
}

template <class C>
static cudaError_t run_diag_any(const ElemParams &P, const void *H, void *ev, int prec,
                                cudaStream_t s, const BatchArgs &B, int64_t nt)
{
    if (prec == TMOP_FP32)
        return run_diag<C, float, float>(P, static_cast<const float *>(H), static_cast<float *>(ev), s,
                                         B, nt);
    if (prec == TMOP_FP64_NATIVE)
        return run_diag<C, double, double>(P, static_cast<const double *>(H),
                                           static_cast<double *>(ev), s, B, nt);
    return run_diag<C, double, df>(P, static_cast<const df *>(H), static_cast<double *>(ev), s, B, nt);
}

cudaError_t launch_diag(int d, int p, int q, const ElemParams &P, const void *H, void *ev, int prec,
                        cudaStream_t s, const BatchArgs *B, int64_t ntiles)
{
    const BatchArgs b0 = B ? *B : BatchArgs{};
#define CASE(D_, P_, Q_) \
    case TMOP_KEY(D_, P_, Q_): return run_diag_any<Cfg<D_, P_, Q_>>(P, H, ev, prec, s, b0, ntiles);
    TMOP_SWITCH(d, p, q, CASE)
#undef CASE
}

}  // namespace tmop
