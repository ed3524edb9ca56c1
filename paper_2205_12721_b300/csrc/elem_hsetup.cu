// Partial-assembly setup kernels: stored d2mu/dT2 data in FP64 (native),
// double-float pairs, or FP32.
#include "elem_launch.cuh"
#include "grad3c.cuh"

namespace tmop {

// Tables of the warp-synchronous set-up for one (NI, NQ), built once per process.
template <int NI, int NQ>
static const GradTab<df, NI, NQ> &hsettab()
{
    static const GradTab<df, NI, NQ> T = [] {
        GradTab<df, NI, NQ> t;
        double B[NQ * NI], G[NQ * NI], w[NQ];
        host_basis_tables(NI, NQ, B, G, w);
        for (int i = 0; i < NQ * NI; ++i) t.B[i] = df(B[i]);
        for (int i = 0; i < NQ * NI; ++i) t.G[i] = df(G[i]);
        for (int i = 0; i < NQ; ++i) t.w[i] = df(w[i]);
        return t;
    }();
    return T;
}

template <class C, class RS, class RH, bool I2>
static cudaError_t run_hsetup_m(const ElemParams &P, const double *x, RH *H, cudaStream_t s,
                                const BatchArgs &B, int64_t ntiles)
{
    const int64_t nb = B.tiles ? ntiles : grid_of<C>(P.E);
    if (nb == 0) return cudaSuccess;
    if constexpr (C::D == 3 && C::NQ * C::NQ <= 32 && std::is_same<RS, df>::value) {
        // the warp-synchronous kernel (the discrete target keeps the block one)
        if (P.target != TGT_DISCRETE) {
            constexpr size_t bytes = Grad3cShape<C>::bytes;
            // register budget: 16 resident warps (12 at n_q = 5); the I2 metrics'
            // point algebra takes the compiler's budget (it would spill)
            auto kern = k_hset3c<C, RH, I2, (I2 ? 1 : (C::NQ >= 5 ? 3 : 4))>;
            cudaError_t e = prepare(kern, bytes);
            if (e != cudaSuccess) return e;
            kern<<<(unsigned)nb, C::NT, bytes, s>>>(P, x, H, B, hsettab<C::NI, C::NQ>());
            count_launch();
            return cudaGetLastError();
        }
    }
    using L = Layout<C, RS>;
    cudaError_t e = prepare(k_hsetup<C, RS, RH, I2>, L::bytes);
    if (e != cudaSuccess) return e;
    k_hsetup<C, RS, RH, I2><<<(unsigned)nb, C::NT, L::bytes, s>>>(P, x, H, B);
    count_launch();
    return cudaGetLastError();
}

// P.metric selects the kernel family (the batch passes its metric here too)
template <class C, class RS, class RH>
static cudaError_t run_hsetup(const ElemParams &P, const double *x, RH *H, cudaStream_t s,
                              const BatchArgs &B, int64_t ntiles)
{
    if (metric_uses_I2(P.metric, C::D)) return run_hsetup_m<C, RS, RH, true>(P, x, H, s, B, ntiles);
    return run_hsetup_m<C, RS, RH, false>(P, x, H, s, B, ntiles);
}

template <class C>
static cudaError_t run_hsetup_any(const ElemParams &P, const double *x, void *H, int prec,
                                  cudaStream_t s, const BatchArgs &B, int64_t nt)
{
    if (prec == TMOP_FP32) return run_hsetup<C, df, float>(P, x, static_cast<float *>(H), s, B, nt);
    if (prec == TMOP_FP64_NATIVE)
        return run_hsetup<C, double, double>(P, x, static_cast<double *>(H), s, B, nt);
    return run_hsetup<C, df, df>(P, x, static_cast<df *>(H), s, B, nt);
}

cudaError_t launch_hsetup(int d, int p, int q, const ElemParams &P, const double *x, void *H,
                          int prec, cudaStream_t s, const BatchArgs *B, int64_t ntiles)
{
    const BatchArgs b0 = B ? *B : BatchArgs{};
#define CASE(D_, P_, Q_) \
    case TMOP_KEY(D_, P_, Q_): return run_hsetup_any<Cfg<D_, P_, Q_>>(P, x, H, prec, s, b0, ntiles);
    TMOP_SWITCH(d, p, q, CASE)
#undef CASE
}

}  // namespace tmop
