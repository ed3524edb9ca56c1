// Partial-assembly setup kernels: stored d2mu/dT2 data in FP64 (native),
// double-float pairs, or FP32.
#include "elem_launch.cuh"

namespace tmop {

template <class C, class RS, class RH, bool I2>
static cudaError_t run_hsetup_m(const ElemParams &P, const double *x, RH *H, cudaStream_t s,
                                const BatchArgs &B, int64_t ntiles)
{
    using L = Layout<C, RS>;
    const int64_t nb = B.tiles ? ntiles : grid_of<C>(P.E);
    if (nb == 0) return cudaSuccess;
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
