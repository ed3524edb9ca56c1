// Partial-assembly setup kernels: stored d2mu/dT2 data in FP64 (native),
// double-float pairs, or FP32.
#include "elem_launch.cuh"

namespace tmop {

template <class C, class RS, class RH>
static cudaError_t run_hsetup(const ElemParams &P, const double *x, RH *H, cudaStream_t s)
{
    using L = Layout<C, RS>;
    const int64_t nb = grid_of<C>(P.E);
    if (nb == 0) return cudaSuccess;
    cudaError_t e = prepare(k_hsetup<C, RS, RH>, L::bytes);
    if (e != cudaSuccess) return e;
    k_hsetup<C, RS, RH><<<(unsigned)nb, C::NT, L::bytes, s>>>(P, x, H);
    count_launch();
    return cudaGetLastError();
}

template <class C>
static cudaError_t run_hsetup_any(const ElemParams &P, const double *x, void *H, int prec,
                                  cudaStream_t s)
{
    if (prec == TMOP_FP32) return run_hsetup<C, df, float>(P, x, static_cast<float *>(H), s);
    if (prec == TMOP_FP64_NATIVE) return run_hsetup<C, double, double>(P, x, static_cast<double *>(H), s);
    return run_hsetup<C, df, df>(P, x, static_cast<df *>(H), s);
}

cudaError_t launch_hsetup(int d, int p, int q, const ElemParams &P, const double *x, void *H,
                          int prec, cudaStream_t s)
{
#define CASE(D_, P_, Q_) \
    case TMOP_KEY(D_, P_, Q_): return run_hsetup_any<Cfg<D_, P_, Q_>>(P, x, H, prec, s);
    TMOP_SWITCH(d, p, q, CASE)
#undef CASE
}

}  // namespace tmop
