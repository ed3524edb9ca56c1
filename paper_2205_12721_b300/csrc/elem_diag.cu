// Hessian-diagonal kernels (Jacobi preconditioner).
#include "elem_launch.cuh"

namespace tmop {

template <class C, class RV, class RC>
static cudaError_t run_diag(const ElemParams &P, const RC *H, RV *ev, cudaStream_t s,
                            const BatchArgs &B, int64_t ntiles)
{
    using L = Layout<C, RC>;
    const int64_t nb = B.tiles ? ntiles : grid_of<C>(P.E);
    if (nb == 0) return cudaSuccess;
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
