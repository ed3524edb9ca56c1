// Hessian-diagonal kernels (Jacobi preconditioner).
#include "elem_launch.cuh"

namespace tmop {

template <class C, class R>
static cudaError_t run_diag(const ElemParams &P, const R *H, R *ev, cudaStream_t s)
{
    using L = Layout<C, R>;
    const int64_t nb = grid_of<C>(P.E);
    if (nb == 0) return cudaSuccess;
    cudaError_t e = prepare(k_diag<C, R>, L::bytes);
    if (e != cudaSuccess) return e;
    k_diag<C, R><<<(unsigned)nb, C::NT, L::bytes, s>>>(P, H, ev);
    count_launch();
    return cudaGetLastError();
}

template <class C>
static cudaError_t run_diag_any(const ElemParams &P, const void *H, void *ev, int prec,
                                cudaStream_t s)
{
    if (prec == TMOP_FP32)
        return run_diag<C, float>(P, static_cast<const float *>(H), static_cast<float *>(ev), s);
    return run_diag<C, double>(P, static_cast<const double *>(H), static_cast<double *>(ev), s);
}

cudaError_t launch_diag(int d, int p, int q, const ElemParams &P, const void *H, void *ev, int prec,
                        cudaStream_t s)
{
#define CASE(D_, P_, Q_) \
    case TMOP_KEY(D_, P_, Q_): return run_diag_any<Cfg<D_, P_, Q_>>(P, H, ev, prec, s);
    TMOP_SWITCH(d, p, q, CASE)
#undef CASE
}

}  // namespace tmop
