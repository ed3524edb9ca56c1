// Energy and gradient kernels: instantiation and launch for every supported
// (dim, order, nq1d).
#include "elem_launch.cuh"

namespace tmop {

template <class C>
static cudaError_t run_energy(const ElemParams &P, const double *x, double *part, cudaStream_t s)
{
    using L = Layout<C, double>;
    const int64_t nb = grid_of<C>(P.E);
    if (nb == 0) return cudaSuccess;
    cudaError_t e = prepare(k_energy<C>, L::bytes);
    if (e != cudaSuccess) return e;
    k_energy<C><<<(unsigned)nb, C::NT, L::bytes, s>>>(P, x, part);
    count_launch();
    return cudaGetLastError();
}

template <class C>
static cudaError_t run_gradient(const ElemParams &P, const double *x, double *ev, cudaStream_t s)
{
    using L = Layout<C, double>;
    const int64_t nb = grid_of<C>(P.E);
    if (nb == 0) return cudaSuccess;
    cudaError_t e = prepare(k_gradient<C>, L::bytes);
    if (e != cudaSuccess) return e;
    k_gradient<C><<<(unsigned)nb, C::NT, L::bytes, s>>>(P, x, ev);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_energy(int d, int p, int q, const ElemParams &P, const double *x, double *part,
                          cudaStream_t s)
{
#define CASE(D_, P_, Q_) \
    case TMOP_KEY(D_, P_, Q_): return run_energy<Cfg<D_, P_, Q_>>(P, x, part, s);
    TMOP_SWITCH(d, p, q, CASE)
#undef CASE
}

cudaError_t launch_gradient(int d, int p, int q, const ElemParams &P, const double *x, double *ev,
                            cudaStream_t s)
{
#define CASE(D_, P_, Q_) \
    case TMOP_KEY(D_, P_, Q_): return run_gradient<Cfg<D_, P_, Q_>>(P, x, ev, s);
    TMOP_SWITCH(d, p, q, CASE)
#undef CASE
}

int64_t elem_blocks(int d, int p, int q, int64_t E)
{
    switch (TMOP_KEY(d, p, q)) {
#define CASE(D_, P_, Q_) \
    case TMOP_KEY(D_, P_, Q_): return grid_of<Cfg<D_, P_, Q_>>(E);
        TMOP_CONFIGS(CASE)
#undef CASE
        default: return -1;
    }
}

bool elem_supported(int d, int p, int q) { return elem_blocks(d, p, q, 1) > 0; }

}  // namespace tmop
