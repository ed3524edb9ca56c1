// Energy and gradient kernels: instantiation and launch for every supported
// (dim, order, nq1d) and both contraction arithmetics (FP64 units or
// double-float on the FP32 units).
#include "elem_launch.cuh"

namespace tmop {

template <class C, class RS>
static cudaError_t run_energy(const ElemParams &P, const double *x, double *part, cudaStream_t s,
                              const BatchArgs &B, int64_t ntiles)
{
    using L = Layout<C, RS>;
    const int64_t nb = B.tiles ? ntiles : grid_of<C>(P.E);
    if (nb == 0) return cudaSuccess;
    cudaError_t e = prepare(k_energy<C, RS>, L::bytes);
    if (e != cudaSuccess) return e;
    k_energy<C, RS><<<(unsigned)nb, C::NT, L::bytes, s>>>(P, x, part, B);
    count_launch();
    return cudaGetLastError();
}

template <class C, class RS>
static cudaError_t run_gradient(const ElemParams &P, const double *x, double *ev, double *part,
                                cudaStream_t s, const BatchArgs &B, int64_t ntiles)
{
    using L = Layout<C, RS>;
    const int64_t nb = B.tiles ? ntiles : grid_of<C>(P.E);
    if (nb == 0) return cudaSuccess;
    cudaError_t e = prepare(k_gradient<C, RS>, L::bytes);
    if (e != cudaSuccess) return e;
    k_gradient<C, RS><<<(unsigned)nb, C::NT, L::bytes, s>>>(P, x, ev, part, B);
    count_launch();
    return cudaGetLastError();
}

template <class C>
static cudaError_t run_energy_any(const ElemParams &P, const double *x, double *part, int arith,
                                  cudaStream_t s, const BatchArgs &B, int64_t nt)
{
    if (arith == ARITH_NATIVE) return run_energy<C, double>(P, x, part, s, B, nt);
    return run_energy<C, df>(P, x, part, s, B, nt);
}

template <class C>
static cudaError_t run_gradient_any(const ElemParams &P, const double *x, double *ev, double *part,
                                    int arith, cudaStream_t s, const BatchArgs &B, int64_t nt)
{
    if (arith == ARITH_NATIVE) return run_gradient<C, double>(P, x, ev, part, s, B, nt);
    return run_gradient<C, df>(P, x, ev, part, s, B, nt);
}

cudaError_t launch_energy(int d, int p, int q, const ElemParams &P, const double *x, double *part,
                          int arith, cudaStream_t s, const BatchArgs *B, int64_t ntiles)
{
    const BatchArgs b0 = B ? *B : BatchArgs{};
#define CASE(D_, P_, Q_) \
    case TMOP_KEY(D_, P_, Q_): return run_energy_any<Cfg<D_, P_, Q_>>(P, x, part, arith, s, b0, ntiles);
    TMOP_SWITCH(d, p, q, CASE)
#undef CASE
}

cudaError_t launch_gradient(int d, int p, int q, const ElemParams &P, const double *x, double *ev,
                            int arith, cudaStream_t s, const BatchArgs *B, int64_t ntiles,
                            double *part)
{
    const BatchArgs b0 = B ? *B : BatchArgs{};
#define CASE(D_, P_, Q_) \
    case TMOP_KEY(D_, P_, Q_): \
        return run_gradient_any<Cfg<D_, P_, Q_>>(P, x, ev, part, arith, s, b0, ntiles);
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
