// Energy and gradient kernels: instantiation and launch for every supported
// (dim, order, nq1d) and both contraction arithmetics (FP64 units or
// double-float on the FP32 units).
#include "elem_launch.cuh"
#include "grad3c.cuh"

namespace tmop {

// Tables of the warp-synchronous gradient for one (NI, NQ), built once per process.
template <int NI, int NQ>
static const GradTab<df, NI, NQ> &gradtab()
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

// The warp-synchronous gradient (3D, an element's n_q x n_q columns in one
// warp, double-float); the register budget of 16 resident warps (12 at n_q = 5,
// whose point algebra would spill at 16).
template <class C>
static cudaError_t run_grad3c(const ElemParams &P, const double *x, double *ev, double *part,
                              cudaStream_t s, const BatchArgs &B, int64_t ntiles)
{
    const int64_t nb = B.tiles ? ntiles : grid_of<C>(P.E);
    if (nb == 0) return cudaSuccess;
    constexpr size_t bytes = Grad3cShape<C>::bytes;
    auto kern = k_grad3c<C, (C::NQ >= 5 ? 3 : 4)>;
    cudaError_t e = prepare(kern, bytes);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)nb, C::NT, bytes, s>>>(P, x, ev, part, B, gradtab<C::NI, C::NQ>());
    count_launch();
    return cudaGetLastError();
}

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
    if constexpr (C::D == 3 && C::NQ * C::NQ <= 32 && std::is_same<RS, df>::value) {
        if (P.target != TGT_DISCRETE) return run_grad3c<C>(P, x, ev, part, s, B, ntiles);
    }
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
