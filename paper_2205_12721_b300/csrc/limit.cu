// Limiting term of the TMOP objective (paper eq. F_full, second term, and
// Sec. 3.5): xi(x - x0, delta) = |x - x0|^2 / delta^2 integrated over the
// target elements.  Its gradient is c_q 2/delta^2 (x - x0)(chi_q) w_i(chi_q)
// and its Hessian the mass-like operator c_q 2/delta^2 w_i w_j delta_ab
// (eq. pa_limiting), applied with value contractions (B (x) B (x) B and its
// transpose) and a stored scalar per quadrature point.  The kernels add
// their element contributions to the element vectors of the main kernels
// (same element, same owner: no race) before the transposed-map assembly.
#include "elem_launch.cuh"

namespace tmop {

namespace {

// Energy partials (2 per CTA: sum, +inf) and, if ev != nullptr, the gradient
// added into the element vector.  c_q = w_q det W(x_q).
template <class C, class RS>
__global__ void __launch_bounds__(C::NT)
k_limit_eg(ElemParams P, const double *__restrict__ x, const double *__restrict__ x0, double lim2,
           double *__restrict__ part, double *__restrict__ ev)
{
    extern __shared__ __align__(16) unsigned char smem[];
    ElemCtx<C, RS> c;
    prologue<C, RS>(P, blockIdx.x, smem, c);
    // d_a(q) = (x - x0)_a(q) in sX (D*NQD); x(q) for the size target in sA
    // blocks D..2D-1 (sA holds DD >= 2D blocks)
    RS *dq = c.sX;
    RS *xq = c.sA + C::D * C::NQD;   // blocks D..2D-1 of sA; the forward scratch uses 0..D-1
    for (int a = 0; a < C::D; ++a) values_at_points<C, RS, double>(P, c, x, x0, a, dq + a * C::NQD);
    if (P.target == TGT_SIZE)
        for (int a = 0; a < C::D; ++a) values_at_points<C, RS, double>(P, c, x, nullptr, a, xq + a * C::NQD);
    if (P.target == TGT_DISCRETE) values_at_points<C, RS, double>(P, c, P.eta, nullptr, 0, xq);
    __syncthreads();
    double esum = 0.0;
    for_my_points<C>(c.tx, c.ty, c.valid, [&](int q, int q3) {
        double xp[3] = {0, 0, 0};
        if (P.target == TGT_SIZE)
#pragma unroll
            for (int k = 0; k < C::D; ++k) xp[k] = to_db(xq[k * C::NQD + q]);
        double ws = target_scale<C::D>(P.target, P.h0, xp);
        if (P.target == TGT_DISCRETE) ws = discrete_scale<C::D>(P.h0, to_db(xq[q]));
        if (!(ws > 0.0)) {                            // no target: no contribution
#pragma unroll
            for (int a = 0; a < C::D; ++a) dq[a * C::NQD + q] = RS(0.0);
            return;
        }
        double wd = ws;
#pragma unroll
        for (int k = 1; k < C::D; ++k) wd *= ws;
        const double cq = point_weight<C>(c.w, c.tx, c.ty, q3) * wd;
        double r2 = 0.0;
#pragma unroll
        for (int a = 0; a < C::D; ++a) {
            const double da = to_db(dq[a * C::NQD + q]);
            r2 += da * da;
            dq[a * C::NQD + q] = from_db<RS>(cq * lim2 * da);
        }
        esum += 0.5 * cq * lim2 * r2;                 // c |d|^2 / delta^2, lim2 = 2/delta^2
    });
    cta_energy_reduce<C>(esum, INFINITY, part, blockIdx.x);
    if (!ev) return;
    __syncthreads();
    for (int a = 0; a < C::D; ++a) {
        values_transpose<C, RS>(c, dq + a * C::NQD);
        if (c.valid)
            for (int i = c.t; i < C::NP; i += C::TPE)
                ev[(int64_t)a * P.E * C::NP + c.e * C::NP + i] += to_db(c.su[i]);
        __syncthreads();
    }
}

// c_q 2/delta^2 at every point (positions of the Hessian set-up).
template <class C>
__global__ void __launch_bounds__(C::NT)
k_limit_setup(ElemParams P, const double *__restrict__ x, double lim2, double *__restrict__ cq_out)
{
    extern __shared__ __align__(16) unsigned char smem[];
    ElemCtx<C, df> c;
    prologue<C, df>(P, blockIdx.x, smem, c);
    if (P.target == TGT_SIZE)
        for (int a = 0; a < C::D; ++a) values_at_points<C, df, double>(P, c, x, nullptr, a, c.sX + a * C::NQD);
    if (P.target == TGT_DISCRETE) values_at_points<C, df, double>(P, c, P.eta, nullptr, 0, c.sX);
    __syncthreads();
    for_my_points<C>(c.tx, c.ty, c.valid, [&](int q, int q3) {
        double xp[3] = {0, 0, 0};
        if (P.target == TGT_SIZE)
#pragma unroll
            for (int k = 0; k < C::D; ++k) xp[k] = to_db(c.sX[k * C::NQD + q]);
        double ws = target_scale<C::D>(P.target, P.h0, xp);
        if (P.target == TGT_DISCRETE) ws = discrete_scale<C::D>(P.h0, to_db(c.sX[q]));
        if (!(ws > 0.0)) {
            cq_out[c.e * C::NQD + q] = 0.0;
            return;
        }
        double wd = ws;
#pragma unroll
        for (int k = 1; k < C::D; ++k) wd *= ws;
        cq_out[c.e * C::NQD + q] = point_weight<C>(c.w, c.tx, c.ty, q3) * wd * lim2;
    });
}

// ev += mass-like action of the stored c_q 2/delta^2 on v (v zero on fixed DOFs).
template <class C, class RV, class RC>
__global__ void __launch_bounds__(C::NT)
k_limit_apply(ElemParams P, const RV *__restrict__ v, const double *__restrict__ cq,
              RV *__restrict__ ev, const int *__restrict__ stop_iter, int k)
{
    if (stop_iter && *stop_iter < iter_of(stop_iter, k)) return;
    extern __shared__ __align__(16) unsigned char smem[];
    ElemCtx<C, RC> c;
    prologue<C, RC>(P, blockIdx.x, smem, c);
    for (int a = 0; a < C::D; ++a) {
        RC *f = c.sX + a * C::NQD;
        values_at_points<C, RC, RV>(P, c, v, nullptr, a, f);
        __syncthreads();
        for_my_points<C>(c.tx, c.ty, c.valid, [&](int q, int) {
            f[q] = prod(RC(cq[c.e * C::NQD + q]), f[q]);
        });
        __syncthreads();
        values_transpose<C, RC>(c, f);
        if (c.valid)
            for (int i = c.t; i < C::NP; i += C::TPE) {
                ev_accum(&ev[(int64_t)a * P.E * C::NP + c.e * C::NP + i], c.su[i]);
            }
        __syncthreads();
    }
}

// ev_a += sum_q c_q 2/delta^2 w_i(q)^2 for every component a.
template <class C, class RV, class RC>
__global__ void __launch_bounds__(C::NT)
k_limit_diag(ElemParams P, const double *__restrict__ cq, RV *__restrict__ ev)
{
    extern __shared__ __align__(16) unsigned char smem[];
    ElemCtx<C, RC> c;
    prologue<C, RC>(P, blockIdx.x, smem, c);
    __shared__ RC bb[C::NQ * C::NI];
    for (int i = threadIdx.x; i < C::NQ * C::NI; i += C::NT) bb[i] = prod(c.B[i], c.B[i]);
    RC *f = c.sX;
    for_my_points<C>(c.tx, c.ty, c.valid, [&](int q, int) { f[q] = RC(cq[c.e * C::NQD + q]); });
    if (c.valid)
        for (int i = c.t; i < C::NP; i += C::TPE) c.su[i] = RC(0.0);
    __syncthreads();
    if (C::D == 3)
        bwd3_tab<C, RC>(bb, bb, bb, f, c.s1, c.s2, c.su, c.tx, c.ty, c.valid);
    else
        bwd2_tab<C, RC>(bb, bb, f, c.s1, c.su, c.tx, c.ty, c.valid);
    if (c.valid)
        for (int a = 0; a < C::D; ++a)
            for (int i = c.t; i < C::NP; i += C::TPE) {
                RV &o = ev[(int64_t)a * P.E * C::NP + c.e * C::NP + i];
                o = RV(to_d(o) + to_d(c.su[i]));
            }
}

template <class C>
int64_t nblk(const ElemParams &P) { return grid_of<C>(P.E); }

}  // namespace

cudaError_t launch_limit_eg(int d, int p, int q, const ElemParams &P, const double *x,
                            const double *x0, double lim2, double *part, double *ev, int arith,
                            cudaStream_t s)
{
    auto run = [&](auto cfg) -> cudaError_t {
        using C = decltype(cfg);
        const int64_t nb = nblk<C>(P);
        if (nb == 0) return cudaSuccess;
        if (arith == ARITH_NATIVE) {
            cudaError_t e = prepare(k_limit_eg<C, double>, Layout<C, double>::bytes);
            if (e != cudaSuccess) return e;
            k_limit_eg<C, double><<<(unsigned)nb, C::NT, Layout<C, double>::bytes, s>>>(P, x, x0, lim2, part, ev);
        } else {
            cudaError_t e = prepare(k_limit_eg<C, df>, Layout<C, df>::bytes);
            if (e != cudaSuccess) return e;
            k_limit_eg<C, df><<<(unsigned)nb, C::NT, Layout<C, df>::bytes, s>>>(P, x, x0, lim2, part, ev);
        }
        count_launch();
        return cudaGetLastError();
    };
#define CASE(D_, P_, Q_) \
    case TMOP_KEY(D_, P_, Q_): return run(Cfg<D_, P_, Q_>{});
    TMOP_SWITCH(d, p, q, CASE)
#undef CASE
}

cudaError_t launch_limit_setup(int d, int p, int q, const ElemParams &P, const double *x, double lim2,
                               double *cq, cudaStream_t s)
{
    auto run = [&](auto cfg) -> cudaError_t {
        using C = decltype(cfg);
        const int64_t nb = nblk<C>(P);
        if (nb == 0) return cudaSuccess;
        cudaError_t e = prepare(k_limit_setup<C>, Layout<C, df>::bytes);
        if (e != cudaSuccess) return e;
        k_limit_setup<C><<<(unsigned)nb, C::NT, Layout<C, df>::bytes, s>>>(P, x, lim2, cq);
        count_launch();
        return cudaGetLastError();
    };
#define CASE(D_, P_, Q_) \
    case TMOP_KEY(D_, P_, Q_): return run(Cfg<D_, P_, Q_>{});
    TMOP_SWITCH(d, p, q, CASE)
#undef CASE
}

cudaError_t launch_limit_apply(int d, int p, int q, const ElemParams &P, const void *v,
                               const double *cq, void *ev, int prec, const int *stop, int k,
                               cudaStream_t s)
{
    auto run = [&](auto cfg) -> cudaError_t {
        using C = decltype(cfg);
        const int64_t nb = nblk<C>(P);
        if (nb == 0) return cudaSuccess;
        cudaError_t e;
        if (prec == TMOP_FP32) {
            e = prepare(k_limit_apply<C, float, float>, Layout<C, float>::bytes);
            if (e != cudaSuccess) return e;
            k_limit_apply<C, float, float><<<(unsigned)nb, C::NT, Layout<C, float>::bytes, s>>>(
                P, static_cast<const float *>(v), cq, static_cast<float *>(ev), stop, k);
        } else if (prec == TMOP_FP64_NATIVE) {
            e = prepare(k_limit_apply<C, double, double>, Layout<C, double>::bytes);
            if (e != cudaSuccess) return e;
            k_limit_apply<C, double, double><<<(unsigned)nb, C::NT, Layout<C, double>::bytes, s>>>(
                P, static_cast<const double *>(v), cq, static_cast<double *>(ev), stop, k);
        } else {
            e = prepare(k_limit_apply<C, double, df>, Layout<C, df>::bytes);
            if (e != cudaSuccess) return e;
            k_limit_apply<C, double, df><<<(unsigned)nb, C::NT, Layout<C, df>::bytes, s>>>(
                P, static_cast<const double *>(v), cq, static_cast<double *>(ev), stop, k);
        }
        count_launch();
        return cudaGetLastError();
    };
#define CASE(D_, P_, Q_) \
    case TMOP_KEY(D_, P_, Q_): return run(Cfg<D_, P_, Q_>{});
    TMOP_SWITCH(d, p, q, CASE)
#undef CASE
}

cudaError_t launch_limit_diag(int d, int p, int q, const ElemParams &P, const double *cq, void *ev,
                              int prec, cudaStream_t s)
{
    auto run = [&](auto cfg) -> cudaError_t {
        using C = decltype(cfg);
        const int64_t nb = nblk<C>(P);
        if (nb == 0) return cudaSuccess;
        cudaError_t e;
        if (prec == TMOP_FP32) {
            e = prepare(k_limit_diag<C, float, float>, Layout<C, float>::bytes);
            if (e != cudaSuccess) return e;
            k_limit_diag<C, float, float><<<(unsigned)nb, C::NT, Layout<C, float>::bytes, s>>>(
                P, cq, static_cast<float *>(ev));
        } else if (prec == TMOP_FP64_NATIVE) {
            e = prepare(k_limit_diag<C, double, double>, Layout<C, double>::bytes);
            if (e != cudaSuccess) return e;
            k_limit_diag<C, double, double><<<(unsigned)nb, C::NT, Layout<C, double>::bytes, s>>>(
                P, cq, static_cast<double *>(ev));
        } else {
            e = prepare(k_limit_diag<C, double, df>, Layout<C, df>::bytes);
            if (e != cudaSuccess) return e;
            k_limit_diag<C, double, df><<<(unsigned)nb, C::NT, Layout<C, df>::bytes, s>>>(
                P, cq, static_cast<double *>(ev));
        }
        count_launch();
        return cudaGetLastError();
    };
#define CASE(D_, P_, Q_) \
    case TMOP_KEY(D_, P_, Q_): return run(Cfg<D_, P_, Q_>{});
    TMOP_SWITCH(d, p, q, CASE)
#undef CASE
}

}  // namespace tmop
