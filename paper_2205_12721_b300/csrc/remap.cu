// Advection remap of the discrete target field (paper Sec. 3.6): the
// partially assembled mass and advection operators of the pseudo-time
// problem  M(x_t) d eta/dt = K(x_t) eta,  x_t = x0 + t v,  v = x1 - x0.
//
//   k_remap_setup  Jacobian of x_t and v at the points; stores
//                  dm = w_q det A_q and dadv_b = w_q (adj(A_q) v_q)_b, since
//                  det A v . A^-T grad_xbar u = (adj(A) v) . grad_xbar u;
//                  per-CTA min det A for the inversion check
//   k_mass_apply   (M u)_e = B^T (dm * B u_e)  (B (x) B (x) B contractions,
//                  compact layout of its own)
//   k_mass_diag    sum_q dm w_i(chi_q)^2 through squared 1D tables
//   k_adv_apply    (K u)_e = B^T (dadv . G u_e)
// Element vectors (one component) are assembled by the transposed-map kernel.
// The Jacobi-CG and RK4 vector kernels are in vec_kernels.cu, the sequencing
// in capi.cu.
#include "elem_launch.cuh"

namespace tmop {

namespace {

template <class C, class R>
__global__ void __launch_bounds__(C::NT)
k_remap_setup(ElemParams P, const double *__restrict__ x0, const double *__restrict__ vel, double t,
              double *__restrict__ dm, double *__restrict__ dadv, double *__restrict__ part)
{
    extern __shared__ __align__(16) unsigned char smem[];
    ElemCtx<C, R> c;
    prologue<C, R>(P, blockIdx.x, smem, c);
    // velocity at the points (sA rows 0..D-1 are scratch here)
    for (int a = 0; a < C::D; ++a) values_at_points<C, R, double>(P, c, vel, nullptr, a, c.sX + a * C::NQD);
    // Jacobian rows of x_t = x0 + t vel
    for (int a = 0; a < C::D; ++a) {
        if (c.valid)
            for (int i = c.t; i < C::NP; i += C::TPE) {
                const int64_t j = a * P.Nx + c.smap[i];
                c.su[i] = R(x0[j] + t * vel[j]);
            }
        __syncthreads();
        R *A0 = c.sA + (a * C::D) * C::NQD;
        if (C::D == 3)
            fwd3<C, R>(c.B, c.G, c.su, c.s1, c.s2, A0, A0 + C::NQD, A0 + 2 * C::NQD, nullptr, c.tx,
                       c.ty, c.valid);
        else
            fwd2<C, R>(c.B, c.G, c.su, c.s1, A0, A0 + C::NQD, nullptr, c.tx, c.ty, c.valid);
    }
    double emin = INFINITY;
    for_my_points<C>(c.tx, c.ty, c.valid, [&](int q, int q3) {
        double A[C::DD], Cf[C::DD];
#pragma unroll
        for (int r = 0; r < C::DD; ++r) A[r] = to_db(c.sA[r * C::NQD + q]);
        cofactor<C::D>(A, Cf);                     // adj(A) = cof(A)^T
        double det = 0.0;
#pragma unroll
        for (int b = 0; b < C::D; ++b) det += A[b] * Cf[b];
        emin = fmin(emin, det);
        const double w = point_weight<C>(c.w, c.tx, c.ty, q3);
        dm[c.e * C::NQD + q] = w * det;
#pragma unroll
        for (int b = 0; b < C::D; ++b) {
            double u = 0.0;
#pragma unroll
            for (int a = 0; a < C::D; ++a) u += Cf[a * C::D + b] * to_db(c.sX[a * C::NQD + q]);
            dadv[((int64_t)b * P.E + c.e) * C::NQD + q] = w * u;
        }
    });
    cta_energy_reduce<C>(0.0, emin, part, blockIdx.x);
}

// ev = element vectors of M u; skipped when *stop < kk (CG iterations after
// convergence).  The mass action is the inner loop of the remap CG and has
// little arithmetic per element, so it runs with its own compact shared
// layout (nodal values and two contraction buffers per element, no
// Jacobian or geometry storage) for a high occupancy, values-only
// contractions, and in 3D the q3 column kept in registers through the last
// forward contraction, the dm scaling and the first transposed one.
template <class C>
struct MassLayout {
    static constexpr int NI = C::NI, NQ = C::NQ;
    static constexpr int SU = C::D == 3 ? NI * NI * NI : NI * NI;
    static constexpr int S1 = C::D == 3 ? NI * NI * NQ : NI * NQ;
    static constexpr int S2 = C::D == 3 ? NI * NQ * NQ : NQ * NQ;
};

template <class C, class R>
__global__ void __launch_bounds__(C::NT)
k_mass_apply(ElemParams P, const double *__restrict__ u, const double *__restrict__ dm,
             double *__restrict__ ev, const int *__restrict__ stop, int kk)
{
    if (stop && *stop < kk) return;
    constexpr int NI = C::NI, NQ = C::NQ;
    using L = MassLayout<C>;
    __shared__ R sB[NQ * NI];
    __shared__ R su_all[C::EPB][L::SU];
    __shared__ R s1_all[C::EPB][L::S1];
    __shared__ R s2_all[C::EPB][L::S2];
    const R *__restrict__ tab = table_of<R>(P);
    for (int i = threadIdx.x; i < NQ * NI; i += C::NT) sB[i] = tab[i];
    const int slot = threadIdx.x / C::TPE;
    const bool act = slot < C::EPB;
    const int sl = act ? slot : 0;
    const int t = threadIdx.x - slot * C::TPE, tx = t % C::MX, ty = t / C::MX;
    const int64_t e = (int64_t)blockIdx.x * C::EPB + sl;
    const bool valid = act && e < P.E;
    R *su = su_all[sl], *s1 = s1_all[sl], *s2 = s2_all[sl];
    // conversions on the integer/FP32 pipes (the FP64 pipe would bound this kernel)
    if (valid)
        for (int i = t; i < C::NP; i += C::TPE) su[i] = from_db<R>(u[P.map[e * C::NP + i]]);
    __syncthreads();
    const double *__restrict__ dme = dm + e * C::NQD;
    if (C::D == 3) {
        if (valid && tx < NQ && ty < NI)                       // i1 -> q1
#pragma unroll
            for (int i3 = 0; i3 < NI; ++i3) {
                R a = R(0.0);
#pragma unroll
                for (int i1 = 0; i1 < NI; ++i1) acc_add(a, sB[tx * NI + i1] * su[(i3 * NI + ty) * NI + i1]);
                s1[(i3 * NI + ty) * NQ + tx] = norm(a);
            }
        __syncthreads();
        if (valid && tx < NQ && ty < NQ)                       // i2 -> q2
#pragma unroll
            for (int i3 = 0; i3 < NI; ++i3) {
                R a = R(0.0);
#pragma unroll
                for (int i2 = 0; i2 < NI; ++i2) acc_add(a, sB[ty * NI + i2] * s1[(i3 * NI + i2) * NQ + tx]);
                s2[(i3 * NQ + ty) * NQ + tx] = norm(a);
            }
        __syncthreads();
        if (valid && tx < NQ && ty < NQ) {                     // i3 -> q3, * dm, q3 -> i3
            R col[NI], acc[NI];
#pragma unroll
            for (int i3 = 0; i3 < NI; ++i3) {
                col[i3] = s2[(i3 * NQ + ty) * NQ + tx];
                acc[i3] = R(0.0);
            }
#pragma unroll
            for (int q3 = 0; q3 < NQ; ++q3) {
                R f = R(0.0);
#pragma unroll
                for (int i3 = 0; i3 < NI; ++i3) acc_add(f, sB[q3 * NI + i3] * col[i3]);
                f = prod(from_db<R>(dme[(q3 * NQ + ty) * NQ + tx]), norm(f));
#pragma unroll
                for (int i3 = 0; i3 < NI; ++i3) acc_add(acc[i3], sB[q3 * NI + i3] * f);
            }
#pragma unroll
            for (int i3 = 0; i3 < NI; ++i3) s2[(i3 * NQ + ty) * NQ + tx] = norm(acc[i3]);
        }
        __syncthreads();
        if (valid && tx < NQ && ty < NI)                       // q2 -> i2
#pragma unroll
            for (int i3 = 0; i3 < NI; ++i3) {
                R a = R(0.0);
#pragma unroll
                for (int q2 = 0; q2 < NQ; ++q2) acc_add(a, sB[q2 * NI + ty] * s2[(i3 * NQ + q2) * NQ + tx]);
                s1[(i3 * NI + ty) * NQ + tx] = norm(a);
            }
        __syncthreads();
        if (valid && tx < NI && ty < NI)                       // q1 -> i1
#pragma unroll
            for (int i3 = 0; i3 < NI; ++i3) {
                R a = R(0.0);
#pragma unroll
                for (int q1 = 0; q1 < NQ; ++q1) acc_add(a, sB[q1 * NI + tx] * s1[(i3 * NI + ty) * NQ + q1]);
                ev[e * C::NP + (i3 * NI + ty) * NI + tx] = to_db(norm(a));
            }
    } else {
        if (valid && tx < NQ && ty < NI) {                     // i1 -> q1
            R a = R(0.0);
#pragma unroll
            for (int i1 = 0; i1 < NI; ++i1) acc_add(a, sB[tx * NI + i1] * su[ty * NI + i1]);
            s1[ty * NQ + tx] = norm(a);
        }
        __syncthreads();
        if (valid && tx < NQ && ty < NQ) {                     // i2 -> q2, * dm
            R a = R(0.0);
#pragma unroll
            for (int i2 = 0; i2 < NI; ++i2) acc_add(a, sB[ty * NI + i2] * s1[i2 * NQ + tx]);
            s2[ty * NQ + tx] = prod(from_db<R>(dme[ty * NQ + tx]), norm(a));
        }
        __syncthreads();
        if (valid && tx < NQ && ty < NI) {                     // q2 -> i2
            R a = R(0.0);
#pragma unroll
            for (int q2 = 0; q2 < NQ; ++q2) acc_add(a, sB[q2 * NI + ty] * s2[q2 * NQ + tx]);
            s1[ty * NQ + tx] = norm(a);
        }
        __syncthreads();
        if (valid && tx < NI && ty < NI) {                     // q1 -> i1
            R a = R(0.0);
#pragma unroll
            for (int q1 = 0; q1 < NQ; ++q1) acc_add(a, sB[q1 * NI + tx] * s1[ty * NQ + q1]);
            ev[e * C::NP + ty * NI + tx] = to_db(norm(a));
        }
    }
}

template <class C, class R>
__global__ void __launch_bounds__(C::NT)
k_mass_diag(ElemParams P, const double *__restrict__ dm, double *__restrict__ ev)
{
    extern __shared__ __align__(16) unsigned char smem[];
    ElemCtx<C, R> c;
    prologue<C, R>(P, blockIdx.x, smem, c);
    __shared__ R bb[C::NQ * C::NI];
    for (int i = threadIdx.x; i < C::NQ * C::NI; i += C::NT) bb[i] = prod(c.B[i], c.B[i]);
    R *f = c.sX;
    for_my_points<C>(c.tx, c.ty, c.valid, [&](int q, int) { f[q] = R(dm[c.e * C::NQD + q]); });
    if (c.valid)
        for (int i = c.t; i < C::NP; i += C::TPE) c.su[i] = R(0.0);
    __syncthreads();
    if (C::D == 3)
        bwd3_tab<C, R>(bb, bb, bb, f, c.s1, c.s2, c.su, c.tx, c.ty, c.valid);
    else
        bwd2_tab<C, R>(bb, bb, f, c.s1, c.su, c.tx, c.ty, c.valid);
    if (c.valid)
        for (int i = c.t; i < C::NP; i += C::TPE) ev[c.e * C::NP + i] = to_d(c.su[i]);
}

template <class C, class R>
__global__ void __launch_bounds__(C::NT)
k_adv_apply(ElemParams P, const double *__restrict__ u, const double *__restrict__ dadv,
            double *__restrict__ ev)
{
    extern __shared__ __align__(16) unsigned char smem[];
    ElemCtx<C, R> c;
    prologue<C, R>(P, blockIdx.x, smem, c);
    // reference gradient of u into sA rows 0..D-1
    if (c.valid)
        for (int i = c.t; i < C::NP; i += C::TPE) c.su[i] = R(u[c.smap[i]]);
    __syncthreads();
    if (C::D == 3)
        fwd3<C, R>(c.B, c.G, c.su, c.s1, c.s2, c.sA, c.sA + C::NQD, c.sA + 2 * C::NQD, nullptr, c.tx,
                   c.ty, c.valid);
    else
        fwd2<C, R>(c.B, c.G, c.su, c.s1, c.sA, c.sA + C::NQD, nullptr, c.tx, c.ty, c.valid);
    R *f = c.sX;
    for_my_points<C>(c.tx, c.ty, c.valid, [&](int q, int) {
        double s = 0.0;
#pragma unroll
        for (int b = 0; b < C::D; ++b)
            s += dadv[((int64_t)b * P.E + c.e) * C::NQD + q] * to_db(c.sA[b * C::NQD + q]);
        f[q] = from_db<R>(s);
    });
    values_transpose<C, R>(c, f);
    if (c.valid)
        for (int i = c.t; i < C::NP; i += C::TPE) ev[c.e * C::NP + i] = to_d(c.su[i]);
}

template <class C>
int64_t nblk(const ElemParams &P) { return grid_of<C>(P.E); }

// Launch kernel template K<C, R> with R = df (ARITH_DW) or double (ARITH_NATIVE).
#define TMOP_REMAP_LAUNCH(KERNEL, ...)                                                        \
    auto run = [&](auto cfg) -> cudaError_t {                                                 \
        using C = decltype(cfg);                                                              \
        const int64_t nb = nblk<C>(P);                                                        \
        if (nb == 0) return cudaSuccess;                                                      \
        cudaError_t e;                                                                        \
        if (arith == ARITH_NATIVE) {                                                          \
            e = prepare(KERNEL<C, double>, Layout<C, double>::bytes);                         \
            if (e != cudaSuccess) return e;                                                   \
            KERNEL<C, double><<<(unsigned)nb, C::NT, Layout<C, double>::bytes, s>>>(__VA_ARGS__); \
        } else {                                                                              \
            e = prepare(KERNEL<C, df>, Layout<C, df>::bytes);                                 \
            if (e != cudaSuccess) return e;                                                   \
            KERNEL<C, df><<<(unsigned)nb, C::NT, Layout<C, df>::bytes, s>>>(__VA_ARGS__);     \
        }                                                                                     \
        count_launch();                                                                       \
        return cudaGetLastError();                                                            \
    };

#define CASE(D_, P_, Q_) \
    case TMOP_KEY(D_, P_, Q_): return run(Cfg<D_, P_, Q_>{});

}  // namespace

cudaError_t launch_remap_setup(int d, int p, int q, const ElemParams &P, const double *x0,
                               const double *vel, double t, double *dm, double *dadv, double *part,
                               int arith, cudaStream_t s)
{
    TMOP_REMAP_LAUNCH(k_remap_setup, P, x0, vel, t, dm, dadv, part)
    TMOP_SWITCH(d, p, q, CASE)
}

cudaError_t launch_mass_apply(int d, int p, int q, const ElemParams &P, const double *u,
                              const double *dm, double *ev, const int *stop, int kk, int arith,
                              cudaStream_t s)
{
    auto run = [&](auto cfg) -> cudaError_t {
        using C = decltype(cfg);
        const int64_t nb = nblk<C>(P);
        if (nb == 0) return cudaSuccess;
        if (arith == ARITH_NATIVE)
            k_mass_apply<C, double><<<(unsigned)nb, C::NT, 0, s>>>(P, u, dm, ev, stop, kk);
        else
            k_mass_apply<C, df><<<(unsigned)nb, C::NT, 0, s>>>(P, u, dm, ev, stop, kk);
        count_launch();
        return cudaGetLastError();
    };
    TMOP_SWITCH(d, p, q, CASE)
}

cudaError_t launch_mass_diag(int d, int p, int q, const ElemParams &P, const double *dm, double *ev,
                             int arith, cudaStream_t s)
{
    TMOP_REMAP_LAUNCH(k_mass_diag, P, dm, ev)
    TMOP_SWITCH(d, p, q, CASE)
}

cudaError_t launch_adv_apply(int d, int p, int q, const ElemParams &P, const double *u,
                             const double *dadv, double *ev, int arith, cudaStream_t s)
{
    TMOP_REMAP_LAUNCH(k_adv_apply, P, u, dadv, ev)
    TMOP_SWITCH(d, p, q, CASE)
}

#undef CASE
#undef TMOP_REMAP_LAUNCH

}  // namespace tmop
