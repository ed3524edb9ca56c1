// Element kernels of the TMOP partial-assembly path (sm_103a).
//
//   k_energy    Jacobians + energy sum_q c_q mu(T) + min det A per CTA
//               (paper Sec. 3.3, eq. D0_expression; line-search check Sec. 2.3)
//   k_gradient  Jacobians + c_q dmu/dT W^-T + transposed contractions to an
//               element vector (Sec. 3.3, eq. vm_pa_grad)
//   k_hsetup    Jacobians + c_q d2mu/dT2 contracted with W^-1 (packed
//               symmetric d^2(d^2+1)/2 values per point) (Sec. 3.4)
//   k_apply     forward contractions of v, pointwise H : dA with the stored
//               data, transposed contractions (Sec. 3.4, eq. vm_pa_hess)
//   k_diag      diagonal of the Hessian from the stored data through
//               products of 1D tables (Sec. 3.4)
// Element vectors (E-vectors) are written as ev[a * E * NP + e * NP + i] and
// assembled to nodes by the transposed-map kernel in vec_kernels.cu.
#pragma once

#include <type_traits>

#include "tmop_device.cuh"

namespace tmop {

template <class C, class R>
struct ElemCtx {
    R *B, *G, *w;
    R *su, *s1, *s2, *sA, *sX;
    int *smap;
    int t, tx, ty;
    int64_t e;
    bool valid;
};

// Stage the tables and the element map; set up the thread's element slot.
template <class C, class R>
__device__ __forceinline__ void prologue(const ElemParams &P, int64_t tile, unsigned char *smem,
                                         ElemCtx<C, R> &c)
{
    using L = Layout<C, R>;
    R *base = reinterpret_cast<R *>(smem);
    const R *__restrict__ tab = table_of<R>(P);
    for (int i = threadIdx.x; i < L::TAB; i += C::NT) base[i] = tab[i];
    c.B = base;
    c.G = base + C::NQ * C::NI;
    c.w = base + 2 * C::NQ * C::NI;
    const int slot = threadIdx.x / C::TPE;
    const bool act = slot < C::EPB;
    const int sl = act ? slot : 0;
    c.t = threadIdx.x - slot * C::TPE;
    c.tx = c.t % C::MX;
    c.ty = c.t / C::MX;
    R *s = base + L::TAB_PAD + sl * L::SLOT;
    c.su = s;
    c.s1 = s + C::SU;
    c.s2 = c.s1 + C::S1;
    c.sA = c.s2 + C::S2;
    c.sX = c.sA + C::DD * C::NQD;
    c.smap = reinterpret_cast<int *>(base + L::TAB_PAD + C::EPB * L::SLOT) + sl * C::NP;
    c.e = tile * C::EPB + sl;
    c.valid = act && c.e < P.E;
    if (c.valid)
        for (int i = c.t; i < C::NP; i += C::TPE) c.smap[i] = P.map[c.e * C::NP + i];
    __syncthreads();
}

// Gather one component of an L-vector into the slot and run the forward
// contractions: sA[(a*D + b)*NQD + q] = d u_a / d xbar_b at q; sX holds the
// interpolated values when xv is requested.  LOCAL (positions): the element's
// first node is subtracted in FP64 before the contractions, so that the
// Jacobian is formed from differences of size h rather than from absolute
// coordinates (sum_i grad w_i = 0 makes it the same A; the interpolated
// values get the offset back).  This removes the cancellation that would
// otherwise scale the rounding of the double-float contractions by |x|/h.
template <class C, class R, class RIN, bool LOCAL = false>
__device__ __forceinline__ void forward_component(const ElemParams &P, ElemCtx<C, R> &c,
                                                  const RIN *__restrict__ u, int a, bool want_x)
{
    double off = 0.0;
    if (LOCAL && c.valid) off = (double)u[a * P.Nx + c.smap[0]];
    if (c.valid)
        for (int i = c.t; i < C::NP; i += C::TPE)
            c.su[i] = LOCAL ? R((double)u[a * P.Nx + c.smap[i]] - off) : R(u[a * P.Nx + c.smap[i]]);
    __syncthreads();
    R *A0 = c.sA + (a * C::D) * C::NQD;
    R *xv = want_x ? c.sX + a * C::NQD : nullptr;
    if (C::D == 3)
        fwd3<C, R>(c.B, c.G, c.su, c.s1, c.s2, A0, A0 + C::NQD, A0 + 2 * C::NQD, xv, c.tx, c.ty,
                   c.valid);
    else
        fwd2<C, R>(c.B, c.G, c.su, c.s1, A0, A0 + C::NQD, xv, c.tx, c.ty, c.valid);
    if (LOCAL && want_x && c.valid && c.tx < C::NQ && c.ty < C::NQ) {
        // each thread restores the points it wrote (its own (q1, q2) column)
        if (C::D == 3) {
            for (int q3 = 0; q3 < C::NQ; ++q3) {
                const int q = (q3 * C::NQ + c.ty) * C::NQ + c.tx;
                xv[q] = R(to_d(xv[q]) + off);
            }
        } else {
            const int q = c.ty * C::NQ + c.tx;
            xv[q] = R(to_d(xv[q]) + off);
        }
    }
}

// Forward pass of the element geometry: the Jacobian rows of x into sA;
// the physical point coordinates into sX for the size target, or the
// interpolated target field eta into sX[0..NQD) for the discrete target
// (its derivative outputs land in sA rows that the x components overwrite).
template <class C, class R>
__device__ __forceinline__ void forward_geometry(const ElemParams &P, ElemCtx<C, R> &c,
                                                 const double *__restrict__ x)
{
    if (P.target == TGT_DISCRETE) {
        if (c.valid)
            for (int i = c.t; i < C::NP; i += C::TPE) c.su[i] = R(P.eta[c.smap[i]]);
        __syncthreads();
        if (C::D == 3)
            fwd3<C, R>(c.B, c.G, c.su, c.s1, c.s2, c.sA, c.sA + C::NQD, c.sA + 2 * C::NQD, c.sX,
                       c.tx, c.ty, c.valid);
        else
            fwd2<C, R>(c.B, c.G, c.su, c.s1, c.sA, c.sA + C::NQD, c.sX, c.tx, c.ty, c.valid);
    }
    const bool want_x = P.target == TGT_SIZE;
    for (int a = 0; a < C::D; ++a) forward_component<C, R, double, true>(P, c, x, a, want_x);
}

// Values at the points of component a of an L-vector u (minus u0 when given):
// the B-only path of the forward contractions, into out[q]; sA rows 0..D-1
// take the discarded derivatives.
template <class C, class R, class RIN>
__device__ __forceinline__ void values_at_points(const ElemParams &P, ElemCtx<C, R> &c,
                                                 const RIN *__restrict__ u, const RIN *__restrict__ u0,
                                                 int a, R *out)
{
    if (c.valid)
        for (int i = c.t; i < C::NP; i += C::TPE) {
            const int64_t j = a * P.Nx + c.smap[i];
            c.su[i] = R(u0 ? (double)u[j] - (double)u0[j] : (double)u[j]);
        }
    __syncthreads();
    if (C::D == 3)
        fwd3<C, R>(c.B, c.G, c.su, c.s1, c.s2, c.sA, c.sA + C::NQD, c.sA + 2 * C::NQD, out, c.tx, c.ty,
                   c.valid);
    else
        fwd2<C, R>(c.B, c.G, c.su, c.s1, c.sA, c.sA + C::NQD, out, c.tx, c.ty, c.valid);
}

// su_i = sum_q f(q) w_i(chi_q) for all element nodes (zeroes su first)
template <class C, class R>
__device__ __forceinline__ void values_transpose(ElemCtx<C, R> &c, const R *f)
{
    if (c.valid)
        for (int i = c.t; i < C::NP; i += C::TPE) c.su[i] = R(0.0);
    __syncthreads();
    if (C::D == 3)
        bwd3_tab<C, R>(c.B, c.B, c.B, f, c.s1, c.s2, c.su, c.tx, c.ty, c.valid);
    else
        bwd2_tab<C, R>(c.B, c.B, f, c.s1, c.su, c.tx, c.ty, c.valid);
}

// Transposed contractions of sA[(a*D + b)*NQD + q] (b = derivative
// direction) and store of the element vector component a.
// ACT: an action element vector (ev_store: float pairs for double-float).
template <class C, class R, class ROUT, bool ACT = false>
__device__ __forceinline__ void backward_component(const ElemParams &P, ElemCtx<C, R> &c,
                                                   ROUT *__restrict__ ev, int a)
{
    const R *Y0 = c.sA + (a * C::D) * C::NQD;
    if (C::D == 3)
        bwd3<C, R>(c.B, c.G, Y0, Y0 + C::NQD, Y0 + 2 * C::NQD, c.s1, c.s2, c.su, c.tx, c.ty,
                   c.valid);
    else
        bwd2<C, R>(c.B, c.G, Y0, Y0 + C::NQD, c.s1, c.su, c.tx, c.ty, c.valid);
    if (c.valid)
        for (int i = c.t; i < C::NP; i += C::TPE)
            if constexpr (ACT)
                ev_store(&ev[(int64_t)a * P.E * C::NP + c.e * C::NP + i], c.su[i]);
            else
                ev[(int64_t)a * P.E * C::NP + c.e * C::NP + i] = ROUT(to_d(c.su[i]));
}

// Iterate over this thread's quadrature points: (q1, q2) = (tx, ty), all q3.
template <class C, class F>
__device__ __forceinline__ void for_my_points(int tx, int ty, bool valid, F &&f)
{
    if (!valid || tx >= C::NQ || ty >= C::NQ) return;
    if (C::D == 3) {
#pragma unroll 1
        for (int q3 = 0; q3 < C::NQ; ++q3) f((q3 * C::NQ + ty) * C::NQ + tx, q3);
    } else {
        f(ty * C::NQ + tx, 0);
    }
}

template <class C, class R>
__device__ __forceinline__ double point_weight(const R *w, int tx, int ty, int q3)
{
    return C::D == 3 ? to_db(w[tx]) * to_db(w[ty]) * to_db(w[q3]) : to_db(w[tx]) * to_db(w[ty]);
}

template <class C, class R>
__device__ __forceinline__ double point_target(const ElemParams &P, const R *sX, int q)
{
    if (P.target == TGT_DISCRETE) return discrete_scale<C::D>(P.h0, to_db(sX[q]));
    double xq[3] = {0, 0, 0};
    if (P.target == TGT_SIZE)
#pragma unroll
        for (int k = 0; k < C::D; ++k) xq[k] = to_db(sX[k * C::NQD + q]);
    return target_scale<C::D>(P.target, P.h0, xq);
}

// Deterministic CTA reduction of (energy sum, min det) into part[2 tile + {0,1}]:
// warps by shuffles, then warp results in order.  Called by all threads.
template <class C>
__device__ __forceinline__ void cta_energy_reduce(double esum, double emin, double *part, int64_t tile)
{
    __shared__ double red_s[C::NT / 32], red_m[C::NT / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        esum += __shfl_down_sync(0xffffffffu, esum, o);
        emin = fmin(emin, __shfl_down_sync(0xffffffffu, emin, o));
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) { red_s[wid] = esum; red_m[wid] = emin; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0, m = INFINITY;
        for (int i = 0; i < C::NT / 32; ++i) { s += red_s[i]; m = fmin(m, red_m[i]); }
        part[2 * tile] = s;
        part[2 * tile + 1] = m;
    }
}

// ---------------------------------------------------------------- energy
// RS: arithmetic of the contractions (double, or df = double-float).
template <class C, class RS>
__global__ void __launch_bounds__(C::NT)
k_energy(ElemParams P, const double *__restrict__ x, double *__restrict__ part, BatchArgs BA)
{
    const void *in = x, *aux = nullptr;
    void *out = part;
    const int *stop = nullptr;
    const int64_t tile = resolve_tile(P, BA, in, aux, out, stop);
    x = static_cast<const double *>(in);
    part = static_cast<double *>(out);
    extern __shared__ __align__(16) unsigned char smem[];
    ElemCtx<C, RS> c;
    prologue<C, RS>(P, tile, smem, c);
    forward_geometry<C, RS>(P, c, x);

    double esum = 0.0, emin = INFINITY;
    // the energy is formed from FP64 invariants (see metric_mu_fp64)
    const bool dw = false;
    const bool use_i2 = metric_uses_I2(P.metric, C::D);
    for_my_points<C>(c.tx, c.ty, c.valid, [&](int q, int q3) {
        double ws = 1.0, iws = 1.0, wd = 1.0;            // identity target: W = I
        if (P.target != TGT_IDENTITY) {
            ws = point_target<C>(P, c.sX, q);
            iws = 1.0 / ws;
            wd = ws;
#pragma unroll
            for (int k = 1; k < C::D; ++k) wd *= ws;
        }
        const double cq = point_weight<C>(c.w, c.tx, c.ty, q3) * wd;
        double I1, tau, I2 = 0.0;
        if constexpr (std::is_same<RS, df>::value) {
            if (dw) {
                df Td[C::DD], Cd[C::DD];
                point_T_dw<C::D, C::NQD>(c.sA, q, iws, P.target == TGT_IDENTITY, Td, Cd, I1, tau);
                if (C::D == 3 && use_i2) {
                    df s(0.0f, 0.0f);
#pragma unroll
                    for (int r = 0; r < C::DD; ++r) acc_add(s, Cd[r] * Cd[r]);
                    I2 = to_db(norm(s));
                }
            }
        }
        if (!dw) {
            double T[C::DD], Cf[C::DD];
#pragma unroll
            for (int r = 0; r < C::DD; ++r) T[r] = to_db(c.sA[r * C::NQD + q]) * iws;
            invariants<C::D>(T, I1, tau, I2, Cf);
        }
        const double detA = ws > 0.0 ? tau * wd : -INFINITY;   // no target: inverted
        if (P.detq) P.detq[c.e * C::NQD + q] = tau * wd;         // det A = det T det W
        emin = fmin(emin, detA);
        if (detA > 0.0) {
            Inv v;
            esum += cq * metric_scalars<C::D>(P.metric, I1, tau, I2, v);
        }
    });

    cta_energy_reduce<C>(esum, emin, part, tile);
}

// ---------------------------------------------------------------- gradient
// The fused energy takes mu at a point from the double-float invariants
// unless |mu| is below this bound: an error in I1 or tau enters mu at first
// order, ~4e-15 on the scale 1 of the metrics' "- 1" (or (tau - 1)^2), so
// near a zero-energy optimum (every |mu| small) the sum would stop at that
// floor and the line search's F(x+) < 1.2 F(x) test would compare noise; there
// the point's mu is recomputed from FP64 invariants of the same T.  The
// decision is per point and per call: a result depends only on x.
constexpr double kMuFp64Below = 1e-6;

// The gradient integrand at one point (and its energy, det A): reads the
// Jacobian A_r at sA[r * ST + q] (r = 0..DD-1), writes c_q dmu/dT(T) W^-T into
// the same slots (zero at an inverted point), adds c_q mu to esum (mu from FP64
// invariants where |mu| < kMuFp64Below, when want_e) and det A to the minimum
// emin.  ws: target scale (W = ws I), iws = 1/ws, wd = ws^D, cq = w_q wd.
template <class C, int ST, class RS>
__device__ __forceinline__ void gradient_point(const ElemParams &P, RS *sA, int q, double ws,
                                               double iws, double wd, double cq, bool want_e,
                                               double &esum, double &emin)
{
    const bool dw = std::is_same<RS, df>::value;
    const bool use_i2 = metric_uses_I2(P.metric, C::D);
    if constexpr (std::is_same<RS, df>::value) {
        if (dw && !use_i2) {      // (I1, tau) metrics: P = 2 f1 T + f_tau cof T on the FP32 pipes
            df Td[C::DD], Cd[C::DD], I1w, tauw;
            double I1, tau;
            point_T_dw<C::D, ST>(sA, q, iws, P.target == TGT_IDENTITY, Td, Cd, I1, tau,
                                     &I1w, &tauw);
            emin = fmin(emin, ws > 0.0 ? tau * wd : -INFINITY);
            if (!(tau > 0.0) || !(ws > 0.0)) {
#pragma unroll
                for (int r = 0; r < C::DD; ++r) sA[r * ST + q] = RS(0.0f, 0.0f);
                return;
            }
            const double sc = cq * iws;
            df a, b;
            double mu_pt;
            if (P.metric == MET_303 || P.metric == MET_303_55) {   // scalars in double-float too
                InvW w;
                mu_pt = to_db(metric303_dw(I1w, tauw, P.metric == MET_303_55, w));
                const df scw = from_db<df>(sc);
                a = dw_mul(scw, df(2.0f * w.f1.h, 2.0f * w.f1.l));
                b = dw_mul(scw, w.ft);
            } else {
                Inv v;
                mu_pt = metric_scalars<C::D>(P.metric, I1, tau, 0.0, v);
                a = from_db<df>(2.0 * v.f1 * sc);
                b = from_db<df>(v.ft * sc);
            }
            if (want_e && fabs(mu_pt) < kMuFp64Below) {
                double Tdb[C::DD];             // energy from FP64 invariants
#pragma unroll
                for (int r = 0; r < C::DD; ++r) Tdb[r] = to_db(Td[r]);
                mu_pt = metric_mu_fp64<C::D>(P.metric, Tdb);
            }
            esum += cq * mu_pt;
#pragma unroll
            for (int r = 0; r < C::DD; ++r) {
                df acc(0.0f, 0.0f);
                acc_add(acc, a * Td[r]);
                acc_add(acc, b * Cd[r]);
                sA[r * ST + q] = norm(acc);
            }
            return;
        }
        if constexpr (C::D == 3) {
            if (dw && use_i2) {   // I2 metrics: + f2 dI2/dT, dI2/dT = 2 (I1 T - T T^T T)
                df Td[9], Cd[9], g2[9], TtT[9], TTt[9], I1w;
                double I1, tau;
                point_T_dw<3, ST>(sA, q, iws, P.target == TGT_IDENTITY, Td, Cd, I1, tau, &I1w);
                emin = fmin(emin, ws > 0.0 ? tau * wd : -INFINITY);
                if (!(tau > 0.0) || !(ws > 0.0)) {
#pragma unroll
                    for (int r = 0; r < 9; ++r) sA[r * ST + q] = RS(0.0f, 0.0f);
                    return;
                }
                const double I2 = i2_dw(Td, Cd, I1w, g2, TtT, TTt);
                Inv v;
                const double mu = metric_scalars<3>(P.metric, I1, tau, I2, v);
                if (want_e && fabs(mu) < kMuFp64Below) {
                    double Tdb[9];             // energy from FP64 invariants
#pragma unroll
                    for (int r = 0; r < 9; ++r) Tdb[r] = to_db(Td[r]);
                    esum += cq * metric_mu_fp64<3>(P.metric, Tdb);
                } else {
                    esum += cq * mu;
                }
                const double sc = cq * iws;
                const df a = from_db<df>(2.0 * v.f1 * sc), b = from_db<df>(v.ft * sc);
                const df c2 = from_db<df>(v.f2 * sc);
#pragma unroll
                for (int r = 0; r < 9; ++r) {
                    df acc(0.0f, 0.0f);
                    acc_add(acc, a * Td[r]);
                    acc_add(acc, b * Cd[r]);
                    acc_add(acc, c2 * g2[r]);
                    sA[r * ST + q] = norm(acc);
                }
                return;
            }
        }
    }
    double T[C::DD], Cf[C::DD], g2[C::DD], TtT[9], TTt[9];
#pragma unroll
    for (int r = 0; r < C::DD; ++r) T[r] = to_db(sA[r * ST + q]) * iws;
    double I1, tau, I2;
    invariants<C::D>(T, I1, tau, I2, Cf);
    emin = fmin(emin, ws > 0.0 ? tau * wd : -INFINITY);
    if (!(tau > 0.0) || !(ws > 0.0)) {                // inverted points contribute 0
#pragma unroll
        for (int r = 0; r < C::DD; ++r) sA[r * ST + q] = RS(0.0);
        return;
    }
    Inv v;
    esum += cq * metric_scalars<C::D>(P.metric, I1, tau, I2, v);
    if (C::D == 3 && v.f2 != 0.0) dI2_3(T, I1, g2, TtT, TTt);
    const double sc = cq * iws;
#pragma unroll
    for (int r = 0; r < C::DD; ++r) {
        double pr = v.f1 * 2.0 * T[r] + v.ft * Cf[r];
        if (C::D == 3 && v.f2 != 0.0) pr += v.f2 * g2[r];
        sA[r * ST + q] = from_db<RS>(sc * pr);
    }}

template <class C, class RS>
__global__ void __launch_bounds__(C::NT)
k_gradient(ElemParams P, const double *__restrict__ x, double *__restrict__ ev, double *part,
           BatchArgs BA)
{
    // part != nullptr: also the energy and min det partials (fused pass)
    const void *in = x, *aux = part;
    void *out = ev;
    const int *stop = nullptr;
    const int64_t tile = resolve_tile(P, BA, in, aux, out, stop);
    x = static_cast<const double *>(in);
    ev = static_cast<double *>(out);
    part = const_cast<double *>(static_cast<const double *>(aux));
    extern __shared__ __align__(16) unsigned char smem[];
    ElemCtx<C, RS> c;
    prologue<C, RS>(P, tile, smem, c);
    forward_geometry<C, RS>(P, c, x);

    double esum = 0.0, emin = INFINITY;
    for_my_points<C>(c.tx, c.ty, c.valid, [&](int q, int q3) {
        double ws = 1.0, iws = 1.0, wd = 1.0;            // identity target: W = I
        if (P.target != TGT_IDENTITY) {
            ws = point_target<C>(P, c.sX, q);
            iws = 1.0 / ws;
            wd = ws;
#pragma unroll
            for (int k = 1; k < C::D; ++k) wd *= ws;
        }
        const double cq = point_weight<C>(c.w, c.tx, c.ty, q3) * wd;
        gradient_point<C, C::NQD, RS>(P, c.sA, q, ws, iws, wd, cq, part != nullptr, esum, emin);
    });
    if (part) cta_energy_reduce<C>(esum, emin, part, tile);   // part is uniform per launch
    __syncthreads();
    for (int a = 0; a < C::D; ++a) backward_component<C, RS, double>(P, c, ev, a);
}

// ---------------------------------------------------------------- Hessian setup
// Two consecutive stored values in one store (an entry pair of the PAIRS
// layout; p aligned to their combined size).
__device__ __forceinline__ void st_pair(df *p, const df &a, const df &b)
{
    *reinterpret_cast<float4 *>(p) = make_float4(a.h, a.l, b.h, b.l);
}
__device__ __forceinline__ void st_pair(float *p, float a, float b)
{
    *reinterpret_cast<float2 *>(p) = make_float2(a, b);
}
__device__ __forceinline__ void st_pair(double *p, double a, double b)
{
    *reinterpret_cast<double2 *>(p) = make_double2(a, b);
}

// The stores of one point's packed entries, made in increasing entry order:
// with the PAIRS layout an even entry is held until its odd partner and the
// two are stored together.
template <class C, class RH>
struct PointStore {
    RH *He;
    int q;
    RH pend;
    __device__ __forceinline__ void put(int k, const RH &v)
    {
        if constexpr (!C::PAIRS) {
            He[C::hoff(k, q)] = v;
        } else {
            if ((C::NS & 1) && k == C::NS - 1) He[C::hoff(k, q)] = v;
            else if ((k & 1) == 0) pend = v;
            else st_pair(He + C::hoff(k - 1, q), pend, v);
        }
    }
};

// HAS_I2 = false: metrics of (I1, tau) only (mu_2, mu_303, mu_55, mu_303 + mu_55,
// and the 2D mu_7, mu_9),
// whose d2mu/dT2 is u (x) g1 + w (x) cof T + 2 f1 Id + f_tau d2tau with
// u = f11 g1 + f1t cof T, w = f1t g1 + ftt cof T: two FMAs per stored entry.
// The stored d2mu/dT2 entries of one point: reads the Jacobian A_r at
// sA[r * ST + q], stores the NS packed entries of c_q W^-1 (d2mu/dT2) W^-T at
// point qh of the element block He (zero at an inverted point).  ws: target
// scale (W = ws I), iws = 1/ws, wd = ws^D, cq = w_q wd.
template <class C, int ST, class RS, class RH, bool HAS_I2>
__device__ __forceinline__ void hsetup_point(const ElemParams &P, const RS *sA, int q, double ws,
                                             double iws, double wd, double cq, RH *He, int qh)
{
    if constexpr (std::is_same<RS, df>::value && !HAS_I2 && !std::is_same<RH, double>::value) {
        // the factored d2mu/dT2 below, on the FP32 pipes
        df Td[C::DD], Cd[C::DD], I1w, tauw;
        double I1, tau;
        point_T_dw<C::D, ST>(sA, q, iws, P.target == TGT_IDENTITY, Td, Cd, I1, tau, &I1w,
                                 &tauw);
        if (!(tau > 0.0) || !(ws > 0.0)) {
#pragma unroll
            for (int s = 0; s < C::NS; ++s) He[C::hoff(s, qh)] = RH(0.0f);
            return;
        }
        const double sc = cq * iws * iws;
        df a1, b1, a2, b2, dg, ft;
        if (P.metric == MET_303 || P.metric == MET_303_55) {     // scalars in double-float too
            InvW w;
            metric303_dw(I1w, tauw, P.metric == MET_303_55, w);
            const df scw = from_db<df>(sc);
            a1 = df(0.0f, 0.0f);                                  // f11 = 0
            b1 = dw_mul(scw, w.f1t);
            a2 = df(2.0f * b1.h, 2.0f * b1.l);
            b2 = dw_mul(scw, w.ftt);
            const df f1s = dw_mul(scw, w.f1);
            dg = df(2.0f * f1s.h, 2.0f * f1s.l);
            ft = dw_mul(scw, w.ft);
        } else {
            Inv v;
            metric_scalars<C::D>(P.metric, I1, tau, 0.0, v);
            a1 = from_db<df>(2.0 * sc * v.f11);
            b1 = from_db<df>(sc * v.f1t);
            a2 = from_db<df>(2.0 * sc * v.f1t);
            b2 = from_db<df>(sc * v.ftt);
            dg = from_db<df>(2.0 * sc * v.f1);
            ft = from_db<df>(sc * v.ft);
        }
        df u[C::DD], w[C::DD];
        PointStore<C, RH> ps{He, qh, RH()};
#pragma unroll
        for (int r = 0; r < C::DD; ++r) {
            df x(0.0f, 0.0f), y(0.0f, 0.0f);
            acc_add(x, a1 * Td[r]);
            acc_add(x, b1 * Cd[r]);
            acc_add(y, a2 * Td[r]);
            acc_add(y, b2 * Cd[r]);
            u[r] = norm(x);
            w[r] = norm(y);
            Td[r] = df(2.0f * Td[r].h, 2.0f * Td[r].l);    // g1 = 2T (exact)
        }
#pragma unroll
        for (int r = 0; r < C::DD; ++r)
#pragma unroll
            for (int s = r; s < C::DD; ++s) {
                const int a = r / C::D, b = r % C::D, cc = s / C::D, e = s % C::D;
                df k(0.0f, 0.0f);
                acc_add(k, u[r] * Td[s]);
                acc_add(k, w[r] * Cd[s]);
                if (r == s) acc_add(k, dprod{dg.h, dg.l});
                if (a != cc && b != e) {
                    if (C::D == 2) {
                        const bool neg = (a == 0) != (b == 0);
                        acc_add(k, neg ? dprod{-ft.h, -ft.l} : dprod{ft.h, ft.l});
                    } else {
                        // T = g1 / 2 at the index of the third row and column
                        const df Tm = df(0.5f * Td[(3 - a - cc) * 3 + (3 - b - e)].h,
                                         0.5f * Td[(3 - a - cc) * 3 + (3 - b - e)].l);
                        const dprod pt = ft * Tm;
                        acc_add(k, eps3(a, cc) * eps3(b, e) > 0.0 ? pt : -pt);
                    }
                }
                ps.put(pidx<C::DD>(r, s), store_dw<RH>(norm(k)));
            }
        return;
    }
    if constexpr (std::is_same<RS, df>::value && HAS_I2 && C::D == 3 &&
                  !std::is_same<RH, double>::value) {
        // I2 metrics (3D): K_rs = u_r g1_s + w_r Cf_s + z_r g2_s + (2 f1 + 2 f2 I1) delta_rs
        //   + f_tau d2tau_rs - 2 f2 (delta_ac TtT_eb + T_ae T_cb + delta_be TTt_ac),
        // u = f11 g1 + f1t Cf + f12 g2 + 2 f2 T, w = f1t g1 + ftt Cf + f2t g2,
        // z = f12 g1 + f2t Cf (f22 = 0), g1 = 2T: d2I2 = 4 T (x) T + 2 I1 Id - ...
        df Td[9], Cd[9], g2w[9], TtTw[9], TTtw[9], I1w;
        PointStore<C, RH> ps{He, qh, RH()};
        double I1, tau;
        point_T_dw<3, ST>(sA, q, iws, P.target == TGT_IDENTITY, Td, Cd, I1, tau, &I1w);
        if (!(tau > 0.0) || !(ws > 0.0)) {
#pragma unroll
            for (int s = 0; s < C::NS; ++s) He[C::hoff(s, qh)] = RH(0.0f);
            return;
        }
        const double I2 = i2_dw(Td, Cd, I1w, g2w, TtTw, TTtw);
        Inv v;
        metric_scalars<3>(P.metric, I1, tau, I2, v);
        const double sc = cq * iws * iws;
        const df k11 = from_db<df>(2.0 * sc * v.f11), k1t = from_db<df>(sc * v.f1t);
        const df k12 = from_db<df>(sc * v.f12), kf2 = from_db<df>(2.0 * sc * v.f2);
        const df l1 = from_db<df>(2.0 * sc * v.f1t), ltt = from_db<df>(sc * v.ftt);
        const df l2t = from_db<df>(sc * v.f2t), m1 = from_db<df>(2.0 * sc * v.f12);
        const df dg = from_db<df>(2.0 * sc * (v.f1 + v.f2 * I1)), ft = from_db<df>(sc * v.ft);
        const df m2 = from_db<df>(-2.0 * sc * v.f2);
        df u[9], w[9], z[9];
#pragma unroll
        for (int r = 0; r < 9; ++r) {
            df x(0.0f, 0.0f), y(0.0f, 0.0f), zz(0.0f, 0.0f);
            acc_add(x, k11 * Td[r]);          // f11 g1 (g1 = 2T)
            acc_add(x, k1t * Cd[r]);
            acc_add(x, k12 * g2w[r]);
            acc_add(x, kf2 * Td[r]);          // 2 f2 T
            acc_add(y, l1 * Td[r]);
            acc_add(y, ltt * Cd[r]);
            acc_add(y, l2t * g2w[r]);
            acc_add(zz, m1 * Td[r]);
            acc_add(zz, l2t * Cd[r]);
            u[r] = norm(x);
            w[r] = norm(y);
            z[r] = norm(zz);
        }
#pragma unroll
        for (int r = 0; r < 9; ++r)
#pragma unroll
            for (int s = r; s < 9; ++s) {
                const int a = r / 3, b = r % 3, cc = s / 3, e = s % 3;
                df k(0.0f, 0.0f);
                acc_add(k, u[r] * df(2.0f * Td[s].h, 2.0f * Td[s].l));
                acc_add(k, w[r] * Cd[s]);
                acc_add(k, z[r] * g2w[s]);
                if (r == s) acc_add(k, dprod{dg.h, dg.l});
                if (a != cc && b != e) {
                    const dprod pt = ft * Td[(3 - a - cc) * 3 + (3 - b - e)];
                    acc_add(k, eps3(a, cc) * eps3(b, e) > 0.0 ? pt : -pt);
                }
                if (a == cc) acc_add(k, m2 * TtTw[e * 3 + b]);
                acc_add(k, m2 * to_df(Td[a * 3 + e] * Td[cc * 3 + b]));
                if (b == e) acc_add(k, m2 * TTtw[a * 3 + cc]);
                ps.put(pidx<9>(r, s), store_dw<RH>(norm(k)));
            }
        return;
    }
    double T[C::DD], Cf[C::DD], g2[9], TtT[9], TTt[9];
#pragma unroll
    for (int r = 0; r < C::DD; ++r) T[r] = to_db(sA[r * ST + q]) * iws;
    double I1, tau, I2;
    invariants<C::D>(T, I1, tau, I2, Cf);
    if (!(tau > 0.0) || !(ws > 0.0)) {                // inverted points store 0
#pragma unroll
        for (int s = 0; s < C::NS; ++s) He[C::hoff(s, qh)] = RH(0.0);
        return;
    }
    Inv v;
    metric_scalars<C::D>(P.metric, I1, tau, I2, v);
    const double sc = cq * iws * iws;
    PointStore<C, RH> ps{He, qh, RH()};
    if constexpr (HAS_I2) {
        if (C::D == 3 && v.f2 != 0.0) dI2_3(T, I1, g2, TtT, TTt);
#pragma unroll
        for (int r = 0; r < C::DD; ++r)
#pragma unroll
            for (int s = r; s < C::DD; ++s)
                ps.put(pidx<C::DD>(r, s),
                       from_db<RH>(sc * metric_K_entry<C::D>(r, s, T, Cf, g2, TtT, TTt, I1, v)));
    } else {
        double u[C::DD], w[C::DD];
#pragma unroll
        for (int r = 0; r < C::DD; ++r) {
            u[r] = sc * (v.f11 * 2.0 * T[r] + v.f1t * Cf[r]);
            w[r] = sc * (v.f1t * 2.0 * T[r] + v.ftt * Cf[r]);
        }
        const double dg = 2.0 * sc * v.f1, ft = sc * v.ft;
#pragma unroll
        for (int r = 0; r < C::DD; ++r)
#pragma unroll
            for (int s = r; s < C::DD; ++s) {
                const int a = r / C::D, b = r % C::D, cc = s / C::D, e = s % C::D;
                double k = u[r] * (2.0 * T[s]) + w[r] * Cf[s];
                if (r == s) k += dg;
                if (a != cc && b != e) {
                    if (C::D == 2) k += ft * ((a == 0 ? 1.0 : -1.0) * (b == 0 ? 1.0 : -1.0));
                    else k += ft * eps3(a, cc) * eps3(b, e) * T[(3 - a - cc) * 3 + (3 - b - e)];
                }
                ps.put(pidx<C::DD>(r, s), from_db<RH>(k));
            }
    }}

template <class C, class RS, class RH, bool HAS_I2>
__global__ void __launch_bounds__(C::NT)
k_hsetup(ElemParams P, const double *__restrict__ x, RH *__restrict__ H, BatchArgs BA)
{
    const void *in = x, *aux = nullptr;
    void *out = H;
    const int *stop = nullptr;
    const int64_t tile = resolve_tile(P, BA, in, aux, out, stop);
    x = static_cast<const double *>(in);
    H = static_cast<RH *>(out);
    extern __shared__ __align__(16) unsigned char smem[];
    ElemCtx<C, RS> c;
    prologue<C, RS>(P, tile, smem, c);
    forward_geometry<C, RS>(P, c, x);

    RH *He = H + c.e * (int64_t)C::HST;
    for_my_points<C>(c.tx, c.ty, c.valid, [&](int q, int q3) {
        double ws = 1.0, iws = 1.0, wd = 1.0;            // identity target: W = I
        if (P.target != TGT_IDENTITY) {
            ws = point_target<C>(P, c.sX, q);
            iws = 1.0 / ws;
            wd = ws;
#pragma unroll
            for (int k = 1; k < C::D; ++k) wd *= ws;
        }
        const double cq = point_weight<C>(c.w, c.tx, c.ty, q3) * wd;
        hsetup_point<C, C::NQD, RS, RH, HAS_I2>(P, c.sA, q, ws, iws, wd, cq, He, q);
    });
}

// ---------------------------------------------------------------- Hessian action
// RV: type of v and of the element vector; RC: arithmetic and stored data
// (double, float, or df with double vectors).  v is expected to be zero on
// fixed DOFs (callers mask it first).  If stop_iter != nullptr and
// *stop_iter < k the launch does nothing (MINRES iterations after
// convergence; k < 0: the device iteration counter, iter_of).
template <class C, class RV, class RC>
__global__ void __launch_bounds__(C::NT)
k_apply(ElemParams P, const RV *__restrict__ v, const RC *__restrict__ H, RV *__restrict__ ev,
        const int *__restrict__ stop_iter, int k, BatchArgs BA)
{
    const void *in = v, *aux = H;
    void *out = ev;
    const int *stop = stop_iter;
    const int64_t tile = resolve_tile(P, BA, in, aux, out, stop);
    v = static_cast<const RV *>(in);
    H = static_cast<const RC *>(aux);
    ev = static_cast<RV *>(out);
    if (stop && *stop < iter_of(stop, k)) return;
    extern __shared__ __align__(16) unsigned char smem[];
    ElemCtx<C, RC> c;
    prologue<C, RC>(P, tile, smem, c);
    for (int a = 0; a < C::D; ++a) forward_component<C, RC, RV>(P, c, v, a, false);

    const RC *He = H + c.e * (int64_t)C::HST;
    for_my_points<C>(c.tx, c.ty, c.valid, [&](int q, int) {
        RC dA[C::DD], h[C::NS];
#pragma unroll
        for (int r = 0; r < C::DD; ++r) dA[r] = c.sA[r * C::NQD + q];
#pragma unroll
        for (int s = 0; s < C::NS; ++s) h[s] = He[C::hoff(s, q)];
#pragma unroll
        for (int r = 0; r < C::DD; ++r) {
            RC y = 0;
#pragma unroll
            for (int s = 0; s < C::DD; ++s) y += h[r <= s ? pidx<C::DD>(r, s) : pidx<C::DD>(s, r)] * dA[s];
            c.sA[r * C::NQD + q] = y;
        }
    });
    __syncthreads();
    for (int a = 0; a < C::D; ++a) backward_component<C, RC, RV, true>(P, c, ev, a);
}

// ---------------------------------------------------------------- diagonal
// diag_{a,i} = sum_q sum_{b,e} H_{ab,ae}(q) d_b w_i(q) d_e w_i(q); the
// product d_b w_i d_e w_i factors per direction k into (B or G)(B or G).
template <class C, class RV, class RC>
__global__ void __launch_bounds__(C::NT)
k_diag(ElemParams P, const RC *__restrict__ H, RV *__restrict__ ev, BatchArgs BA)
{
    const void *in = nullptr, *aux = H;
    void *out = ev;
    const int *stop = nullptr;
    const int64_t tile = resolve_tile(P, BA, in, aux, out, stop);
    H = static_cast<const RC *>(aux);
    ev = static_cast<RV *>(out);
    extern __shared__ __align__(16) unsigned char smem[];
    ElemCtx<C, RC> c;
    prologue<C, RC>(P, tile, smem, c);
    __shared__ RC tbl[3][C::NQ * C::NI];          // B*B, B*G, G*G (elementwise)
    for (int i = threadIdx.x; i < C::NQ * C::NI; i += C::NT) {
        tbl[0][i] = prod(c.B[i], c.B[i]);
        tbl[1][i] = prod(c.B[i], c.G[i]);
        tbl[2][i] = prod(c.G[i], c.G[i]);
    }
    __syncthreads();
    const RC *He = H + c.e * (int64_t)C::HST;
    if constexpr (C::D == 3) {
        // The six (b <= e) pairs of each component a in one pass per
        // contraction stage (3 barriers per component): the thread's q3
        // column of each pair is read straight from the stored data and
        // contracted in registers, then q2 and q1 through shared memory,
        // with the pairs summed in the last stage.  Scratch: sA and sX
        // (12 NQ^3 values >= 6 NI NQ^2 + 6 NI^2 NQ since NQ >= NI).
        constexpr int NI = C::NI, NQ = C::NQ, GA = NI * NQ * NQ, HB = NI * NI * NQ;
        constexpr int PB[6] = {0, 0, 0, 1, 1, 2}, PE[6] = {0, 1, 2, 1, 2, 2};
        static_assert(6 * GA + 6 * HB <= (C::DD + C::D) * C::NQD, "diag scratch");
        RC *g = c.sA, *h = c.sA + 6 * GA;
        for (int a = 0; a < 3; ++a) {
            if (c.valid && c.tx < NQ && c.ty < NQ) {          // q3 -> i3
#pragma unroll
                for (int p = 0; p < 6; ++p) {
                    const RC *T3 = tbl[(PB[p] == 2) + (PE[p] == 2)];
                    const int hs = pidx<C::DD>(a * 3 + PB[p], a * 3 + PE[p]);
                    RC col[NQ];
#pragma unroll
                    for (int q3 = 0; q3 < NQ; ++q3) {
                        const RC v = He[C::hoff(hs, (q3 * NQ + c.ty) * NQ + c.tx)];
                        col[q3] = PB[p] == PE[p] ? v : twice(v);
                    }
#pragma unroll
                    for (int i3 = 0; i3 < NI; ++i3) {
                        RC z = RC(0.0);
#pragma unroll
                        for (int q3 = 0; q3 < NQ; ++q3) acc_add(z, T3[q3 * NI + i3] * col[q3]);
                        g[p * GA + (i3 * NQ + c.ty) * NQ + c.tx] = norm(z);
                    }
                }
            }
            __syncthreads();
            if (c.valid && c.tx < NQ && c.ty < NI) {          // q2 -> i2
#pragma unroll
                for (int p = 0; p < 6; ++p) {
                    const RC *T2 = tbl[(PB[p] == 1) + (PE[p] == 1)];
#pragma unroll
                    for (int i3 = 0; i3 < NI; ++i3) {
                        RC z = RC(0.0);
#pragma unroll
                        for (int q2 = 0; q2 < NQ; ++q2)
                            acc_add(z, T2[q2 * NI + c.ty] * g[p * GA + (i3 * NQ + q2) * NQ + c.tx]);
                        h[p * HB + (i3 * NI + c.ty) * NQ + c.tx] = norm(z);
                    }
                }
            }
            __syncthreads();
            if (c.valid && c.tx < NI && c.ty < NI) {          // q1 -> i1, pairs summed
#pragma unroll
                for (int i3 = 0; i3 < NI; ++i3) {
                    RC o = RC(0.0);
#pragma unroll
                    for (int p = 0; p < 6; ++p) {
                        const RC *T1 = tbl[(PB[p] == 0) + (PE[p] == 0)];
#pragma unroll
                        for (int q1 = 0; q1 < NQ; ++q1)
                            acc_add(o, T1[q1 * NI + c.tx] * h[p * HB + (i3 * NI + c.ty) * NQ + q1]);
                        o = norm(o);
                    }
                    RV &out = ev[(int64_t)a * P.E * C::NP + c.e * C::NP + (i3 * NI + c.ty) * NI + c.tx];
                    if constexpr (std::is_same<RV, float>::value) out = o;
                    else out = to_db(o);
                }
            }
            __syncthreads();
        }
        return;
    }
    RC *f = c.sA;
    for (int a = 0; a < C::D; ++a) {
        if (c.valid)
            for (int i = c.t; i < C::NP; i += C::TPE) c.su[i] = RC(0.0);
        for (int b = 0; b < C::D; ++b)
            for (int e2 = b; e2 < C::D; ++e2) {
                const int r = a * C::D + b, s = a * C::D + e2;
                const RC scale = (b == e2) ? RC(1.0) : RC(2.0);
                for_my_points<C>(c.tx, c.ty, c.valid, [&](int q, int) {
                    f[q] = prod(scale, He[C::hoff(pidx<C::DD>(r, s), q)]);
                });
                __syncthreads();
                const RC *T1 = tbl[(b == 0) + (e2 == 0)];
                const RC *T2 = tbl[(b == 1) + (e2 == 1)];
                if (C::D == 3) {
                    const RC *T3 = tbl[(b == 2) + (e2 == 2)];
                    bwd3_tab<C, RC>(T1, T2, T3, f, c.s1, c.s2, c.su, c.tx, c.ty, c.valid);
                } else {
                    bwd2_tab<C, RC>(T1, T2, f, c.s1, c.su, c.tx, c.ty, c.valid);
                }
            }
        if (c.valid)
            for (int i = c.t; i < C::NP; i += C::TPE)
                ev[(int64_t)a * P.E * C::NP + c.e * C::NP + i] = RV(to_d(c.su[i]));
        __syncthreads();
    }
}

}  // namespace tmop
