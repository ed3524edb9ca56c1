// 3D energy gradient, one element per group of lanes of one warp (sm_103a).
//
// g = B^T [c_q dmu/dT(T) W^-T] (paper Sec. 3.3, eq. vm_pa_grad), with the
// fused energy sum_q c_q mu(T_q) and min det A of the CTA's element tile.  The
// Jacobian A at the points is sum-factorised with B and G (A_{c0} = G1 B2 B3 u,
// A_{c1} = B1 G2 B3 u, A_{c2} = B1 B2 G3 u) from the element's positions minus
// its first node (sum_i grad w_i = 0 makes it the same A and removes the |x|/h
// cancellation from the double-float rounding): the collocated derivative
// (D applied to the values at the points) would amplify the rounding of those
// values by the row sums of |D|, and dmu/dT near a shape optimum is a small
// difference of O(1) terms, so the gradient needs the more accurate A.  The
// integrand per point is gradient_point, shared with the sum-factorised
// kernel; the transposed pass is sum-factorised with B^T and G^T as well (the
// collocated D^T would again scale the rounding by the row sums of |D|, above
// the scale of the sum).  The lane mapping and the per-warp shared-memory
// columns are those of k_apply3c, the contraction buffers lie in columns that
// are dead at the time; the CTA is one element tile of four warps, so the
// energy partials keep the tile order.  Against the sum-factorised kernel it
// runs warp-synchronous (no CTA barrier between stages) with every contraction
// along q3 in registers.
#pragma once

#include "apply3c.cuh"

namespace tmop {

// The 1D tables B, G (and D) and the Gauss weights, in the kernel parameter space.
template <class R, int NI, int NQ>
struct GradTab {
    R B[NQ * NI];                                           // B[q * NI + i] = w_i(chi_q)
    R G[NQ * NI];                                           // G[q * NI + i] = w_i'(chi_q)
    R w[NQ];
};

template <class C>
struct Grad3cShape {
    using S = Apply3cShape<C, 4>;
    static constexpr int TAB = 2 * C::NQ * C::NI;           // B, G (an even count)
    // forward buffers of an element: the gathered nodes, B1 u and G1 u
    static constexpr int FB = C::NP + 2 * C::NI * C::NI * C::NQ;
    static_assert(S::EPW * FB <= 3 * C::NQ * 32, "forward buffers in three column rows");
    // tables, the 9 Jacobian / integrand columns and the 3 physical-coordinate
    // columns of every thread
    static constexpr size_t bytes =
        sizeof(df) * (size_t)(TAB + 9 * C::NQ * S::NT + 3 * C::NQ * S::NT);
};

// Forward pass of the warp-synchronous geometry kernels: the Jacobian A_{c b}
// at the points of element e into the warp's columns cs [(3 c + b) NQ + q3]
// and the physical point coordinates into xs [c NQ + q3] (32-lane stride), by
// B/G sum factorisation of the positions minus the element's first node, with
// every partial sum renormalised; fu, fb, fg: the element's buffers (in column
// rows 6-8, dead until component 2 is stored).
template <class C>
__device__ __forceinline__ void grad3c_forward(const ElemParams &P, const double *__restrict__ x,
                                               int64_t e, bool valid, int t, int tx, int ty,
                                               int lane, const int *m, int m0, const df *Bs,
                                               const df *Gs, const GradTab<df, C::NI, C::NQ> &T,
                                               df *cs, df *xs, df *fu, df *fb, df *fg)
{
    using S = Apply3cShape<C, 4>;
    using RC = df;
    constexpr int NI = C::NI, NQ = C::NQ, NP = C::NP;
#pragma unroll 1
    for (int c = 0; c < 3; ++c) {
        const double off = valid ? x[c * P.Nx + m0] : 0.0;
#pragma unroll
        for (int j = 0; j < S::NPL; ++j) {
            const int i = t + j * S::TPE;
            if (valid && i < NP) fu[i] = RC(x[c * P.Nx + m[j]] - off);
        }
        __syncwarp();
        if (valid && ty < NI) {                             // i1 -> q1: B1 u and G1 u
            RC Bx[NI], Gx[NI];
#pragma unroll
            for (int i = 0; i < NI; ++i) {
                Bx[i] = Bs[tx * NI + i];
                Gx[i] = Gs[tx * NI + i];
            }
#pragma unroll
            for (int i3 = 0; i3 < NI; ++i3) {
                const RC *u = fu + (i3 * NI + ty) * NI;
                RC a = mul1(Bx[0], u[0]);
                RC g = mul1(Gx[0], u[0]);
#pragma unroll
                for (int i1 = 1; i1 < NI; ++i1) {
                    a += Bx[i1] * u[i1];
                    g += Gx[i1] * u[i1];
                }
                fb[(i3 * NI + ty) * NQ + tx] = a;
                fg[(i3 * NI + ty) * NQ + tx] = g;
            }
        }
        __syncwarp();
        RC g0[NQ], g1[NQ], g2[NQ];
        if (valid) {
            RC By[NI], Gy[NI], sbb[NI], sbg[NI], sgb[NI];   // B2 B1 u, G2 B1 u, B2 G1 u
#pragma unroll
            for (int i = 0; i < NI; ++i) {
                By[i] = Bs[ty * NI + i];
                Gy[i] = Gs[ty * NI + i];
            }
#pragma unroll
            for (int i3 = 0; i3 < NI; ++i3) {               // i2 -> q2
                const RC *wb = fb + i3 * NI * NQ + tx;
                const RC *wg = fg + i3 * NI * NQ + tx;
                RC a = mul1(By[0], wb[0]);
                RC b = mul1(Gy[0], wb[0]);
                RC d = mul1(By[0], wg[0]);
#pragma unroll
                for (int i2 = 1; i2 < NI; ++i2) {
                    a += By[i2] * wb[i2 * NQ];
                    b += Gy[i2] * wb[i2 * NQ];
                    d += By[i2] * wg[i2 * NQ];
                }
                sbb[i3] = a;
                sbg[i3] = b;
                sgb[i3] = d;
            }
#pragma unroll
            for (int q3 = 0; q3 < NQ; ++q3) {               // i3 -> q3 (registers)
                RC u = mul1(T.B[q3 * NI], sbb[0]);        // values at the points
                RC a0 = mul1(T.B[q3 * NI], sgb[0]);
                RC a1 = mul1(T.B[q3 * NI], sbg[0]);
                RC a2 = mul1(T.G[q3 * NI], sbb[0]);
#pragma unroll
                for (int i3 = 1; i3 < NI; ++i3) {
                    u += T.B[q3 * NI + i3] * sbb[i3];
                    a0 += T.B[q3 * NI + i3] * sgb[i3];
                    a1 += T.B[q3 * NI + i3] * sbg[i3];
                    a2 += T.G[q3 * NI + i3] * sbb[i3];
                }
                xs[(c * NQ + q3) * 32 + lane] = norm(u + RC(off));   // physical coordinate
                g0[q3] = a0;
                g1[q3] = a1;
                g2[q3] = a2;
            }
        }
        if (c == 2) __syncwarp();                           // rows 6-8 held the buffers
        if (valid) {
#pragma unroll
            for (int q3 = 0; q3 < NQ; ++q3) {
                cs[((c * 3 + 0) * NQ + q3) * 32 + lane] = g0[q3];
                cs[((c * 3 + 1) * NQ + q3) * 32 + lane] = g1[q3];
                cs[((c * 3 + 2) * NQ + q3) * 32 + lane] = g2[q3];
            }
        }
        __syncwarp();                                       // the buffers are reused by the next gather
    }

}

template <class C, int MINB>
__global__ void __launch_bounds__(128, MINB)
k_grad3c(ElemParams P, const double *__restrict__ x, double *__restrict__ ev, double *part,
         BatchArgs BA, const GradTab<df, C::NI, C::NQ> T)
{
    static_assert(C::D == 3, "3D kernel");
    using S = Apply3cShape<C, 4>;
    using RC = df;
    static_assert(S::NT == C::NT && S::EPB == C::EPB, "the CTA is one element tile");
    constexpr int NI = C::NI, NQ = C::NQ, NP = C::NP;

    // part != nullptr (or a batch aux role): also the energy and min det partials
    const void *in = x, *aux = part;
    void *out = ev;
    const int *stop = nullptr;
    const int64_t tile = resolve_tile(P, BA, in, aux, out, stop);
    x = static_cast<const double *>(in);
    ev = static_cast<double *>(out);
    part = const_cast<double *>(static_cast<const double *>(aux));

    using G3 = Grad3cShape<C>;
    extern __shared__ __align__(16) unsigned char smem[];
    RC *Bs = reinterpret_cast<RC *>(smem);                  // B[q * NI + i]
    RC *Gs = Bs + NQ * NI;                                  // G[q * NI + i]
    if (threadIdx.x == 0) {                                 // compile-time indices only
#pragma unroll
        for (int i = 0; i < NQ * NI; ++i) Bs[i] = T.B[i];
#pragma unroll
        for (int i = 0; i < NQ * NI; ++i) Gs[i] = T.G[i];
    }
    __syncthreads();

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int slot = lane / S::TPE;
    const bool act = slot < S::EPW;
    const int t = lane - slot * S::TPE;
    const int tx = t % NQ, ty = t / NQ;
    const int64_t e = tile * C::EPB + warp * S::EPW + (act ? slot : 0);
    const bool valid = act && e < P.E;
    // the warp's columns [(r * NQ + q3) * 32 + lane]: Jacobian then integrand
    // rows r = 3 c + b, and the physical point coordinates (size target)
    RC *cs = Bs + G3::TAB + warp * 9 * NQ * 32;
    RC *xs = Bs + G3::TAB + 9 * NQ * S::NT + warp * 3 * NQ * 32;
    // forward buffers in rows 6-8: nodes u, B1 u, G1 u [(i3 * NI + i2) * NQ + q1]
    RC *fu = cs + 6 * NQ * 32 + (act ? slot : 0) * G3::FB;
    RC *fb = fu + NP;
    RC *fg = fb + NI * NI * NQ;
    int m[S::NPL];
#pragma unroll
    for (int j = 0; j < S::NPL; ++j) {
        const int i = t + j * S::TPE;
        m[j] = (valid && i < NP) ? P.map[e * NP + i] : 0;
    }
    const int m0 = valid ? P.map[e * NP] : 0;              // the element's first node

    grad3c_forward<C>(P, x, e, valid, t, tx, ty, lane, m, m0, Bs, Gs, T, cs, xs, fu, fb, fg);

    // ---- pointwise: the integrand c_q dmu/dT W^-T over the Jacobian columns
    double esum = 0.0, emin = INFINITY;
    if (valid) {
#pragma unroll 1
        for (int q3 = 0; q3 < NQ; ++q3) {
            double ws = 1.0, iws = 1.0, wd = 1.0;           // identity target: W = I
            if (P.target != TGT_IDENTITY) {
                double xq[3];
#pragma unroll
                for (int k = 0; k < 3; ++k) xq[k] = to_db(xs[(k * NQ + q3) * 32 + lane]);
                ws = target_scale<3>(P.target, P.h0, xq);
                iws = 1.0 / ws;
                wd = ws * ws * ws;
            }
            const double cq = to_db(T.w[tx]) * to_db(T.w[ty]) * to_db(T.w[q3]) * wd;
            gradient_point<C, NQ * 32, RC>(P, cs + lane, q3 * 32, ws, iws, wd, cq, part != nullptr,
                                           esum, emin);
        }
    }
    if (part) cta_energy_reduce<C>(esum, emin, part, tile);   // part is uniform per launch

    // ---- transposed, sum-factorised with B and G:
    // g_c = G1^T B2^T B3^T Y0 + B1^T G2^T B3^T Y1 + B1^T B2^T G3^T Y2
    // (Y_b = the integrand rows 3 c + b); buffers: the three q3 -> i3 results
    // in rows 0-2 (dead once component 0 is read), the two q2 -> i2 results in
    // the physical-coordinate columns (dead after the pointwise phase)
    constexpr int TBE = 3 * NI * NQ * NQ, SRE = 2 * NI * NI * NQ;
    static_assert(S::EPW * TBE <= 3 * NQ * 32 && S::EPW * SRE <= 3 * NQ * 32, "backward buffers");
    RC *tb0 = cs + (act ? slot : 0) * TBE;                  // [(i3 * NQ + q2) * NQ + q1]
    RC *tb1 = tb0 + NI * NQ * NQ, *tb2 = tb1 + NI * NQ * NQ;
    RC *sb = xs + (act ? slot : 0) * SRE;                   // [(i3 * NI + i2) * NQ + q1]
    RC *rb = sb + NI * NI * NQ;
#pragma unroll 1
    for (int c = 0; c < 3; ++c) {
        RC Y0[NQ], Y1[NQ], Y2[NQ];
#pragma unroll
        for (int q3 = 0; q3 < NQ; ++q3) {
            Y0[q3] = cs[((c * 3 + 0) * NQ + q3) * 32 + lane];
            Y1[q3] = cs[((c * 3 + 1) * NQ + q3) * 32 + lane];
            Y2[q3] = cs[((c * 3 + 2) * NQ + q3) * 32 + lane];
        }
        if (c == 0) __syncwarp();                           // rows 0-2 become the buffers
        if (valid) {
#pragma unroll
            for (int i3 = 0; i3 < NI; ++i3) {               // q3 -> i3 (registers)
                RC a = mul1(T.B[i3], Y0[0]);
                RC b = mul1(T.B[i3], Y1[0]);
                RC g = mul1(T.G[i3], Y2[0]);
#pragma unroll
                for (int q3 = 1; q3 < NQ; ++q3) {
                    acc_add(a, T.B[q3 * NI + i3] * Y0[q3]);
                    acc_add(b, T.B[q3 * NI + i3] * Y1[q3]);
                    acc_add(g, T.G[q3 * NI + i3] * Y2[q3]);
                }
                tb0[(i3 * NQ + ty) * NQ + tx] = a;
                tb1[(i3 * NQ + ty) * NQ + tx] = b;
                tb2[(i3 * NQ + ty) * NQ + tx] = g;
            }
        }
        __syncwarp();
        if (valid && ty < NI) {                             // q2 -> i2
            RC BTy[NQ], GTy[NQ];
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                BTy[q] = Bs[q * NI + ty];
                GTy[q] = Gs[q * NI + ty];
            }
#pragma unroll
            for (int i3 = 0; i3 < NI; ++i3) {
                const RC *w0 = tb0 + i3 * NQ * NQ + tx;
                const RC *w1 = tb1 + i3 * NQ * NQ + tx;
                const RC *w2 = tb2 + i3 * NQ * NQ + tx;
                RC a = mul1(BTy[0], w0[0]);
                RC r = mul1(GTy[0], w1[0]);
#pragma unroll
                for (int q2 = 1; q2 < NQ; ++q2) {
                    acc_add(a, BTy[q2] * w0[q2 * NQ]);
                    acc_add(r, GTy[q2] * w1[q2 * NQ]);
                }
#pragma unroll
                for (int q2 = 0; q2 < NQ; ++q2) acc_add(r, BTy[q2] * w2[q2 * NQ]);
                sb[(i3 * NI + ty) * NQ + tx] = a;
                rb[(i3 * NI + ty) * NQ + tx] = r;
            }
        }
        __syncwarp();
        if (valid && tx < NI && ty < NI) {                  // q1 -> i1
            RC BTx[NQ], GTx[NQ];
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                BTx[q] = Bs[q * NI + tx];
                GTx[q] = Gs[q * NI + tx];
            }
            double *o_e = ev + (int64_t)c * P.E * NP + e * NP;
#pragma unroll
            for (int i3 = 0; i3 < NI; ++i3) {
                const RC *ws = sb + (i3 * NI + ty) * NQ;
                const RC *wr = rb + (i3 * NI + ty) * NQ;
                RC a = mul1(GTx[0], ws[0]);
#pragma unroll
                for (int q1 = 1; q1 < NQ; ++q1) acc_add(a, GTx[q1] * ws[q1]);
#pragma unroll
                for (int q1 = 0; q1 < NQ; ++q1) acc_add(a, BTx[q1] * wr[q1]);
                o_e[(i3 * NI + ty) * NI + tx] = cvt_out(a);
            }
        }
        __syncwarp();                                       // the buffers are reused by the next component
    }
}


// Partial-assembly set-up on the same forward pass: the stored d2mu/dT2 entries
// of every point (hsetup_point, shared with the block kernel k_hsetup), each
// lane storing its own points (entry pairs: one 8- or 16-byte store per two
// entries across consecutive lanes).  Paper Sec. 3.4.
template <class C, class RH, bool HAS_I2, int MINB>
__global__ void __launch_bounds__(128, MINB)
k_hset3c(ElemParams P, const double *__restrict__ x, RH *__restrict__ H, BatchArgs BA,
         const GradTab<df, C::NI, C::NQ> T)
{
    static_assert(C::D == 3, "3D kernel");
    using S = Apply3cShape<C, 4>;
    using RC = df;
    static_assert(S::NT == C::NT && S::EPB == C::EPB, "the CTA is one element tile");
    constexpr int NI = C::NI, NQ = C::NQ, NP = C::NP;

    const void *in = x, *aux = nullptr;
    void *out = H;
    const int *stop = nullptr;
    const int64_t tile = resolve_tile(P, BA, in, aux, out, stop);
    x = static_cast<const double *>(in);
    H = static_cast<RH *>(out);

    using G3 = Grad3cShape<C>;
    extern __shared__ __align__(16) unsigned char smem[];
    RC *Bs = reinterpret_cast<RC *>(smem);                  // B[q * NI + i]
    RC *Gs = Bs + NQ * NI;                                  // G[q * NI + i]
    if (threadIdx.x == 0) {                                 // compile-time indices only
#pragma unroll
        for (int i = 0; i < NQ * NI; ++i) Bs[i] = T.B[i];
#pragma unroll
        for (int i = 0; i < NQ * NI; ++i) Gs[i] = T.G[i];
    }
    __syncthreads();

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int slot = lane / S::TPE;
    const bool act = slot < S::EPW;
    const int t = lane - slot * S::TPE;
    const int tx = t % NQ, ty = t / NQ;
    const int64_t e = tile * C::EPB + warp * S::EPW + (act ? slot : 0);
    const bool valid = act && e < P.E;
    RC *cs = Bs + G3::TAB + warp * 9 * NQ * 32;
    RC *xs = Bs + G3::TAB + 9 * NQ * S::NT + warp * 3 * NQ * 32;
    RC *fu = cs + 6 * NQ * 32 + (act ? slot : 0) * G3::FB;
    RC *fb = fu + NP;
    RC *fg = fb + NI * NI * NQ;
    int m[S::NPL];
#pragma unroll
    for (int j = 0; j < S::NPL; ++j) {
        const int i = t + j * S::TPE;
        m[j] = (valid && i < NP) ? P.map[e * NP + i] : 0;
    }
    const int m0 = valid ? P.map[e * NP] : 0;
    grad3c_forward<C>(P, x, e, valid, t, tx, ty, lane, m, m0, Bs, Gs, T, cs, xs, fu, fb, fg);
    if (!valid) return;                                     // no barrier follows

    RH *He = H + e * (int64_t)C::HST;
    const int pt = ty * NQ + tx;
#pragma unroll 1
    for (int q3 = 0; q3 < NQ; ++q3) {
        double ws = 1.0, iws = 1.0, wd = 1.0;               // identity target: W = I
        if (P.target != TGT_IDENTITY) {
            double xq[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) xq[k] = to_db(xs[(k * NQ + q3) * 32 + lane]);
            ws = target_scale<3>(P.target, P.h0, xq);
            iws = 1.0 / ws;
            wd = ws * ws * ws;
        }
        const double cq = to_db(T.w[tx]) * to_db(T.w[ty]) * to_db(T.w[q3]) * wd;
        hsetup_point<C, NQ * 32, RC, RH, HAS_I2>(P, cs + lane, q3 * 32, ws, iws, wd, cq, He,
                                                 q3 * NQ * NQ + pt);
    }
}

}  // namespace tmop
