// Vector kernels of the TMOP Newton step: deterministic assembly of element
// vectors through the transposed element map, fixed-DOF masks, FP64
// reductions with fixed block order, and the fused Jacobi-preconditioned
// MINRES updates (Paige & Saunders 1975, the inner solver of paper Sec. 2.3
// and 3.4) whose scalar recurrences run in one-thread kernels so that the
// host never has to read them inside an iteration.
#include <climits>
#include <cmath>

#include "dfloat.cuh"
#include "minres_scalar.cuh"
#include "tmop_device.cuh"
#include "tmop_internal.h"

namespace tmop {

namespace {

constexpr int VT = 256;           // threads per block of the vector kernels
constexpr int RED_MAX = 1184;     // 8 CTAs per SM on 148 SMs

__device__ __forceinline__ double block_sum(double v, double *sh)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += sh[i];
    return s;   // valid on thread 0
}


// y[dof] = sum over the element entries of the node (fixed order), then the
// fixed-DOF rule: mode 0 -> 0, mode 1 -> vfix[dof] (or 0), mode 2 -> 1.
template <class RI, class RO>
__global__ void k_assemble(const RI *__restrict__ ev, const int32_t *__restrict__ ptr,
                           const int32_t *__restrict__ idx, const uint8_t *__restrict__ fixed,
                           const RO *__restrict__ vfix, int mode, int64_t Nx, int D, int64_t ENP,
                           RO *__restrict__ out, const int *__restrict__ stop, int k)
{
    if (stop && *stop < iter_of(stop, k)) return;
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= Nx) return;
    const int b = ptr[n], e = ptr[n + 1];
    // entries in fixed order; the D component loads of an entry are independent
    typename AsmAcc<RI>::T s[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) asm_zero(s[a]);
    for (int j = b; j < e; ++j) {
        const int64_t t = __ldg(idx + j);
#pragma unroll
        for (int a = 0; a < 3; ++a)
            if (a < D) asm_add(s[a], ld_entry(ev + a * ENP + t));
        if (((j - b) & 7) == 7)
#pragma unroll
            for (int a = 0; a < 3; ++a) asm_renorm(s[a]);
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (a >= D) break;
        const int64_t dof = a * Nx + n;
        RO r = asm_out<RO>(s[a]);
        if (fixed && fixed[dof]) r = (mode == 0) ? RO(0) : (mode == 1 ? (vfix ? vfix[dof] : RO(0)) : RO(1));
        out[dof] = r;
    }
}

template <class R>
__global__ void k_mask(const R *__restrict__ v, const uint8_t *__restrict__ fixed, int64_t n,
                       R *__restrict__ out)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (fixed && fixed[i]) ? R(0) : v[i];
}

__global__ void k_trial(const double *__restrict__ x, const double *__restrict__ dx, double alpha,
                        int64_t n, double *__restrict__ out)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = x[i] - alpha * dx[i];
}

// *flag = 1 when a and b differ in any bit of any entry (left untouched
// otherwise); every writer stores the same value.
__global__ void k_differs(const double *__restrict__ a, const double *__restrict__ b, int64_t n,
                          double *__restrict__ flag)
{
    bool d = false;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        d |= __double_as_longlong(a[i]) != __double_as_longlong(b[i]);
    if (__any_sync(0xffffffffu, d) && (threadIdx.x & 31) == 0) *flag = 1.0;
}

template <class R>
__global__ void k_dot(const R *__restrict__ a, const R *__restrict__ b, int64_t n,
                      double *__restrict__ part)
{
    __shared__ double sh[VT / 32];
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        s += (double)a[i] * (double)b[i];
    s = block_sum(s, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void k_finalize_sum(const double *__restrict__ part, int nb, double *__restrict__ out)
{
    __shared__ double sh[VT / 32];
    double s = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) s += part[i];
    s = block_sum(s, sh);
    if (threadIdx.x == 0) *out = s;
}

// part holds (sum, min) pairs; out = (sum, min).
__global__ void k_finalize_energy(const double *__restrict__ part, int64_t nb, double *__restrict__ out)
{
    __shared__ double sh[VT / 32], shm[VT / 32];
    double s = 0.0, m = INFINITY;
    for (int64_t i = threadIdx.x; i < nb; i += blockDim.x) {
        s += part[2 * i];
        m = fmin(m, part[2 * i + 1]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmin(m, __shfl_down_sync(0xffffffffu, m, o));
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) shm[wid] = m;
    s = block_sum(s, sh);     // contains a __syncthreads, publishing shm
    if (threadIdx.x == 0) {
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) m = fmin(m, shm[i]);
        out[0] = s;
        out[1] = m;
    }
}

template <class R>
__global__ void k_jacobi(const R *__restrict__ diag, int64_t n, R *__restrict__ minv)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double a = fabs((double)diag[i]);
        minv[i] = (R)(a < 1e-300 ? 1.0 : 1.0 / a);
    }
}

// ---------------------------------------------------------------- MINRES
// r1 = r2 = b, y = M^-1 b; partial dot(b, y).
template <class R>
__global__ void k_minres_init(const double *__restrict__ b, const R *__restrict__ minv, int64_t n,
                              R *__restrict__ r1, R *__restrict__ r2, R *__restrict__ y,
                              double *__restrict__ part)
{
    __shared__ double sh[VT / 32];
    double s;
    VecDot<R> dot;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const R bi = (R)b[i];
        const R yi = minv[i] * bi;
        r1[i] = bi;
        r2[i] = bi;
        y[i] = yi;
        dot.add(bi, yi);
    }
    s = block_sum(dot.get(), sh);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void k_minres_start(const double *__restrict__ part, int nb, MinresState *st)
{
    __shared__ double sh[VT / 32];
    double s = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) s += part[i];
    s = block_sum(s, sh);
    if (threadIdx.x == 0) minres_start_scalars(st, s);
}

// v = y / beta (first Lanczos vector).
template <class R>
__global__ void k_minres_scale(const R *__restrict__ y, const MinresState *__restrict__ st, int64_t n,
                               R *__restrict__ v)
{
    if (st->stop_iter < 1) return;
    const VecS<R> ib = (VecS<R>)(1.0 / st->beta);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        v[i] = (R)((VecS<R>)y[i] * ib);
}

// y = z - (beta/beta_old) r1 (k >= 2), in place in z; partial dot(v, y).
template <class R>
__global__ void k_lanczos_a(R *__restrict__ z, const R *__restrict__ r1, const R *__restrict__ v,
                            const MinresState *__restrict__ st, int64_t n, int k,
                            double *__restrict__ part)
{
    if (k < 0) k = st->k;                                  // device iteration counter
    if (st->stop_iter < k) return;
    __shared__ double sh[VT / 32];
    using S = VecS<R>;
    const S c = (S)((k >= 2) ? st->beta / st->beta_old : 0.0);
    VecDot<R> dot;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const R yi = (R)((S)z[i] - c * (S)r1[i]);
        z[i] = yi;
        dot.add(v[i], yi);
    }
    const double s = block_sum(dot.get(), sh);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// The assembly of the action's element vectors (fixed DOFs -> 0) fused with
// the first Lanczos update: y = z - (beta/beta_old) r1 and the partial
// dot(v, y), one node (all components) per thread, grid-stride over nb
// blocks.  Saves the write and re-read of z.
template <class RI, class R>
__global__ void k_assemble_lanczos_a(const RI *__restrict__ ev, const int32_t *__restrict__ ptr,
                                     const int32_t *__restrict__ idx, const uint8_t *__restrict__ fixed,
                                     int64_t Nx, int D, int64_t ENP, R *__restrict__ y,
                                     const R *__restrict__ r1, const R *__restrict__ v,
                                     const MinresState *__restrict__ st, int k, double *__restrict__ part)
{
    if (k < 0) k = st->k;                                  // device iteration counter
    if (st->stop_iter < k) return;
    __shared__ double sh[VT / 32];
    using S = VecS<R>;
    const S c = (S)((k >= 2) ? st->beta / st->beta_old : 0.0);
    VecDot<R> dot;
    for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < Nx; n += (int64_t)gridDim.x * blockDim.x) {
        const int b = ptr[n], e = ptr[n + 1];
        typename AsmAcc<RI>::T s[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) asm_zero(s[a]);
        for (int j = b; j < e; ++j) {
            const int64_t t = __ldg(idx + j);
#pragma unroll
            for (int a = 0; a < 3; ++a)
                if (a < D) asm_add(s[a], ld_entry(ev + a * ENP + t));
            if (((j - b) & 7) == 7)
#pragma unroll
                for (int a = 0; a < 3; ++a) asm_renorm(s[a]);
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (a >= D) break;
            const int64_t dof = a * Nx + n;
            const R z = (fixed && fixed[dof]) ? R(0) : asm_out<R>(s[a]);
            const R yi = (R)((S)z - c * (S)r1[dof]);
            y[dof] = yi;
            dot.add(v[dof], yi);
        }
    }
    const double dsum = block_sum(dot.get(), sh);
    if (threadIdx.x == 0) part[blockIdx.x] = dsum;
}

__global__ void k_iter_next(MinresState *st) { st->k += 1; }

__global__ void k_fin_alpha(const double *__restrict__ part, int nb, MinresState *st, int k)
{
    if (k < 0) k = st->k;                                  // device iteration counter
    if (st->stop_iter < k) return;
    __shared__ double sh[VT / 32];
    double s = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) s += part[i];
    s = block_sum(s, sh);
    if (threadIdx.x == 0) st->alpha = s;
}

// y -= (alpha/beta) r2 (in place); ynew = M^-1 y; partial dot(y, ynew).
template <class R>
__global__ void k_lanczos_b(R *__restrict__ y, const R *__restrict__ r2, const R *__restrict__ minv,
                            const MinresState *__restrict__ st, int64_t n, int k,
                            R *__restrict__ ynew, double *__restrict__ part)
{
    if (k < 0) k = st->k;                                  // device iteration counter
    if (st->stop_iter < k) return;
    __shared__ double sh[VT / 32];
    using S = VecS<R>;
    const S c = (S)(st->alpha / st->beta);
    VecDot<R> dot;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const R yi = (R)((S)y[i] - c * (S)r2[i]);
        const R zi = minv[i] * yi;
        y[i] = yi;
        ynew[i] = zi;
        dot.add(yi, zi);
    }
    const double s = block_sum(dot.get(), sh);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// beta_{k+1}, the Givens rotations of the tridiagonal QR, phi and the stop test.
__global__ void k_fin_beta(const double *__restrict__ part, int nb, MinresState *st, int k,
                           double rtol, int fixed_its)
{
    if (k < 0) k = st->k;                                  // device iteration counter
    if (st->stop_iter < k) return;
    __shared__ double sh[VT / 32];
    double s = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) s += part[i];
    s = block_sum(s, sh);
    if (threadIdx.x == 0) minres_beta_scalars(st, s, k, rtol, fixed_its);
}

// wnew = (v - eps_old w1 - delta w2) / gamma; dx += phi wnew; v = ynew / beta.
template <class R>
__global__ void k_minres_update(R *__restrict__ v, const R *__restrict__ w1, const R *__restrict__ w2,
                                R *__restrict__ wnew, double *__restrict__ dx,
                                const R *__restrict__ ynew, const MinresState *__restrict__ st,
                                int64_t n, int k)
{
    if (k < 0) k = st->k;                                  // device iteration counter
    if (st->stop_iter < k) return;
    using S = VecS<R>;
    const S eo = (S)st->eps_old, de = (S)st->delta, ig = (S)(1.0 / st->gamma);
    const double ph = st->phi;
    const S ib = (S)((st->beta > 0.0) ? 1.0 / st->beta : 0.0);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const S wn = ((S)v[i] - eo * (S)w1[i] - de * (S)w2[i]) * ig;
        wnew[i] = (R)wn;
        dx[i] += ph * (double)wn;                           // the solution stays FP64
        v[i] = (R)((S)ynew[i] * ib);
    }
}

inline unsigned grid_for(int64_t n)
{
    int64_t g = (n + VT - 1) / VT;
    if (g > RED_MAX) g = RED_MAX;
    return (unsigned)(g < 1 ? 1 : g);
}

// Vector algebra for callers that drive their own Krylov iteration.
__global__ void k_lincomb(int64_t n, double a, const double *__restrict__ x, double b,
                          const double *__restrict__ y, double c, const double *__restrict__ z,
                          double *__restrict__ out)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double v = a * x[i];
        if (y) v += b * y[i];
        if (z) v += c * z[i];
        out[i] = v;
    }
}

__global__ void k_vmul(int64_t n, const double *__restrict__ x, const double *__restrict__ y,
                       double *__restrict__ out)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = x[i] * y[i];
}

// partial sums of x_i y_i over the entries with mask_i != 0 (all when mask is null)
__global__ void k_dot_masked(const double *__restrict__ a, const double *__restrict__ b,
                             const uint8_t *__restrict__ mask, int64_t n, double *__restrict__ part)
{
    __shared__ double sh[VT / 32];
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        if (!mask || mask[i]) s += a[i] * b[i];
    s = block_sum(s, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void k_vgather(int64_t m, const int32_t *__restrict__ idx, const double *__restrict__ src,
                          double *__restrict__ dst)
{
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < m; k += (int64_t)gridDim.x * blockDim.x)
        dst[k] = src[idx[k]];
}

// dst[idx[k]] += vals[k]; the indices of one call are distinct (no atomics)
__global__ void k_vscatter_add(int64_t m, const int32_t *__restrict__ idx,
                               const double *__restrict__ vals, double *__restrict__ dst)
{
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < m; k += (int64_t)gridDim.x * blockDim.x)
        dst[idx[k]] += vals[k];
}

}  // namespace

cudaError_t launch_vgather(int64_t m, const int32_t *idx, const double *src, double *dst,
                           cudaStream_t s)
{
    if (m == 0) return cudaSuccess;
    k_vgather<<<grid_for(m), VT, 0, s>>>(m, idx, src, dst);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_vscatter_add(int64_t m, const int32_t *idx, const double *vals, double *dst,
                                cudaStream_t s)
{
    if (m == 0) return cudaSuccess;
    k_vscatter_add<<<grid_for(m), VT, 0, s>>>(m, idx, vals, dst);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_lincomb(int64_t n, double a, const double *x, double b, const double *y,
                           double c, const double *z, double *out, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    k_lincomb<<<grid_for(n), VT, 0, s>>>(n, a, x, b, y, c, z, out);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_vmul(int64_t n, const double *x, const double *y, double *out, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    k_vmul<<<grid_for(n), VT, 0, s>>>(n, x, y, out);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_dot_masked(const double *a, const double *b, const uint8_t *mask, int64_t n,
                              double *part, int nb, cudaStream_t s)
{
    k_dot_masked<<<nb, VT, 0, s>>>(a, b, mask, n, part);
    count_launch();
    return cudaGetLastError();
}

// ---------------------------------------------------------------- remap CG / RK4
// Jacobi-preconditioned CG for the mass solves of the advection remap
// (Sec. 3.6).  The scalars live in CgState on the device; iteration kk
// (1-based) runs only while st->stop >= kk, so a fixed launch sequence
// stops doing work once the solve has converged.
namespace {

// k = 0, r = b, z = dinv r, p = z; partial r.z
__global__ void k_cg_init(const double *__restrict__ b, const double *__restrict__ dinv, int64_t n,
                          double *__restrict__ k, double *__restrict__ r, double *__restrict__ z,
                          double *__restrict__ p, double *__restrict__ part)
{
    __shared__ double sh[VT / 32];
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double bi = b[i], zi = dinv[i] * bi;
        k[i] = 0.0;
        r[i] = bi;
        z[i] = zi;
        p[i] = zi;
        s += bi * zi;
    }
    s = block_sum(s, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void k_cg_start(const double *__restrict__ part, int nb, double rtol, CgState *st)
{
    __shared__ double sh[VT / 32];
    double s = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) s += part[i];
    s = block_sum(s, sh);
    if (threadIdx.x == 0) {
        st->rz = s;
        st->rz_stop = rtol * rtol * s;
        st->stop = (s > st->rz_stop && s > 0.0) ? INT_MAX : 0;
        st->its = 0;
        st->alpha = st->beta = 0.0;
    }
}

// Mp = assembly of the one-component element vectors ev (fixed entry order,
// no fixed DOFs) and the partial p.Mp, in one pass
__global__ void k_cg_assemble_dot(const double *__restrict__ ev, const int32_t *__restrict__ ptr,
                                  const int32_t *__restrict__ idx, int64_t n,
                                  const double *__restrict__ p, double *__restrict__ q,
                                  double *__restrict__ part, const CgState *__restrict__ st, int kk)
{
    if (st->stop < kk) return;
    __shared__ double sh[VT / 32];
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int b = ptr[i], e = ptr[i + 1];
        double a = 0.0;
        for (int j = b; j < e; ++j) a += __ldg(ev + __ldg(idx + j));
        q[i] = a;
        s += p[i] * a;
    }
    s = block_sum(s, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// alpha = r.z / p.Mp; a non-positive p.Mp (mass operator of an inverted
// mesh) ends the solve before the update
__global__ void k_cg_alpha(const double *__restrict__ part, int nb, CgState *st, int kk)
{
    if (st->stop < kk) return;
    __shared__ double sh[VT / 32];
    double s = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) s += part[i];
    s = block_sum(s, sh);
    if (threadIdx.x == 0) {
        if (s > 0.0) {
            st->alpha = st->rz / s;
        } else {
            st->alpha = 0.0;
            st->stop = kk - 1;
        }
    }
}

// k += alpha p, r -= alpha Mp, z = dinv r; partial r.z
__global__ void k_cg_update(double *__restrict__ k, double *__restrict__ r, double *__restrict__ z,
                            const double *__restrict__ p, const double *__restrict__ q,
                            const double *__restrict__ dinv, int64_t n, double *__restrict__ part,
                            const CgState *__restrict__ st, int kk)
{
    if (st->stop < kk) return;
    __shared__ double sh[VT / 32];
    const double a = st->alpha;
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        k[i] += a * p[i];
        const double ri = r[i] - a * q[i];
        const double zi = dinv[i] * ri;
        r[i] = ri;
        z[i] = zi;
        s += ri * zi;
    }
    s = block_sum(s, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// new r.z, beta, convergence (or the iteration cap) -> stop = kk
__global__ void k_cg_beta(const double *__restrict__ part, int nb, CgState *st, int kk, int max_it)
{
    if (st->stop < kk) return;
    __shared__ double sh[VT / 32];
    double s = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) s += part[i];
    s = block_sum(s, sh);
    if (threadIdx.x == 0) {
        st->beta = s / st->rz;
        st->rz = s;
        st->its = kk;
        if (!(s > st->rz_stop) || !(s > 0.0) || kk >= max_it) st->stop = kk;
    }
}

// p = z + beta p
__global__ void k_cg_dir(double *__restrict__ p, const double *__restrict__ z, int64_t n,
                         const CgState *__restrict__ st, int kk)
{
    if (st->stop <= kk) return;         // no further iteration uses p
    const double b = st->beta;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = z[i] + b * p[i];
}

// out = u + c k
__global__ void k_axpy(const double *__restrict__ u, const double *__restrict__ k, double c, int64_t n,
                       double *__restrict__ out)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = u[i] + c * k[i];
}

// u += dt/6 (k1 + 2 k2 + 2 k3 + k4)
__global__ void k_rk4_combine(double *__restrict__ u, const double *__restrict__ k1,
                              const double *__restrict__ k2, const double *__restrict__ k3,
                              const double *__restrict__ k4, double dt, int64_t n)
{
    const double h = dt / 6.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        u[i] += h * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]);
}

__global__ void k_recip(const double *__restrict__ d, int64_t n, double *__restrict__ out)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = 1.0 / d[i];
}

// acc = min(acc, min over the (sum, min) pairs of part); reset: acc = min over part
__global__ void k_min_accum(const double *__restrict__ part, int64_t nb, double *acc, int reset)
{
    __shared__ double shm[VT / 32];
    double m = INFINITY;
    for (int64_t i = threadIdx.x; i < nb; i += blockDim.x) m = fmin(m, part[2 * i + 1]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmin(m, __shfl_down_sync(0xffffffffu, m, o));
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) shm[wid] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) m = fmin(m, shm[i]);
        *acc = reset ? m : fmin(*acc, m);
    }
}

}  // namespace

int reduce_blocks(int64_t n) { return (int)grid_for(n); }

cudaError_t launch_assemble(const void *ev, int ev_prec, const int32_t *ptr, const int32_t *idx,
                            const uint8_t *fixed, const void *vfix, int mode, int64_t Nx, int D,
                            int64_t ENP, void *out, int out_prec, const int *stop, int k,
                            cudaStream_t s)
{
    if (Nx == 0) return cudaSuccess;
    const unsigned g = (unsigned)((Nx + VT - 1) / VT);
    if (ev_prec == TMOP_FP64 && out_prec == TMOP_FP64)
        k_assemble<double, double><<<g, VT, 0, s>>>((const double *)ev, ptr, idx, fixed,
                                                    (const double *)vfix, mode, Nx, D, ENP,
                                                    (double *)out, stop, k);
    else if (ev_prec == TMOP_FP32 && out_prec == TMOP_FP32)
        k_assemble<float, float><<<g, VT, 0, s>>>((const float *)ev, ptr, idx, fixed,
                                                  (const float *)vfix, mode, Nx, D, ENP,
                                                  (float *)out, stop, k);
    else if (ev_prec == EV_DF_PAIR && out_prec == TMOP_FP64)
        k_assemble<df, double><<<g, VT, 0, s>>>((const df *)ev, ptr, idx, fixed,
                                                (const double *)vfix, mode, Nx, D, ENP,
                                                (double *)out, stop, k);
    else
        return cudaErrorInvalidValue;
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_mask(const void *v, const uint8_t *fixed, int64_t n, void *out, int prec,
                        cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    if (prec == TMOP_FP32)
        k_mask<float><<<grid_for(n), VT, 0, s>>>((const float *)v, fixed, n, (float *)out);
    else
        k_mask<double><<<grid_for(n), VT, 0, s>>>((const double *)v, fixed, n, (double *)out);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_trial(const double *x, const double *dx, double alpha, int64_t n, double *out,
                         cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    k_trial<<<grid_for(n), VT, 0, s>>>(x, dx, alpha, n, out);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_differs(const double *a, const double *b, int64_t n, double *flag, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(flag, 0, sizeof(double), s);
    if (e != cudaSuccess || n == 0) return e;
    k_differs<<<grid_for(n), VT, 0, s>>>(a, b, n, flag);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_dot(const void *a, const void *b, int prec, int64_t n, double *part, int nb,
                       cudaStream_t s)
{
    if (prec == TMOP_FP32)
        k_dot<float><<<nb, VT, 0, s>>>((const float *)a, (const float *)b, n, part);
    else
        k_dot<double><<<nb, VT, 0, s>>>((const double *)a, (const double *)b, n, part);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_finalize_sum(const double *part, int nb, double *out, cudaStream_t s)
{
    k_finalize_sum<<<1, VT, 0, s>>>(part, nb, out);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_finalize_energy(const double *part, int64_t nb, double *out, cudaStream_t s)
{
    k_finalize_energy<<<1, VT, 0, s>>>(part, nb, out);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_jacobi(const void *diag, int prec, int64_t n, void *minv, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    if (prec == TMOP_FP32)
        k_jacobi<float><<<grid_for(n), VT, 0, s>>>((const float *)diag, n, (float *)minv);
    else
        k_jacobi<double><<<grid_for(n), VT, 0, s>>>((const double *)diag, n, (double *)minv);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_minres_init(const double *b, const void *minv, int prec, int64_t n, void *r1,
                               void *r2, void *y, double *part, int nb, cudaStream_t s)
{
    if (prec == TMOP_FP32)
        k_minres_init<float><<<nb, VT, 0, s>>>(b, (const float *)minv, n, (float *)r1, (float *)r2,
                                              (float *)y, part);
    else
        k_minres_init<double><<<nb, VT, 0, s>>>(b, (const double *)minv, n, (double *)r1,
                                               (double *)r2, (double *)y, part);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_minres_start(const double *part, int nb, MinresState *st, int, cudaStream_t s)
{
    k_minres_start<<<1, VT, 0, s>>>(part, nb, st);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_minres_scale(const void *y, const MinresState *st, int prec, int64_t n, void *v,
                                cudaStream_t s)
{
    if (prec == TMOP_FP32)
        k_minres_scale<float><<<grid_for(n), VT, 0, s>>>((const float *)y, st, n, (float *)v);
    else
        k_minres_scale<double><<<grid_for(n), VT, 0, s>>>((const double *)y, st, n, (double *)v);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_lanczos_a(void *z, const void *r1, const void *v, const MinresState *st,
                             int prec, int64_t n, int k, double *part, int nb, cudaStream_t s)
{
    if (prec == TMOP_FP32)
        k_lanczos_a<float><<<nb, VT, 0, s>>>((float *)z, (const float *)r1, (const float *)v, st, n,
                                            k, part);
    else
        k_lanczos_a<double><<<nb, VT, 0, s>>>((double *)z, (const double *)r1, (const double *)v,
                                             st, n, k, part);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_assemble_lanczos_a(const void *ev, const int32_t *ptr, const int32_t *idx,
                                      const uint8_t *fixed, int64_t Nx, int D, int64_t ENP, void *y,
                                      const void *r1, const void *v, const MinresState *st, int prec,
                                      int k, double *part, int nb, cudaStream_t s)
{
    if (prec == TMOP_FP32)
        k_assemble_lanczos_a<float, float><<<nb, VT, 0, s>>>(
            (const float *)ev, ptr, idx, fixed, Nx, D, ENP, (float *)y, (const float *)r1,
            (const float *)v, st, k, part);
    else if (prec == EV_DF_PAIR)                      // float-pair entries, FP64 vectors
        k_assemble_lanczos_a<df, double><<<nb, VT, 0, s>>>(
            (const df *)ev, ptr, idx, fixed, Nx, D, ENP, (double *)y, (const double *)r1,
            (const double *)v, st, k, part);
    else
        k_assemble_lanczos_a<double, double><<<nb, VT, 0, s>>>(
            (const double *)ev, ptr, idx, fixed, Nx, D, ENP, (double *)y, (const double *)r1,
            (const double *)v, st, k, part);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_iter_next(MinresState *st, cudaStream_t s)
{
    k_iter_next<<<1, 1, 0, s>>>(st);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_fin_alpha(const double *part, int nb, MinresState *st, int k, cudaStream_t s)
{
    k_fin_alpha<<<1, VT, 0, s>>>(part, nb, st, k);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_lanczos_b(void *y, const void *r2, const void *minv, const MinresState *st,
                             int prec, int64_t n, int k, void *ynew, double *part, int nb,
                             cudaStream_t s)
{
    if (prec == TMOP_FP32)
        k_lanczos_b<float><<<nb, VT, 0, s>>>((float *)y, (const float *)r2, (const float *)minv, st,
                                            n, k, (float *)ynew, part);
    else
        k_lanczos_b<double><<<nb, VT, 0, s>>>((double *)y, (const double *)r2,
                                             (const double *)minv, st, n, k, (double *)ynew, part);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_fin_beta(const double *part, int nb, MinresState *st, int k, double rtol,
                            int fixed_its, cudaStream_t s)
{
    k_fin_beta<<<1, VT, 0, s>>>(part, nb, st, k, rtol, fixed_its);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_minres_update(void *v, const void *w1, const void *w2, void *wnew, double *dx,
                                 const void *ynew, const MinresState *st, int prec, int64_t n,
                                 int k, cudaStream_t s)
{
    if (prec == TMOP_FP32)
        k_minres_update<float><<<grid_for(n), VT, 0, s>>>((float *)v, (const float *)w1,
                                                         (const float *)w2, (float *)wnew, dx,
                                                         (const float *)ynew, st, n, k);
    else
        k_minres_update<double><<<grid_for(n), VT, 0, s>>>((double *)v, (const double *)w1,
                                                          (const double *)w2, (double *)wnew, dx,
                                                          (const double *)ynew, st, n, k);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_cg_init(const double *b, const double *dinv, int64_t n, double *k, double *r,
                           double *z, double *p, double *part, int nb, double rtol, CgState *st,
                           cudaStream_t s)
{
    k_cg_init<<<nb, VT, 0, s>>>(b, dinv, n, k, r, z, p, part);
    k_cg_start<<<1, VT, 0, s>>>(part, nb, rtol, st);
    count_launch(2);
    return cudaGetLastError();
}

cudaError_t launch_cg_iter(const double *ev, const int32_t *ptr, const int32_t *idx, double *p,
                           double *Mp, double *k, double *r, double *z, const double *dinv, int64_t n,
                           double *part, int nb, CgState *st, int kk, int max_it, cudaStream_t s)
{
    k_cg_assemble_dot<<<nb, VT, 0, s>>>(ev, ptr, idx, n, p, Mp, part, st, kk);
    k_cg_alpha<<<1, VT, 0, s>>>(part, nb, st, kk);
    k_cg_update<<<nb, VT, 0, s>>>(k, r, z, p, Mp, dinv, n, part, st, kk);
    k_cg_beta<<<1, VT, 0, s>>>(part, nb, st, kk, max_it);
    k_cg_dir<<<nb, VT, 0, s>>>(p, z, n, st, kk);
    count_launch(5);
    return cudaGetLastError();
}

cudaError_t launch_axpy(const double *u, const double *k, double c, int64_t n, double *out,
                        cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    k_axpy<<<grid_for(n), VT, 0, s>>>(u, k, c, n, out);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_rk4_combine(double *u, const double *k1, const double *k2, const double *k3,
                               const double *k4, double dt, int64_t n, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    k_rk4_combine<<<grid_for(n), VT, 0, s>>>(u, k1, k2, k3, k4, dt, n);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_recip(const double *d, int64_t n, double *out, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    k_recip<<<grid_for(n), VT, 0, s>>>(d, n, out);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_min_accum(const double *part, int64_t nb, double *acc, int reset, cudaStream_t s)
{
    k_min_accum<<<1, VT, 0, s>>>(part, nb, acc, reset);
    count_launch();
    return cudaGetLastError();
}

}  // namespace tmop
