// Internal declarations shared by the host code and the kernel launchers.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/tmop.h"

namespace tmop {

// Supported (dim, order, nq1d) triples: every p in 1..4 with nq1d in {p+1, p+2},
// and in 3D also nq1d = 9 (the 9^3-point rule of the paper's Kershaw runs).
#define TMOP_CONFIGS(X)                                                                    \
    X(2, 1, 2) X(2, 1, 3) X(2, 2, 3) X(2, 2, 4) X(2, 3, 4) X(2, 3, 5) X(2, 4, 5) X(2, 4, 6) \
    X(3, 1, 2) X(3, 1, 3) X(3, 2, 3) X(3, 2, 4) X(3, 3, 4) X(3, 3, 5) X(3, 4, 5) X(3, 4, 6) \
    X(3, 1, 9) X(3, 2, 9) X(3, 3, 9) X(3, 4, 9)
#define TMOP_KEY(d, p, q) ((d) * 100 + (p) * 10 + (q))

struct ElemParams;
struct BatchArgs;

// Arithmetic of the FP64-accuracy contractions (energy, gradient, setup).
enum { ARITH_DW = 0, ARITH_NATIVE = 1 };

// Element-vector format of the double-float Hessian action (TMOP_FP64): float
// pairs in 8-byte slots (dfloat.cuh, EvPair), an ev_prec of launch_assemble.
enum { EV_DF_PAIR = 16 };
// Values of stored d2mu/dT2 per element (Cfg::HST: ns entries at nqd points;
// in 3D with nq^2 <= 32, the entry-pair layout, rounded up to a multiple of 4).
inline int64_t h_stride(int d, int nq, int ns, int nqd)
{
    const int64_t n = (int64_t)ns * nqd;
    return (d == 3 && nq * nq <= 32) ? (n + 3) & ~(int64_t)3 : n;
}
// Element-vector format written by the Hessian action of a precision.
inline int action_ev_format(int hess_precision)
{
    return hess_precision == TMOP_FP64 ? (int)EV_DF_PAIR
                                       : (hess_precision == TMOP_FP32 ? (int)TMOP_FP32 : (int)TMOP_FP64);
}

// Element-kernel launchers (one translation unit each).  Return the launch
// error.  nblocks() is the grid size a launch over E elements uses.
int64_t elem_blocks(int d, int p, int q, int64_t E);
bool elem_supported(int d, int p, int q);
// B (optional): batched launch over ntiles (mesh, tile) CTAs; the pointer
// arguments are then taken from the per-mesh role buffers.
cudaError_t launch_energy(int d, int p, int q, const ElemParams &P, const double *x, double *part,
                          int arith, cudaStream_t s, const BatchArgs *B = nullptr, int64_t ntiles = 0);
// part != nullptr (or a batch aux role): fused energy + min det partials.
cudaError_t launch_gradient(int d, int p, int q, const ElemParams &P, const double *x, double *ev,
                            int arith, cudaStream_t s, const BatchArgs *B = nullptr,
                            int64_t ntiles = 0, double *part = nullptr);
cudaError_t launch_hsetup(int d, int p, int q, const ElemParams &P, const double *x, void *H,
                          int prec, cudaStream_t s, const BatchArgs *B = nullptr, int64_t ntiles = 0);
cudaError_t launch_apply(int d, int p, int q, const ElemParams &P, const void *v, const void *H,
                         void *ev, int prec, const int *stop_iter, int k, cudaStream_t s,
                         const BatchArgs *B = nullptr, int64_t ntiles = 0);
// Action kernel variants (elem_apply_impl.cuh): count for a configuration,
// the one in use for (config, precision), and its override (-1 = table default).
int apply_variant_count(int d, int p, int q);
int apply_variant(int d, int p, int q, int prec);
bool set_apply_variant(int d, int p, int q, int prec, int variant);
cudaError_t launch_diag(int d, int p, int q, const ElemParams &P, const void *H, void *ev, int prec,
                        cudaStream_t s, const BatchArgs *B = nullptr, int64_t ntiles = 0);

// Limiting term |x - x0|^2 / delta^2 (limit.cu); lim2 = 2 / delta^2.
cudaError_t launch_limit_eg(int d, int p, int q, const ElemParams &P, const double *x,
                            const double *x0, double lim2, double *part, double *ev, int arith,
                            cudaStream_t s);
cudaError_t launch_limit_setup(int d, int p, int q, const ElemParams &P, const double *x, double lim2,
                               double *cq, cudaStream_t s);
cudaError_t launch_limit_apply(int d, int p, int q, const ElemParams &P, const void *v,
                               const double *cq, void *ev, int prec, const int *stop, int k,
                               cudaStream_t s);
cudaError_t launch_limit_diag(int d, int p, int q, const ElemParams &P, const double *cq, void *ev,
                              int prec, cudaStream_t s);

// Advection remap of the discrete target field (remap.cu), arith as above.
cudaError_t launch_remap_setup(int d, int p, int q, const ElemParams &P, const double *x0,
                               const double *vel, double t, double *dm, double *dadv, double *part,
                               int arith, cudaStream_t s);
cudaError_t launch_mass_apply(int d, int p, int q, const ElemParams &P, const double *u,
                              const double *dm, double *ev, const int *stop, int kk, int arith,
                              cudaStream_t s);
cudaError_t launch_mass_diag(int d, int p, int q, const ElemParams &P, const double *dm, double *ev,
                             int arith, cudaStream_t s);
cudaError_t launch_adv_apply(int d, int p, int q, const ElemParams &P, const double *u,
                             const double *dadv, double *ev, int arith, cudaStream_t s);

// Host tables: Gauss-Legendre rule on [0,1], GLL nodes, Lagrange B/G.
void host_gauss_legendre(int n, double *x, double *w);
void host_gll_nodes(int n, double *x);
void host_basis_tables(int ni, int nq, double *B, double *G, double *w1d);
void host_colloc_deriv(int nq, double *D);

// MINRES scalar state kept on the device.
struct MinresState {
    double beta, beta_old, beta1, alpha, dbar, eps, eps_old, phibar, cs, sn, gamma, delta, phi;
    int stop_iter;   // first iteration after which nothing changes (INT_MAX while running)
    int k;           // the current iteration (device counter; follows stop_iter)
    int breakdown;
    int iters;
};
static_assert(offsetof(MinresState, k) == offsetof(MinresState, stop_iter) + sizeof(int),
              "iter_of reads the iteration counter right after the stop iteration");


// CG scalar state of one remap mass solve, kept on the device.
struct CgState {
    int stop;        // iterations done when the solve ended (INT_MAX while running)
    int its;
    double rz, rz_stop, alpha, beta;
};

// Vector / reduction launchers (vec_kernels.cu).
int reduce_blocks(int64_t n);
cudaError_t launch_assemble(const void *ev, int ev_prec, const int32_t *ptr, const int32_t *idx,
                            const uint8_t *fixed, const void *vfix, int mode, int64_t Nx, int D,
                            int64_t ENP, void *out, int out_prec, const int *stop, int k,
                            cudaStream_t s);
cudaError_t launch_mask(const void *v, const uint8_t *fixed, int64_t n, void *out, int prec,
                        cudaStream_t s);
cudaError_t launch_trial(const double *x, const double *dx, double alpha, int64_t n, double *out,
                         cudaStream_t s);
// *flag (device) = 1.0 when a and b differ bitwise in some entry, else 0.0.
cudaError_t launch_differs(const double *a, const double *b, int64_t n, double *flag, cudaStream_t s);
cudaError_t launch_dot(const void *a, const void *b, int prec, int64_t n, double *part, int nb,
                       cudaStream_t s);
cudaError_t launch_dot_masked(const double *a, const double *b, const uint8_t *mask, int64_t n,
                              double *part, int nb, cudaStream_t s);
cudaError_t launch_lincomb(int64_t n, double a, const double *x, double b, const double *y,
                           double c, const double *z, double *out, cudaStream_t s);
cudaError_t launch_vmul(int64_t n, const double *x, const double *y, double *out, cudaStream_t s);
cudaError_t launch_vgather(int64_t m, const int32_t *idx, const double *src, double *dst,
                           cudaStream_t s);
cudaError_t launch_vscatter_add(int64_t m, const int32_t *idx, const double *vals, double *dst,
                                cudaStream_t s);
cudaError_t launch_finalize_sum(const double *part, int nb, double *out, cudaStream_t s);
cudaError_t launch_finalize_energy(const double *part, int64_t nb, double *out, cudaStream_t s);
cudaError_t launch_jacobi(const void *diag, int prec, int64_t n, void *minv, cudaStream_t s);
cudaError_t launch_minres_init(const double *b, const void *minv, int prec, int64_t n, void *r1,
                               void *r2, void *y, double *part, int nb, cudaStream_t s);
cudaError_t launch_minres_start(const double *part, int nb, MinresState *st, int max_it,
                                cudaStream_t s);
cudaError_t launch_minres_scale(const void *y, const MinresState *st, int prec, int64_t n, void *v,
                                cudaStream_t s);
cudaError_t launch_lanczos_a(void *z, const void *r1, const void *v, const MinresState *st,
                             int prec, int64_t n, int k, double *part, int nb, cudaStream_t s);
// Assembly of the action's element vectors fused with launch_lanczos_a
// (y = z - (beta/beta_old) r1, partial dot(v, y) over nb blocks).
cudaError_t launch_assemble_lanczos_a(const void *ev, const int32_t *ptr, const int32_t *idx,
                                      const uint8_t *fixed, int64_t Nx, int D, int64_t ENP, void *y,
                                      const void *r1, const void *v, const MinresState *st, int prec,
                                      int k, double *part, int nb, cudaStream_t s);
cudaError_t launch_fin_alpha(const double *part, int nb, MinresState *st, int k, cudaStream_t s);
// st->k += 1: the start of a MINRES iteration whose launches take k = -1.
cudaError_t launch_iter_next(MinresState *st, cudaStream_t s);
cudaError_t launch_lanczos_b(void *y, const void *r2, const void *minv, const MinresState *st,
                             int prec, int64_t n, int k, void *ynew, double *part, int nb,
                             cudaStream_t s);
cudaError_t launch_fin_beta(const double *part, int nb, MinresState *st, int k, double rtol,
                            int fixed_its, cudaStream_t s);
cudaError_t launch_minres_update(void *v, const void *w1, const void *w2, void *wnew, double *dx,
                                 const void *ynew, const MinresState *st, int prec, int64_t n,
                                 int k, cudaStream_t s);

// Remap CG and RK4 vector kernels (vec_kernels.cu).  One CG iteration kk
// (1-based) is the mass action into element vectors ev (remap.cu) followed by
// launch_cg_iter (assembly of Mp fused with p.Mp, then the CG updates).
cudaError_t launch_cg_init(const double *b, const double *dinv, int64_t n, double *k, double *r,
                           double *z, double *p, double *part, int nb, double rtol, CgState *st,
                           cudaStream_t s);
cudaError_t launch_cg_iter(const double *ev, const int32_t *ptr, const int32_t *idx, double *p,
                           double *Mp, double *k, double *r, double *z, const double *dinv, int64_t n,
                           double *part, int nb, CgState *st, int kk, int max_it, cudaStream_t s);
cudaError_t launch_axpy(const double *u, const double *k, double c, int64_t n, double *out,
                        cudaStream_t s);
cudaError_t launch_rk4_combine(double *u, const double *k1, const double *k2, const double *k3,
                               const double *k4, double dt, int64_t n, cudaStream_t s);
cudaError_t launch_recip(const double *d, int64_t n, double *out, cudaStream_t s);
cudaError_t launch_min_accum(const double *part, int64_t nb, double *acc, int reset, cudaStream_t s);

// Global launch counter (instrumentation).
void count_launch(int n = 1);
// This thread's launch count, and the removal of n counted launches (the
// launches recorded by a graph capture are counted when the graph runs).
int64_t thread_launches();
void uncount_launches(int n);

// Text returned by tmop_last_error() on the calling thread.
void set_last_error(const std::string &msg);

}  // namespace tmop
