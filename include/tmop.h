/*
 * tmop.h: C ABI of the B300 (sm_103a) TMOP partial-assembly library.
 *
 * The library computes the data-parallel hot path of the target-matrix
 * optimization paradigm (TMOP) for high-order quadrilateral (2D) and
 * hexahedral (3D) meshes of order p = 1..4, as described in "Accelerating
 * High-Order Mesh Optimization Using Finite Element Partial Assembly on
 * GPUs" (Camier et al.):
 *   - Jacobians A = sum_i x_{E,i} grad(w_i)^T at the quadrature points by
 *     sum factorisation, T = A W^-1 (Sec. 2.2 eq. A and eq. T, Sec. 3.2);
 *   - the energy F = sum_E sum_q w_q det(W) mu(T) (eq. F_full, Sec. 3.3);
 *   - its nodal gradient dF/dx (eq. vm_pa_grad, Sec. 3.3);
 *   - partial assembly of d2mu/dT2 at every quadrature point, the Hessian
 *     action and its diagonal (eq. vm_pa_hess, Sec. 3.4);
 *   - the Newton step with Jacobi-preconditioned MINRES and the backtracking
 *     line search that keeps det(A) > 0 (Sec. 2.3, eq. nodal_solve/dx).
 *
 * Conventions shared by every call
 *   - Every array argument is a DEVICE pointer unless marked "host".  The
 *     caller owns every array it passes; the context owns everything it
 *     allocates (stored Hessian data, tables, maps, work vectors) and frees it
 *     in tmop_destroy.
 *   - Positions and vectors are component-major: x[a * num_nodes + node],
 *     length dim * num_nodes ("DOF" = dim * num_nodes, the paper's count of
 *     unique degrees of freedom, Sec. 4.1 table).
 *   - elem_to_node is num_elems x (order+1)^dim int32 in lexicographic local
 *     order i = i1 + (p+1) i2 + (p+1)^2 i3 (Sec. 3.1).
 *   - Reference element [0,1]^dim, Gauss-Legendre quadrature with nq1d points
 *     per direction, Lagrange basis on Gauss-Lobatto-Legendre nodes.
 *   - All work is enqueued on the stream given to tmop_setup.  Calls that
 *     return host scalars synchronise that stream; the others do not.
 *   - No call aborts or traps: each returns a tmop_status, and
 *     tmop_last_error() gives a one-line description of the last failure on
 *     the calling thread.
 *   - A context is not thread-safe; use one context per host thread.
 */
#ifndef TMOP_H
#define TMOP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    TMOP_OK = 0,
    TMOP_ERR_ARG = 1,          /* invalid argument or unsupported size */
    TMOP_ERR_INVERTED = 2,     /* det(A) <= 0 at some quadrature point */
    TMOP_ERR_CUDA = 3,         /* a CUDA runtime call failed */
    TMOP_ERR_OOM = 4,          /* device allocation failed */
    TMOP_ERR_MINRES = 5,       /* MINRES breakdown */
    TMOP_ERR_LINESEARCH = 6,   /* no step length passed the line search */
    TMOP_ERR_TIMEOUT = 7,      /* a bounded device wait gave up */
    TMOP_ERR_UNSUPPORTED = 8   /* (dim, order, nq1d, metric) not built */
} tmop_status;

/* Quality metrics (Sec. 2.2; mu_303 in Sec. 4.1).  T = A W^-1, tau = det T.
 *   TMOP_METRIC_2     (2D) mu = |T|^2 / (2 tau) - 1                 shape
 *   TMOP_METRIC_302   (3D) mu = |T|^2 |T^-1|^2 / 9 - 1              shape
 *   TMOP_METRIC_303   (3D) mu = |T|^2 / (3 tau^(2/3)) - 1            shape
 *   TMOP_METRIC_55    (2D/3D) mu = (tau - 1)^2                       size
 *   TMOP_METRIC_303_55 (3D) mu_303 + mu_55                          shape+size
 *   TMOP_METRIC_7     (2D/3D) mu = |T - T^-t|^2                      shape+size
 *   TMOP_METRIC_9     (2D/3D) mu = tau |T - T^-t|^2                  shape+size */
enum { TMOP_METRIC_2 = 2, TMOP_METRIC_7 = 7, TMOP_METRIC_9 = 9, TMOP_METRIC_55 = 55,
       TMOP_METRIC_302 = 302, TMOP_METRIC_303 = 303, TMOP_METRIC_303_55 = 30355 };

/* Targets W (eq. W).  IDENTITY: W = I.  SIZE_FIELD: W = h0 s(x)^(1/dim) I
 * with s(x) = 1 + 0.5 prod_k sin(2 pi x_k) evaluated at the current physical
 * quadrature point; W is recomputed whenever positions change and dW/dx is
 * not differentiated (Sec. 3.6).  DISCRETE: W = h0 eta(x_q)^(1/dim) I with
 * eta a finite element field of the mesh's own space (nodal values, one per
 * node), interpolated to the points by the same contractions as the
 * positions (Sec. 3.6); eta is set by tmop_set_target_field, or remapped to
 * every new position by tmop_newton_step after tmop_set_remap_source.  A
 * point with eta(x_q) <= 0 has no target and counts as inverted. */
enum { TMOP_TARGET_IDENTITY = 0, TMOP_TARGET_SIZE_FIELD = 1, TMOP_TARGET_DISCRETE = 2 };

/* Precision of the stored d2mu/dT2 data, the Hessian action, its diagonal
 * and the inner MINRES vectors.  Energy, gradient, det(A), the line search
 * and the outer convergence test always have FP64 inputs, outputs and
 * accuracy.
 *   TMOP_FP64         FP64 vectors; contractions and stored data in
 *                     double-float pairs on the FP32 units (48-bit
 *                     significand, relative rounding ~4e-15), because B300
 *                     issues FP64 arithmetic ~60x slower than FP32.
 *   TMOP_FP32         FP32 stored data, action, diagonal and Krylov vectors;
 *                     energy/gradient/setup contractions in double-float.
 *   TMOP_FP64_NATIVE  every contraction on the FP64 units (reference path). */
enum { TMOP_FP64 = 0, TMOP_FP32 = 1, TMOP_FP64_NATIVE = 2 };

typedef struct {
    int dim;             /* 2 or 3 */
    int order;           /* p, 1..4 */
    int nq1d;            /* quadrature points per direction: p+1, p+2, or 9 (3D) */
    int64_t num_elems;
    int64_t num_nodes;   /* N_x */
    int metric;          /* TMOP_METRIC_* valid for dim */
    int target;          /* TMOP_TARGET_* */
    double target_h0;    /* h0 of the size and discrete targets (ignored for IDENTITY) */
    int hess_precision;  /* TMOP_FP64, TMOP_FP32 or TMOP_FP64_NATIVE */
    double limit_delta;  /* > 0: add the limiting term |x - x0|^2 / delta^2 (Sec. 3.5,
                            eq. F_full); x0 is given by tmop_set_limit_reference.  0: off */
} tmop_desc;

typedef struct {
    double minres_rtol;     /* stop when ||r||_{M^-1} <= rtol ||b||_{M^-1} */
    int minres_max_it;      /* iteration cap (the paper uses 50, Sec. 4.1) */
    int minres_fixed_its;   /* 1: run exactly minres_max_it iterations */
    double ls_factor;       /* 1.2 in the paper (Sec. 2.3) */
    int ls_max_halvings;    /* alpha = 1, 1/2, ..., 2^-ls_max_halvings */
} tmop_solver_opts;

typedef struct {
    double energy;         /* F(x) before the step */
    double grad_norm;      /* |dF(x)| before the step (l2, free DOFs) */
    double energy_new;     /* F(x+) of the accepted step */
    double grad_norm_new;  /* |dF(x+)| of the accepted step */
    double alpha;          /* accepted step length (0 if none) */
    double min_det;        /* min det(A) over quadrature points of x+ */
    double minres_resid;   /* final ||r||_{M^-1} / ||b||_{M^-1} */
    int minres_iters;
    int halvings;
    int status;            /* tmop_status of the step */
} tmop_step_report;

typedef struct tmop_ctx tmop_ctx;

/* Build a context for one mesh (Sec. 2.1 mesh, Sec. 3 PA operator
 * decomposition): 1D tables B1D/G1D (eq. B_G_1D), a device copy of the
 * element-to-node map, and its transpose (node -> element entries) used for
 * the deterministic, atomics-free E-vector to L-vector assembly.
 *   desc          host; sizes and options (see tmop_desc).
 *   elem_to_node  device int32, num_elems * (order+1)^dim; copied.
 *   fixed         device uint8, dim * num_nodes (1 = Dirichlet DOF), or NULL
 *                 for none; copied.  The gradient is zero and the Hessian
 *                 row/column is the identity on fixed DOFs.
 *   cuda_stream   a cudaStream_t (NULL = legacy default stream).
 *   out           host; receives the context.
 * Errors: TMOP_ERR_ARG (bad sizes, map entry out of range),
 * TMOP_ERR_UNSUPPORTED, TMOP_ERR_OOM, TMOP_ERR_CUDA. */
tmop_status tmop_setup(const tmop_desc *desc, const int32_t *elem_to_node, const uint8_t *fixed,
                       void *cuda_stream, tmop_ctx **out);

/* Energy F(x) = 1^T D0(B G x) (Sec. 3.3, eq. D0_expression) and the minimum
 * of det(A) over all quadrature points.
 *   x        device FP64, dim * num_nodes.
 *   F        host; F(x), or +inf when the mesh is inverted.
 *   min_det  host (may be NULL); min over quadrature points of det(A).
 * Synchronises the stream.  Returns TMOP_ERR_INVERTED when min det <= 0. */
tmop_status tmop_energy(tmop_ctx *ctx, const double *x, double *F, double *min_det);

/* Gradient g = dF/dx (Sec. 3.3, eq. vm_pa_grad, general W: the quadrature
 * data is c_q P(T) W^-T with c_q = w_q det W), assembled to nodes, zero on
 * fixed DOFs.
 *   x  device FP64, dim * num_nodes;  g  device FP64, same length (output).
 * Asynchronous.  An inverted point contributes nothing; call tmop_energy to
 * detect inversion. */
tmop_status tmop_gradient(tmop_ctx *ctx, const double *x, double *g);

/* Partial-assembly setup (Sec. 3.4): store, at every quadrature point, the
 * A-space second derivative H_{ab,ce} = c_q sum_{n,f} d2mu/dT_an dT_cf
 * W^-1_bn W^-1_ef, d^4 values of which the d^2 (d^2+1)/2 symmetric ones are
 * kept, in the context's precision.  x: device FP64.  Asynchronous. */
tmop_status tmop_hessian_setup(tmop_ctx *ctx, const double *x);

/* Hessian action y = d2F v from the stored data (Sec. 3.4, eq. vm_pa_hess):
 * forward contractions B G v, pointwise H : dA, transposed contractions,
 * deterministic assembly.  Fixed DOFs: v is treated as zero there on input
 * and y = v there on output.
 *   v, y  device, dim * num_nodes, double* for TMOP_FP64 / TMOP_FP64_NATIVE
 *         contexts and float* for TMOP_FP32 contexts; must not alias.
 * Requires a previous tmop_hessian_setup.  Asynchronous. */
tmop_status tmop_hessian_apply(tmop_ctx *ctx, const void *v, void *y);

/* Diagonal of d2F from the stored data by tensor contractions (Sec. 3.4,
 * Jacobi preconditioning); 1 on fixed DOFs.
 *   diag  device, dim * num_nodes, double* (FP64 contexts) or float* (FP32).
 * Requires a previous tmop_hessian_setup.  Asynchronous. */
tmop_status tmop_hessian_diag(tmop_ctx *ctx, void *diag);

/* One Newton step (Sec. 2.3): dx = [d2F]^-1 dF by Jacobi-preconditioned
 * MINRES (x0 = 0, M^-1 = 1/|diag|), then x+ = x - alpha dx with alpha = 1,
 * 1/2, ... until det A(x+) > 0 at every point, F(x+) < ls_factor F(x) and
 * |dF(x+)| < ls_factor |dF(x)|.
 *   x     device FP64, dim * num_nodes; overwritten only by an accepted step.
 *   opts  host (NULL = rtol 1e-8, 50 iterations, factor 1.2, 20 halvings).
 *   rep   host (may be NULL).
 * Synchronises.  Returns TMOP_ERR_INVERTED if x is inverted,
 * TMOP_ERR_LINESEARCH if no step length passed (x unchanged),
 * TMOP_ERR_MINRES on breakdown.  A stationary x (dF = 0) returns TMOP_OK
 * with alpha = 0.  The energy, min det and gradient the line search computed
 * at the accepted positions are kept with a copy of them: the next step
 * takes them instead of evaluating again when its x is bitwise equal to
 * that copy (one compare pass over x) and no call that changes the energy
 * (tmop_set_limit_reference, tmop_set_target_field, tmop_set_remap_source)
 * came in between; steps with a remap source always evaluate.  The same
 * kernels on the same input give the same bits, so results do not depend on
 * the reuse. */
tmop_status tmop_newton_step(tmop_ctx *ctx, double *x, const tmop_solver_opts *opts,
                             tmop_step_report *rep);
/* Number of Newton steps of this context that reused the evaluation at the
 * previous step's accepted positions (diagnostics). */
int64_t tmop_step_reuses(const tmop_ctx *ctx);

/* det(A) at every quadrature point of the mesh x (Sec. 2.2, eq. A:
 * A = sum_i x_{E,i} grad(w_i)^T, the Jacobian of the reference-to-physical
 * map; det A > 0 everywhere is the validity condition that the line search of
 * Sec. 2.3 enforces).  A diagnostic export of the quantity whose minimum
 * tmop_energy returns.
 *   x    device FP64, dim * num_nodes.
 *   det  device FP64, num_elems * nq1d^dim, caller-owned:
 *        det[e * nq1d^dim + q] with q = q1 + nq1d q2 (+ nq1d^2 q3), the
 *        lexicographic point index.  Computed as det(T) det(W) from the FP64
 *        invariants of T = A W^-1 (W = I for the identity target).
 * Asynchronous.  Errors: TMOP_ERR_ARG (NULL pointer, discrete target without
 * a field). */
tmop_status tmop_det(tmop_ctx *ctx, const double *x, double *det);

/* Energy and min det(A) without allocating anything (the paper has no
 * counterpart: this exists for callers of this library that cannot call
 * cudaMalloc, e.g. code running inside an application whose memory pool has
 * claimed the device memory, or latency-bound loops where cudaMalloc/cudaFree
 * would synchronise the device).  It computes what tmop_energy computes, with
 * no context: the per-CTA partial sums and the 1D basis tables live in one
 * file-scope device array of about 1 MiB (65,536 partial pairs + the tables of
 * every supported (order, nq1d)), which every GPU that loads the library
 * holds until the process exits.
 *   desc          host; sizes, metric and target as for tmop_setup;
 *                 hess_precision selects the contraction arithmetic as there
 *                 (TMOP_FP64_NATIVE: FP64 units; otherwise double-float).
 *   elem_to_node  device int32, num_elems * (order+1)^dim, in range (not checked).
 *   x             device FP64, dim * num_nodes.
 *   out           device FP64[2]; receives F(x) and min det(A).  F is the sum
 *                 over points with det A > 0: check out[1] > 0 (otherwise the
 *                 mesh is inverted and F is meaningless).
 *   cuda_stream   stream of the two launches.
 * Meshes needing more than 65,536 CTAs (e.g. more than 524,288 elements for
 * 3D p = 3 with 4^3 points) are rejected with TMOP_ERR_ARG before anything
 * is launched; use tmop_energy.  The first call on a device looks up the
 * array's device address and writes the tables into it with one synchronous
 * copy (once per device, with that device current); make that first call
 * before any stream capture.  Every later call is asynchronous: two kernel
 * launches on cuda_stream, no copy.  All calls share the array and it keeps
 * the last call's partial sums; every value a call reads is written by that
 * call (or is a table), so nothing is cleared.  Calls that overlap on the
 * GPU (different streams, or different host threads) race on the partial
 * sums.  Never calls cudaMalloc, cudaFree or any allocating routine. */
tmop_status tmop_energy_noalloc(const tmop_desc *desc, const int32_t *elem_to_node,
                                const double *x, double *out, void *cuda_stream);

/* ---- Batches of meshes (many small problems in shared launches) --------
 * A batch holds up to max_meshes independent meshes that share dim, order,
 * nq1d, metric, target and precision but not their sizes.  Each mesh keeps
 * its own resident state (positions, map, stored Hessian data, Krylov
 * vectors) on the device; tmop_batch_step runs one Newton step (Sec. 2.3) of
 * every active mesh with shared kernel launches over all of their elements
 * and DOFs, with per-mesh scalars, per-mesh MINRES recurrences and per-mesh
 * line searches.  A mesh stops when |dF(x)|/|dF(x0)| <= newton_rtol, after
 * newton_max_it steps, or on an error (its status).  Meshes can be added and
 * removed between steps (continuous batching).  A mesh's results do not
 * depend on the other meshes of the batch (per-mesh reductions in a fixed
 * order). */
typedef struct {
    int dim, order, nq1d, metric, target, hess_precision;
    int max_meshes;              /* slot capacity */
    tmop_solver_opts solver;     /* MINRES and line-search options */
    double newton_rtol;          /* stop when |dF| <= newton_rtol |dF(x0)| */
    int newton_max_it;           /* Newton step cap per mesh */
} tmop_batch_desc;

typedef struct {
    int done;          /* 1 when the mesh needs no more steps */
    int status;        /* tmop_status of the mesh (TMOP_OK if converged or capped) */
    int newton_its;    /* accepted Newton steps */
    int minres_its;    /* total MINRES iterations */
    double energy0, energy, grad_norm0, grad_norm, min_det, alpha;
} tmop_mesh_state;

typedef struct tmop_batch tmop_batch;

/* Create an empty batch working on the given stream.  Errors as tmop_setup. */
tmop_status tmop_batch_create(const tmop_batch_desc *desc, void *cuda_stream, tmop_batch **out);

/* Add a mesh: elem_to_node (device int32), fixed (device uint8 dim*num_nodes
 * or NULL) and the initial positions x (device FP64) are copied into a new
 * device slab owned by the batch; target_h0 is the mesh's size-target scale.
 * slot (host) receives its handle.  Synchronises the stream.  Errors:
 * TMOP_ERR_ARG (full batch, bad map), TMOP_ERR_OOM. */
tmop_status tmop_batch_add(tmop_batch *b, int64_t num_elems, int64_t num_nodes,
                           const int32_t *elem_to_node, const uint8_t *fixed, const double *x,
                           double target_h0, int *slot);

/* One Newton step of every active mesh.  n_active (host, may be NULL)
 * receives the number of meshes still active afterwards.  Synchronises. */
tmop_status tmop_batch_step(tmop_batch *b, int *n_active);

/* State of one mesh after the last step (host struct). */
tmop_status tmop_batch_state(tmop_batch *b, int slot, tmop_mesh_state *st);

/* Copy a mesh's current positions to x_out (device FP64, dim*num_nodes);
 * asynchronous on the batch stream. */
tmop_status tmop_batch_positions(tmop_batch *b, int slot, double *x_out);

/* Free a mesh's slab and its slot (between steps). */
tmop_status tmop_batch_remove(tmop_batch *b, int slot);

/* Device bytes a mesh of this size would take in this batch, and the bytes
 * the batch holds now (for admission by a memory budget). */
int64_t tmop_batch_mesh_bytes(const tmop_batch *b, int64_t num_elems, int64_t num_nodes);
int64_t tmop_batch_device_bytes(const tmop_batch *b);

/* Free the batch and all its meshes.  NULL is accepted. */
void tmop_batch_destroy(tmop_batch *b);

/* Reference positions x0 of the limiting term xi = |x - x0|^2 / delta^2
 * (paper Sec. 3.5; its Hessian is the mass-like operator of eq.
 * pa_limiting).  x0: device FP64, dim * num_nodes; copied.  Required before
 * any evaluation of a context created with limit_delta > 0; TMOP_ERR_ARG
 * for a context without the term.  Asynchronous. */
tmop_status tmop_set_limit_reference(tmop_ctx *ctx, const double *x0);

/* ---------------------------------------------------------------------------
 * Adaptive discrete target and its advection remap (Sec. 3.6).
 *
 * eta is known on positions x0; its values on positions x1 follow from the
 * pseudo-time advection d eta/dt = v . grad eta, v = x1 - x0,
 * x_t = x0 + t v, t in [0, 1], discretised by Galerkin in the mesh's space:
 *     M(x_t) d eta/dt = K(x_t) eta,  M_ij = int w_i w_j,
 *     K_ij = int w_i v . grad w_j  (on the mesh x_t, the mesh's quadrature),
 * with the partially assembled mass and advection operators (w_q det A_q
 * and w_q adj(A_q) v_q stored per point) and classical RK4 with `steps`
 * uniform steps; every stage solves M k = K eta by Jacobi-preconditioned CG
 * from k = 0, stopping when sqrt(r.z) <= cg_rtol sqrt(b.z0) or after
 * cg_max_it iterations.  All arithmetic runs on the device; the host reads
 * the CG stop flag once per chunk of iterations.
 * --------------------------------------------------------------------------- */
typedef struct {
    int steps;           /* RK4 steps, >= 1 */
    double cg_rtol;      /* relative preconditioned residual of the mass solves */
    int cg_max_it;       /* >= 1 */
} tmop_remap_opts;

typedef struct {
    int cg_iters;        /* CG iterations over all stages */
    int solves;          /* mass solves (4 per step) */
    double min_det;      /* min det A over the intermediate meshes x_t */
    int status;          /* tmop_status */
} tmop_remap_report;

/* The field eta of a TMOP_TARGET_DISCRETE context on the current mesh.
 * eta: device FP64, num_nodes values; copied.  Asynchronous.  TMOP_ERR_ARG
 * for a context with another target. */
tmop_status tmop_set_target_field(tmop_ctx *ctx, const double *eta);

/* Remap source of a TMOP_TARGET_DISCRETE context: eta0 given on positions
 * x0 (device FP64, num_nodes and dim * num_nodes values; copied).  From now
 * on tmop_newton_step remaps eta from (x0, eta0) to x at its start and to
 * every line-search trial (a trial whose intermediate mesh inverts is
 * rejected); the field of the accepted positions stays in the context.
 * eta0 = NULL switches the remap off.  opts NULL: {4, 1e-12, 200}. */
tmop_status tmop_set_remap_source(tmop_ctx *ctx, const double *x0, const double *eta0,
                                  const tmop_remap_opts *opts);

/* eta1 = eta0 remapped from positions x0 to x1 on this context's mesh (any
 * target).  Device FP64 pointers: x0, x1 dim * num_nodes; eta0, eta1
 * num_nodes (eta1 may equal eta0).  Synchronous.  rep may be NULL.  Errors:
 * TMOP_ERR_ARG, TMOP_ERR_INVERTED (det A <= 0 on some x_t; eta1 undefined),
 * TMOP_ERR_OOM / TMOP_ERR_CUDA. */
tmop_status tmop_remap(tmop_ctx *ctx, const double *x0, const double *x1, const double *eta0,
                       double *eta1, const tmop_remap_opts *opts, tmop_remap_report *rep);

/* Free the context and everything it owns.  NULL is accepted. */
void tmop_destroy(tmop_ctx *ctx);

/* Static string for a status code. */
const char *tmop_status_string(tmop_status st);

/* Description of the last failure on the calling thread ("" if none). */
const char *tmop_last_error(void);

/* ---- Instrumentation (not part of the paper's method) ------------------ */

/* Number of kernels this library has launched since load (all contexts). */
int64_t tmop_launch_count(void);

/* Kernel classes for per-class device timing. */
enum { TMOP_K_ENERGY = 0, TMOP_K_GRADIENT = 1, TMOP_K_HSETUP = 2, TMOP_K_APPLY = 3,
       TMOP_K_DIAG = 4, TMOP_K_ASSEMBLE = 5, TMOP_K_VECTOR = 6,
       TMOP_K_REMAP_SETUP = 7,   /* remap operator data at x_t (+ mass diagonal) */
       TMOP_K_MASS = 8,          /* remap mass action (element kernel) */
       TMOP_K_ADVECT = 9,        /* remap advection action (element kernel) */
       TMOP_K_NCLASS = 10 };

/* Enable (1) or disable (0) CUDA-event timing of every element kernel
 * launch on the context's stream, and reset the accumulated figures. */
tmop_status tmop_profile_enable(tmop_ctx *ctx, int on);

/* Run the MINRES iterations of tmop_newton_step as CUDA graphs (1, the
 * default) or as separate launches (0).  A graph holds 4 iterations (the
 * launches of an iteration read the iteration index from a device counter);
 * one graph per phase of the work-vector rotation is captured on first use
 * and replayed while its parameters (output vector, tolerance, kernel
 * variant, limiting term) stay the same.  Graphs are not used while
 * profiling is enabled.  When the context's stream is the legacy default
 * stream (which cannot be captured), the MINRES solve runs on a stream the
 * context creates, ordered after the work queued before the call and before
 * the work queued after it (events).  Results are the same either way (the
 * same kernels in the same order). */
tmop_status tmop_set_graphs(tmop_ctx *ctx, int on);
/* Number of MINRES graph launches of this context so far (diagnostics). */
int64_t tmop_graph_launches(const tmop_ctx *ctx);

/* Accumulated device time (ms) and launch count of one kernel class since
 * profiling was enabled.  Synchronises the stream. */
tmop_status tmop_profile_read(tmop_ctx *ctx, int kernel_class, double *total_ms,
                              int64_t *launches);

/* Bytes of device memory the context holds. */
int64_t tmop_device_bytes(const tmop_ctx *ctx);

/* ---- Vector algebra for a caller-driven Krylov iteration ---------------
 * The element-partitioned Newton step of several ranks (the P operator of
 * Sec. 3 applied per rank, interface sums between ranks; see dist.py) runs
 * its Jacobi-MINRES (Sec. 2.3) on the host, with these kernels for the
 * vector work on each rank's local DOFs.  Device FP64 arrays of n values,
 * enqueued on the context's stream; out may alias an input.
 *   tmop_vec_lincomb  out = a x + b y + c z  (y or z NULL: term absent)
 *   tmop_vec_mul      out = x .* y
 *   tmop_vec_dot      *out (host) = sum_i x_i y_i over the entries with
 *                     mask_i != 0 (mask: device uint8, or NULL for all);
 *                     a fixed summation order; synchronises.
 * Errors: TMOP_ERR_ARG for NULL inputs or n < 0. */
tmop_status tmop_vec_lincomb(tmop_ctx *ctx, int64_t n, double a, const double *x, double b,
                             const double *y, double c, const double *z, double *out);
tmop_status tmop_vec_mul(tmop_ctx *ctx, int64_t n, const double *x, const double *y, double *out);
tmop_status tmop_vec_dot(tmop_ctx *ctx, int64_t n, const double *x, const double *y,
                         const uint8_t *mask, double *out);

/* The Jacobi preconditioner of the Newton step's MINRES (Sec. 3.4):
 * minv_i = 1/|diag_i|, 1 where |diag_i| < 1e-300. */
tmop_status tmop_vec_jacobi(tmop_ctx *ctx, int64_t n, const double *diag, double *minv);

/* Interface-sum packing: dst[k] = src[idx[k]] (gather) and
 * dst[idx[k]] += vals[k] (scatter-add; the m indices must be distinct).
 * idx: device int32, m entries in range (not checked). */
tmop_status tmop_vec_gather(tmop_ctx *ctx, int64_t m, const int32_t *idx, const double *src,
                            double *dst);
tmop_status tmop_vec_scatter_add(tmop_ctx *ctx, int64_t m, const int32_t *idx, const double *vals,
                                 double *dst);

/* ---- Fault injection for the tests of the failure paths (host side) -----
 * No GPU fault is involved: the library pretends, on the host, that a
 * computation failed, and the tests check what the caller then sees. */
enum { TMOP_FAULT_NONE = 0, TMOP_FAULT_MINRES_BREAKDOWN = 1 };

/* The next Newton step of the context (tmop_inject_fault) or of one mesh of
 * a batch (tmop_batch_inject_fault) treats its MINRES solve, after running
 * it, as broken down (as if a preconditioned inner product had been negative
 * or not finite, which valid inputs never produce with M^-1 = 1/|diag|): the
 * step returns TMOP_ERR_MINRES with x unchanged; the batch mesh is retired
 * with that status, the other meshes are not affected.  Applies once;
 * TMOP_FAULT_NONE cancels.  TMOP_ERR_ARG for an unknown fault or slot. */
tmop_status tmop_inject_fault(tmop_ctx *ctx, int fault);
tmop_status tmop_batch_inject_fault(tmop_batch *b, int slot, int fault);

/* MINRES iterations of tmop_batch_step as CUDA graphs of 4 iterations (1,
 * the default) or separate launches (0), as tmop_set_graphs; a graph is
 * captured again when the stepped subset of meshes, its tile tables or the
 * kernel variant change.  No graphs on the legacy default stream. */
tmop_status tmop_batch_set_graphs(tmop_batch *b, int on);
/* Number of MINRES graph launches of this batch so far (diagnostics). */
int64_t tmop_batch_graph_launches(const tmop_batch *b);

/* ---- Kernel-variant autotuning (not part of the paper's method) ----------
 * The Hessian action (the dominant kernel, Sec. 3.4) has several kernel
 * variants for some configurations (3D with nq1d^2 <= 32): the
 * sum-factorised kernel (variant 0) and collocated-derivative kernels that
 * keep the per-point values in registers or shared memory, with 2, 4 or 8
 * warps per CTA.  All compute the same action.  A process-wide table gives
 * the variant per (dim, order, nq1d, precision); its defaults were measured
 * on a B300 by the autotuner, and every context and batch of the process
 * uses it at each launch.  Changing an entry while another host thread
 * launches actions of that configuration is allowed (the entry is atomic);
 * a launch uses the value it reads. */

/* Number of action variants of a configuration (1 = only variant 0; 0 =
 * unsupported configuration). */
int tmop_apply_variants(int dim, int order, int nq1d);

/* The variant in use for (dim, order, nq1d, precision), and its override
 * (variant -1 restores the measured default).  TMOP_ERR_ARG for an
 * unsupported configuration or a variant out of range. */
tmop_status tmop_get_apply_variant(int dim, int order, int nq1d, int precision, int *variant);
tmop_status tmop_set_apply_variant(int dim, int order, int nq1d, int precision, int variant);

/* Time every action variant on this context's own mesh and stored data
 * (reps launches each after one warm-up, CUDA events on the context's
 * stream, input vector zero), install the fastest in the process-wide table
 * and return it.  Requires a previous tmop_hessian_setup.
 *   variant  host (may be NULL): the chosen variant.
 *   ms       host (may be NULL): tmop_apply_variants(...) entries, the mean
 *            time of one launch of each variant.
 * Synchronises; overwrites the context's internal work vectors. */
tmop_status tmop_autotune(tmop_ctx *ctx, int reps, int *variant, double *ms);

#ifdef __cplusplus
}
#endif

#endif /* TMOP_H */
