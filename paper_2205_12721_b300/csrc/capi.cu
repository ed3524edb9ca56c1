// C ABI of the TMOP partial-assembly library: context set-up, the seven
// entry points of the hot path and the host-driven Newton / MINRES loop.
// Every arithmetic step runs in the kernels of elem_*.cu and vec_kernels.cu;
// this file validates arguments, owns device memory and sequences launches.
#include <algorithm>
#include <atomic>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "tmop_device.cuh"
#include "tmop_internal.h"

using namespace tmop;

namespace {

thread_local std::string g_last_error;
std::atomic<int64_t> g_launches{0};
thread_local int64_t t_launches = 0;          // this thread's launches (graph node counts)

tmop_status fail(tmop_status st, const std::string &msg)
{
    g_last_error = msg;
    return st;
}

tmop_status cuda_fail(cudaError_t e, const char *where)
{
    g_last_error = std::string(where) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? TMOP_ERR_OOM : TMOP_ERR_CUDA;
}

#define CK(call)                                              \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);   \
    } while (0)

#define TRY(expr)                                 \
    do {                                          \
        tmop_status s_ = (expr);                  \
        if (s_ != TMOP_OK) return s_;             \
    } while (0)

struct ProfRec {
    int cls;
    cudaEvent_t a, b;
};

}  // namespace

namespace tmop {
void count_launch(int n)
{
    g_launches.fetch_add(n, std::memory_order_relaxed);
    t_launches += n;
}

int64_t thread_launches() { return t_launches; }

void uncount_launches(int n)
{
    g_launches.fetch_sub(n, std::memory_order_relaxed);
    t_launches -= n;
}
void set_last_error(const std::string &msg) { g_last_error = msg; }
}  // namespace tmop

struct tmop_ctx {
    tmop_desc desc{};
    int d = 0, p = 0, nq = 0, ni = 0, np = 0, nqd = 0, ns = 0, prec = 0;
    int vprec = 0;               // vector type of the action / MINRES: FP32 or FP64
    int arith = 0;               // ARITH_DW or ARITH_NATIVE for energy/gradient/setup
    int64_t E = 0, Nx = 0, ndof = 0, ENP = 0;
    size_t rsz = 8;
    cudaStream_t stream = nullptr;
    // mesh data
    int32_t *map = nullptr, *csr_ptr = nullptr, *csr_idx = nullptr;
    uint8_t *fixed = nullptr;
    double *tab = nullptr;
    float *tabf = nullptr;
    df *tabw = nullptr;
    // partial assembly data and element vectors
    void *H = nullptr;
    bool h_ready = false;
    double *ev64 = nullptr;
    void *evR = nullptr;
    // reductions
    double *part = nullptr;
    int64_t part_n = 0;
    double *scal = nullptr;      // device scalars
    double *hscal = nullptr;     // pinned host mirror
    // Newton / MINRES work
    double *g = nullptr, *dx = nullptr, *xt = nullptr;
    // F, min det and |g| at the positions the last Newton step accepted (kept
    // in xt, the gradient in g): the next step reuses them when its x equals
    // xt bitwise and nothing that defines the energy changed in between
    bool fg_valid = false;
    double fg_F = 0.0, fg_md = 0.0, fg_gn = 0.0;
    int64_t reused_fg = 0;             // steps that took them (tmop_step_reuses)
    void *vm = nullptr, *diagR = nullptr, *minv = nullptr;
    void *kv[8] = {nullptr};     // v, R1, R2, Z, W1, W2, W3, spare
    MinresState *st = nullptr, *hst = nullptr;
    int check_every = 4;
    // CUDA graphs of 4 MINRES iterations, one per phase of the 3-buffer
    // rotation (the 4-buffer rotation returns to its start every 4 iterations)
    bool graphs = true;
    int64_t graph_launches = 0;
    // the context's own stream for graph-captured solves when its stream is the
    // legacy default stream (which cannot be captured), and the handoff event
    cudaStream_t gstream = nullptr;
    cudaEvent_t gev = nullptr;
    struct MinresGraph {
        cudaGraphExec_t exec = nullptr;
        const double *dx = nullptr;
        double rtol = 0.0;
        int fixed_its = 0, variant = -1, lim = 0, nodes = 0;
    } mg[3];
    // limiting term
    double lim2 = 0.0;                 // 2 / delta^2, 0 when off
    double *x0 = nullptr, *lim_cq = nullptr, *part2 = nullptr;
    bool x0_set = false;
    // discrete target field and its remap (allocated on first use)
    double *eta = nullptr, *eta_t = nullptr;
    bool eta_set = false;
    int fault = TMOP_FAULT_NONE;     // host-side fault of the next Newton step (tests)
    double *rsrc_x0 = nullptr, *rsrc_eta0 = nullptr;
    bool remap_on = false;
    tmop_remap_opts remap_opts{4, 1e-12, 200};
    struct Remap {
        bool ready = false;
        double *vel = nullptr, *dm[2] = {nullptr, nullptr}, *dadv[2] = {nullptr, nullptr};
        double *dinv[2] = {nullptr, nullptr}, *k[4] = {nullptr}, *es = nullptr, *rhs = nullptr;
        double *r = nullptr, *z = nullptr, *pv = nullptr, *Mp = nullptr, *mind = nullptr;
        CgState *cg = nullptr, *hcg = nullptr;   // device state, pinned host mirror
        double *hmind = nullptr;
        int last_its = 8;
    } rm;
    // instrumentation
    bool prof = false;
    std::vector<ProfRec> pending;
    std::vector<cudaEvent_t> pool;
    double prof_ms[TMOP_K_NCLASS] = {0};
    int64_t prof_n[TMOP_K_NCLASS] = {0};
    int64_t bytes = 0;
    std::vector<void *> allocs;

    ElemParams params() const
    {
        ElemParams P;
        P.map = map;
        P.E = E;
        P.Nx = Nx;
        P.tab = tab;
        P.tabf = tabf;
        P.tabw = tabw;
        P.metric = desc.metric;
        P.target = desc.target;
        P.h0 = desc.target_h0;
        P.eta = eta;
        return P;
    }

    template <class T>
    tmop_status alloc(T **ptr, size_t count)
    {
        *ptr = nullptr;
        if (count == 0) count = 1;
        void *q = nullptr;
        cudaError_t e = cudaMalloc(&q, count * sizeof(T));
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            return fail(TMOP_ERR_OOM, "cudaMalloc of " + std::to_string(count * sizeof(T)) + " bytes failed");
        }
        allocs.push_back(q);
        bytes += (int64_t)(count * sizeof(T));
        *ptr = static_cast<T *>(q);
        return TMOP_OK;
    }
    tmop_status alloc_raw(void **ptr, size_t nbytes)
    {
        char *q = nullptr;
        TRY(alloc(&q, nbytes));
        *ptr = q;
        return TMOP_OK;
    }

    cudaEvent_t event()
    {
        if (!pool.empty()) {
            cudaEvent_t e = pool.back();
            pool.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        cudaEventCreate(&e);
        return e;
    }
};

namespace {

// Run one launch, timing it with events on the context stream when enabled.
template <class F>
tmop_status timed(tmop_ctx *c, int cls, const char *what, F &&launch)
{
    cudaEvent_t a = nullptr, b = nullptr;
    if (c->prof) {
        a = c->event();
        b = c->event();
        cudaEventRecord(a, c->stream);
    }
    cudaError_t e = launch();
    if (e != cudaSuccess) return cuda_fail(e, what);
    if (c->prof) {
        cudaEventRecord(b, c->stream);
        c->pending.push_back({cls, a, b});
    }
    return TMOP_OK;
}

tmop_status prof_resolve(tmop_ctx *c)
{
    if (c->pending.empty()) return TMOP_OK;
    CK(cudaStreamSynchronize(c->stream));
    for (auto &r : c->pending) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, r.a, r.b));
        c->prof_ms[r.cls] += ms;
        c->prof_n[r.cls] += 1;
        c->pool.push_back(r.a);
        c->pool.push_back(r.b);
    }
    c->pending.clear();
    return TMOP_OK;
}

bool metric_ok(int m, int d) { return metric_valid(m, d); }

tmop_status limit_ready(tmop_ctx *c)
{
    if (c->lim2 > 0.0 && !c->x0_set)
        return fail(TMOP_ERR_ARG, "limit_delta > 0 but tmop_set_limit_reference has not been called");
    return TMOP_OK;
}

tmop_status target_ready(tmop_ctx *c)
{
    if (c->desc.target == TMOP_TARGET_DISCRETE && !c->eta_set)
        return fail(TMOP_ERR_ARG, "discrete target: call tmop_set_target_field or tmop_set_remap_source");
    return TMOP_OK;
}

// Limiting energy into scal[4] (and its gradient added into ev64 when ev).
tmop_status limit_eg_async(tmop_ctx *c, const double *x, double *ev)
{
    if (c->lim2 <= 0.0) return TMOP_OK;
    const ElemParams P = c->params();
    const int64_t nb = elem_blocks(c->d, c->p, c->nq, c->E);
    CK(launch_limit_eg(c->d, c->p, c->nq, P, x, c->x0, c->lim2, c->part2, ev, c->arith, c->stream));
    CK(launch_finalize_energy(c->part2, nb, c->scal + 4, c->stream));
    return TMOP_OK;
}

// Energy + min det into ctx->scal[0..1] (device), no sync.
tmop_status energy_async(tmop_ctx *c, const double *x)
{
    TRY(limit_ready(c));
    TRY(target_ready(c));
    const ElemParams P = c->params();
    const int64_t nb = elem_blocks(c->d, c->p, c->nq, c->E);
    TRY(timed(c, TMOP_K_ENERGY, "energy kernel",
              [&] { return launch_energy(c->d, c->p, c->nq, P, x, c->part, c->arith, c->stream); }));
    CK(launch_finalize_energy(c->part, nb, c->scal, c->stream));
    TRY(limit_eg_async(c, x, nullptr));
    return TMOP_OK;
}

tmop_status read_scalars(tmop_ctx *c, int n)
{
    CK(cudaMemcpyAsync(c->hscal, c->scal, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return TMOP_OK;
}

tmop_status energy_sync(tmop_ctx *c, const double *x, double *F, double *md)
{
    TRY(energy_async(c, x));
    TRY(read_scalars(c, 6));
    *md = c->hscal[1];
    if (!(c->hscal[1] > 0.0) && c->E > 0) {
        *F = INFINITY;
        return fail(TMOP_ERR_INVERTED, "det(A) <= 0 at some quadrature point");
    }
    *F = c->hscal[0] + (c->lim2 > 0.0 ? c->hscal[4] : 0.0);
    return TMOP_OK;
}

tmop_status gradient_async(tmop_ctx *c, const double *x, double *g)
{
    TRY(limit_ready(c));
    TRY(target_ready(c));
    const ElemParams P = c->params();
    TRY(timed(c, TMOP_K_GRADIENT, "gradient kernel",
              [&] { return launch_gradient(c->d, c->p, c->nq, P, x, c->ev64, c->arith, c->stream); }));
    TRY(limit_eg_async(c, x, c->ev64));
    TRY(timed(c, TMOP_K_ASSEMBLE, "assemble", [&] {
        return launch_assemble(c->ev64, TMOP_FP64, c->csr_ptr, c->csr_idx, c->fixed, nullptr, 0,
                               c->Nx, c->d, c->ENP, g, TMOP_FP64, nullptr, 0, c->stream);
    }));
    return TMOP_OK;
}

// Fused energy + min det + gradient (one forward pass): g on the device,
// F and min det on the host (synchronises).
tmop_status energy_grad_sync(tmop_ctx *c, const double *x, double *g, double *F, double *md)
{
    TRY(limit_ready(c));
    TRY(target_ready(c));
    const ElemParams P = c->params();
    const int64_t nb = elem_blocks(c->d, c->p, c->nq, c->E);
    TRY(timed(c, TMOP_K_GRADIENT, "energy+gradient kernel", [&] {
        return launch_gradient(c->d, c->p, c->nq, P, x, c->ev64, c->arith, c->stream, nullptr, 0,
                               c->part);
    }));
    CK(launch_finalize_energy(c->part, nb, c->scal, c->stream));
    TRY(limit_eg_async(c, x, c->ev64));
    TRY(timed(c, TMOP_K_ASSEMBLE, "assemble", [&] {
        return launch_assemble(c->ev64, TMOP_FP64, c->csr_ptr, c->csr_idx, c->fixed, nullptr, 0,
                               c->Nx, c->d, c->ENP, g, TMOP_FP64, nullptr, 0, c->stream);
    }));
    TRY(read_scalars(c, 6));
    *md = c->hscal[1];
    if (!(c->hscal[1] > 0.0) && c->E > 0) {
        *F = INFINITY;
        return fail(TMOP_ERR_INVERTED, "det(A) <= 0 at some quadrature point");
    }
    *F = c->hscal[0] + (c->lim2 > 0.0 ? c->hscal[4] : 0.0);
    return TMOP_OK;
}

// ||a||_2 for an FP64 vector (synchronises).
tmop_status norm_sync(tmop_ctx *c, const double *a, double *out)
{
    const int nb = reduce_blocks(c->ndof);
    CK(launch_dot(a, a, TMOP_FP64, c->ndof, c->part, nb, c->stream));
    CK(launch_finalize_sum(c->part, nb, c->scal + 2, c->stream));
    CK(cudaMemcpyAsync(c->hscal + 2, c->scal + 2, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    *out = std::sqrt(std::fmax(c->hscal[2], 0.0));
    return TMOP_OK;
}

tmop_status hsetup_async(tmop_ctx *c, const double *x)
{
    TRY(limit_ready(c));
    TRY(target_ready(c));
    const ElemParams P = c->params();
    TRY(timed(c, TMOP_K_HSETUP, "hessian setup kernel",
              [&] { return launch_hsetup(c->d, c->p, c->nq, P, x, c->H, c->prec, c->stream); }));
    if (c->lim2 > 0.0) CK(launch_limit_setup(c->d, c->p, c->nq, P, x, c->lim2, c->lim_cq, c->stream));
    c->h_ready = true;
    return TMOP_OK;
}

// Element vectors of H v (shape term + limiting term) for a v already zero
// on fixed DOFs.
tmop_status apply_elements(tmop_ctx *c, const void *v, const int *stop, int k)
{
    const ElemParams P = c->params();
    TRY(timed(c, TMOP_K_APPLY, "apply kernel", [&] {
        return launch_apply(c->d, c->p, c->nq, P, v, c->H, c->evR, c->prec, stop, k, c->stream);
    }));
    if (c->lim2 > 0.0)
        CK(launch_limit_apply(c->d, c->p, c->nq, P, v, c->lim_cq, c->evR, c->prec, stop, k, c->stream));
    return TMOP_OK;
}

// ---------------------------------------------------------------- remap (Sec. 3.6)
tmop_status remap_alloc(tmop_ctx *c)
{
    auto &R = c->rm;
    if (R.ready) return TMOP_OK;
    const size_t nq = (size_t)c->E * c->nqd;
    TRY(c->alloc(&R.vel, c->ndof));
    for (int i = 0; i < 2; ++i) {
        TRY(c->alloc(&R.dm[i], nq));
        TRY(c->alloc(&R.dadv[i], (size_t)c->d * nq));
        TRY(c->alloc(&R.dinv[i], c->Nx));
    }
    for (int i = 0; i < 4; ++i) TRY(c->alloc(&R.k[i], c->Nx));
    TRY(c->alloc(&R.es, c->Nx));
    TRY(c->alloc(&R.rhs, c->Nx));
    TRY(c->alloc(&R.r, c->Nx));
    TRY(c->alloc(&R.z, c->Nx));
    TRY(c->alloc(&R.pv, c->Nx));
    TRY(c->alloc(&R.Mp, c->Nx));
    TRY(c->alloc(&R.mind, 1));
    TRY(c->alloc((double **)&R.cg, sizeof(CgState) / sizeof(double) + 1));
    if (!R.hcg) CK(cudaMallocHost((void **)&R.hcg, sizeof(CgState)));
    if (!R.hmind) CK(cudaMallocHost((void **)&R.hmind, sizeof(double)));
    R.ready = true;
    return TMOP_OK;
}

// Mass data, advection data and the inverse mass diagonal of x_t into set i;
// min det A of x_t folded into rm.mind.
tmop_status remap_setup(tmop_ctx *c, const double *x0, double t, int i, bool reset)
{
    auto &R = c->rm;
    const ElemParams P = c->params();
    const int64_t nb = elem_blocks(c->d, c->p, c->nq, c->E);
    TRY(timed(c, TMOP_K_REMAP_SETUP, "remap setup kernel", [&] {
        return launch_remap_setup(c->d, c->p, c->nq, P, x0, R.vel, t, R.dm[i], R.dadv[i], c->part,
                                  c->arith, c->stream);
    }));
    CK(launch_min_accum(c->part, nb, R.mind, reset ? 1 : 0, c->stream));
    CK(launch_mass_diag(c->d, c->p, c->nq, P, R.dm[i], c->ev64, c->arith, c->stream));
    CK(launch_assemble(c->ev64, TMOP_FP64, c->csr_ptr, c->csr_idx, nullptr, nullptr, 0, c->Nx, 1,
                       c->ENP, R.rhs, TMOP_FP64, nullptr, 0, c->stream));
    CK(launch_recip(R.rhs, c->Nx, R.dinv[i], c->stream));
    return TMOP_OK;
}

// kout = M_i^-1 K_i u by Jacobi-CG; the host reads the stop flag once per
// chunk of iterations (the first chunk as long as the previous solve).
tmop_status remap_stage(tmop_ctx *c, const double *u, int i, double *kout, const tmop_remap_opts &o,
                        int *its)
{
    auto &R = c->rm;
    const ElemParams P = c->params();
    const int nb = reduce_blocks(c->Nx);
    TRY(timed(c, TMOP_K_ADVECT, "advection kernel", [&] {
        return launch_adv_apply(c->d, c->p, c->nq, P, u, R.dadv[i], c->ev64, c->arith, c->stream);
    }));
    CK(launch_assemble(c->ev64, TMOP_FP64, c->csr_ptr, c->csr_idx, nullptr, nullptr, 0, c->Nx, 1,
                       c->ENP, R.rhs, TMOP_FP64, nullptr, 0, c->stream));
    CK(launch_cg_init(R.rhs, R.dinv[i], c->Nx, kout, R.r, R.z, R.pv, c->part, nb, o.cg_rtol, R.cg,
                      c->stream));
    const int *stop = &R.cg->stop;
    int k = 0, chunk = std::max(4, R.last_its);
    while (true) {
        const int kend = std::min(o.cg_max_it, k + chunk);
        for (int kk = k + 1; kk <= kend; ++kk) {
            TRY(timed(c, TMOP_K_MASS, "mass kernel", [&] {
                return launch_mass_apply(c->d, c->p, c->nq, P, R.pv, R.dm[i], c->ev64, stop, kk,
                                         c->arith, c->stream);
            }));
            CK(launch_cg_iter(c->ev64, c->csr_ptr, c->csr_idx, R.pv, R.Mp, kout, R.r, R.z, R.dinv[i],
                              c->Nx, c->part, nb, R.cg, kk, o.cg_max_it, c->stream));
        }
        CK(cudaMemcpyAsync(R.hcg, R.cg, sizeof(CgState), cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        if (R.hcg->stop <= kend || kend >= o.cg_max_it) break;
        k = kend;
        chunk = 4;
    }
    *its = R.hcg->its;
    R.last_its = std::max(1, R.hcg->its);
    return TMOP_OK;
}

// eta1 = eta0 advected from x0 to x1: RK4 with o.steps uniform pseudo-time
// steps; stage times (n + c_s) dt with c = 0, 1/2, 1/2, 1; the operators at
// (n+1) dt serve the last stage of step n and the first of step n+1.
tmop_status remap_run(tmop_ctx *c, const double *x0, const double *x1, const double *eta0,
                      double *eta1, const tmop_remap_opts &o, tmop_remap_report *rep)
{
    tmop_remap_report r{0, 0, INFINITY, TMOP_OK};
    if (o.steps < 1 || o.cg_max_it < 1 || !(o.cg_rtol >= 0.0))
        return fail(TMOP_ERR_ARG, "remap: steps >= 1, cg_max_it >= 1, cg_rtol >= 0 required");
    TRY(remap_alloc(c));
    auto &R = c->rm;
    CK(launch_trial(x1, x0, 1.0, c->ndof, R.vel, c->stream));          // v = x1 - x0
    if (eta1 != eta0)
        CK(cudaMemcpyAsync(eta1, eta0, sizeof(double) * c->Nx, cudaMemcpyDeviceToDevice, c->stream));
    const double dt = 1.0 / o.steps;
    int its = 0;
    TRY(remap_setup(c, x0, 0.0, 0, true));
    for (int n = 0; n < o.steps; ++n) {
        TRY(remap_stage(c, eta1, 0, R.k[0], o, &its));
        r.cg_iters += its;
        TRY(remap_setup(c, x0, (n + 0.5) * dt, 1, false));
        CK(launch_axpy(eta1, R.k[0], 0.5 * dt, c->Nx, R.es, c->stream));
        TRY(remap_stage(c, R.es, 1, R.k[1], o, &its));
        r.cg_iters += its;
        CK(launch_axpy(eta1, R.k[1], 0.5 * dt, c->Nx, R.es, c->stream));
        TRY(remap_stage(c, R.es, 1, R.k[2], o, &its));
        r.cg_iters += its;
        TRY(remap_setup(c, x0, (n + 1.0) * dt, 0, false));
        CK(launch_axpy(eta1, R.k[2], dt, c->Nx, R.es, c->stream));
        TRY(remap_stage(c, R.es, 0, R.k[3], o, &its));
        r.cg_iters += its;
        CK(launch_rk4_combine(eta1, R.k[0], R.k[1], R.k[2], R.k[3], dt, c->Nx, c->stream));
        r.solves += 4;
    }
    CK(cudaMemcpyAsync(R.hmind, R.mind, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    r.min_det = *R.hmind;
    if (!(r.min_det > 0.0) && c->E > 0) {
        r.status = TMOP_ERR_INVERTED;
        if (rep) *rep = r;
        return fail(TMOP_ERR_INVERTED, "remap: det(A) <= 0 on an intermediate mesh");
    }
    if (rep) *rep = r;
    return TMOP_OK;
}

tmop_status eta_alloc(tmop_ctx *c)
{
    if (!c->eta) TRY(c->alloc(&c->eta, c->Nx));
    if (!c->eta_t) TRY(c->alloc(&c->eta_t, c->Nx));
    return TMOP_OK;
}

tmop_status diag_async(tmop_ctx *c, void *diag)
{
    const ElemParams P = c->params();
    TRY(timed(c, TMOP_K_DIAG, "diag kernel", [&] {
        return launch_diag(c->d, c->p, c->nq, P, c->H, c->evR, c->prec, c->stream);
    }));
    if (c->lim2 > 0.0) CK(launch_limit_diag(c->d, c->p, c->nq, P, c->lim_cq, c->evR, c->prec, c->stream));
    TRY(timed(c, TMOP_K_ASSEMBLE, "assemble", [&] {
        return launch_assemble(c->evR, c->vprec, c->csr_ptr, c->csr_idx, c->fixed, nullptr, 2,
                               c->Nx, c->d, c->ENP, diag, c->vprec, nullptr, 0, c->stream);
    }));
    return TMOP_OK;
}

// Jacobi-preconditioned MINRES for H dx = b (b FP64, zero on fixed DOFs), on
// the context's stream.
tmop_status minres_on(tmop_ctx *c, const double *b, double *dx, double rtol, int max_it,
                      int fixed_its, int *iters, double *resid, int *breakdown)
{
    const int64_t n = c->ndof;
    const int pr = c->vprec;
    const size_t vb = c->rsz * (size_t)n;
    const int nb = reduce_blocks(n);
    // The assembly fused with the first Lanczos update (one pass less over z)
    // for FP32 vectors (0.43 -> 0.40 ms per iteration at 48^3 Q3) and for the
    // float-pair element vectors of the double-float action (Newton step
    // 28.87 -> 28.72 ms); with FP64 element vectors (native FP64) the fused
    // grid-stride gather measured no faster than the one-node-per-thread
    // assembly followed by the update.
    const bool fuse = pr == TMOP_FP32 || action_ev_format(c->prec) == EV_DF_PAIR;
    void *v = c->kv[0], *R1 = c->kv[1], *R2 = c->kv[2], *Z = c->kv[3];
    void *W1 = c->kv[4], *W2 = c->kv[5], *W3 = c->kv[6];
    CK(cudaMemsetAsync(dx, 0, sizeof(double) * n, c->stream));
    CK(cudaMemsetAsync(W1, 0, vb, c->stream));
    CK(cudaMemsetAsync(W2, 0, vb, c->stream));
    CK(launch_minres_init(b, c->minv, pr, n, R1, R2, Z, c->part, nb, c->stream));
    CK(launch_minres_start(c->part, nb, c->st, max_it, c->stream));
    CK(launch_minres_scale(Z, c->st, pr, n, v, c->stream));
    // (R1, R2, Y) rotate; the first Y is Z
    void *Y = Z;
    Z = c->kv[7];
    // The launches of one iteration, all with k = -1: the kernels take the
    // iteration from the device counter st->k, advanced by the first launch.
    constexpr int KD = -1;
    auto launch_iteration = [&]() -> tmop_status {
        CK(launch_iter_next(c->st, c->stream));
        TRY(apply_elements(c, v, &c->st->stop_iter, KD));
        if (fuse) {
            TRY(timed(c, TMOP_K_ASSEMBLE, "assemble + lanczos", [&] {
                return launch_assemble_lanczos_a(c->evR, c->csr_ptr, c->csr_idx, c->fixed, c->Nx,
                                                 c->d, c->ENP, Z, R1, v, c->st,
                                                 pr == TMOP_FP32 ? pr : action_ev_format(c->prec), KD,
                                                 c->part, nb, c->stream);
            }));
        } else {
            TRY(timed(c, TMOP_K_ASSEMBLE, "assemble", [&] {
                return launch_assemble(c->evR, action_ev_format(c->prec), c->csr_ptr, c->csr_idx,
                                       c->fixed, nullptr, 1, c->Nx, c->d, c->ENP, Z, c->vprec,
                                       &c->st->stop_iter, KD, c->stream);
            }));
            CK(launch_lanczos_a(Z, R1, v, c->st, pr, n, KD, c->part, nb, c->stream));
        }
        CK(launch_fin_alpha(c->part, nb, c->st, KD, c->stream));
        // Z holds y; new y = M^-1 y goes to the old R1
        CK(launch_lanczos_b(Z, R2, c->minv, c->st, pr, n, KD, R1, c->part, nb, c->stream));
        CK(launch_fin_beta(c->part, nb, c->st, KD, rtol, fixed_its, c->stream));
        CK(launch_minres_update(v, W1, W2, W3, dx, R1, c->st, pr, n, KD, c->stream));
        return TMOP_OK;
    };
    // rotate: r1 <- r2, r2 <- y(Z), ynew lives in old R1 (consumed), freed old Y buffer
    auto rotate = [&] {
        void *oR1 = R1;
        R1 = R2;
        R2 = Z;
        Z = Y;
        Y = oR1;
        void *oW1 = W1;
        W1 = W2;
        W2 = W3;
        W3 = oW1;
    };
    // Blocks of 4 iterations as CUDA graphs (not with per-kernel profiling,
    // whose events are host-side records, nor on the legacy stream); the graph
    // of a phase is captured once and replayed while its parameters hold.
    const bool graphs = c->graphs && !c->prof && c->stream != nullptr;
    const int variant = apply_variant(c->d, c->p, c->nq, c->prec);
    int k = 0;
    while (k < max_it) {
        if (graphs && max_it - k >= 4) {
            tmop_ctx::MinresGraph &g = c->mg[(k / 4) % 3];
            if (!g.exec || g.dx != dx || g.rtol != rtol || g.fixed_its != fixed_its ||
                g.variant != variant || g.lim != (c->lim2 > 0.0)) {
                if (g.exec) cudaGraphExecDestroy(g.exec);
                g.exec = nullptr;
                cudaGraph_t graph = nullptr;
                CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
                const int64_t l0 = t_launches;
                tmop_status st = TMOP_OK;
                for (int j = 0; j < 4 && st == TMOP_OK; ++j) {
                    st = launch_iteration();
                    rotate();
                }
                const cudaError_t ec = cudaStreamEndCapture(c->stream, &graph);
                if (st != TMOP_OK) {
                    if (graph) cudaGraphDestroy(graph);
                    return st;
                }
                if (ec != cudaSuccess) return cuda_fail(ec, "cudaStreamEndCapture");
                const cudaError_t ei = cudaGraphInstantiate(&g.exec, graph, 0);
                cudaGraphDestroy(graph);
                if (ei != cudaSuccess) {
                    g.exec = nullptr;
                    return cuda_fail(ei, "cudaGraphInstantiate");
                }
                g.dx = dx;
                g.rtol = rtol;
                g.fixed_its = fixed_its;
                g.variant = variant;
                g.lim = c->lim2 > 0.0;
                g.nodes = (int)(t_launches - l0);
                uncount_launches(g.nodes);                    // counted at each graph launch
            } else {
                for (int j = 0; j < 4; ++j) rotate();
            }
            CK(cudaGraphLaunch(g.exec, c->stream));
            count_launch(g.nodes);
            ++c->graph_launches;
            k += 4;
        } else {
            TRY(launch_iteration());
            rotate();
            ++k;
        }
        if (!fixed_its && (k % c->check_every == 0) && k < max_it) {
            CK(cudaMemcpyAsync(c->hst, c->st, sizeof(MinresState), cudaMemcpyDeviceToHost, c->stream));
            CK(cudaStreamSynchronize(c->stream));
            if (c->hst->stop_iter <= k) break;
        }
    }
    CK(cudaMemcpyAsync(c->hst, c->st, sizeof(MinresState), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    *iters = c->hst->iters;
    *resid = (c->hst->beta1 > 0.0) ? c->hst->phibar / c->hst->beta1 : 0.0;
    *breakdown = c->hst->breakdown;
    return TMOP_OK;
}

// MINRES; with graphs on and the legacy default stream as the context's
// stream, the solve runs on the context's own non-blocking stream, after the
// work already queued on the legacy stream and before the work queued later
// (event handoff both ways).
tmop_status minres(tmop_ctx *c, const double *b, double *dx, double rtol, int max_it,
                   int fixed_its, int *iters, double *resid, int *breakdown)
{
    if (!(c->graphs && !c->prof && c->stream == nullptr))
        return minres_on(c, b, dx, rtol, max_it, fixed_its, iters, resid, breakdown);
    if (!c->gstream) {
        CK(cudaStreamCreateWithFlags(&c->gstream, cudaStreamNonBlocking));
        CK(cudaEventCreateWithFlags(&c->gev, cudaEventDisableTiming));
    }
    CK(cudaEventRecord(c->gev, nullptr));
    CK(cudaStreamWaitEvent(c->gstream, c->gev, 0));
    c->stream = c->gstream;
    const tmop_status st = minres_on(c, b, dx, rtol, max_it, fixed_its, iters, resid, breakdown);
    c->stream = nullptr;
    CK(cudaEventRecord(c->gev, c->gstream));
    CK(cudaStreamWaitEvent(nullptr, c->gev, 0));
    return st;
}

}  // namespace

extern "C" {

const char *tmop_status_string(tmop_status st)
{
    switch (st) {
        case TMOP_OK: return "ok";
        case TMOP_ERR_ARG: return "invalid argument";
        case TMOP_ERR_INVERTED: return "inverted element (det(A) <= 0)";
        case TMOP_ERR_CUDA: return "CUDA error";
        case TMOP_ERR_OOM: return "out of device memory";
        case TMOP_ERR_MINRES: return "MINRES breakdown";
        case TMOP_ERR_LINESEARCH: return "line search failed";
        case TMOP_ERR_TIMEOUT: return "device wait timed out";
        case TMOP_ERR_UNSUPPORTED: return "unsupported configuration";
    }
    return "unknown status";
}

const char *tmop_last_error(void) { return g_last_error.c_str(); }

int64_t tmop_launch_count(void) { return g_launches.load(); }

void tmop_destroy(tmop_ctx *ctx)
{
    if (!ctx) return;
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    for (auto &g : ctx->mg)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    if (ctx->gstream) {
        cudaStreamSynchronize(ctx->gstream);
        cudaStreamDestroy(ctx->gstream);
    }
    if (ctx->gev) cudaEventDestroy(ctx->gev);
    for (auto &r : ctx->pending) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
    for (auto e : ctx->pool) cudaEventDestroy(e);
    for (void *q : ctx->allocs) cudaFree(q);
    if (ctx->hscal) cudaFreeHost(ctx->hscal);
    if (ctx->hst) cudaFreeHost(ctx->hst);
    if (ctx->rm.hcg) cudaFreeHost(ctx->rm.hcg);
    if (ctx->rm.hmind) cudaFreeHost(ctx->rm.hmind);
    delete ctx;
}

tmop_status tmop_setup(const tmop_desc *desc, const int32_t *elem_to_node, const uint8_t *fixed,
                       void *cuda_stream, tmop_ctx **out)
{
    if (!desc || !out) return fail(TMOP_ERR_ARG, "desc and out must not be NULL");
    *out = nullptr;
    const tmop_desc &D = *desc;
    if (D.dim != 2 && D.dim != 3) return fail(TMOP_ERR_ARG, "dim must be 2 or 3");
    if (D.order < 1 || D.order > 4) return fail(TMOP_ERR_UNSUPPORTED, "order must be 1..4");
    if (!elem_supported(D.dim, D.order, D.nq1d))
        return fail(TMOP_ERR_UNSUPPORTED, "nq1d must be order+1, order+2 (or 9 in 3D)");
    if (D.num_elems < 0 || D.num_nodes <= 0) return fail(TMOP_ERR_ARG, "bad mesh sizes");
    if (!metric_ok(D.metric, D.dim)) return fail(TMOP_ERR_UNSUPPORTED, "metric not defined for this dim");
    if (D.target != TMOP_TARGET_IDENTITY && D.target != TMOP_TARGET_SIZE_FIELD &&
        D.target != TMOP_TARGET_DISCRETE)
        return fail(TMOP_ERR_ARG, "unknown target");
    if (D.target != TMOP_TARGET_IDENTITY && !(D.target_h0 > 0.0))
        return fail(TMOP_ERR_ARG, "target_h0 must be > 0");
    if (D.limit_delta < 0.0 || D.limit_delta != D.limit_delta)
        return fail(TMOP_ERR_ARG, "limit_delta must be >= 0");
    if (D.hess_precision != TMOP_FP64 && D.hess_precision != TMOP_FP32 &&
        D.hess_precision != TMOP_FP64_NATIVE)
        return fail(TMOP_ERR_ARG, "hess_precision must be TMOP_FP64, TMOP_FP32 or TMOP_FP64_NATIVE");
    if (D.num_elems > 0 && !elem_to_node) return fail(TMOP_ERR_ARG, "elem_to_node is NULL");
    const int64_t ndof = (int64_t)D.dim * D.num_nodes;
    int np = 1;
    for (int k = 0; k < D.dim; ++k) np *= D.order + 1;
    if (D.num_elems * (int64_t)np >= INT_MAX) return fail(TMOP_ERR_ARG, "mesh too large (E*NP >= 2^31)");

    tmop_ctx *c = new tmop_ctx();
    c->desc = D;
    c->d = D.dim;
    c->p = D.order;
    c->nq = D.nq1d;
    c->ni = D.order + 1;
    c->np = np;
    c->nqd = 1;
    for (int k = 0; k < D.dim; ++k) c->nqd *= D.nq1d;
    c->ns = (c->d * c->d) * (c->d * c->d + 1) / 2;
    c->prec = D.hess_precision;
    c->vprec = c->prec == TMOP_FP32 ? TMOP_FP32 : TMOP_FP64;
    c->arith = c->prec == TMOP_FP64_NATIVE ? ARITH_NATIVE : ARITH_DW;
    c->rsz = c->prec == TMOP_FP32 ? 4 : 8;
    c->E = D.num_elems;
    c->Nx = D.num_nodes;
    c->ndof = ndof;
    c->ENP = D.num_elems * (int64_t)np;
    c->stream = static_cast<cudaStream_t>(cuda_stream);

    auto bail = [&](tmop_status st) {
        std::string m = g_last_error;
        tmop_destroy(c);
        g_last_error = m;
        return st;
    };
#define STRY(expr)                                 \
    do {                                           \
        tmop_status s_ = (expr);                   \
        if (s_ != TMOP_OK) return bail(s_);        \
    } while (0)
#define SCK(call)                                                  \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return bail(cuda_fail(e_, #call));  \
    } while (0)

    // element map: validate on the host and build its transpose (CSR)
    std::vector<int32_t> hmap((size_t)c->ENP);
    if (c->ENP > 0) {
        SCK(cudaMemcpyAsync(hmap.data(), elem_to_node, sizeof(int32_t) * c->ENP,
                            cudaMemcpyDeviceToHost, c->stream));
        SCK(cudaStreamSynchronize(c->stream));
    }
    std::vector<int32_t> ptr((size_t)c->Nx + 1, 0), idx((size_t)c->ENP);
    for (int64_t j = 0; j < c->ENP; ++j) {
        const int32_t nd = hmap[j];
        if (nd < 0 || nd >= c->Nx) {
            delete c;
            return fail(TMOP_ERR_ARG, "elem_to_node entry " + std::to_string(j) + " = " +
                                          std::to_string(nd) + " out of range");
        }
        ptr[nd + 1]++;
    }
    for (int64_t i = 0; i < c->Nx; ++i) ptr[i + 1] += ptr[i];
    {
        std::vector<int32_t> fill(ptr.begin(), ptr.end() - 1);
        for (int64_t j = 0; j < c->ENP; ++j) idx[fill[hmap[j]]++] = (int32_t)j;
    }
    STRY(c->alloc(&c->map, c->ENP));
    STRY(c->alloc(&c->csr_ptr, c->Nx + 1));
    STRY(c->alloc(&c->csr_idx, c->ENP));
    if (c->ENP > 0) {
        SCK(cudaMemcpyAsync(c->map, hmap.data(), sizeof(int32_t) * c->ENP, cudaMemcpyHostToDevice, c->stream));
        SCK(cudaMemcpyAsync(c->csr_idx, idx.data(), sizeof(int32_t) * c->ENP, cudaMemcpyHostToDevice, c->stream));
    }
    SCK(cudaMemcpyAsync(c->csr_ptr, ptr.data(), sizeof(int32_t) * (c->Nx + 1), cudaMemcpyHostToDevice, c->stream));
    if (fixed) {
        STRY(c->alloc(&c->fixed, ndof));
        SCK(cudaMemcpyAsync(c->fixed, fixed, ndof, cudaMemcpyDeviceToDevice, c->stream));
    }
    // 1D tables: B, G, weights
    const int tabn = 2 * c->nq * c->ni + c->nq;
    std::vector<double> tab(tabn);
    std::vector<float> tabf(tabn);
    std::vector<df> tabw(tabn);
    host_basis_tables(c->ni, c->nq, tab.data(), tab.data() + c->nq * c->ni,
                      tab.data() + 2 * c->nq * c->ni);
    for (int i = 0; i < tabn; ++i) {
        tabf[i] = (float)tab[i];
        tabw[i] = df(tab[i]);
    }
    STRY(c->alloc(&c->tab, tabn));
    STRY(c->alloc(&c->tabf, tabn));
    STRY(c->alloc(&c->tabw, tabn));
    SCK(cudaMemcpyAsync(c->tabw, tabw.data(), sizeof(df) * tabn, cudaMemcpyHostToDevice, c->stream));
    SCK(cudaMemcpyAsync(c->tab, tab.data(), sizeof(double) * tabn, cudaMemcpyHostToDevice, c->stream));
    SCK(cudaMemcpyAsync(c->tabf, tabf.data(), sizeof(float) * tabn, cudaMemcpyHostToDevice, c->stream));
    // stored Hessian data, element vectors, reductions, work vectors
    // padded to a 256-byte multiple: the action kernels prefetch whole 16-byte lines
    STRY(c->alloc_raw(&c->H, ((c->rsz * (size_t)c->E * h_stride(c->d, c->nq, c->ns, c->nqd) + 255) / 256) * 256 + 256));
    STRY(c->alloc(&c->ev64, (size_t)c->d * c->ENP));
    if (c->vprec == TMOP_FP32) STRY(c->alloc_raw(&c->evR, 4 * (size_t)c->d * c->ENP));
    else c->evR = c->ev64;
    const int64_t eb = elem_blocks(c->d, c->p, c->nq, c->E);
    c->part_n = std::max<int64_t>(2 * eb, 2 * 1184);
    STRY(c->alloc(&c->part, c->part_n));
    STRY(c->alloc(&c->scal, 8));
    STRY(c->alloc((double **)&c->st, sizeof(MinresState) / sizeof(double) + 1));
    STRY(c->alloc(&c->g, ndof));
    STRY(c->alloc(&c->dx, ndof));
    STRY(c->alloc(&c->xt, ndof));
    STRY(c->alloc_raw(&c->vm, c->rsz * ndof));
    STRY(c->alloc_raw(&c->diagR, c->rsz * ndof));
    STRY(c->alloc_raw(&c->minv, c->rsz * ndof));
    for (int i = 0; i < 8; ++i) STRY(c->alloc_raw(&c->kv[i], c->rsz * ndof));
    if (D.limit_delta > 0.0) {
        c->lim2 = 2.0 / (D.limit_delta * D.limit_delta);
        STRY(c->alloc(&c->x0, ndof));
        STRY(c->alloc(&c->lim_cq, (size_t)c->E * c->nqd));
        STRY(c->alloc(&c->part2, c->part_n));
    }
    SCK(cudaMallocHost((void **)&c->hscal, 8 * sizeof(double)));
    SCK(cudaMallocHost((void **)&c->hst, sizeof(MinresState)));
    SCK(cudaStreamSynchronize(c->stream));
#undef STRY
#undef SCK
    *out = c;
    return TMOP_OK;
}

tmop_status tmop_energy(tmop_ctx *ctx, const double *x, double *F, double *min_det)
{
    if (!ctx || !x || !F) return fail(TMOP_ERR_ARG, "NULL argument");
    double md = INFINITY;
    tmop_status st = energy_sync(ctx, x, F, &md);
    if (min_det) *min_det = md;
    return st;
}

tmop_status tmop_det(tmop_ctx *ctx, const double *x, double *det)
{
    if (!ctx || !x || !det) return fail(TMOP_ERR_ARG, "NULL argument");
    TRY(target_ready(ctx));
    ElemParams P = ctx->params();
    P.detq = det;
    TRY(timed(ctx, TMOP_K_ENERGY, "det kernel", [&] {
        return launch_energy(ctx->d, ctx->p, ctx->nq, P, x, ctx->part, ctx->arith, ctx->stream);
    }));
    return TMOP_OK;
}

tmop_status tmop_gradient(tmop_ctx *ctx, const double *x, double *g)
{
    if (!ctx || !x || !g) return fail(TMOP_ERR_ARG, "NULL argument");
    return gradient_async(ctx, x, g);
}

tmop_status tmop_hessian_setup(tmop_ctx *ctx, const double *x)
{
    if (!ctx || !x) return fail(TMOP_ERR_ARG, "NULL argument");
    return hsetup_async(ctx, x);
}

tmop_status tmop_hessian_apply(tmop_ctx *ctx, const void *v, void *y)
{
    if (!ctx || !v || !y) return fail(TMOP_ERR_ARG, "NULL argument");
    if (v == y) return fail(TMOP_ERR_ARG, "v and y must not alias");
    if (!ctx->h_ready) return fail(TMOP_ERR_ARG, "tmop_hessian_setup has not been called");
    CK(launch_mask(v, ctx->fixed, ctx->ndof, ctx->vm, ctx->vprec, ctx->stream));
    const ElemParams P = ctx->params();
    TRY(timed(ctx, TMOP_K_APPLY, "apply kernel", [&] {
        return launch_apply(ctx->d, ctx->p, ctx->nq, P, ctx->vm, ctx->H, ctx->evR, ctx->prec,
                            nullptr, 0, ctx->stream);
    }));
    if (ctx->lim2 > 0.0)
        CK(launch_limit_apply(ctx->d, ctx->p, ctx->nq, P, ctx->vm, ctx->lim_cq, ctx->evR, ctx->prec,
                              nullptr, 0, ctx->stream));
    TRY(timed(ctx, TMOP_K_ASSEMBLE, "assemble", [&] {
        return launch_assemble(ctx->evR, action_ev_format(ctx->prec), ctx->csr_ptr, ctx->csr_idx,
                               ctx->fixed, v, 1, ctx->Nx, ctx->d, ctx->ENP, y, ctx->vprec, nullptr,
                               0, ctx->stream);
    }));
    return TMOP_OK;
}

tmop_status tmop_hessian_diag(tmop_ctx *ctx, void *diag)
{
    if (!ctx || !diag) return fail(TMOP_ERR_ARG, "NULL argument");
    if (!ctx->h_ready) return fail(TMOP_ERR_ARG, "tmop_hessian_setup has not been called");
    return diag_async(ctx, diag);
}

tmop_status tmop_newton_step(tmop_ctx *c, double *x, const tmop_solver_opts *opts,
                             tmop_step_report *rep)
{
    if (!c || !x) return fail(TMOP_ERR_ARG, "NULL argument");
    tmop_solver_opts o = {1e-8, 50, 0, 1.2, 20};
    if (opts) o = *opts;
    if (o.minres_max_it < 0 || o.ls_max_halvings < 0) return fail(TMOP_ERR_ARG, "negative iteration limit");
    tmop_step_report r;
    std::memset(&r, 0, sizeof(r));
    auto finish = [&](tmop_status st) {
        r.status = st;
        if (rep) *rep = r;
        return st;
    };
    double F0 = 0, md0 = 0;
    tmop_status st = TMOP_OK;
    if (c->remap_on) {      // discrete target: eta follows the positions (Sec. 3.6)
        st = remap_run(c, c->rsrc_x0, x, c->rsrc_eta0, c->eta, c->remap_opts, nullptr);
        if (st != TMOP_OK) return finish(st);
    }
    // F, min det and g at x: those of the previous step's accepted trial when
    // x is still those positions (the same kernels on the same input give
    // the same bits), else evaluated
    bool reuse = false;
    if (c->fg_valid && !c->remap_on) {
        CK(launch_differs(x, c->xt, c->ndof, c->scal + 7, c->stream));
        CK(cudaMemcpyAsync(c->hscal + 7, c->scal + 7, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        reuse = c->hscal[7] == 0.0;
    }
    c->fg_valid = false;
    double g0 = 0;
    if (reuse) {
        F0 = c->fg_F;
        md0 = c->fg_md;
        g0 = c->fg_gn;
        r.energy = F0;
        r.min_det = md0;
        c->reused_fg += 1;
    } else {
        st = energy_grad_sync(c, x, c->g, &F0, &md0);
        r.energy = F0;
        r.min_det = md0;
        if (st != TMOP_OK) return finish(st);
        st = norm_sync(c, c->g, &g0);
        if (st != TMOP_OK) return finish(st);
    }
    r.grad_norm = g0;
    if (g0 == 0.0) {
        r.energy_new = F0;
        r.grad_norm_new = 0.0;
        return finish(TMOP_OK);
    }
    if ((st = hsetup_async(c, x)) != TMOP_OK) return finish(st);
    if ((st = diag_async(c, c->diagR)) != TMOP_OK) return finish(st);
    {
        cudaError_t e = launch_jacobi(c->diagR, c->vprec, c->ndof, c->minv, c->stream);
        if (e != cudaSuccess) return finish(cuda_fail(e, "jacobi"));
    }
    int its = 0, brk = 0;
    double res = 0;
    st = minres(c, c->g, c->dx, o.minres_rtol, o.minres_max_it, o.minres_fixed_its, &its, &res, &brk);
    if (st != TMOP_OK) return finish(st);
    r.minres_iters = its;
    r.minres_resid = res;
    if (c->fault == TMOP_FAULT_MINRES_BREAKDOWN) {          // injected by tmop_inject_fault
        c->fault = TMOP_FAULT_NONE;
        brk = 1;
    }
    if (brk)
        return finish(fail(TMOP_ERR_MINRES, "MINRES breakdown (a preconditioned inner product was "
                                            "negative or not finite)"));
    double alpha = 1.0;
    for (int h = 0; h <= o.ls_max_halvings; ++h, alpha *= 0.5) {
        cudaError_t e = launch_trial(x, c->dx, alpha, c->ndof, c->xt, c->stream);
        if (e != cudaSuccess) return finish(cuda_fail(e, "trial"));
        // with the remap, the trial is evaluated with eta remapped to it; the
        // field of the accepted trial stays in c->eta
        bool swapped = false;
        auto restore = [&] { if (swapped) std::swap(c->eta, c->eta_t); swapped = false; };
        if (c->remap_on) {
            st = remap_run(c, c->rsrc_x0, c->xt, c->rsrc_eta0, c->eta_t, c->remap_opts, nullptr);
            if (st == TMOP_ERR_INVERTED) continue;        // x_t inverted on the way
            if (st != TMOP_OK) return finish(st);
            std::swap(c->eta, c->eta_t);
            swapped = true;
        }
        double F1 = 0, md1 = 0;
        st = energy_grad_sync(c, c->xt, c->g, &F1, &md1);
        if (st == TMOP_ERR_INVERTED) { restore(); continue; }   // det A(x+) > 0 required
        if (st != TMOP_OK) { restore(); return finish(st); }
        if (!(F1 < o.ls_factor * F0)) { restore(); continue; }  // energy test
        double g1 = 0;
        if ((st = norm_sync(c, c->g, &g1)) != TMOP_OK) { restore(); return finish(st); }
        if (!(g1 < o.ls_factor * g0)) { restore(); continue; }  // gradient test
        e = cudaMemcpyAsync(x, c->xt, sizeof(double) * c->ndof, cudaMemcpyDeviceToDevice, c->stream);
        if (e != cudaSuccess) return finish(cuda_fail(e, "accept"));
        e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) return finish(cuda_fail(e, "accept"));
        r.alpha = alpha;
        r.halvings = h;
        r.energy_new = F1;
        r.grad_norm_new = g1;
        r.min_det = md1;
        c->fg_valid = true;                                     // xt = x, g at xt
        c->fg_F = F1;
        c->fg_md = md1;
        c->fg_gn = g1;
        g_last_error.clear();
        return finish(TMOP_OK);
    }
    return finish(fail(TMOP_ERR_LINESEARCH, "no step length passed the line search"));
}

tmop_status tmop_set_limit_reference(tmop_ctx *ctx, const double *x0)
{
    if (!ctx || !x0) return fail(TMOP_ERR_ARG, "NULL argument");
    if (ctx->lim2 <= 0.0) return fail(TMOP_ERR_ARG, "context has no limiting term (limit_delta = 0)");
    CK(cudaMemcpyAsync(ctx->x0, x0, sizeof(double) * ctx->ndof, cudaMemcpyDeviceToDevice, ctx->stream));
    ctx->x0_set = true;
    ctx->fg_valid = false;
    return TMOP_OK;
}

tmop_status tmop_set_target_field(tmop_ctx *ctx, const double *eta)
{
    if (!ctx || !eta) return fail(TMOP_ERR_ARG, "NULL argument");
    if (ctx->desc.target != TMOP_TARGET_DISCRETE) return fail(TMOP_ERR_ARG, "context target is not DISCRETE");
    TRY(eta_alloc(ctx));
    CK(cudaMemcpyAsync(ctx->eta, eta, sizeof(double) * ctx->Nx, cudaMemcpyDeviceToDevice, ctx->stream));
    ctx->eta_set = true;
    ctx->fg_valid = false;
    return TMOP_OK;
}

tmop_status tmop_set_remap_source(tmop_ctx *ctx, const double *x0, const double *eta0,
                                  const tmop_remap_opts *opts)
{
    if (!ctx) return fail(TMOP_ERR_ARG, "NULL context");
    if (ctx->desc.target != TMOP_TARGET_DISCRETE) return fail(TMOP_ERR_ARG, "context target is not DISCRETE");
    ctx->fg_valid = false;
    if (!eta0) {
        ctx->remap_on = false;
        return TMOP_OK;
    }
    if (!x0) return fail(TMOP_ERR_ARG, "x0 is NULL");
    tmop_remap_opts o{4, 1e-12, 200};
    if (opts) o = *opts;
    if (o.steps < 1 || o.cg_max_it < 1 || !(o.cg_rtol >= 0.0))
        return fail(TMOP_ERR_ARG, "remap: steps >= 1, cg_max_it >= 1, cg_rtol >= 0 required");
    TRY(eta_alloc(ctx));
    if (!ctx->rsrc_x0) TRY(ctx->alloc(&ctx->rsrc_x0, ctx->ndof));
    if (!ctx->rsrc_eta0) TRY(ctx->alloc(&ctx->rsrc_eta0, ctx->Nx));
    CK(cudaMemcpyAsync(ctx->rsrc_x0, x0, sizeof(double) * ctx->ndof, cudaMemcpyDeviceToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->rsrc_eta0, eta0, sizeof(double) * ctx->Nx, cudaMemcpyDeviceToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->eta, eta0, sizeof(double) * ctx->Nx, cudaMemcpyDeviceToDevice, ctx->stream));
    ctx->remap_opts = o;
    ctx->remap_on = true;
    ctx->eta_set = true;
    return TMOP_OK;
}

tmop_status tmop_remap(tmop_ctx *ctx, const double *x0, const double *x1, const double *eta0,
                       double *eta1, const tmop_remap_opts *opts, tmop_remap_report *rep)
{
    if (!ctx || !x0 || !x1 || !eta0 || !eta1) return fail(TMOP_ERR_ARG, "NULL argument");
    tmop_remap_opts o{4, 1e-12, 200};
    if (opts) o = *opts;
    tmop_status st = remap_run(ctx, x0, x1, eta0, eta1, o, rep);
    if (st == TMOP_OK) g_last_error.clear();
    return st;
}

tmop_status tmop_set_graphs(tmop_ctx *ctx, int on)
{
    if (!ctx) return fail(TMOP_ERR_ARG, "NULL context");
    ctx->graphs = on != 0;
    return TMOP_OK;
}

int64_t tmop_graph_launches(const tmop_ctx *ctx) { return ctx ? ctx->graph_launches : 0; }
int64_t tmop_step_reuses(const tmop_ctx *ctx) { return ctx ? ctx->reused_fg : 0; }

tmop_status tmop_profile_enable(tmop_ctx *ctx, int on)
{
    if (!ctx) return fail(TMOP_ERR_ARG, "NULL context");
    TRY(prof_resolve(ctx));
    for (int i = 0; i < TMOP_K_NCLASS; ++i) { ctx->prof_ms[i] = 0; ctx->prof_n[i] = 0; }
    ctx->prof = on != 0;
    return TMOP_OK;
}

tmop_status tmop_profile_read(tmop_ctx *ctx, int cls, double *total_ms, int64_t *launches)
{
    if (!ctx || cls < 0 || cls >= TMOP_K_NCLASS) return fail(TMOP_ERR_ARG, "bad argument");
    TRY(prof_resolve(ctx));
    if (total_ms) *total_ms = ctx->prof_ms[cls];
    if (launches) *launches = ctx->prof_n[cls];
    return TMOP_OK;
}

int64_t tmop_device_bytes(const tmop_ctx *ctx) { return ctx ? ctx->bytes : 0; }

tmop_status tmop_vec_lincomb(tmop_ctx *ctx, int64_t n, double a, const double *x, double b,
                             const double *y, double c, const double *z, double *out)
{
    if (!ctx || !x || !out || n < 0) return fail(TMOP_ERR_ARG, "NULL argument or n < 0");
    CK(launch_lincomb(n, a, x, b, y, c, z, out, ctx->stream));
    return TMOP_OK;
}

tmop_status tmop_vec_mul(tmop_ctx *ctx, int64_t n, const double *x, const double *y, double *out)
{
    if (!ctx || !x || !y || !out || n < 0) return fail(TMOP_ERR_ARG, "NULL argument or n < 0");
    CK(launch_vmul(n, x, y, out, ctx->stream));
    return TMOP_OK;
}

tmop_status tmop_vec_dot(tmop_ctx *ctx, int64_t n, const double *x, const double *y,
                         const uint8_t *mask, double *out)
{
    if (!ctx || !x || !y || !out || n < 0) return fail(TMOP_ERR_ARG, "NULL argument or n < 0");
    const int nb = reduce_blocks(n);
    CK(launch_dot_masked(x, y, mask, n, ctx->part, nb, ctx->stream));
    CK(launch_finalize_sum(ctx->part, nb, ctx->scal + 3, ctx->stream));
    CK(cudaMemcpyAsync(ctx->hscal + 3, ctx->scal + 3, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    *out = ctx->hscal[3];
    return TMOP_OK;
}

tmop_status tmop_vec_jacobi(tmop_ctx *ctx, int64_t n, const double *diag, double *minv)
{
    if (!ctx || !diag || !minv || n < 0) return fail(TMOP_ERR_ARG, "NULL argument or n < 0");
    CK(launch_jacobi(diag, TMOP_FP64, n, minv, ctx->stream));
    return TMOP_OK;
}

tmop_status tmop_vec_gather(tmop_ctx *ctx, int64_t m, const int32_t *idx, const double *src,
                            double *dst)
{
    if (!ctx || m < 0 || (m > 0 && (!idx || !src || !dst))) return fail(TMOP_ERR_ARG, "NULL argument or m < 0");
    CK(launch_vgather(m, idx, src, dst, ctx->stream));
    return TMOP_OK;
}

tmop_status tmop_vec_scatter_add(tmop_ctx *ctx, int64_t m, const int32_t *idx, const double *vals,
                                 double *dst)
{
    if (!ctx || m < 0 || (m > 0 && (!idx || !vals || !dst))) return fail(TMOP_ERR_ARG, "NULL argument or m < 0");
    CK(launch_vscatter_add(m, idx, vals, dst, ctx->stream));
    return TMOP_OK;
}

tmop_status tmop_inject_fault(tmop_ctx *ctx, int fault)
{
    if (!ctx || (fault != TMOP_FAULT_NONE && fault != TMOP_FAULT_MINRES_BREAKDOWN))
        return fail(TMOP_ERR_ARG, "NULL context or unknown fault");
    ctx->fault = fault;
    return TMOP_OK;
}

int tmop_apply_variants(int dim, int order, int nq1d)
{
    if (!elem_supported(dim, order, nq1d)) return 0;
    return apply_variant_count(dim, order, nq1d);
}

tmop_status tmop_get_apply_variant(int dim, int order, int nq1d, int precision, int *variant)
{
    if (!variant || !elem_supported(dim, order, nq1d) || precision < 0 || precision > 2)
        return fail(TMOP_ERR_ARG, "bad configuration, precision or NULL output");
    *variant = apply_variant(dim, order, nq1d, precision);
    return TMOP_OK;
}

tmop_status tmop_set_apply_variant(int dim, int order, int nq1d, int precision, int variant)
{
    if (!elem_supported(dim, order, nq1d) || !set_apply_variant(dim, order, nq1d, precision, variant))
        return fail(TMOP_ERR_ARG, "bad configuration, precision or variant");
    return TMOP_OK;
}

tmop_status tmop_autotune(tmop_ctx *c, int reps, int *variant, double *ms)
{
    if (!c || reps < 1) return fail(TMOP_ERR_ARG, "NULL context or reps < 1");
    if (!c->h_ready) return fail(TMOP_ERR_ARG, "tmop_hessian_setup has not been called");
    const int n = apply_variant_count(c->d, c->p, c->nq);
    const ElemParams P = c->params();
    CK(cudaMemsetAsync(c->vm, 0, c->rsz * (size_t)c->ndof, c->stream));
    cudaEvent_t a = nullptr, b = nullptr;
    CK(cudaEventCreate(&a));
    cudaError_t e = cudaEventCreate(&b);
    if (e != cudaSuccess) { cudaEventDestroy(a); return cuda_fail(e, "cudaEventCreate"); }
    int best = -1;
    double best_ms = 0.0;
    for (int v = 0; v < n && e == cudaSuccess; ++v) {
        set_apply_variant(c->d, c->p, c->nq, c->prec, v);
        auto launch = [&] {
            return launch_apply(c->d, c->p, c->nq, P, c->vm, c->H, c->evR, c->prec, nullptr, 0,
                                c->stream);
        };
        if ((e = launch()) != cudaSuccess) break;             // warm-up (and kernel attributes)
        if ((e = cudaEventRecord(a, c->stream)) != cudaSuccess) break;
        for (int r = 0; r < reps && e == cudaSuccess; ++r) e = launch();
        if (e != cudaSuccess || (e = cudaEventRecord(b, c->stream)) != cudaSuccess ||
            (e = cudaEventSynchronize(b)) != cudaSuccess)
            break;
        float t = 0.f;
        if ((e = cudaEventElapsedTime(&t, a, b)) != cudaSuccess) break;
        const double per = (double)t / reps;
        if (ms) ms[v] = per;
        if (best < 0 || per < best_ms) {
            best = v;
            best_ms = per;
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    set_apply_variant(c->d, c->p, c->nq, c->prec, e == cudaSuccess ? best : -1);
    if (e != cudaSuccess) return cuda_fail(e, "autotune");
    if (variant) *variant = best;
    return TMOP_OK;
}

}  // extern "C"
