// Batched and continuously batched TMOP Newton steps.
//
// A tmop_batch holds up to max_meshes independent meshes of the same
// (dim, order, nq1d, metric, target, precision).  Every mesh keeps its own
// resident state (map and transposed map, positions, stored d2mu/dT2 data,
// element vectors, Krylov vectors, partial sums) in one device slab; one
// Newton step of all active meshes is a fixed sequence of shared launches
// whose grids cover the (mesh, tile) pairs of the active meshes.  Per-mesh
// scalars (energies, norms, MINRES recurrences, line-search decisions) live
// on the device, one block or thread per mesh.  Reductions are per mesh in a
// fixed order, so a mesh's results do not depend on which other meshes share
// the launches.  Meshes can be added and removed between steps (continuous
// batching); that edits only the per-mesh descriptor table.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#include "minres_scalar.cuh"
#include "tmop_device.cuh"
#include "tmop_internal.h"

namespace tmop {

struct BState {
    MinresState ms;
    double F0, g0, gfirst, F1, g1, md0, md1, alpha, energy_first;
    int status, done, have_fg, acc_h, work, newton_its, minres_total, halvings, first, pad;
};

namespace {

constexpr int BT = 256;       // threads per block of the batched vector kernels
constexpr int VCH = 4096;     // DOFs per vector tile
constexpr int NCH = 256;      // nodes per assembly tile

__device__ __forceinline__ double bsum(double v, double *sh)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < BT / 32; ++i) s += sh[i];
    return s;
}

template <class T>
__device__ __forceinline__ T *rp(const BMesh &m, int role) { return static_cast<T *>(m.ptr[role]); }

// chunk of DOFs [i0, i1) of the tile's mesh
__device__ __forceinline__ void chunk_range(const BMesh &m, int chunk, int64_t &i0, int64_t &i1)
{
    i0 = (int64_t)chunk * VCH;
    i1 = i0 + VCH < m.ndof ? i0 + VCH : m.ndof;
}

// ---------------------------------------------------------------- per-mesh reductions
__global__ void b_energy_final(const BMesh *M, BState *S, const int *mlist, int which)
{
    const int m = mlist[blockIdx.x];
    const BMesh &bm = M[m];
    const double *part = rp<double>(bm, ROLE_PART);
    __shared__ double sh[BT / 32], shm[BT / 32];
    double s = 0.0, mn = INFINITY;
    for (int i = threadIdx.x; i < bm.ntile_e; i += BT) {
        s += part[2 * i];
        mn = fmin(mn, part[2 * i + 1]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mn = fmin(mn, __shfl_down_sync(0xffffffffu, mn, o));
    if ((threadIdx.x & 31) == 0) shm[threadIdx.x >> 5] = mn;
    s = bsum(s, sh);
    if (threadIdx.x == 0) {
        for (int i = 0; i < BT / 32; ++i) mn = fmin(mn, shm[i]);
        if (which == 0) { S[m].F0 = s; S[m].md0 = mn; }
        else { S[m].F1 = s; S[m].md1 = mn; }
    }
}

__global__ void b_norm_final(const BMesh *M, BState *S, const int *mlist, int which)
{
    const int m = mlist[blockIdx.x];
    const BMesh &bm = M[m];
    const double *part = rp<double>(bm, ROLE_VPART);
    __shared__ double sh[BT / 32];
    double s = 0.0;
    for (int i = threadIdx.x; i < bm.nchunk; i += BT) s += part[i];
    s = bsum(s, sh);
    if (threadIdx.x == 0) {
        const double g = sqrt(fmax(s, 0.0));
        if (which == 0) { S[m].g0 = g; S[m].have_fg = 1; }
        else S[m].g1 = g;
    }
}

// ---------------------------------------------------------------- vector tiles
template <class RA, class RB>
__global__ void b_dot(const BMesh *M, const int2 *tiles, int ra, int rb)
{
    const int2 t = tiles[blockIdx.x];
    const BMesh &bm = M[t.x];
    int64_t i0, i1;
    chunk_range(bm, t.y, i0, i1);
    const RA *a = rp<RA>(bm, ra);
    const RB *b = rp<RB>(bm, rb);
    __shared__ double sh[BT / 32];
    double s = 0.0;
    for (int64_t i = i0 + threadIdx.x; i < i1; i += BT) s += (double)a[i] * (double)b[i];
    s = bsum(s, sh);
    if (threadIdx.x == 0) rp<double>(bm, ROLE_VPART)[t.y] = s;
}

// out = sum of element entries per node (fixed order) + fixed-DOF rule
// (mode 0 -> 0, 1 -> 0, 2 -> 1); skipped for meshes whose MINRES stopped.
template <class RI, class RO>
__global__ void b_assemble(const BMesh *M, const int2 *tiles, int ev_role, int out_role, int mode,
                           int D, int NP, const BState *S, int k)
{
    const int2 t = tiles[blockIdx.x];
    const BMesh &bm = M[t.x];
    if (S && S[t.x].ms.stop_iter < (k >= 0 ? k : S[t.x].ms.k)) return;
    const int64_t n = (int64_t)t.y * NCH + threadIdx.x;
    const int64_t Nx = bm.P.Nx;
    if (n >= Nx) return;
    const RI *ev = rp<RI>(bm, ev_role);
    RO *out = rp<RO>(bm, out_role);
    const int64_t ENP = bm.P.E * NP;
    const int b = bm.csr_ptr[n], e = bm.csr_ptr[n + 1];
    typename AsmAcc<RI>::T s[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) asm_zero(s[a]);
    for (int j = b; j < e; ++j) {
        const int64_t t = bm.csr_idx[j];
#pragma unroll
        for (int a = 0; a < 3; ++a)
            if (a < D) asm_add(s[a], ld_plain(ev + a * ENP + t));
        if (((j - b) & 7) == 7)
#pragma unroll
            for (int a = 0; a < 3; ++a) asm_renorm(s[a]);
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (a >= D) break;
        const int64_t dof = a * Nx + n;
        out[dof] = (bm.fixed && bm.fixed[dof]) ? RO((mode == 2) ? 1.0 : 0.0) : asm_out<RO>(s[a]);
    }
}

template <class R>
__global__ void b_jacobi(const BMesh *M, const int2 *tiles)
{
    const int2 t = tiles[blockIdx.x];
    const BMesh &bm = M[t.x];
    int64_t i0, i1;
    chunk_range(bm, t.y, i0, i1);
    const R *dg = rp<R>(bm, ROLE_DIAG);
    R *mi = rp<R>(bm, ROLE_MINV);
    for (int64_t i = i0 + threadIdx.x; i < i1; i += BT) {
        const double a = fabs((double)dg[i]);
        mi[i] = (R)(a < 1e-300 ? 1.0 : 1.0 / a);
    }
}

// ---------------------------------------------------------------- MINRES
template <class R>
__global__ void b_minres_init(const BMesh *M, const int2 *tiles, int r1, int r2, int y)
{
    const int2 t = tiles[blockIdx.x];
    const BMesh &bm = M[t.x];
    int64_t i0, i1;
    chunk_range(bm, t.y, i0, i1);
    const double *b = rp<double>(bm, ROLE_G);
    const R *mi = rp<R>(bm, ROLE_MINV);
    R *R1 = rp<R>(bm, ROLE_KV0 + r1), *R2 = rp<R>(bm, ROLE_KV0 + r2), *Y = rp<R>(bm, ROLE_KV0 + y);
    __shared__ double sh[BT / 32];
    VecDot<R> dot;
    for (int64_t i = i0 + threadIdx.x; i < i1; i += BT) {
        const R bi = (R)b[i];
        const R yi = mi[i] * bi;
        R1[i] = bi;
        R2[i] = bi;
        Y[i] = yi;
        dot.add(bi, yi);
    }
    const double s = bsum(dot.get(), sh);
    if (threadIdx.x == 0) rp<double>(bm, ROLE_VPART)[t.y] = s;
}

__global__ void b_minres_start(const BMesh *M, BState *S, const int *mlist)
{
    const int m = mlist[blockIdx.x];
    const BMesh &bm = M[m];
    const double *part = rp<double>(bm, ROLE_VPART);
    __shared__ double sh[BT / 32];
    double s = 0.0;
    for (int i = threadIdx.x; i < bm.nchunk; i += BT) s += part[i];
    s = bsum(s, sh);
    if (threadIdx.x == 0) minres_start_scalars(&S[m].ms, s);
}

template <class R>
__global__ void b_minres_scale(const BMesh *M, const int2 *tiles, const BState *S, int y, int v)
{
    const int2 t = tiles[blockIdx.x];
    const BMesh &bm = M[t.x];
    const MinresState &ms = S[t.x].ms;
    if (ms.stop_iter < 1) return;
    int64_t i0, i1;
    chunk_range(bm, t.y, i0, i1);
    const R *Y = rp<R>(bm, ROLE_KV0 + y);
    R *V = rp<R>(bm, ROLE_KV0 + v);
    const VecS<R> ib = (VecS<R>)(1.0 / ms.beta);
    for (int64_t i = i0 + threadIdx.x; i < i1; i += BT) V[i] = (R)((VecS<R>)Y[i] * ib);
}

template <class R>
__global__ void b_lanczos_a(const BMesh *M, const int2 *tiles, const BState *S, int z, int r1, int v,
                            int k)
{
    const int2 t = tiles[blockIdx.x];
    const BMesh &bm = M[t.x];
    const MinresState &ms = S[t.x].ms;
    if (k < 0) k = ms.k;                                   // device iteration counter
    if (ms.stop_iter < k) return;
    int64_t i0, i1;
    chunk_range(bm, t.y, i0, i1);
    R *Z = rp<R>(bm, ROLE_KV0 + z);
    const R *R1 = rp<R>(bm, ROLE_KV0 + r1), *V = rp<R>(bm, ROLE_KV0 + v);
    using SR = VecS<R>;
    const SR c = (SR)((k >= 2) ? ms.beta / ms.beta_old : 0.0);
    __shared__ double sh[BT / 32];
    VecDot<R> dot;
    for (int64_t i = i0 + threadIdx.x; i < i1; i += BT) {
        const R yi = (R)((SR)Z[i] - c * (SR)R1[i]);
        Z[i] = yi;
        dot.add(V[i], yi);
    }
    const double s = bsum(dot.get(), sh);
    if (threadIdx.x == 0) rp<double>(bm, ROLE_VPART)[t.y] = s;
}

__global__ void b_fin_alpha(const BMesh *M, BState *S, const int *mlist, int k)
{
    const int m = mlist[blockIdx.x];
    if (k < 0) k = S[m].ms.k;
    if (S[m].ms.stop_iter < k) return;
    const BMesh &bm = M[m];
    const double *part = rp<double>(bm, ROLE_VPART);
    __shared__ double sh[BT / 32];
    double s = 0.0;
    for (int i = threadIdx.x; i < bm.nchunk; i += BT) s += part[i];
    s = bsum(s, sh);
    if (threadIdx.x == 0) S[m].ms.alpha = s;
}

template <class R>
__global__ void b_lanczos_b(const BMesh *M, const int2 *tiles, const BState *S, int y, int r2,
                            int ynew, int k)
{
    const int2 t = tiles[blockIdx.x];
    const BMesh &bm = M[t.x];
    const MinresState &ms = S[t.x].ms;
    if (k < 0) k = ms.k;
    if (ms.stop_iter < k) return;
    int64_t i0, i1;
    chunk_range(bm, t.y, i0, i1);
    R *Y = rp<R>(bm, ROLE_KV0 + y), *YN = rp<R>(bm, ROLE_KV0 + ynew);
    const R *R2 = rp<R>(bm, ROLE_KV0 + r2), *mi = rp<R>(bm, ROLE_MINV);
    using SR = VecS<R>;
    const SR c = (SR)(ms.alpha / ms.beta);
    __shared__ double sh[BT / 32];
    VecDot<R> dot;
    for (int64_t i = i0 + threadIdx.x; i < i1; i += BT) {
        const R yi = (R)((SR)Y[i] - c * (SR)R2[i]);
        const R zi = mi[i] * yi;
        Y[i] = yi;
        YN[i] = zi;
        dot.add(yi, zi);
    }
    const double s = bsum(dot.get(), sh);
    if (threadIdx.x == 0) rp<double>(bm, ROLE_VPART)[t.y] = s;
}

__global__ void b_fin_beta(const BMesh *M, BState *S, const int *mlist, int k, double rtol,
                           int fixed_its)
{
    const int m = mlist[blockIdx.x];
    if (k < 0) k = S[m].ms.k;
    if (S[m].ms.stop_iter < k) return;
    const BMesh &bm = M[m];
    const double *part = rp<double>(bm, ROLE_VPART);
    __shared__ double sh[BT / 32];
    double s = 0.0;
    for (int i = threadIdx.x; i < bm.nchunk; i += BT) s += part[i];
    s = bsum(s, sh);
    if (threadIdx.x == 0) minres_beta_scalars(&S[m].ms, s, k, rtol, fixed_its);
}

template <class R>
__global__ void b_minres_update(const BMesh *M, const int2 *tiles, const BState *S, int v, int w1,
                                int w2, int wnew, int ynew, int k)
{
    const int2 t = tiles[blockIdx.x];
    const BMesh &bm = M[t.x];
    const MinresState &ms = S[t.x].ms;
    if (k < 0) k = ms.k;
    if (ms.stop_iter < k) return;
    int64_t i0, i1;
    chunk_range(bm, t.y, i0, i1);
    R *V = rp<R>(bm, ROLE_KV0 + v), *WN = rp<R>(bm, ROLE_KV0 + wnew);
    const R *W1 = rp<R>(bm, ROLE_KV0 + w1), *W2 = rp<R>(bm, ROLE_KV0 + w2);
    const R *YN = rp<R>(bm, ROLE_KV0 + ynew);
    double *dx = rp<double>(bm, ROLE_DX);
    using SR = VecS<R>;
    const SR eo = (SR)ms.eps_old, de = (SR)ms.delta, ig = (SR)(1.0 / ms.gamma);
    const double ph = ms.phi;
    const SR ib = (SR)((ms.beta > 0.0) ? 1.0 / ms.beta : 0.0);
    for (int64_t i = i0 + threadIdx.x; i < i1; i += BT) {
        const SR wn = ((SR)V[i] - eo * (SR)W1[i] - de * (SR)W2[i]) * ig;
        WN[i] = (R)wn;
        dx[i] += ph * (double)wn;                           // the solution stays FP64
        V[i] = (R)((SR)YN[i] * ib);
    }
}

// S[m].ms.k += 1 for the meshes of the subset: the start of a MINRES
// iteration whose launches take k = -1.
__global__ void b_iter_next(BState *S, const int *mlist, int nm)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < nm) S[mlist[j]].ms.k += 1;
}

template <class R>
__global__ void b_zero(const BMesh *M, const int2 *tiles, int w1, int w2)
{
    const int2 t = tiles[blockIdx.x];
    const BMesh &bm = M[t.x];
    int64_t i0, i1;
    chunk_range(bm, t.y, i0, i1);
    R *A = rp<R>(bm, ROLE_KV0 + w1), *B = rp<R>(bm, ROLE_KV0 + w2);
    double *dx = rp<double>(bm, ROLE_DX);
    for (int64_t i = i0 + threadIdx.x; i < i1; i += BT) {
        A[i] = R(0);
        B[i] = R(0);
        dx[i] = 0.0;
    }
}

// ---------------------------------------------------------------- Newton control
// One thread per listed mesh: convergence test |g|/|g0| <= rtol and caps.
__global__ void b_prep(BState *S, const int *mlist, int n, double rtol, int max_newton)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    BState &st = S[mlist[j]];
    st.work = 0;
    st.acc_h = -1;
    if (st.done) return;
    if (!(st.md0 > 0.0)) {
        st.status = TMOP_ERR_INVERTED;
        st.done = 1;
        return;
    }
    if (st.first) {
        st.gfirst = st.g0;
        st.energy_first = st.F0;
        st.first = 0;
    }
    if (st.g0 == 0.0 || st.g0 <= rtol * st.gfirst || st.newton_its >= max_newton) {
        st.done = 1;
        return;
    }
    st.work = 1;
}

__global__ void b_trial(const BMesh *M, const int2 *tiles, const BState *S, int h)
{
    const int2 t = tiles[blockIdx.x];
    const BMesh &bm = M[t.x];
    if (S[t.x].acc_h >= 0) return;
    int64_t i0, i1;
    chunk_range(bm, t.y, i0, i1);
    const double *x = rp<double>(bm, ROLE_X), *dx = rp<double>(bm, ROLE_DX);
    double *xt = rp<double>(bm, ROLE_XT);
    const double alpha = ldexp(1.0, -h);
    for (int64_t i = i0 + threadIdx.x; i < i1; i += BT) xt[i] = x[i] - alpha * dx[i];
}

// Line-search tests of the paper (Sec. 2.3): det A(x+) > 0, F(x+) < f F(x),
// |g(x+)| < f |g(x)|.
__global__ void b_ls_decide(BState *S, const int *mlist, int n, double factor, int h)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    BState &st = S[mlist[j]];
    if (!st.work || st.acc_h >= 0) return;
    if (st.md1 > 0.0 && st.F1 < factor * st.F0 && st.g1 < factor * st.g0) {
        st.acc_h = h;
        st.alpha = ldexp(1.0, -h);
    }
}

__global__ void b_accept_copy(const BMesh *M, const int2 *tiles, const BState *S, int h)
{
    const int2 t = tiles[blockIdx.x];
    const BMesh &bm = M[t.x];
    if (S[t.x].acc_h != h) return;
    int64_t i0, i1;
    chunk_range(bm, t.y, i0, i1);
    double *x = rp<double>(bm, ROLE_X);
    const double *xt = rp<double>(bm, ROLE_XT);
    for (int64_t i = i0 + threadIdx.x; i < i1; i += BT) x[i] = xt[i];
}

__global__ void b_finish(BState *S, const int *mlist, int n)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    BState &st = S[mlist[j]];
    if (!st.work) return;
    st.minres_total += st.ms.iters;
    if (st.ms.breakdown) {
        st.status = TMOP_ERR_MINRES;
        st.done = 1;
    } else if (st.acc_h >= 0) {
        st.newton_its += 1;
        st.halvings = st.acc_h;
        st.F0 = st.F1;
        st.g0 = st.g1;
        st.md0 = st.md1;
        st.have_fg = 1;
    } else {
        st.status = TMOP_ERR_LINESEARCH;
        st.done = 1;
    }
    st.work = 0;
}

inline unsigned blocks_for(int n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace
}  // namespace tmop

using namespace tmop;

struct tmop_batch {
    tmop_batch_desc desc{};
    int d = 0, p = 0, nq = 0, np = 0, nqd = 0, ns = 0, vprec = 0, arith = 0;
    size_t rsz = 8;
    cudaStream_t stream = nullptr;
    double *tab = nullptr;
    float *tabf = nullptr;
    df *tabw = nullptr;
    BMesh *dM = nullptr;                 // device descriptors [capacity]
    BState *dS = nullptr;                // device states [capacity]
    BState *hS = nullptr;                // pinned mirror
    std::vector<BMesh> hM;
    std::vector<void *> slab;            // per-slot device slab
    std::vector<int64_t> slab_bytes;
    std::vector<char> used;
    // tile tables of the current subset
    int2 *dtile_e = nullptr, *dtile_n = nullptr, *dtile_v = nullptr;
    int *dmlist = nullptr;
    size_t cap_e = 0, cap_n = 0, cap_v = 0;
    int *hmlist = nullptr;
    int2 *hbuf = nullptr;
    size_t hbuf_cap = 0;
    int nt_e = 0, nt_n = 0, nt_v = 0, nm = 0;
    int64_t bytes = 0;
    std::vector<int> fault;              // host-side fault of a mesh's next step (tests)
    // the subset whose tables are on the device (valid while no mesh joins or leaves)
    std::vector<int> cur;
    bool cur_valid = false;
    int64_t mesh_ver = 0;                // counts joins and leaves
    // CUDA graphs of 4 MINRES iterations, one per phase of the 3-buffer rotation
    bool graphs = true;
    int64_t graph_launches = 0;
    struct BGraph {
        cudaGraphExec_t exec = nullptr;
        std::vector<int> subset;
        int64_t ver = -1;
        const void *te = nullptr, *tn = nullptr, *tv = nullptr;
        int variant = -1, nodes = 0;
    } bg[3];
};

namespace {

tmop_status bfail(tmop_status st, const std::string &m)
{
    set_last_error(m);
    return st;
}

#define BCK(call)                                                                          \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess) {                                                           \
            (void)cudaGetLastError();                                                      \
            return bfail(e_ == cudaErrorMemoryAllocation ? TMOP_ERR_OOM : TMOP_ERR_CUDA,   \
                         std::string(#call) + ": " + cudaGetErrorString(e_));              \
        }                                                                                  \
    } while (0)

// layout of one mesh slab: offsets of every buffer, 256-byte aligned
struct SlabPlan {
    int64_t off[24];
    int64_t map, ptr, idx, fixed;
    int64_t total;
};

SlabPlan plan_slab(const tmop_batch *b, int64_t E, int64_t Nx, bool has_fixed)
{
    SlabPlan s;
    int64_t o = 0;
    auto take = [&](int64_t bytes) {
        const int64_t r = o;
        o += ((bytes + 255) / 256) * 256;
        return r;
    };
    const int64_t ndof = (int64_t)b->d * Nx, ENP = E * b->np;
    const int64_t ntile = std::max<int64_t>(elem_blocks(b->d, b->p, b->nq, E), 1);
    const int64_t nchunk = std::max<int64_t>((ndof + VCH - 1) / VCH, 1);
    for (int i = 0; i < 24; ++i) s.off[i] = -1;
    s.map = take(4 * ENP);
    s.ptr = take(4 * (Nx + 1));
    s.idx = take(4 * ENP);
    s.fixed = has_fixed ? take(ndof) : -1;
    s.off[ROLE_X] = take(8 * ndof);
    s.off[ROLE_XT] = take(8 * ndof);
    s.off[ROLE_G] = take(8 * ndof);
    s.off[ROLE_DX] = take(8 * ndof);
    s.off[ROLE_H] = take((int64_t)b->rsz * E * h_stride(b->d, b->nq, b->ns, b->nqd) + 256);
    s.off[ROLE_EV64] = take(8 * b->d * ENP);
    s.off[ROLE_EVR] = (b->vprec == TMOP_FP32) ? take(4 * b->d * ENP) : s.off[ROLE_EV64];
    s.off[ROLE_DIAG] = take((int64_t)b->rsz * ndof);
    s.off[ROLE_MINV] = take((int64_t)b->rsz * ndof);
    s.off[ROLE_PART] = take(16 * ntile);
    s.off[ROLE_VPART] = take(8 * nchunk);
    for (int i = 0; i < 8; ++i) s.off[ROLE_KV0 + i] = take((int64_t)b->rsz * ndof);
    s.total = o;
    return s;
}

template <class T>
tmop_status ensure(T **dptr, size_t *cap, size_t need)
{
    if (need <= *cap) return TMOP_OK;
    if (*dptr) cudaFree(*dptr);
    *dptr = nullptr;
    BCK(cudaMalloc((void **)dptr, sizeof(T) * need));
    *cap = need;
    return TMOP_OK;
}

// Upload the tile tables of the meshes in ms (element, node and vector tiles).
tmop_status set_subset(tmop_batch *b, const std::vector<int> &ms)
{
    if (b->cur_valid && ms == b->cur) return TMOP_OK;     // the tables are on the device
    size_t ne = 0, nn = 0, nv = 0;
    for (int m : ms) {
        ne += b->hM[m].ntile_e;
        nn += (b->hM[m].P.Nx + NCH - 1) / NCH;
        nv += b->hM[m].nchunk;
    }
    const size_t tot = ne + nn + nv + ms.size();
    if (tot > b->hbuf_cap) {
        if (b->hbuf) cudaFreeHost(b->hbuf);
        b->hbuf = nullptr;
        BCK(cudaMallocHost((void **)&b->hbuf, sizeof(int2) * (tot + 16)));
        b->hbuf_cap = tot + 16;
    }
    int2 *te = b->hbuf, *tn = te + ne, *tv = tn + nn;
    int *ml = reinterpret_cast<int *>(tv + nv);
    size_t ie = 0, in = 0, iv = 0;
    for (size_t j = 0; j < ms.size(); ++j) {
        const int m = ms[j];
        for (int t = 0; t < b->hM[m].ntile_e; ++t) te[ie++] = make_int2(m, t);
        const int nnt = (int)((b->hM[m].P.Nx + NCH - 1) / NCH);
        for (int t = 0; t < nnt; ++t) tn[in++] = make_int2(m, t);
        for (int t = 0; t < b->hM[m].nchunk; ++t) tv[iv++] = make_int2(m, t);
        ml[j] = m;
    }
    tmop_status st;
    if ((st = ensure(&b->dtile_e, &b->cap_e, std::max<size_t>(ne, 1))) != TMOP_OK) return st;
    if ((st = ensure(&b->dtile_n, &b->cap_n, std::max<size_t>(nn, 1))) != TMOP_OK) return st;
    if ((st = ensure(&b->dtile_v, &b->cap_v, std::max<size_t>(nv, 1))) != TMOP_OK) return st;
    if (!b->dmlist) BCK(cudaMalloc((void **)&b->dmlist, sizeof(int) * b->desc.max_meshes));
    BCK(cudaStreamSynchronize(b->stream));   // previous launches may still read the tables
    if (ne) BCK(cudaMemcpyAsync(b->dtile_e, te, sizeof(int2) * ne, cudaMemcpyHostToDevice, b->stream));
    if (nn) BCK(cudaMemcpyAsync(b->dtile_n, tn, sizeof(int2) * nn, cudaMemcpyHostToDevice, b->stream));
    if (nv) BCK(cudaMemcpyAsync(b->dtile_v, tv, sizeof(int2) * nv, cudaMemcpyHostToDevice, b->stream));
    if (!ms.empty())
        BCK(cudaMemcpyAsync(b->dmlist, ml, sizeof(int) * ms.size(), cudaMemcpyHostToDevice, b->stream));
    BCK(cudaStreamSynchronize(b->stream));   // the pinned staging buffer is reused next time
    b->nt_e = (int)ne;
    b->nt_n = (int)nn;
    b->nt_v = (int)nv;
    b->nm = (int)ms.size();
    b->cur = ms;
    b->cur_valid = true;
    return TMOP_OK;
}

tmop_status read_states(tmop_batch *b)
{
    BCK(cudaMemcpyAsync(b->hS, b->dS, sizeof(BState) * b->desc.max_meshes, cudaMemcpyDeviceToHost,
                        b->stream));
    BCK(cudaStreamSynchronize(b->stream));
    return TMOP_OK;
}

BatchArgs bargs(const tmop_batch *b, int in, int aux, int out, bool stop)
{
    BatchArgs a;
    a.tiles = b->dtile_e;
    a.meshes = b->dM;
    a.in = in;
    a.aux = aux;
    a.out = out;
    a.stop = stop ? &b->dS[0].ms.stop_iter : nullptr;
    a.stop_stride = (int)(sizeof(BState) / sizeof(int));
    return a;
}

// energy and gradient of the current subset at role xr into (F, md) (which) and ROLE_G, g
tmop_status eval_fg(tmop_batch *b, int xr, int which)
{
    ElemParams P0{};
    // fused pass: energy / min det partials (aux role) and the element gradient
    BatchArgs a = bargs(b, xr, ROLE_PART, ROLE_EV64, false);
    BCK(launch_gradient(b->d, b->p, b->nq, P0, nullptr, nullptr, b->arith, b->stream, &a, b->nt_e));
    b_energy_final<<<b->nm, BT, 0, b->stream>>>(b->dM, b->dS, b->dmlist, which);
    count_launch();
    b_assemble<double, double><<<b->nt_n, NCH, 0, b->stream>>>(b->dM, b->dtile_n, ROLE_EV64, ROLE_G,
                                                                0, b->d, b->np, nullptr, 0);
    b_dot<double, double><<<b->nt_v, BT, 0, b->stream>>>(b->dM, b->dtile_v, ROLE_G, ROLE_G);
    b_norm_final<<<b->nm, BT, 0, b->stream>>>(b->dM, b->dS, b->dmlist, which);
    count_launch(4);
    BCK(cudaGetLastError());
    return TMOP_OK;
}

template <class R>
tmop_status setup_and_minres(tmop_batch *b)
{
    const tmop_batch_desc &D = b->desc;
    ElemParams P0{};
    P0.metric = b->desc.metric;            // selects the set-up kernel family
    BatchArgs a = bargs(b, ROLE_X, -1, ROLE_H, false);
    BCK(launch_hsetup(b->d, b->p, b->nq, P0, nullptr, nullptr, b->desc.hess_precision, b->stream, &a,
                      b->nt_e));
    a = bargs(b, -1, ROLE_H, ROLE_EVR, false);
    BCK(launch_diag(b->d, b->p, b->nq, P0, nullptr, nullptr, b->desc.hess_precision, b->stream, &a,
                    b->nt_e));
    b_assemble<R, R><<<b->nt_n, NCH, 0, b->stream>>>(b->dM, b->dtile_n, ROLE_EVR, ROLE_DIAG, 2, b->d,
                                                      b->np, nullptr, 0);
    b_jacobi<R><<<b->nt_v, BT, 0, b->stream>>>(b->dM, b->dtile_v);
    // buffers: v=0, R1=1, R2=2, Y=3, Z=7, W1=4, W2=5, W3=6
    int v = 0, R1 = 1, R2 = 2, Y = 3, Z = 7, W1 = 4, W2 = 5, W3 = 6;
    b_zero<R><<<b->nt_v, BT, 0, b->stream>>>(b->dM, b->dtile_v, W1, W2);
    b_minres_init<R><<<b->nt_v, BT, 0, b->stream>>>(b->dM, b->dtile_v, R1, R2, Y);
    b_minres_start<<<b->nm, BT, 0, b->stream>>>(b->dM, b->dS, b->dmlist);
    b_minres_scale<R><<<b->nt_v, BT, 0, b->stream>>>(b->dM, b->dtile_v, b->dS, Y, v);
    count_launch(6);
    BCK(cudaGetLastError());
    const int max_it = D.solver.minres_max_it;
    // The launches of one iteration, all with k = -1: the kernels take the
    // iteration from the per-mesh device counters, advanced by the first launch.
    constexpr int KD = -1;
    auto launch_iteration = [&]() -> tmop_status {
        b_iter_next<<<blocks_for(b->nm, 128), 128, 0, b->stream>>>(b->dS, b->dmlist, b->nm);
        count_launch();
        a = bargs(b, ROLE_KV0 + v, ROLE_H, ROLE_EVR, true);
        BCK(launch_apply(b->d, b->p, b->nq, P0, nullptr, nullptr, nullptr, b->desc.hess_precision,
                         nullptr, KD, b->stream, &a, b->nt_e));
        if constexpr (std::is_same<R, double>::value) {
            if (D.hess_precision == TMOP_FP64)      // float-pair element vectors
                b_assemble<df, double><<<b->nt_n, NCH, 0, b->stream>>>(
                    b->dM, b->dtile_n, ROLE_EVR, ROLE_KV0 + Z, 1, b->d, b->np, b->dS, KD);
            else
                b_assemble<R, R><<<b->nt_n, NCH, 0, b->stream>>>(b->dM, b->dtile_n, ROLE_EVR,
                                                                  ROLE_KV0 + Z, 1, b->d, b->np,
                                                                  b->dS, KD);
        } else {
            b_assemble<R, R><<<b->nt_n, NCH, 0, b->stream>>>(b->dM, b->dtile_n, ROLE_EVR, ROLE_KV0 + Z,
                                                              1, b->d, b->np, b->dS, KD);
        }
        b_lanczos_a<R><<<b->nt_v, BT, 0, b->stream>>>(b->dM, b->dtile_v, b->dS, Z, R1, v, KD);
        b_fin_alpha<<<b->nm, BT, 0, b->stream>>>(b->dM, b->dS, b->dmlist, KD);
        b_lanczos_b<R><<<b->nt_v, BT, 0, b->stream>>>(b->dM, b->dtile_v, b->dS, Z, R2, R1, KD);
        b_fin_beta<<<b->nm, BT, 0, b->stream>>>(b->dM, b->dS, b->dmlist, KD, D.solver.minres_rtol,
                                                D.solver.minres_fixed_its);
        b_minres_update<R><<<b->nt_v, BT, 0, b->stream>>>(b->dM, b->dtile_v, b->dS, v, W1, W2, W3, R1,
                                                           KD);
        count_launch(6);
        BCK(cudaGetLastError());
        return TMOP_OK;
    };
    auto rotate = [&] {
        const int oR1 = R1;
        R1 = R2;
        R2 = Z;
        Z = Y;
        Y = oR1;
        const int oW1 = W1;
        W1 = W2;
        W2 = W3;
        W3 = oW1;
    };
    // Blocks of 4 iterations as CUDA graphs (not on the legacy stream); the
    // graph of a phase is captured once and replayed while the subset, its
    // tables and the kernel variant stay the same.
    const bool graphs = b->graphs && b->stream != nullptr;
    const int variant = apply_variant(b->d, b->p, b->nq, D.hess_precision);
    int k = 0;
    while (k < max_it) {
        if (graphs && max_it - k >= 4) {
            tmop_batch::BGraph &g = b->bg[(k / 4) % 3];
            if (!g.exec || g.subset != b->cur || g.ver != b->mesh_ver || g.te != b->dtile_e ||
                g.tn != b->dtile_n || g.tv != b->dtile_v || g.variant != variant) {
                if (g.exec) cudaGraphExecDestroy(g.exec);
                g.exec = nullptr;
                cudaGraph_t graph = nullptr;
                BCK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
                const int64_t l0 = thread_launches();
                tmop_status st = TMOP_OK;
                for (int j = 0; j < 4 && st == TMOP_OK; ++j) {
                    st = launch_iteration();
                    rotate();
                }
                const cudaError_t ec = cudaStreamEndCapture(b->stream, &graph);
                if (st != TMOP_OK) {
                    if (graph) cudaGraphDestroy(graph);
                    return st;
                }
                BCK(ec);
                const cudaError_t ei = cudaGraphInstantiate(&g.exec, graph, 0);
                cudaGraphDestroy(graph);
                if (ei != cudaSuccess) {
                    g.exec = nullptr;
                    BCK(ei);
                }
                g.subset = b->cur;
                g.ver = b->mesh_ver;
                g.te = b->dtile_e;
                g.tn = b->dtile_n;
                g.tv = b->dtile_v;
                g.variant = variant;
                g.nodes = (int)(thread_launches() - l0);
                uncount_launches(g.nodes);                    // counted at each graph launch
            } else {
                for (int j = 0; j < 4; ++j) rotate();
            }
            BCK(cudaGraphLaunch(g.exec, b->stream));
            count_launch(g.nodes);
            ++b->graph_launches;
            k += 4;
        } else {
            tmop_status st = launch_iteration();
            if (st != TMOP_OK) return st;
            rotate();
            ++k;
        }
        if (!D.solver.minres_fixed_its && k % 4 == 0 && k < max_it) {
            tmop_status st = read_states(b);
            if (st != TMOP_OK) return st;
            bool all = true;
            for (int m = 0; m < D.max_meshes; ++m)
                if (b->used[m] && b->hS[m].work && b->hS[m].ms.stop_iter > k) all = false;
            if (all) break;
        }
    }
    return TMOP_OK;
}

template <class R>
tmop_status line_search(tmop_batch *b, std::vector<int> pending)
{
    const tmop_batch_desc &D = b->desc;
    for (int h = 0; h <= D.solver.ls_max_halvings && !pending.empty(); ++h) {
        tmop_status st = set_subset(b, pending);
        if (st != TMOP_OK) return st;
        b_trial<<<b->nt_v, BT, 0, b->stream>>>(b->dM, b->dtile_v, b->dS, h);
        count_launch();
        if ((st = eval_fg(b, ROLE_XT, 1)) != TMOP_OK) return st;
        b_ls_decide<<<blocks_for(b->nm, 128), 128, 0, b->stream>>>(b->dS, b->dmlist, b->nm,
                                                                  D.solver.ls_factor, h);
        b_accept_copy<<<b->nt_v, BT, 0, b->stream>>>(b->dM, b->dtile_v, b->dS, h);
        count_launch(2);
        if ((st = read_states(b)) != TMOP_OK) return st;
        std::vector<int> next;
        for (int m : pending)
            if (b->hS[m].acc_h < 0) next.push_back(m);
        pending.swap(next);
    }
    return TMOP_OK;
}

}  // namespace

extern "C" {

tmop_status tmop_batch_create(const tmop_batch_desc *desc, void *cuda_stream, tmop_batch **out)
{
    if (!desc || !out) return bfail(TMOP_ERR_ARG, "desc and out must not be NULL");
    *out = nullptr;
    const tmop_batch_desc &D = *desc;
    if (D.dim != 2 && D.dim != 3) return bfail(TMOP_ERR_ARG, "dim must be 2 or 3");
    if (!elem_supported(D.dim, D.order, D.nq1d))
        return bfail(TMOP_ERR_UNSUPPORTED, "order must be 1..4 and nq1d order+1, order+2 (or 9 in 3D)");
    const bool mok = metric_valid(D.metric, D.dim);
    if (!mok) return bfail(TMOP_ERR_UNSUPPORTED, "metric not defined for this dim");
    if (D.target == TMOP_TARGET_DISCRETE)
        return bfail(TMOP_ERR_UNSUPPORTED, "the discrete target needs a field per mesh: tmop_setup only");
    if (D.target != TMOP_TARGET_IDENTITY && D.target != TMOP_TARGET_SIZE_FIELD)
        return bfail(TMOP_ERR_ARG, "unknown target");
    if (D.hess_precision != TMOP_FP64 && D.hess_precision != TMOP_FP32 &&
        D.hess_precision != TMOP_FP64_NATIVE)
        return bfail(TMOP_ERR_ARG, "bad hess_precision");
    if (D.max_meshes < 1 || D.max_meshes > (1 << 20)) return bfail(TMOP_ERR_ARG, "bad max_meshes");
    if (D.solver.minres_max_it < 0 || D.solver.ls_max_halvings < 0)
        return bfail(TMOP_ERR_ARG, "negative iteration limit");
    tmop_batch *b = new tmop_batch();
    b->desc = D;
    b->d = D.dim;
    b->p = D.order;
    b->nq = D.nq1d;
    b->np = 1;
    b->nqd = 1;
    for (int k = 0; k < D.dim; ++k) {
        b->np *= D.order + 1;
        b->nqd *= D.nq1d;
    }
    b->ns = (b->d * b->d) * (b->d * b->d + 1) / 2;
    b->vprec = D.hess_precision == TMOP_FP32 ? TMOP_FP32 : TMOP_FP64;
    b->arith = D.hess_precision == TMOP_FP64_NATIVE ? ARITH_NATIVE : ARITH_DW;
    b->rsz = b->vprec == TMOP_FP32 ? 4 : 8;
    b->stream = static_cast<cudaStream_t>(cuda_stream);
    b->hM.resize(D.max_meshes);
    b->slab.assign(D.max_meshes, nullptr);
    b->slab_bytes.assign(D.max_meshes, 0);
    b->used.assign(D.max_meshes, 0);
    b->fault.assign(D.max_meshes, TMOP_FAULT_NONE);
    auto bail = [&](tmop_status st) {
        tmop_batch_destroy(b);
        return st;
    };
    const int tabn = 2 * b->nq * (b->p + 1) + b->nq;
    std::vector<double> tab(tabn);
    std::vector<float> tabf(tabn);
    std::vector<df> tabw(tabn);
    host_basis_tables(b->p + 1, b->nq, tab.data(), tab.data() + b->nq * (b->p + 1),
                      tab.data() + 2 * b->nq * (b->p + 1));
    for (int i = 0; i < tabn; ++i) {
        tabf[i] = (float)tab[i];
        tabw[i] = df(tab[i]);
    }
    cudaError_t e = cudaSuccess;
    if ((e = cudaMalloc((void **)&b->tab, 8 * tabn)) || (e = cudaMalloc((void **)&b->tabf, 4 * tabn)) ||
        (e = cudaMalloc((void **)&b->tabw, 8 * tabn)) ||
        (e = cudaMalloc((void **)&b->dM, sizeof(BMesh) * D.max_meshes)) ||
        (e = cudaMalloc((void **)&b->dS, sizeof(BState) * D.max_meshes)) ||
        (e = cudaMallocHost((void **)&b->hS, sizeof(BState) * D.max_meshes)) ||
        (e = cudaMemcpy(b->tab, tab.data(), 8 * tabn, cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy(b->tabf, tabf.data(), 4 * tabn, cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy(b->tabw, tabw.data(), 8 * tabn, cudaMemcpyHostToDevice)) ||
        (e = cudaMemset(b->dS, 0, sizeof(BState) * D.max_meshes))) {
        (void)cudaGetLastError();
        set_last_error(std::string("batch allocation: ") + cudaGetErrorString(e));
        return bail(e == cudaErrorMemoryAllocation ? TMOP_ERR_OOM : TMOP_ERR_CUDA);
    }
    std::memset(b->hS, 0, sizeof(BState) * D.max_meshes);
    *out = b;
    return TMOP_OK;
}

int64_t tmop_batch_mesh_bytes(const tmop_batch *b, int64_t num_elems, int64_t num_nodes)
{
    if (!b || num_elems < 0 || num_nodes <= 0) return -1;
    return plan_slab(b, num_elems, num_nodes, true).total;
}

int64_t tmop_batch_device_bytes(const tmop_batch *b) { return b ? b->bytes : 0; }

tmop_status tmop_batch_add(tmop_batch *b, int64_t num_elems, int64_t num_nodes,
                           const int32_t *elem_to_node, const uint8_t *fixed, const double *x,
                           double target_h0, int *slot_out)
{
    if (!b || !x || !slot_out || num_nodes <= 0 || num_elems < 0)
        return bfail(TMOP_ERR_ARG, "bad argument");
    if (num_elems > 0 && !elem_to_node) return bfail(TMOP_ERR_ARG, "elem_to_node is NULL");
    if (b->desc.target == TMOP_TARGET_SIZE_FIELD && !(target_h0 > 0.0))
        return bfail(TMOP_ERR_ARG, "target_h0 must be > 0");
    if (num_elems * (int64_t)b->np >= INT_MAX) return bfail(TMOP_ERR_ARG, "mesh too large");
    int slot = -1;
    for (int m = 0; m < b->desc.max_meshes; ++m)
        if (!b->used[m]) { slot = m; break; }
    if (slot < 0) return bfail(TMOP_ERR_ARG, "batch is full");
    const int64_t ndof = (int64_t)b->d * num_nodes, ENP = num_elems * b->np;
    // element map -> host, validate, transpose
    std::vector<int32_t> hmap((size_t)ENP);
    if (ENP) {
        BCK(cudaMemcpyAsync(hmap.data(), elem_to_node, 4 * ENP, cudaMemcpyDeviceToHost, b->stream));
        BCK(cudaStreamSynchronize(b->stream));
    }
    std::vector<int32_t> ptr((size_t)num_nodes + 1, 0), idx((size_t)ENP);
    for (int64_t j = 0; j < ENP; ++j) {
        if (hmap[j] < 0 || hmap[j] >= num_nodes)
            return bfail(TMOP_ERR_ARG, "elem_to_node entry out of range");
        ptr[hmap[j] + 1]++;
    }
    for (int64_t i = 0; i < num_nodes; ++i) ptr[i + 1] += ptr[i];
    {
        std::vector<int32_t> fill(ptr.begin(), ptr.end() - 1);
        for (int64_t j = 0; j < ENP; ++j) idx[fill[hmap[j]]++] = (int32_t)j;
    }
    const SlabPlan sp = plan_slab(b, num_elems, num_nodes, fixed != nullptr);
    char *base = nullptr;
    BCK(cudaMalloc((void **)&base, sp.total));
    b->slab[slot] = base;
    b->slab_bytes[slot] = sp.total;
    b->bytes += sp.total;
    BMesh M;
    std::memset(&M, 0, sizeof(M));
    M.P.map = reinterpret_cast<const int32_t *>(base + sp.map);
    M.P.E = num_elems;
    M.P.Nx = num_nodes;
    M.P.tab = b->tab;
    M.P.tabf = b->tabf;
    M.P.tabw = b->tabw;
    M.P.metric = b->desc.metric;
    M.P.target = b->desc.target;
    M.P.h0 = target_h0;
    M.csr_ptr = reinterpret_cast<const int32_t *>(base + sp.ptr);
    M.csr_idx = reinterpret_cast<const int32_t *>(base + sp.idx);
    M.fixed = fixed ? reinterpret_cast<const uint8_t *>(base + sp.fixed) : nullptr;
    for (int i = 0; i < 24; ++i) M.ptr[i] = sp.off[i] >= 0 ? base + sp.off[i] : nullptr;
    M.ndof = ndof;
    M.ntile_e = (int)std::max<int64_t>(elem_blocks(b->d, b->p, b->nq, num_elems), 0);
    M.nchunk = (int)((ndof + VCH - 1) / VCH);
    if (ENP) {
        BCK(cudaMemcpyAsync(base + sp.map, hmap.data(), 4 * ENP, cudaMemcpyHostToDevice, b->stream));
        BCK(cudaMemcpyAsync(base + sp.idx, idx.data(), 4 * ENP, cudaMemcpyHostToDevice, b->stream));
    }
    BCK(cudaMemcpyAsync(base + sp.ptr, ptr.data(), 4 * (num_nodes + 1), cudaMemcpyHostToDevice, b->stream));
    if (fixed) BCK(cudaMemcpyAsync(base + sp.fixed, fixed, ndof, cudaMemcpyDeviceToDevice, b->stream));
    BCK(cudaMemcpyAsync(M.ptr[ROLE_X], x, 8 * ndof, cudaMemcpyDeviceToDevice, b->stream));
    BCK(cudaMemcpyAsync(&b->dM[slot], &M, sizeof(BMesh), cudaMemcpyHostToDevice, b->stream));
    BState S0;
    std::memset(&S0, 0, sizeof(S0));
    S0.first = 1;
    S0.acc_h = -1;
    BCK(cudaMemcpyAsync(&b->dS[slot], &S0, sizeof(BState), cudaMemcpyHostToDevice, b->stream));
    BCK(cudaStreamSynchronize(b->stream));   // host staging (hmap, idx, ptr, M, S0) goes out of scope
    b->hM[slot] = M;
    b->hS[slot] = S0;
    b->used[slot] = 1;
    b->cur_valid = false;
    ++b->mesh_ver;
    b->fault[slot] = TMOP_FAULT_NONE;
    *slot_out = slot;
    return TMOP_OK;
}

tmop_status tmop_batch_remove(tmop_batch *b, int slot)
{
    if (!b || slot < 0 || slot >= b->desc.max_meshes || !b->used[slot])
        return bfail(TMOP_ERR_ARG, "bad slot");
    BCK(cudaStreamSynchronize(b->stream));
    cudaFree(b->slab[slot]);
    b->bytes -= b->slab_bytes[slot];
    b->slab[slot] = nullptr;
    b->slab_bytes[slot] = 0;
    b->used[slot] = 0;
    b->cur_valid = false;
    ++b->mesh_ver;
    return TMOP_OK;
}

tmop_status tmop_batch_step(tmop_batch *b, int *n_active)
{
    if (!b) return bfail(TMOP_ERR_ARG, "NULL batch");
    tmop_status st;
    std::vector<int> act, need;
    for (int m = 0; m < b->desc.max_meshes; ++m)
        if (b->used[m] && !b->hS[m].done) {
            act.push_back(m);
            if (!b->hS[m].have_fg) need.push_back(m);
        }
    if (n_active) *n_active = 0;
    if (act.empty()) return TMOP_OK;
    if (!need.empty()) {
        if ((st = set_subset(b, need)) != TMOP_OK) return st;
        if ((st = eval_fg(b, ROLE_X, 0)) != TMOP_OK) return st;
    }
    if ((st = set_subset(b, act)) != TMOP_OK) return st;
    b_prep<<<blocks_for(b->nm, 128), 128, 0, b->stream>>>(b->dS, b->dmlist, b->nm,
                                                        b->desc.newton_rtol, b->desc.newton_max_it);
    count_launch();
    BCK(cudaGetLastError());
    if ((st = read_states(b)) != TMOP_OK) return st;
    std::vector<int> work;
    for (int m : act)
        if (b->hS[m].work) work.push_back(m);
    if (!work.empty()) {
        if ((st = set_subset(b, work)) != TMOP_OK) return st;
        st = (b->vprec == TMOP_FP32) ? setup_and_minres<float>(b) : setup_and_minres<double>(b);
        if (st != TMOP_OK) return st;
        if ((st = read_states(b)) != TMOP_OK) return st;
        // a mesh whose MINRES broke down takes no line search: its positions stay
        // as they are and b_finish retires it with TMOP_ERR_MINRES
        std::vector<int> search;
        for (int m : work) {
            if (b->fault[m] == TMOP_FAULT_MINRES_BREAKDOWN) {     // tmop_batch_inject_fault
                b->fault[m] = TMOP_FAULT_NONE;
                b->hS[m].ms.breakdown = 1;
                BCK(cudaMemcpyAsync(&b->dS[m].ms.breakdown, &b->hS[m].ms.breakdown, sizeof(int),
                                    cudaMemcpyHostToDevice, b->stream));
            }
            if (!b->hS[m].ms.breakdown) search.push_back(m);
        }
        if (!search.empty()) {
            st = (b->vprec == TMOP_FP32) ? line_search<float>(b, search)
                                         : line_search<double>(b, search);
            if (st != TMOP_OK) return st;
        }
        if ((st = set_subset(b, work)) != TMOP_OK) return st;
        b_finish<<<blocks_for(b->nm, 128), 128, 0, b->stream>>>(b->dS, b->dmlist, b->nm);
        count_launch();
        BCK(cudaGetLastError());
        if ((st = read_states(b)) != TMOP_OK) return st;
    }
    int n = 0;
    for (int m = 0; m < b->desc.max_meshes; ++m)
        if (b->used[m] && !b->hS[m].done) ++n;
    if (n_active) *n_active = n;
    return TMOP_OK;
}

tmop_status tmop_batch_set_graphs(tmop_batch *b, int on)
{
    if (!b) return bfail(TMOP_ERR_ARG, "NULL batch");
    b->graphs = on != 0;
    return TMOP_OK;
}

int64_t tmop_batch_graph_launches(const tmop_batch *b) { return b ? b->graph_launches : 0; }

tmop_status tmop_batch_inject_fault(tmop_batch *b, int slot, int fault)
{
    if (!b || slot < 0 || slot >= b->desc.max_meshes || !b->used[slot] ||
        (fault != TMOP_FAULT_NONE && fault != TMOP_FAULT_MINRES_BREAKDOWN))
        return bfail(TMOP_ERR_ARG, "bad slot or unknown fault");
    b->fault[slot] = fault;
    return TMOP_OK;
}

tmop_status tmop_batch_state(tmop_batch *b, int slot, tmop_mesh_state *out)
{
    if (!b || !out || slot < 0 || slot >= b->desc.max_meshes || !b->used[slot])
        return bfail(TMOP_ERR_ARG, "bad slot");
    const BState &s = b->hS[slot];
    out->done = s.done;
    out->status = s.status;
    out->newton_its = s.newton_its;
    out->minres_its = s.minres_total;
    out->energy0 = s.energy_first;
    out->energy = s.F0;
    out->grad_norm0 = s.gfirst;
    out->grad_norm = s.g0;
    out->min_det = s.md0;
    out->alpha = s.alpha;
    return TMOP_OK;
}

tmop_status tmop_batch_positions(tmop_batch *b, int slot, double *x_out)
{
    if (!b || !x_out || slot < 0 || slot >= b->desc.max_meshes || !b->used[slot])
        return bfail(TMOP_ERR_ARG, "bad slot");
    BCK(cudaMemcpyAsync(x_out, b->hM[slot].ptr[ROLE_X], 8 * b->hM[slot].ndof, cudaMemcpyDeviceToDevice,
                        b->stream));
    return TMOP_OK;
}

void tmop_batch_destroy(tmop_batch *b)
{
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    for (auto &g : b->bg)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    for (void *p : b->slab)
        if (p) cudaFree(p);
    cudaFree(b->tab);
    cudaFree(b->tabf);
    cudaFree(b->tabw);
    cudaFree(b->dM);
    cudaFree(b->dS);
    cudaFree(b->dtile_e);
    cudaFree(b->dtile_n);
    cudaFree(b->dtile_v);
    cudaFree(b->dmlist);
    if (b->hS) cudaFreeHost(b->hS);
    if (b->hbuf) cudaFreeHost(b->hbuf);
    delete b;
}

}  // extern "C"
