// tmop_energy_noalloc: the energy / min det(A) computation for callers that
// must not allocate device memory.  It runs the same energy kernel and final
// reduction as tmop_energy, but its scratch (per-CTA partial sums and the 1D
// basis tables) lives in one file-scope device array instead of memory a
// context allocates.
#include <cmath>
#include <mutex>
#include <string>

#include "tmop_device.cuh"
#include "tmop_internal.h"

namespace {

constexpr int kMaxCtas = 65536;                   // partial (sum, min) pairs
constexpr int kTableOffset = 2 * kMaxCtas;        // 1D tables follow the partials
constexpr int kTableMax = 128;                    // B, G, w of one (p+1, nq) pair, FP64
static_assert(2 * 9 * 5 + 9 <= kTableMax, "the 9-point rule at p = 4 must fit a table slot");
// One slot per (p+1, nq) pair of the supported configurations: the FP64
// tables, then the same values as double-float pairs (8 bytes each).
constexpr int kSlots = 12;
constexpr int kSlotDoubles = 2 * kTableMax;
constexpr int kScratchDoubles = kTableOffset + kSlots * kSlotDoubles;

// Shared by every call in the process on this device; holds the last call's
// partial sums (and the tables, written once) until the library is unloaded.
static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double *g_scratch_addr[kMaxDevices] = {nullptr};

tmop_status set_error(tmop_status st, const std::string &m)
{
    tmop::set_last_error(m);
    return st;
}

// Table slot of a (p+1, nq) pair, -1 if none.
int slot_of(int ni, int nq)
{
    static const int pairs[kSlots][2] = {{2, 2}, {2, 3}, {3, 3}, {3, 4}, {4, 4}, {4, 5},
                                         {5, 5}, {5, 6}, {2, 9}, {3, 9}, {4, 9}, {5, 9}};
    for (int i = 0; i < kSlots; ++i)
        if (pairs[i][0] == ni && pairs[i][1] == nq) return i;
    return -1;
}

// Device address of the scratch array for the current device.  The first
// call on a device looks it up (host code cannot use the symbol itself as a
// device pointer) and writes the tables of every configuration into their
// slots with one synchronous copy; later calls only read them.
tmop_status scratch_for_current_device(double **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return set_error(TMOP_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return set_error(TMOP_ERR_ARG, "device index too large");
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess)
            return set_error(TMOP_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        static double host[kSlots * kSlotDoubles];
        for (int ni = 2; ni <= 5; ++ni)
            for (int nq = 2; nq <= 9; ++nq) {
                const int sl = slot_of(ni, nq);
                if (sl < 0) continue;
                double *tab = host + sl * kSlotDoubles;
                tmop::host_basis_tables(ni, nq, tab, tab + nq * ni, tab + 2 * nq * ni);
                tmop::df *tabw = reinterpret_cast<tmop::df *>(tab + kTableMax);
                for (int i = 0; i < 2 * nq * ni + nq; ++i) tabw[i] = tmop::df(tab[i]);
            }
        e = cudaMemcpy(static_cast<double *>(p) + kTableOffset, host, sizeof(host),
                       cudaMemcpyHostToDevice);
        if (e != cudaSuccess)
            return set_error(TMOP_ERR_CUDA, std::string("table upload: ") + cudaGetErrorString(e));
        g_scratch_addr[dev] = static_cast<double *>(p);
    }
    *out = g_scratch_addr[dev];
    return TMOP_OK;
}

}  // namespace

extern "C" tmop_status tmop_energy_noalloc(const tmop_desc *desc, const int32_t *elem_to_node,
                                           const double *x, double *out, void *cuda_stream)
{
    using namespace tmop;
    if (!desc || !x || !out) return set_error(TMOP_ERR_ARG, "desc, x and out must not be NULL");
    const tmop_desc &D = *desc;
    if (D.dim != 2 && D.dim != 3) return set_error(TMOP_ERR_ARG, "dim must be 2 or 3");
    if (!elem_supported(D.dim, D.order, D.nq1d))
        return set_error(TMOP_ERR_UNSUPPORTED, "order must be 1..4 and nq1d order+1, order+2 (or 9 in 3D)");
    const bool metric_ok = metric_valid(D.metric, D.dim);
    if (!metric_ok) return set_error(TMOP_ERR_UNSUPPORTED, "metric not defined for this dim");
    if (D.target == TMOP_TARGET_DISCRETE)
        return set_error(TMOP_ERR_UNSUPPORTED, "the discrete target needs a field per mesh: tmop_setup only");
    if (D.target != TMOP_TARGET_IDENTITY && D.target != TMOP_TARGET_SIZE_FIELD)
        return set_error(TMOP_ERR_ARG, "unknown target");
    if (D.target == TMOP_TARGET_SIZE_FIELD && !(D.target_h0 > 0.0))
        return set_error(TMOP_ERR_ARG, "target_h0 must be > 0");
    if (D.num_elems < 0 || D.num_nodes <= 0) return set_error(TMOP_ERR_ARG, "bad mesh sizes");
    if (D.limit_delta != 0.0)
        return set_error(TMOP_ERR_UNSUPPORTED, "the limiting term is not available without a context");
    if (D.hess_precision != TMOP_FP64 && D.hess_precision != TMOP_FP32 &&
        D.hess_precision != TMOP_FP64_NATIVE)
        return set_error(TMOP_ERR_ARG, "hess_precision must be TMOP_FP64, TMOP_FP32 or TMOP_FP64_NATIVE");
    const int64_t nb = elem_blocks(D.dim, D.order, D.nq1d, D.num_elems);
    if (nb > kMaxCtas)
        return set_error(TMOP_ERR_ARG, "mesh too large for tmop_energy_noalloc: needs " +
                                           std::to_string(nb) + " CTAs, the static scratch holds " +
                                           std::to_string(kMaxCtas) + "; use tmop_energy");
    if (D.num_elems > 0 && !elem_to_node) return set_error(TMOP_ERR_ARG, "elem_to_node is NULL");
    const int sl = slot_of(D.order + 1, D.nq1d);
    if (sl < 0) return set_error(TMOP_ERR_UNSUPPORTED, "no table slot for this (order, nq1d)");

    double *scratch = nullptr;
    tmop_status st = scratch_for_current_device(&scratch);
    if (st != TMOP_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);

    // the tables of this configuration, written by the first call on the device
    const double *tab = scratch + kTableOffset + sl * kSlotDoubles;
    ElemParams P;
    P.map = elem_to_node;
    P.E = D.num_elems;
    P.Nx = D.num_nodes;
    P.tab = tab;
    P.tabf = nullptr;
    P.tabw = reinterpret_cast<const df *>(tab + kTableMax);
    P.metric = D.metric;
    P.target = D.target;
    P.h0 = D.target_h0;
    // every partial slot the reduction reads is written by this launch, so
    // nothing in the scratch needs clearing first
    const int arith = D.hess_precision == TMOP_FP64_NATIVE ? ARITH_NATIVE : ARITH_DW;
    cudaError_t e = launch_energy(D.dim, D.order, D.nq1d, P, x, scratch, arith, s);
    if (e == cudaSuccess) e = launch_finalize_energy(scratch, nb, out, s);
    if (e != cudaSuccess) return set_error(TMOP_ERR_CUDA, std::string("energy launch: ") + cudaGetErrorString(e));
    return TMOP_OK;
}
