// Hessian-action dispatch: precision, configuration and the kernel variant of
// the process-wide table (autotune_table.h defaults, tmop_set_apply_variant /
// tmop_autotune updates).
#include <atomic>

#include "autotune_table.h"
#include "elem_launch.cuh"

namespace tmop {

cudaError_t launch_apply_df(int d, int p, int q, const ElemParams &P, const void *v, const void *H,
                            void *ev, const int *stop, int k, cudaStream_t s, const BatchArgs *B,
                            int64_t ntiles, int variant);
cudaError_t launch_apply_f32(int d, int p, int q, const ElemParams &P, const void *v, const void *H,
                             void *ev, const int *stop, int k, cudaStream_t s, const BatchArgs *B,
                             int64_t ntiles, int variant);
cudaError_t launch_apply_f64(int d, int p, int q, const ElemParams &P, const void *v, const void *H,
                             void *ev, const int *stop, int k, cudaStream_t s, const BatchArgs *B,
                             int64_t ntiles, int variant);

namespace {

constexpr int kSlots = (TMOP_KEY(3, 4, 9) + 1) * 3;
std::atomic<int> g_variant[kSlots];           // 0 = not set, else variant + 1

int slot_of(int d, int p, int q, int prec) { return TMOP_KEY(d, p, q) * 3 + prec; }

}  // namespace

int apply_variant_count(int d, int p, int q)
{
    switch (TMOP_KEY(d, p, q)) {
#define CASE(D_, P_, Q_) \
    case TMOP_KEY(D_, P_, Q_): return (D_ == 3 && Q_ * Q_ <= 32) ? 19 : 1;
        TMOP_CONFIGS(CASE)
#undef CASE
        default: return 0;
    }
}

int apply_variant(int d, int p, int q, int prec)
{
    const int n = apply_variant_count(d, p, q);
    if (n <= 1 || prec < 0 || prec > 2) return 0;
    const int set = g_variant[slot_of(d, p, q, prec)].load(std::memory_order_relaxed);
    if (set > 0) return set - 1;
    for (const ApplyTuned &t : kApplyTuned)
        if (t.d == d && t.p == p && t.q == q && t.prec == prec && t.variant < n) return t.variant;
    return 3;                                  // shared-memory columns, 4 warps per CTA
}

bool set_apply_variant(int d, int p, int q, int prec, int variant)
{
    const int n = apply_variant_count(d, p, q);
    if (n == 0 || prec < 0 || prec > 2 || variant < -1 || variant >= n) return false;
    g_variant[slot_of(d, p, q, prec)].store(variant + 1, std::memory_order_relaxed);
    return true;
}

cudaError_t launch_apply(int d, int p, int q, const ElemParams &P, const void *v, const void *H,
                         void *ev, int prec, const int *stop_iter, int k, cudaStream_t s,
                         const BatchArgs *B, int64_t ntiles)
{
    const int var = apply_variant(d, p, q, prec);
    if (prec == TMOP_FP32)
        return launch_apply_f32(d, p, q, P, v, H, ev, stop_iter, k, s, B, ntiles, var);
    if (prec == TMOP_FP64_NATIVE)
        return launch_apply_f64(d, p, q, P, v, H, ev, stop_iter, k, s, B, ntiles, var);
    return launch_apply_df(d, p, q, P, v, H, ev, stop_iter, k, s, B, ntiles, var);
}

}  // namespace tmop
