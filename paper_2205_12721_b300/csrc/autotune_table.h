// Hessian-action kernel variant per (dim, order, nq1d, precision), measured
// on a B300 by the autotuner (bench.py --workload autotune); generated by
// paper_2205_12721_b300/autotune_gen.py from autotune_table.json.  prec:
// 0 = TMOP_FP64 (double-float), 1 = TMOP_FP32, 2 = TMOP_FP64_NATIVE.  Variant
// numbers: elem_apply_impl.cuh.
#pragma once

namespace tmop {

struct ApplyTuned {
    int d, p, q, prec, variant;
};

static const ApplyTuned kApplyTuned[] = {
    {3, 1, 2, 0, 14},
    {3, 1, 2, 1, 4},
    {3, 1, 2, 2, 1},
    {3, 1, 3, 0, 3},
    {3, 1, 3, 1, 4},
    {3, 1, 3, 2, 0},
    {3, 2, 3, 0, 18},
    {3, 2, 3, 1, 17},
    {3, 2, 3, 2, 2},
    {3, 2, 4, 0, 18},
    {3, 2, 4, 1, 2},
    {3, 2, 4, 2, 1},
    {3, 3, 4, 0, 13},
    {3, 3, 4, 1, 17},
    {3, 3, 4, 2, 2},
    {3, 3, 5, 0, 5},
    {3, 3, 5, 1, 17},
    {3, 3, 5, 2, 0},
    {3, 4, 5, 0, 7},
    {3, 4, 5, 1, 17},
    {3, 4, 5, 2, 6},
};

}  // namespace tmop
