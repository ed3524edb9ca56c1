"""Write csrc/autotune_table.h (the compiled-in defaults of the Hessian-action
kernel variant per configuration) from autotune_table.json, the rows that
``bench.py --workload autotune`` measured on a B300:

    python -m paper_2205_12721_b300.autotune_gen [autotune_table.json]
"""
from __future__ import annotations

import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))


def write_header(rows, path=os.path.join(HERE, "csrc", "autotune_table.h")):
    ents = sorted({(r["d"], r["p"], r["nq"], r["prec"], r["variant"]) for r in rows})
    body = ",\n".join("    {%d, %d, %d, %d, %d}" % e for e in ents)
    text = f"""// Hessian-action kernel variant per (dim, order, nq1d, precision), measured
// on a B300 by the autotuner (bench.py --workload autotune); generated by
// paper_2205_12721_b300/autotune_gen.py from autotune_table.json.  prec:
// 0 = TMOP_FP64 (double-float), 1 = TMOP_FP32, 2 = TMOP_FP64_NATIVE.  Variant
// numbers: elem_apply_impl.cuh.
#pragma once

namespace tmop {{

struct ApplyTuned {{
    int d, p, q, prec, variant;
}};

static const ApplyTuned kApplyTuned[] = {{
{body},
}};

}}  // namespace tmop
"""
    with open(path, "w") as f:
        f.write(text)
    return path


def main(argv):
    src = argv[1] if len(argv) > 1 else os.path.join(HERE, "autotune_table.json")
    with open(src) as f:
        data = json.load(f)
    rows = data["rows"] if isinstance(data, dict) else data
    print(write_header(rows))


if __name__ == "__main__":
    main(sys.argv)
