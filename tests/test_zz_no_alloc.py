"""tmop_energy_noalloc against tmop_energy and the FP64 oracle, through the C
ABI.

tmop_energy_noalloc serves callers that cannot call cudaMalloc (for example
code embedded in an application whose pool allocator already owns the device
memory, or latency-bound loops where an allocation would synchronise the
device).  It keeps its scratch in a static device array instead of a
context, so two calls in a row must both reproduce the context-based result
and the oracle's, in every arithmetic (double-float and native FP64) and
target it accepts; a mesh too large for that array, or an unknown
precision, must be refused up front.  This file is collected last so that a
failure here cannot hide the other tests."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2205_12721_b300 import capi, meshgen

pytestmark = pytest.mark.gpu

TOL = 1e-12


def _check_case(m, metric, nq=None, target=capi.TARGET_IDENTITY, h0=1.0, prec=capi.FP64):
    nq = nq or m.order + 1
    desc = capi.Desc(m.dim, m.order, nq, m.num_elems, m.num_nodes, metric, target, h0, prec)
    emap = torch.from_numpy(np.ascontiguousarray(m.map)).cuda()
    fixed = torch.from_numpy(m.fixed).cuda()
    x = torch.from_numpy(m.x).cuda()
    ctx = capi.tmop_setup(desc, emap, fixed)
    try:
        st, F_ref, md_ref = capi.tmop_energy(ctx, x)
        assert st == capi.OK
    finally:
        capi.tmop_destroy(ctx)
    om = O.Mesh(m.dim, m.order, nq, m.map, m.num_nodes, metric, m.fixed, target, h0)
    st_o, F_o, md_o, S = O.energy(om, m.x)
    assert st_o == 0
    for _ in range(2):                        # two calls in a row share the scratch
        out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
        st = capi.tmop_energy_noalloc(desc, emap, x, out)
        assert st == capi.OK, capi.last_error()
        torch.cuda.synchronize()
        F, md = out.tolist()
        assert abs(F - F_ref) <= TOL * max(abs(F_ref), S), (F, F_ref)
        assert abs(F - F_o) <= TOL * max(abs(F_o), S), (F, F_o)
        assert abs(md - md_ref) <= TOL * abs(md_ref), (md, md_ref)
        assert abs(md - md_o) <= TOL * abs(md_o), (md, md_o)


def test_noalloc_matches_context_energy_and_oracle():
    _check_case(meshgen.config_mesh(1), capi.METRIC_2)
    _check_case(meshgen.config_mesh(3, n_e=12), capi.METRIC_303)
    _check_case(meshgen.config_mesh(2, n_e=10), capi.METRIC_302, nq=4)


def test_noalloc_native_fp64_size_target_and_nine_point_rule():
    m = meshgen.config_mesh(3, n_e=6, order=2)
    _check_case(m, capi.METRIC_303, prec=capi.FP64_NATIVE)
    _check_case(m, capi.METRIC_303_55, target=capi.TARGET_SIZE_FIELD, h0=1.0 / 6)
    fine = meshgen.perturb_smooth(meshgen.structured(3, 4, 4), seed=12, amp_smooth=0.03,
                                  amp_noise=0.015)
    _check_case(fine, capi.METRIC_303, nq=9)


def test_noalloc_rejects_meshes_beyond_its_scratch_and_bad_precision():
    m = meshgen.structured(3, 3, 2)
    emap = torch.from_numpy(np.ascontiguousarray(m.map)).cuda()
    x = torch.from_numpy(m.x).cuda()
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    # more elements than 65,536 CTAs hold for any elements-per-CTA value (at most
    # 32), and no map: a size check that passed by mistake would still return
    # TMOP_ERR_ARG (NULL map) and launch nothing
    desc = capi.Desc(3, 3, 4, 65536 * 256 + 1, m.num_nodes, capi.METRIC_303,
                     capi.TARGET_IDENTITY, 1.0, capi.FP64)
    st = capi.tmop_energy_noalloc(desc, None, x, out)
    assert st == capi.ERR_ARG
    assert "too large" in capi.last_error()
    bad = capi.Desc(3, 3, 4, m.num_elems, m.num_nodes, capi.METRIC_303, capi.TARGET_IDENTITY,
                    1.0, 7)
    assert capi.tmop_energy_noalloc(bad, emap, x, out) == capi.ERR_ARG
    assert "hess_precision" in capi.last_error()
    torch.cuda.synchronize()
    assert out.abs().sum().item() == 0.0      # nothing was launched
