"""tmop_energy_noalloc against tmop_energy, through the C ABI.

tmop_energy_noalloc serves callers that cannot call cudaMalloc (for example
code embedded in an application whose pool allocator already owns the device
memory, or latency-bound loops where an allocation would synchronise the
device).  It keeps its scratch in a static device array instead of a
context, so two calls in a row must both reproduce the context-based result,
and a mesh too large for that array must be refused up front.  This file is
collected last so that a failure here cannot hide the other tests."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2205_12721_b300 import capi, meshgen

pytestmark = pytest.mark.gpu

TOL = 1e-12


def _check_case(m, metric, nq=None, target=capi.TARGET_IDENTITY, h0=1.0):
    desc = capi.Desc(m.dim, m.order, nq or m.order + 1, m.num_elems, m.num_nodes, metric,
                     target, h0, capi.FP64)
    emap = torch.from_numpy(np.ascontiguousarray(m.map)).cuda()
    fixed = torch.from_numpy(m.fixed).cuda()
    x = torch.from_numpy(m.x).cuda()
    ctx = capi.tmop_setup(desc, emap, fixed)
    try:
        st, F_ref, md_ref = capi.tmop_energy(ctx, x)
        assert st == capi.OK
    finally:
        capi.tmop_destroy(ctx)
    scale = max(abs(F_ref), m.num_elems)      # sum_q |w_q det W| = E for W = I
    for _ in range(2):                        # two calls in a row share the scratch
        out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
        st = capi.tmop_energy_noalloc(desc, emap, x, out)
        assert st == capi.OK, capi.last_error()
        torch.cuda.synchronize()
        F, md = out.tolist()
        assert abs(F - F_ref) <= TOL * scale, (F, F_ref)
        assert abs(md - md_ref) <= TOL * abs(md_ref), (md, md_ref)


def test_noalloc_matches_context_energy():
    _check_case(meshgen.config_mesh(1), capi.METRIC_2)
    _check_case(meshgen.config_mesh(3, n_e=12), capi.METRIC_303)
    _check_case(meshgen.config_mesh(2, n_e=10), capi.METRIC_302, nq=4)


def test_noalloc_rejects_meshes_beyond_its_scratch():
    m = meshgen.structured(3, 3, 2)
    emap = torch.from_numpy(np.ascontiguousarray(m.map)).cuda()
    x = torch.from_numpy(m.x).cuda()
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    # 3D p=3 with 4^3 points packs 8 elements per CTA: 65,536 CTAs at most
    desc = capi.Desc(3, 3, 4, 65536 * 8 + 1, m.num_nodes, capi.METRIC_303,
                     capi.TARGET_IDENTITY, 1.0, capi.FP64)
    st = capi.tmop_energy_noalloc(desc, emap, x, out)
    assert st == capi.ERR_ARG
    assert "too large" in capi.last_error()
    assert out.abs().sum().item() == 0.0      # nothing was launched
