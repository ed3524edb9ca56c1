"""Reuse of the line search's evaluation at the accepted positions
(tmop_newton_step): consecutive steps on one context take F, min det and the
gradient of the previous step's accepted trial instead of evaluating them
again.  The trajectory is bitwise that of a fresh context started at each
step's positions (which must evaluate), and the reuse is dropped when x
changed by one bit or when the energy's definition changed
(tmop_set_limit_reference)."""
import numpy as np
import pytest
import torch

from gpu_common import dev, host, make_case
from paper_2205_12721_b300 import capi
from paper_2205_12721_b300.mesh_opt import TmopMesh

pytestmark = pytest.mark.gpu

CASES = [
    (3, 2, 302, (4, 3, 3), "fp64", 0.0),
    (3, 3, 303, (3, 3, 2), "fp32", 0.0),
    (2, 2, 2, (8, 8), "fp64", 0.05),
]
IDS = ["3d-p2-fp64", "3d-p3-fp32", "2d-p2-limit"]
OPTS = dict(minres_rtol=1e-8, minres_max_it=50)


def _mesh(m, metric, precision, limit):
    return TmopMesh(m.dim, m.order, m.map, m.num_nodes, metric, fixed=m.fixed, precision=precision,
                    limit_delta=limit, x0=m.x if limit > 0 else None)


def _fresh_step(m, metric, precision, limit, x_host):
    gm = _mesh(m, metric, precision, limit)
    try:
        x = dev(x_host)
        r = gm.newton_step(x, **OPTS)
        assert capi.tmop_step_reuses(gm.ctx) == 0
        return host(x), r
    finally:
        gm.close()


def _same_report(a, b):
    for k in ("status", "energy", "grad_norm", "min_det", "alpha", "minres_iters", "halvings",
              "energy_new", "grad_norm_new", "minres_resid"):
        assert a[k] == b[k], k


@pytest.mark.parametrize("d,p,metric,shape,precision,limit", CASES, ids=IDS)
def test_consecutive_steps_equal_fresh_contexts(d, p, metric, shape, precision, limit):
    m = make_case(d, p, shape, seed=90 + p)
    gm = _mesh(m, metric, precision, limit)
    try:
        x = dev(m.x)
        steps = 4
        for i in range(steps):
            before = host(x)
            r = gm.newton_step(x, **OPTS)
            assert r["status"] == capi.OK
            xf, rf = _fresh_step(m, metric, precision, limit, before)
            assert np.array_equal(host(x), xf)
            _same_report(r, rf)
        assert capi.tmop_step_reuses(gm.ctx) == steps - 1
    finally:
        gm.close()


def test_changed_positions_are_evaluated():
    d, p, metric, shape, precision, limit = CASES[0]
    m = make_case(d, p, shape, seed=93)
    gm = _mesh(m, metric, precision, limit)
    try:
        x = dev(m.x)
        assert gm.newton_step(x, **OPTS)["status"] == capi.OK
        xh = host(x)
        free = np.flatnonzero(np.asarray(m.fixed).reshape(-1) == 0)   # node or DOF flags
        i = int(free[len(free) // 2])                      # component 0 of a free node / DOF
        xh[i] = np.nextafter(xh[i], np.inf)                  # one bit of one DOF
        x.copy_(torch.from_numpy(xh))
        r = gm.newton_step(x, **OPTS)
        assert capi.tmop_step_reuses(gm.ctx) == 0
        xf, rf = _fresh_step(m, metric, precision, limit, xh)
        assert np.array_equal(host(x), xf)
        _same_report(r, rf)
    finally:
        gm.close()


def test_limit_reference_change_drops_the_reuse():
    d, p, metric, shape, precision, limit = CASES[2]
    m = make_case(d, p, shape, seed=94)
    gm = _mesh(m, metric, precision, limit)
    try:
        x = dev(m.x)
        assert gm.newton_step(x, **OPTS)["status"] == capi.OK
        x0 = dev(m.x)
        capi.tmop_set_limit_reference(gm.ctx, x0)            # same values, still a change
        xh = host(x)
        r = gm.newton_step(x, **OPTS)
        torch.cuda.synchronize()
        assert capi.tmop_step_reuses(gm.ctx) == 0
        xf, rf = _fresh_step(m, metric, precision, limit, xh)
        assert np.array_equal(host(x), xf)
        _same_report(r, rf)
    finally:
        gm.close()
