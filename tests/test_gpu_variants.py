"""Every Hessian-action kernel variant (the autotuner's search space) against
the FP64 oracle (paper Sec. 3.4, eq. vm_pa_hess), and the collocated
variants against each other: they differ only in where the per-point values
live and in warps per CTA, with the same arithmetic in the same order, so
their actions and batched Newton trajectories are bitwise equal.

Meshes: 60 elements (5 x 4 x 3), so every warps-per-CTA choice leaves a
ragged last CTA and, in a batch, CTAs that span two meshes' tiles."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2205_12721_b300 import capi, meshgen as mg
from paper_2205_12721_b300.batch import TmopBatch

from gpu_common import TOL, assert_vec_close, dev, gpu_mesh, host, make_case, oracle_mesh

pytestmark = pytest.mark.gpu

CONFIGS = [(1, 2), (1, 3), (2, 3), (2, 4), (3, 4), (3, 5), (4, 5)]
PRECS = {"fp64": (capi.FP64, TOL), "fp64-native": (capi.FP64_NATIVE, TOL), "fp32": (capi.FP32, 2e-6)}


@pytest.fixture(autouse=True)
def _restore_defaults():
    yield
    for p, nq in CONFIGS:
        for prec, _ in PRECS.values():
            capi.tmop_set_apply_variant(3, p, nq, prec, -1)


@pytest.mark.parametrize("p,nq", CONFIGS, ids=[f"p{p}q{q}" for p, q in CONFIGS])
@pytest.mark.parametrize("precision", list(PRECS))
def test_every_variant_matches_oracle(p, nq, precision):
    prec, tol = PRECS[precision]
    n = capi.tmop_apply_variants(3, p, nq)
    assert n == 19
    metric = 303 if p % 2 else 302
    m = make_case(3, p, (5, 4, 3), seed=50 + p)
    om = oracle_mesh(m, metric, nq)
    gm = gpu_mesh(m, metric, nq, precision=precision)
    x = dev(m.x)
    gm.hessian_setup(x)
    v = np.random.default_rng(p * 10 + nq).standard_normal(m.ndof)
    y_o, ya = O.hessian_apply(om, m.x, v, with_abs=True)
    rd = torch.float32 if precision == "fp32" else torch.float64
    ys = {}
    for var in range(n):
        capi.tmop_set_apply_variant(3, p, nq, prec, var)
        assert capi.tmop_get_apply_variant(3, p, nq, prec) == var
        y = host(gm.hessian_apply(dev(v, rd)))
        assert_vec_close(y, y_o, ya, tol=tol, what=f"variant {var}")
        assert np.array_equal(y[m.fixed != 0], v.astype(np.float32 if precision == "fp32"
                                                         else np.float64)[m.fixed != 0])
        ys[var] = y
    for var in range(2, n):                      # collocated variants: bitwise equal
        assert np.array_equal(ys[var], ys[1]), var
    gm.close()


def test_variant_table_api():
    assert capi.tmop_apply_variants(2, 2, 3) == 1
    assert capi.tmop_apply_variants(3, 4, 6) == 1          # 36 lanes: no collocated kernel
    assert capi.tmop_apply_variants(3, 3, 4) == 19
    assert capi.tmop_apply_variants(3, 5, 6) == 0          # unsupported
    with pytest.raises(capi.TmopError):
        capi.tmop_set_apply_variant(3, 3, 4, capi.FP64, 19)
    with pytest.raises(capi.TmopError):
        capi.tmop_set_apply_variant(2, 2, 3, capi.FP64, 1)
    d0 = capi.tmop_get_apply_variant(3, 3, 4, capi.FP64)
    capi.tmop_set_apply_variant(3, 3, 4, capi.FP64, 2)
    assert capi.tmop_get_apply_variant(3, 3, 4, capi.FP64) == 2
    capi.tmop_set_apply_variant(3, 3, 4, capi.FP64, -1)
    assert capi.tmop_get_apply_variant(3, 3, 4, capi.FP64) == d0


def test_autotune_installs_the_fastest():
    m = make_case(3, 3, (8, 8, 8), seed=3)
    gm = gpu_mesh(m, 303, 4)
    x = dev(m.x)
    gm.hessian_setup(x)
    best, ms = capi.tmop_autotune(gm.ctx, 3)
    assert len(ms) == 19 and all(t > 0 for t in ms)
    assert ms[best] == min(ms)
    assert capi.tmop_get_apply_variant(3, 3, 4, capi.FP64) == best
    gm.close()


@pytest.mark.parametrize("variant", [1, 2, 3, 5, 7, 9, 10, 11, 12, 13, 16, 17])
def test_batched_trajectory_same_for_every_collocated_variant(variant):
    """Meshes of 3 x 3 x 2 = 18 elements against 8-element tiles: with 2 or 8
    warps per CTA a CTA covers half a tile or two tiles of different meshes."""
    d, p, metric = 3, 3, 303
    meshes = [mg.perturb_smooth(mg.structured(d, p, s), seed=60 + i, amp_smooth=0.03, amp_noise=0.015)
              for i, s in enumerate([(3, 3, 2), (2, 2, 3), (3, 2, 2)])]

    def run(var):
        capi.tmop_set_apply_variant(d, p, p + 1, capi.FP64, var)
        b = TmopBatch(d, p, metric, max_meshes=4, minres_max_it=30, minres_fixed_its=True)
        slots = [b.add_structured(mm) for mm in meshes]
        for _ in range(2):
            b.step()
        xs = [b.positions(s).cpu().numpy() for s in slots]
        b.close()
        return xs

    ref = run(1)
    got = run(variant)
    for a, bb in zip(ref, got):
        assert np.array_equal(a, bb)
