"""Batched Newton steps (many meshes in shared launches) through the C ABI.

* per-step parity of every mesh of a mixed-size batch with the FP64 oracle;
* a mesh's trajectory is bitwise the same alone and inside a batch (per-mesh
  reductions in a fixed order), also when meshes join and leave between steps;
* mixed precision (FP32 stored d2mu/dT2 and Krylov vectors) reaches the FP64
  batch's final energy within 1e-8 relative on the size-target metric."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2205_12721_b300 import capi, meshgen as mg
from paper_2205_12721_b300.batch import TmopBatch

pytestmark = pytest.mark.gpu


def _mesh(d, p, shape, seed, amp=0.03):
    return mg.perturb_smooth(mg.structured(d, p, shape), seed=seed, amp_smooth=amp, amp_noise=amp / 2)


def _x(b, slot):
    return b.positions(slot).cpu().numpy()


@pytest.mark.parametrize("d,p,metric,shapes", [
    (3, 2, 302, [(4, 3, 3), (3, 3, 2), (5, 4, 3)]),
    (2, 2, 2, [(6, 5), (8, 8), (4, 7)]),
    (3, 3, 303, [(3, 3, 2), (4, 2, 2)]),
])
def test_batch_step_matches_oracle(d, p, metric, shapes):
    # a fixed number of MINRES iterations on both sides: with a stop test, two
    # solves that stop one iteration apart differ by about the tolerance times
    # the condition number, far above rounding (no tie in the stop test here)
    meshes = [_mesh(d, p, s, 30 + i) for i, s in enumerate(shapes)]
    its = 40
    b = TmopBatch(d, p, metric, max_meshes=8, minres_max_it=its, minres_fixed_its=True)
    slots = [b.add_structured(m) for m in meshes]
    for step in range(2):
        xs = {s: _x(b, s) for s in slots}
        b.step()
        for s, m in zip(slots, meshes):
            om = O.Mesh(d, p, p + 1, m.map, m.num_nodes, metric, m.fixed)
            xo = xs[s].copy()
            ro = O.newton_step(om, xo, 0.0, its, minres_fixed_its=True)
            st = b.state(s)
            assert ro["status"] == 0 and st["status"] == 0
            assert ro["minres_iters"] == its
            assert np.abs(_x(b, s) - xo).max() <= 1e-10 * m.h, (step, s)
            assert st["newton_its"] == step + 1
    b.close()


def test_batch_alone_equals_mixed_and_continuous_membership():
    d, p, metric = 3, 2, 302
    meshes = [_mesh(d, p, s, 40 + i) for i, s in enumerate([(3, 3, 3), (4, 3, 2), (2, 2, 2), (5, 3, 3)])]
    steps = 3
    alone = []
    for m in meshes:
        b1 = TmopBatch(d, p, metric, max_meshes=1, minres_max_it=60)
        s = b1.add_structured(m)
        for _ in range(steps):
            b1.step()
        alone.append((_x(b1, s), b1.state(s)))
        b1.close()
    # mixed: meshes 0, 1 from the start, 2 joins after one step, 3 after two;
    # a finished mesh leaves and its slot is reused
    bm = TmopBatch(d, p, metric, max_meshes=3, minres_max_it=60)
    s0, s1 = bm.add_structured(meshes[0]), bm.add_structured(meshes[1])
    bm.step()
    s2 = bm.add_structured(meshes[2])
    bm.step()
    bm.step()                                    # meshes 0, 1 have done 3 steps
    x0, st0 = _x(bm, s0), bm.state(s0)
    x1, st1 = _x(bm, s1), bm.state(s1)
    bm.remove(s0)
    s3 = bm.add_structured(meshes[3])           # reuses slot s0
    assert s3 == s0
    bm.step()                                    # mesh 2: 3 steps
    x2 = _x(bm, s2)
    bm.step()
    bm.step()                                    # mesh 3: 3 steps
    x3 = _x(bm, s3)
    for got, (ref, rst) in zip([x0, x1, x2, x3], alone):
        assert np.array_equal(got, ref)
    assert st0["energy"] == alone[0][1]["energy"] and st1["minres_its"] == alone[1][1]["minres_its"]
    bm.close()


@pytest.mark.parametrize("p", [1, 2])
def test_mixed_precision_final_energy(p):
    """Shape + size metric with the size target (mu_303 + mu_55,
    W = h0 s(x)^(1/3) I): the FP32 stored-Hessian / FP32-Krylov solve ends at
    the FP64 solve's energy within 1e-8 relative."""
    shapes = [(4, 4, 4), (5, 4, 3), (3, 3, 4)]
    meshes = [_mesh(3, p, s, 50 + i, amp=0.05) for i, s in enumerate(shapes)]
    finals = {}
    for prec in ("fp64", "fp32"):
        b = TmopBatch(3, p, capi.METRIC_303_55, target=capi.TARGET_SIZE_FIELD, precision=prec,
                      max_meshes=4, minres_max_it=100, newton_rtol=1e-10, newton_max_it=40)
        slots = [b.add_structured(m, h0=1.0 / max(m.n)) for m in meshes]
        b.solve(60)
        finals[prec] = [b.state(s) for s in slots]
        b.close()
    for m, a, c in zip(meshes, finals["fp64"], finals["fp32"]):
        assert a["status"] == 0 and c["status"] == 0
        assert a["energy"] < a["energy0"]
        assert abs(a["energy"] - c["energy"]) <= 1e-8 * max(abs(a["energy"]), 1e-8 * m.num_elems), (a, c)


def test_batch_rtol_stopped_minres_matches_oracle():
    """The batched per-mesh MINRES stop test (phibar <= rtol beta1, Sec. 2.3)
    against the oracle's: meshes perturbed mildly enough that MINRES converges
    to rtol 1e-8 well before its cap (no tie in the stop test), the same
    iteration count per step and iterates to 1e-10 h."""
    d, p, metric = 3, 2, 302
    meshes = [_mesh(d, p, s, 80 + i, amp=0.02) for i, s in enumerate([(3, 3, 2), (4, 3, 2), (2, 3, 3)])]
    b = TmopBatch(d, p, metric, max_meshes=4, minres_rtol=1e-8, minres_max_it=200)
    slots = [b.add_structured(m) for m in meshes]
    for step in range(2):
        xs = {s: _x(b, s) for s in slots}
        its0 = {s: b.state(s)["minres_its"] for s in slots}
        b.step()
        for s, m in zip(slots, meshes):
            om = O.Mesh(d, p, p + 1, m.map, m.num_nodes, metric, m.fixed)
            xo = xs[s].copy()
            ro = O.newton_step(om, xo, 1e-8, 200)
            st = b.state(s)
            assert ro["status"] == 0 and st["status"] == 0
            assert ro["minres_iters"] < 200
            assert st["minres_its"] - its0[s] == ro["minres_iters"], (step, s)
            assert np.abs(_x(b, s) - xo).max() <= 1e-10 * m.h, (step, s)
    b.close()
