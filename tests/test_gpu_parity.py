"""GPU (sm_103a library, through the C ABI) against the FP64 oracle, element
by element on the same seeded meshes.

Tolerances (FP64 path): energy |dF| <= 1e-12 max(|F|, S_F) with
S_F = sum_q |w_q det W|; gradient, Hessian action and diagonal
||d||_2 <= 1e-12 max(||ref||_2, ||abs-sum scale||_2); min det(A) relative
1e-12.  Mesh shapes give element counts that leave a ragged last CTA for
every elements-per-CTA value the kernels use, and span several CTAs."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2205_12721_b300 import capi

from gpu_common import (TOL, assert_vec_close, dev, gpu_mesh, host, make_case, oracle_mesh)

pytestmark = pytest.mark.gpu

SHAPES = {2: [(9, 7), (11, 6)], 3: [(5, 4, 3), (7, 2, 2)]}
CASES = []
for p in (1, 2, 3, 4):
    for dq in (1, 2):
        CASES.append((2, p, p + dq, 2, 0))
        CASES.append((3, p, p + dq, 303 if p % 2 else 302, 0))
CASES += [(2, 2, 3, 55, 0), (3, 2, 3, 55, 0), (3, 3, 4, 30355, 1), (3, 1, 2, 30355, 1),
          (3, 4, 5, 30355, 1), (2, 3, 4, 55, 1), (3, 2, 3, 302, 1),
          # the 9^3-point rule of the paper's Kershaw runs
          (3, 1, 9, 303, 0), (3, 2, 9, 302, 0), (3, 4, 9, 303, 0),
          # shape+size metrics mu_7 = |T - T^-t|^2, mu_9 = tau |T - T^-t|^2
          (2, 2, 3, 7, 1), (2, 3, 4, 9, 0), (2, 1, 3, 9, 1), (3, 2, 3, 7, 1), (3, 3, 4, 9, 1),
          (3, 1, 2, 7, 0), (3, 4, 5, 9, 1)]


def _ids(c):
    return f"d{c[0]}p{c[1]}q{c[2]}m{c[3]}t{c[4]}"


NATIVE_CASES = [(2, 2, 3, 2, 0), (2, 4, 6, 2, 0), (3, 1, 2, 302, 0), (3, 3, 4, 303, 0),
                (3, 4, 5, 302, 0), (3, 2, 3, 30355, 1), (3, 3, 9, 303, 0), (3, 2, 3, 9, 1),
                (2, 2, 3, 7, 1)]
PARAMS = [(c, "fp64") for c in CASES] + [(c, "fp64-native") for c in NATIVE_CASES]


@pytest.mark.parametrize("case,precision", PARAMS, ids=[f"{_ids(c)}-{p}" for c, p in PARAMS])
def test_fp64_parity(case, precision):
    """FP64-class contexts: double-float contractions (default) and the
    native FP64-unit path."""
    d, p, nq, metric, target = case
    for si, shape in enumerate(SHAPES[d]):
        m = make_case(d, p, shape, seed=10 + si)
        h0 = 1.0 / max(shape)
        om = oracle_mesh(m, metric, nq, target, h0)
        gm = gpu_mesh(m, metric, nq, target, h0, precision=precision)
        x = dev(m.x)
        # energy and min det
        st_o, F_o, md_o, S = O.energy(om, m.x)
        assert st_o == 0
        st, F, md = gm.energy(x)
        assert st == capi.OK
        assert abs(F - F_o) <= TOL * max(abs(F_o), S), (F, F_o, S)
        assert abs(md - md_o) <= TOL * abs(md_o)
        # det A at every quadrature point (relative, per point)
        det_o = O.det(om, m.x)
        det = host(gm.det(x))
        assert det.shape == det_o.shape
        assert np.all(np.abs(det - det_o) <= TOL * np.abs(det_o)), np.abs(det / det_o - 1).max()
        assert det.min() == md
        # gradient
        g_o, ga = O.gradient(om, m.x, with_abs=True)
        g = host(gm.gradient(x))
        assert_vec_close(g, g_o, ga, what="gradient")
        assert np.all(g[m.fixed != 0] == 0)
        # Hessian action (v nonzero on fixed DOFs: they must act as identity)
        gm.hessian_setup(x)
        v = np.random.default_rng(3 + si).standard_normal(m.ndof)
        y_o, ya = O.hessian_apply(om, m.x, v, with_abs=True)
        y = host(gm.hessian_apply(dev(v)))
        assert_vec_close(y, y_o, ya, what="hessian_apply")
        assert np.array_equal(y[m.fixed != 0], v[m.fixed != 0])
        # diagonal
        dg_o, dga = O.hessian_diag(om, m.x, with_abs=True)
        dg = host(gm.hessian_diag())
        assert_vec_close(dg, dg_o, dga, what="diag")
        gm.close()


@pytest.mark.parametrize("case", [(2, 2, 3, 2, 0), (3, 2, 3, 302, 0), (3, 3, 4, 303, 0),
                                  (3, 4, 5, 303, 0), (3, 2, 3, 30355, 1), (3, 3, 4, 7, 1)],
                         ids=_ids)
def test_fp32_hessian_data(case):
    """FP32 stored d2mu/dT2 and FP32 action: error stated against the FP64
    oracle (single-precision rounding of H, v and the contractions)."""
    d, p, nq, metric, target = case
    shape = SHAPES[d][0]
    m = make_case(d, p, shape, seed=21)
    h0 = 1.0 / max(shape)
    om = oracle_mesh(m, metric, nq, target, h0)
    gm = gpu_mesh(m, metric, nq, target, h0, precision="fp32")
    x = dev(m.x)
    gm.hessian_setup(x)
    v = np.random.default_rng(5).standard_normal(m.ndof)
    y_o, ya = O.hessian_apply(om, m.x, v, with_abs=True)
    y = host(gm.hessian_apply(dev(v, torch.float32)))
    assert_vec_close(y, y_o, ya, tol=2e-6, what="fp32 apply")
    dg = host(gm.hessian_diag())
    dg_o, dga = O.hessian_diag(om, m.x, with_abs=True)
    assert_vec_close(dg, dg_o, dga, tol=2e-6, what="fp32 diag")
    # energy and gradient stay FP64 in the mixed mode
    st_o, F_o, _, S = O.energy(om, m.x)
    st, F, _ = gm.energy(x)
    assert abs(F - F_o) <= TOL * max(abs(F_o), S)
    g_o, ga = O.gradient(om, m.x, with_abs=True)
    assert_vec_close(host(gm.gradient(x)), g_o, ga, what="fp32-mode gradient")
    gm.close()


def test_ideal_and_single_element():
    from paper_2205_12721_b300 import meshgen as mg
    for d, p, metric in [(2, 3, 2), (3, 2, 302), (3, 4, 303)]:
        m = mg.structured(d, p, 3)
        gm = gpu_mesh(m, metric)
        st, F, md = gm.energy(dev(m.x))
        assert st == 0 and abs(F) < 1e-13 * m.num_elems
        assert np.abs(host(gm.gradient(dev(m.x)))).max() < 1e-12
        gm.close()
        one = mg.structured(d, p, 1)
        R = mg.random_rotation(d, 4)
        x1 = mg.rigid_map(one, R @ np.diag(np.linspace(1, 2, d)), 1.0)
        om = oracle_mesh(one, metric)
        gm1 = gpu_mesh(one, metric, fixed=False)
        _, F_o, md_o, S = O.energy(om, x1)
        st, F, md = gm1.energy(dev(x1))
        assert abs(F - F_o) <= TOL * max(F_o, S) and abs(md - md_o) <= TOL * md_o
        gm1.close()


def test_error_paths():
    from paper_2205_12721_b300 import meshgen as mg
    m = mg.structured(2, 1, 3)
    x = m.x.copy()
    x[5 + 4 * 1] += 0.7                      # invert the elements around one node
    gm = gpu_mesh(m, 2)
    st, F, md = gm.energy(dev(x))
    assert st == capi.ERR_INVERTED and F == float("inf") and md <= 0
    xd = dev(x)
    before = xd.clone()
    r = gm.newton_step(xd)
    assert r["status"] == capi.ERR_INVERTED and torch.equal(xd, before)
    # apply before setup
    with pytest.raises(capi.TmopError):
        gm.hessian_apply(dev(np.zeros(m.ndof)))
    gm.close()
    bad = m.map.copy()
    bad[0, 0] = m.num_nodes
    with pytest.raises(capi.TmopError) as ei:
        from paper_2205_12721_b300.mesh_opt import TmopMesh
        TmopMesh(2, 1, bad, m.num_nodes, 2, fixed=m.fixed)
    assert ei.value.status == capi.ERR_ARG
    with pytest.raises(capi.TmopError) as ei:
        gpu_mesh(m, 2, nq=5)
    assert ei.value.status == capi.ERR_UNSUPPORTED
    with pytest.raises(capi.TmopError) as ei:
        gpu_mesh(m, 303)
    assert ei.value.status == capi.ERR_UNSUPPORTED


def _newton_parity(m, metric, steps, target=0, h0=1.0, nq=None, max_it=200):
    """Per-step parity: both sides take one Newton step from the same x (the
    GPU's), MINRES run to its rtol (1e-8); the accepted step must agree to
    1e-10 h.  Also follows the two trajectories side by side."""
    om = oracle_mesh(m, metric, nq, target, h0)
    gm = gpu_mesh(m, metric, nq, target, h0)
    xo = m.x.copy()
    xg = dev(m.x)
    g_first = None
    for k in range(steps):
        x_start = host(xg)
        xs = x_start.copy()
        S = O.energy(om, xs)[3]                          # scale sum_q |c_q|
        ro = O.newton_step(om, xs, 1e-8, max_it)
        rg = gm.newton_step(xg, 1e-8, max_it)
        g_first = g_first or ro["grad_norm"]
        if ro["grad_norm"] < 1e-8 * g_first or abs(ro["energy"]) <= 1e-12 * S:
            break        # converged: F is at rounding level, line-search tests are ties
        assert ro["status"] == 0 and rg["status"] == 0, (k, ro, rg)
        assert ro["minres_iters"] < max_it, "case must be well conditioned (MINRES converges)"
        assert rg["halvings"] == ro["halvings"], (k, ro, rg)
        assert abs(rg["minres_iters"] - ro["minres_iters"]) <= 1, (k, ro, rg)
        assert abs(rg["energy"] - ro["energy"]) <= TOL * max(ro["energy"], S)
        err = np.abs(host(xg) - xs).max()
        assert err <= 1e-10 * m.h, (k, err)
        O.newton_step(om, xo, 1e-8, max_it)             # the oracle's own trajectory
        assert np.abs(host(xg) - xo).max() <= 1e-10 * m.h
    gm.close()
    return xo


def test_newton_iterates_2d():
    """2D 8x8 Q2, mu_2, MINRES rtol 1e-8 (converged at every step)."""
    from paper_2205_12721_b300 import meshgen as mg
    _newton_parity(mg.perturb_uniform(mg.structured(2, 2, 8), 0.08, 20260102), 2, 6)


def test_newton_iterates_3d():
    from paper_2205_12721_b300 import meshgen as mg
    _newton_parity(mg.perturb_smooth(mg.structured(3, 2, 4), 20260103, 0.03, 0.015), 302, 4)
    _newton_parity(mg.perturb_smooth(mg.structured(3, 3, (4, 3, 3)), 5, 0.03, 0.015), 303, 3)
    _newton_parity(mg.perturb_smooth(mg.structured(3, 2, 4), 6, 0.03, 0.015), 30355, 3,
                   target=1, h0=0.25)


def test_newton_iterates_shape_size_metrics():
    """mu_7 and mu_9 with the size target (their 3D forms use I2 = |cof T|^2)."""
    from paper_2205_12721_b300 import meshgen as mg
    _newton_parity(mg.perturb_smooth(mg.structured(3, 2, 4), 7, 0.03, 0.015), 7, 3,
                   target=1, h0=0.25)
    _newton_parity(mg.perturb_smooth(mg.structured(3, 3, (3, 3, 4)), 8, 0.03, 0.015), 9, 3,
                   target=1, h0=0.25)
    _newton_parity(mg.perturb_smooth(mg.structured(2, 3, 6), 9, 0.05, 0.02), 9, 3,
                   target=1, h0=1.0 / 6)


def test_cfg1_solve_reaches_uniform_mesh():
    """The 2D 8x8 Q2 configuration (+-0.15h, mu_2, 10 Newton steps, MINRES
    rtol 1e-8 / 50 iterations).  Its first Hessians are indefinite and MINRES
    stops at 50 iterations, where the truncated iterate is sensitive to
    rounding (1e-13 relative changes move it by ~1e-3), so intermediate
    iterates are compared through their reports and both solves must end at
    the uniform mesh, which the paper states is the optimum."""
    from paper_2205_12721_b300 import meshgen as mg
    m = mg.config_mesh(1)
    ideal = mg.structured(2, 2, 8).x
    om = oracle_mesh(m, 2)
    gm = gpu_mesh(m, 2)
    xo = m.x.copy()
    xg = dev(m.x)
    for k in range(10):
        ro = O.newton_step(om, xo, 1e-8, 50)
        rg = gm.newton_step(xg, 1e-8, 50)
        assert ro["status"] == 0 and rg["status"] == 0
        if k == 0:
            assert abs(rg["energy"] - ro["energy"]) <= 1e-12 * ro["energy"]
            assert abs(rg["grad_norm"] - ro["grad_norm"]) <= 1e-12 * ro["grad_norm"]
    assert np.abs(xo - ideal).max() <= 1e-10 * m.h
    assert np.abs(host(xg) - ideal).max() <= 1e-10 * m.h
    gm.close()


def test_cfg1_newton_steps_fixed_minres():
    """Per-step iterates on the 2D 8x8 Q2 configuration itself (+-0.15h, mu_2,
    10 Newton steps).  Each step starts both sides from the same x (the
    oracle's) and runs exactly 10 MINRES iterations (paper Sec. 2.3 with a
    fixed inner iteration count), where the Krylov iterate is not yet
    sensitive to rounding; the accepted x+ must agree to 1e-10 h, and the step
    reports (energy, |dF|, halvings) must agree.  |dF| is compared at 1e-12 of
    max(|dF|, ||abs-sum scale||) plus 1e-13 |dF(x0)|: near the optimum
    dmu/dT -> 0 by cancellation of terms of size |T|/tau that do not shrink,
    so its rounding stays at the level of the first gradient."""
    from paper_2205_12721_b300 import meshgen as mg
    m = mg.config_mesh(1)
    om = oracle_mesh(m, 2)
    gm = gpu_mesh(m, 2)
    xo = m.x.copy()
    g_first = None
    for k in range(10):
        S = O.energy(om, xo)[3]
        ga = O.gradient(om, xo, with_abs=True)[1]       # abs-sum scale of dF
        xg = dev(xo)
        ro = O.newton_step(om, xo, 0.0, 10, True)
        rg = gm.newton_step(xg, 0.0, 10, True)
        assert ro["status"] == 0 and rg["status"] == 0, (k, ro, rg)
        assert ro["minres_iters"] == rg["minres_iters"] == 10
        assert rg["halvings"] == ro["halvings"], (k, ro, rg)
        assert abs(rg["energy"] - ro["energy"]) <= TOL * max(ro["energy"], S)
        g_first = g_first or ro["grad_norm"]
        assert abs(rg["grad_norm"] - ro["grad_norm"]) <= (TOL * max(ro["grad_norm"], np.linalg.norm(ga))
                                                          + 1e-13 * g_first), k
        err = np.abs(host(xg) - xo).max()
        assert err <= 1e-10 * m.h, (k, err)
    gm.close()


@pytest.mark.parametrize("p,nq,prec", [(1, 9, "fp64"), (2, 9, "fp64"), (3, 5, "fp64"), (2, 9, "fp32")])
def test_kershaw_solve_reaches_uniform_mesh(p, nq, prec):
    """The Kershaw mesh (sliding boundary) solved on the GPU ends at the
    uniform mesh, as the paper states and the oracle confirms."""
    from paper_2205_12721_b300 import meshgen as mg
    m = mg.kershaw(p, (6, 2, 2), 0.3, 0.3)
    u = mg.structured(3, p, (6, 2, 2))
    gm = gpu_mesh(m, 303, nq, precision=prec)
    x = dev(m.x)
    reps = gm.solve(x, max_newton=40, rtol=1e-11, minres_rtol=1e-10, minres_max_it=200)
    assert all(r["status"] == 0 for r in reps)
    tol = 1e-9 if prec == "fp64" else 1e-5
    assert np.abs(host(x) - u.x).max() < tol / 6
    gm.close()


LIMIT_CASES = [((2, 2, 3, 2, 0), "fp64"), ((3, 2, 3, 303, 0), "fp64"), ((3, 3, 4, 302, 0), "fp64"),
               ((3, 2, 3, 30355, 1), "fp64"), ((3, 2, 3, 303, 0), "fp32"),
               ((3, 3, 4, 303, 0), "fp64-native"), ((2, 3, 5, 2, 1), "fp64")]


@pytest.mark.parametrize("case,precision", LIMIT_CASES, ids=[f"{_ids(c)}-{p}" for c, p in LIMIT_CASES])
def test_limiting_term_parity(case, precision):
    """Objective with the limiting term |x - x0|^2 / delta^2 (Sec. 3.5):
    energy, gradient, Hessian action (shape part + mass-like part) and
    diagonal against the oracle; one Newton step from the same x."""
    from paper_2205_12721_b300 import meshgen as mg
    from paper_2205_12721_b300.mesh_opt import TmopMesh
    d, p, nq, metric, target = case
    shape = SHAPES[d][0]
    base = mg.structured(d, p, shape)
    m = mg.perturb_smooth(base, seed=17, amp_smooth=0.05, amp_noise=0.025)
    h0, delta = 1.0 / max(shape), 0.05
    om = O.Mesh(d, p, nq, m.map, m.num_nodes, metric, m.fixed, target, h0, delta, base.x)
    gm = TmopMesh(d, p, m.map, m.num_nodes, metric, fixed=m.fixed, nq1d=nq, target=target,
                  target_h0=h0, precision=precision, limit_delta=delta, x0=base.x)
    tol = 2e-6 if precision == "fp32" else TOL
    x = dev(m.x)
    st_o, F_o, _, S = O.energy(om, m.x)
    st, F, _ = gm.energy(x)
    assert st == 0 and abs(F - F_o) <= TOL * max(abs(F_o), S)
    g_o, ga = O.gradient(om, m.x, with_abs=True)
    assert_vec_close(host(gm.gradient(x)), g_o, ga, what="gradient + limiting")
    gm.hessian_setup(x)
    v = np.random.default_rng(9).standard_normal(m.ndof)
    y_o, ya = O.hessian_apply(om, m.x, v, with_abs=True)
    rd = torch.float32 if precision == "fp32" else torch.float64
    assert_vec_close(host(gm.hessian_apply(dev(v, rd))), y_o, ya, tol=tol, what="apply + limiting")
    dg_o, dga = O.hessian_diag(om, m.x, with_abs=True)
    assert_vec_close(host(gm.hessian_diag()), dg_o, dga, tol=tol, what="diag + limiting")
    if precision != "fp32":
        # a fixed number of MINRES iterations on both sides (no stop-test tie)
        xo = m.x.copy()
        ro = O.newton_step(om, xo, 0.0, 30, minres_fixed_its=True)
        rg = gm.newton_step(x, 0.0, 30, minres_fixed_its=True)
        assert ro["status"] == 0 and rg["status"] == 0
        assert np.abs(host(x) - xo).max() <= 1e-10 * m.h
    gm.close()


def test_limiting_requires_reference():
    from paper_2205_12721_b300 import meshgen as mg
    from paper_2205_12721_b300.mesh_opt import TmopMesh
    m = mg.structured(2, 2, 3)
    gm = TmopMesh(2, 2, m.map, m.num_nodes, 2, fixed=m.fixed, limit_delta=0.1)
    with pytest.raises(capi.TmopError) as ei:
        gm.gradient(dev(m.x))
    assert ei.value.status == capi.ERR_ARG
    gm.set_limit_reference(m.x)
    g = host(gm.gradient(dev(m.x)))
    assert np.abs(g).max() < 1e-12            # ideal mesh at its own reference
    gm.close()
    plain = TmopMesh(2, 2, m.map, m.num_nodes, 2, fixed=m.fixed)
    with pytest.raises(capi.TmopError):
        plain.set_limit_reference(m.x)
    plain.close()
