"""Adaptive discrete target and advection remap (paper Sec. 3.6) on the GPU,
through the C ABI, against the FP64 oracle.

* discrete target W = h0 eta(x_q)^(1/d) I: energy, gradient, Hessian action
  and diagonal with the parity tolerances of the other FP64 tests (1e-12,
  condition-aware; 2e-6 for FP32 stored data);
* remap: eta1 against the oracle's remap with the same RK4 steps and CG
  tolerance.  Both sides stop CG at a relative preconditioned residual of
  1e-14, so eta1 agrees to 1e-11 of max |eta|; linear fields are moved
  exactly (a property of the method, independent of the oracle);
* Newton with the remap source: per-step positions within 1e-10 h;
* an inverted intermediate mesh and an undefined target are reported, and
  the discrete target is refused where it has no field (batches)."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2205_12721_b300 import capi, meshgen as mg
from paper_2205_12721_b300.mesh_opt import TmopMesh

from gpu_common import TOL, assert_vec_close, dev, host

pytestmark = pytest.mark.gpu

SHAPES = {2: (7, 5), 3: (4, 3, 3)}


def _field(m, x):
    N = m.num_nodes
    X = [x[a * N:(a + 1) * N] for a in range(m.dim)]
    f = 1.0 + 0.35 * np.sin(2 * np.pi * X[0]) * np.cos(np.pi * X[1])
    if m.dim == 3:
        f = f * (1.0 + 0.2 * np.sin(np.pi * X[2]))
    return f


def _pair(m, metric, nq, h0, eta, precision="fp64", **okw):
    om = O.Mesh(m.dim, m.order, nq, m.map, m.num_nodes, metric, m.fixed, O.TARGET_DISCRETE, h0,
                eta=eta, **okw)
    gm = TmopMesh(m.dim, m.order, m.map, m.num_nodes, metric, fixed=m.fixed, nq1d=nq,
                  target=capi.TARGET_DISCRETE, target_h0=h0, precision=precision)
    return om, gm


CASES = [((2, 2, 3, 2), "fp64"), ((2, 3, 4, 55), "fp64"), ((2, 4, 6, 9), "fp64"),
         ((3, 1, 2, 303), "fp64"), ((3, 2, 3, 30355), "fp64"), ((3, 3, 4, 7), "fp64"),
         ((3, 4, 5, 302), "fp64"), ((3, 2, 9, 303), "fp64"), ((3, 2, 3, 303), "fp64-native"),
         ((2, 2, 3, 2), "fp64-native"), ((3, 3, 4, 30355), "fp32"), ((2, 3, 4, 2), "fp32")]


@pytest.mark.parametrize("case,precision", CASES,
                         ids=[f"d{c[0]}p{c[1]}q{c[2]}m{c[3]}-{p}" for c, p in CASES])
def test_discrete_target_parity(case, precision):
    d, p, nq, metric = case
    shape = SHAPES[d]
    m = mg.perturb_smooth(mg.structured(d, p, shape), seed=21, amp_smooth=0.04, amp_noise=0.02)
    h0 = 1.0 / max(shape)
    eta = _field(m, m.x)
    om, gm = _pair(m, metric, nq, h0, eta, precision)
    gm.set_target_field(eta)
    x = dev(m.x)
    st_o, F_o, md_o, S = O.energy(om, m.x)
    st, F, md = gm.energy(x)
    assert st_o == 0 and st == capi.OK
    assert abs(F - F_o) <= TOL * max(abs(F_o), S), (F, F_o)
    assert abs(md - md_o) <= TOL * abs(md_o)
    g_o, ga = O.gradient(om, m.x, with_abs=True)
    assert_vec_close(host(gm.gradient(x)), g_o, ga, what="gradient")
    gm.hessian_setup(x)
    tol = 2e-6 if precision == "fp32" else TOL
    rd = torch.float32 if precision == "fp32" else torch.float64
    v = np.random.default_rng(5).standard_normal(m.ndof)
    y_o, ya = O.hessian_apply(om, m.x, v, with_abs=True)
    assert_vec_close(host(gm.hessian_apply(dev(v, rd))), y_o, ya, tol=tol, what="apply")
    dg_o, dga = O.hessian_diag(om, m.x, with_abs=True)
    assert_vec_close(host(gm.hessian_diag()), dg_o, dga, tol=tol, what="diag")
    gm.close()


def test_discrete_target_with_limiting_term():
    d, p, nq, metric = 2, 2, 3, 2
    base = mg.structured(d, p, SHAPES[d])
    m = mg.perturb_smooth(base, seed=22, amp_smooth=0.04, amp_noise=0.02)
    h0, delta = 1.0 / 7, 0.05
    eta = _field(m, m.x)
    om = O.Mesh(d, p, nq, m.map, m.num_nodes, metric, m.fixed, O.TARGET_DISCRETE, h0, delta, base.x,
                eta=eta)
    gm = TmopMesh(d, p, m.map, m.num_nodes, metric, fixed=m.fixed, nq1d=nq,
                  target=capi.TARGET_DISCRETE, target_h0=h0, limit_delta=delta, x0=base.x)
    gm.set_target_field(eta)
    x = dev(m.x)
    st_o, F_o, _, S = O.energy(om, m.x)
    assert abs(gm.energy(x)[1] - F_o) <= TOL * max(abs(F_o), S)
    g_o, ga = O.gradient(om, m.x, with_abs=True)
    assert_vec_close(host(gm.gradient(x)), g_o, ga, what="gradient")
    gm.hessian_setup(x)
    dg_o, dga = O.hessian_diag(om, m.x, with_abs=True)
    assert_vec_close(host(gm.hessian_diag()), dg_o, dga, what="diag")
    gm.close()


def test_undefined_target_is_inverted():
    m = mg.structured(2, 2, (4, 4))
    eta = np.ones(m.num_nodes)
    eta[m.num_nodes // 2] = -5.0
    om, gm = _pair(m, 55, 3, 0.25, eta)
    gm.set_target_field(eta)
    st_o, F_o, md_o, _ = O.energy(om, m.x)
    st, F, md = gm.energy(dev(m.x))
    assert st_o == O.ERR_INVERTED and st == capi.ERR_INVERTED
    assert F == np.inf and md == -np.inf and md_o == -np.inf
    gm.close()


REMAP = [(2, 1, 3, "fp64"), (2, 2, 2, "fp64"), (2, 4, 1, "fp64"), (3, 1, 2, "fp64"), (3, 2, 2, "fp64"),
         (3, 3, 1, "fp64"), (3, 2, 2, "fp64-native"), (2, 3, 2, "fp64-native")]


@pytest.mark.parametrize("d,p,steps,precision", REMAP)
def test_remap_parity(d, p, steps, precision):
    shape = SHAPES[d]
    x0m = mg.structured(d, p, shape)
    m = mg.perturb_smooth(mg.structured(d, p, shape), seed=23, amp_smooth=0.05 if p < 3 else 0.03,
                          amp_noise=0.02 if p < 3 else 0.01)
    om = O.Mesh(d, p, p + 1, m.map, m.num_nodes, 303 if d == 3 else 2, m.fixed)
    gm = TmopMesh(d, p, m.map, m.num_nodes, 303 if d == 3 else 2, fixed=m.fixed, precision=precision)
    eta0 = _field(x0m, x0m.x)
    st_o, eta_o, its_o = O.remap(om, x0m.x, m.x, eta0, steps=steps, cg_rtol=1e-14, cg_max_it=500)
    eta_g, rep = gm.remap(x0m.x, m.x, eta0, steps=steps, cg_rtol=1e-14, cg_max_it=500)
    assert st_o == 0 and rep["status"] == capi.OK
    assert rep["solves"] == 4 * steps and rep["min_det"] > 0
    assert abs(rep["cg_iters"] - its_o) <= 4 * steps, (rep, its_o)
    err = np.abs(host(eta_g) - eta_o).max()
    assert err <= 1e-11 * np.abs(eta_o).max(), err
    # linear fields move exactly (method property)
    N = m.num_nodes
    lin = lambda x: 0.7 + sum((0.9, -1.3, 0.4)[a] * x[a * N:(a + 1) * N] for a in range(d))
    eta_l, rep = gm.remap(x0m.x, m.x, lin(x0m.x), steps=steps, cg_rtol=1e-14, cg_max_it=500)
    assert np.abs(host(eta_l) - lin(m.x)).max() < 1e-12
    gm.close()


def test_remap_reports_inverted_intermediate_mesh():
    d, p = 2, 2
    x0m = mg.structured(d, p, (4, 4))
    m = mg.structured(d, p, (4, 4))
    x1 = m.x.copy()
    N = m.num_nodes
    c = N // 2                                   # an interior node pushed through its neighbours
    x1[c] += 0.6
    om = O.Mesh(d, p, p + 1, m.map, N, 2, m.fixed)
    st_o, _, _ = O.remap(om, x0m.x, x1, np.ones(N), steps=2)
    gm = TmopMesh(d, p, m.map, N, 2, fixed=m.fixed)
    _, rep = gm.remap(x0m.x, x1, np.ones(N), steps=2)
    assert st_o == O.ERR_INVERTED and rep["status"] == capi.ERR_INVERTED and rep["min_det"] <= 0
    # the context stays usable
    eta_g, rep = gm.remap(x0m.x, x0m.x, np.ones(N), steps=1)
    assert rep["status"] == capi.OK and np.array_equal(host(eta_g), np.ones(N))
    gm.close()


@pytest.mark.parametrize("d,p,shape,metric,steps", [(2, 2, (6, 6), 2, 4), (3, 2, (3, 3, 3), 30355, 3),
                                                    (3, 1, (4, 4, 3), 7, 3)])
def test_newton_with_remap_parity(d, p, shape, metric, steps):
    """eta0 given on the uniform mesh; both sides remap it to x and to every
    line-search trial; per-step positions agree to 1e-10 h."""
    x0m = mg.structured(d, p, shape)
    m = mg.perturb_smooth(mg.structured(d, p, shape), seed=24, amp_smooth=0.04, amp_noise=0.02)
    h0 = 1.0 / max(shape)
    eta0 = _field(x0m, x0m.x)
    om, gm = _pair(m, metric, p + 1, h0, eta0, remap_x0=x0m.x, remap_eta0=eta0, remap_steps=2,
                   remap_cg_rtol=1e-14, remap_cg_max_it=500)
    gm.set_remap_source(x0m.x, eta0, steps=2, cg_rtol=1e-14, cg_max_it=500)
    x = dev(m.x)
    g_first = None
    for k in range(steps):
        xs = host(x)
        x_start = xs.copy()
        ro = O.newton_step(om, xs, 1e-9, 300)
        rg = gm.newton_step(x, 1e-9, 300)
        g_first = g_first or ro["grad_norm"]
        if ro["grad_norm"] < 1e-8 * g_first or abs(ro["energy"]) <= 1e-12 * O.energy(om, x_start)[3]:
            break        # F at rounding level: the line-search tests are ties
        assert ro["status"] == 0 and rg["status"] == 0, (k, ro, rg)
        assert ro["minres_iters"] < 300
        assert rg["halvings"] == ro["halvings"]
        S = O.energy(om, x_start)[3]              # scale sum_q |c_q| (eta0 targets)
        assert abs(rg["energy"] - ro["energy"]) <= 1e-11 * max(abs(ro["energy"]), S)
        assert np.abs(host(x) - xs).max() <= 1e-10 * m.h, k
    gm.close()


def test_discrete_target_errors():
    m = mg.structured(2, 2, (3, 3))
    gm = TmopMesh(2, 2, m.map, m.num_nodes, 2, fixed=m.fixed, target=capi.TARGET_DISCRETE,
                  target_h0=1 / 3)
    with pytest.raises(capi.TmopError) as ei:
        capi.tmop_energy(gm.ctx, dev(m.x))
    assert ei.value.status == capi.ERR_ARG
    with pytest.raises(capi.TmopError):
        gm.remap(m.x, m.x, np.ones(m.num_nodes), steps=0)
    gm.close()
    plain = TmopMesh(2, 2, m.map, m.num_nodes, 2, fixed=m.fixed)
    with pytest.raises(capi.TmopError) as ei:
        plain.set_target_field(np.ones(m.num_nodes))
    assert ei.value.status == capi.ERR_ARG
    plain.close()
    from paper_2205_12721_b300.batch import TmopBatch
    with pytest.raises(capi.TmopError) as ei:
        TmopBatch(2, 2, 2, target=capi.TARGET_DISCRETE)
    assert ei.value.status == capi.ERR_UNSUPPORTED
