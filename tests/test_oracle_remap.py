"""Pins for the oracle's adaptive discrete target and advection remap
(paper Sec. 3.6).

What fixes each value independently of the oracle's own code:
* the mass operator integrates: 1^T M(x) 1 is the mesh volume (1 for the unit
  cube with fixed boundary), u^T M u = int u^2 for a linear u (quadrature
  exact at the chosen n_q); M is symmetric positive definite and its
  diagonal is the diagonal;
* the advection operator maps constants to 0, and for a linear field
  a . x it equals the mass operator applied to a . v node by node (grad of
  a linear field is a, so a wrong Jacobian transpose fails);
* the remap moves linear fields exactly (their semi-discrete solution is
  exact and RK4 reproduces it), keeps constants, and is the identity for
  zero velocity;
* for a smooth field the remap error against the exact nodal values falls
  with mesh refinement, and the pseudo-time error falls as dt^4 (RK4);
* the discrete target with a constant field c gives the closed-form energy
  c (1/c - 1)^2 of mu_55 on the ideal mesh, and a field interpolating the
  size function approaches the analytic size target's energy;
* the gradient of the discrete-target energy matches finite differences
  (eta is a fixed nodal field, so F is smooth in x).
"""
import numpy as np
import pytest

from paper_2205_12721_b300 import meshgen as mg


def _om(O, m, nq=None, metric=2, **kw):
    return O.Mesh(m.dim, m.order, nq or m.order + 1, m.map, m.num_nodes, metric, m.fixed, **kw)


def _pert(d, p, n, seed=3, amp=0.05):
    return mg.perturb_smooth(mg.structured(d, p, n), seed=seed, amp_smooth=amp, amp_noise=amp / 2)


def _comp(m, x, a):
    return x[a * m.num_nodes:(a + 1) * m.num_nodes]


@pytest.mark.parametrize("d,p,n,nq", [(2, 1, 5, 4), (2, 2, 4, 4), (2, 3, 3, 6), (3, 1, 3, 3),
                                      (3, 2, 2, 6)])
def test_mass_operator_integrates(oracle_mod, d, p, n, nq):
    O = oracle_mod
    m = _pert(d, p, n)
    om = _om(O, m, nq=nq, metric=2 if d == 2 else 303)
    N = m.num_nodes
    st, M1 = O.mass_apply(om, m.x, np.ones(N))
    assert st == 0
    assert abs(M1.sum() - 1.0) < 1e-13                   # volume of the unit square / cube
    # u = x_0: u^T M u = int x_0^2 = 1/3 (the physical domain is the unit cube)
    u = _comp(m, m.x, 0)
    st, Mu = O.mass_apply(om, m.x, u)
    assert abs(u @ Mu - 1.0 / 3.0) < 1e-13


@pytest.mark.parametrize("d,p", [(2, 2), (3, 1)])
def test_mass_dense_spd_and_diagonal(oracle_mod, d, p):
    O = oracle_mod
    m = _pert(d, p, 2, amp=0.1)
    om = _om(O, m, metric=2 if d == 2 else 303)
    N = m.num_nodes
    Md = np.column_stack([O.mass_apply(om, m.x, np.eye(N)[j])[1] for j in range(N)])
    np.testing.assert_allclose(Md, Md.T, rtol=0, atol=1e-15 * np.abs(Md).max())
    assert np.linalg.eigvalsh(Md).min() > 0
    st, dg = O.mass_diag(om, m.x)
    np.testing.assert_allclose(dg, np.diag(Md), rtol=1e-13)


@pytest.mark.parametrize("d,p,n", [(2, 2, 4), (2, 4, 3), (3, 2, 2), (3, 3, 2)])
def test_advection_operator_linear_fields(oracle_mod, d, p, n):
    O = oracle_mod
    m = _pert(d, p, n, seed=5)
    om = _om(O, m, metric=2 if d == 2 else 303)
    N = m.num_nodes
    rng = np.random.default_rng(1)
    vel = 0.05 * rng.standard_normal(d * N)
    st, K1 = O.advect_apply(om, m.x, vel, np.ones(N))
    assert st == 0 and np.abs(K1).max() < 1e-15
    a = rng.standard_normal(d)
    u = sum(a[k] * _comp(m, m.x, k) for k in range(d))
    _, Ku = O.advect_apply(om, m.x, vel, u)
    av = sum(a[k] * _comp(m, vel, k) for k in range(d))
    _, Mav = O.mass_apply(om, m.x, av)
    np.testing.assert_allclose(Ku, Mav, rtol=0, atol=1e-13 * np.abs(Mav).max())


@pytest.mark.parametrize("d,p,n,steps", [(2, 1, 6, 1), (2, 2, 4, 3), (2, 4, 3, 2), (3, 2, 2, 2),
                                         (3, 3, 2, 1)])
def test_remap_exact_for_linear_fields(oracle_mod, d, p, n, steps):
    O = oracle_mod
    x0 = mg.structured(d, p, n)
    m = _pert(d, p, n, seed=7, amp=0.08 if p <= 2 else 0.03)
    om = _om(O, m, metric=2 if d == 2 else 303)
    N = m.num_nodes
    a = np.array([1.7, -0.4, 0.9][:d])
    lin = lambda x: 0.3 + sum(a[k] * _comp(m, x, k) for k in range(d))
    st, eta1, its = O.remap(om, x0.x, m.x, lin(x0.x), steps=steps, cg_rtol=1e-14, cg_max_it=500)
    assert st == 0 and its > 0
    np.testing.assert_allclose(eta1, lin(m.x), rtol=0, atol=2e-13)
    st, c1, _ = O.remap(om, x0.x, m.x, np.full(N, 2.5), steps=steps)
    np.testing.assert_allclose(c1, 2.5, rtol=0, atol=1e-14)
    eta = np.random.default_rng(2).uniform(1, 2, N)
    st, same, its0 = O.remap(om, m.x, m.x, eta, steps=steps)
    assert np.array_equal(same, eta) and its0 == 0


def _smooth(m, x):
    X, Y = _comp(m, x, 0), _comp(m, x, 1)
    return 1.5 + np.sin(2 * np.pi * X) * np.cos(np.pi * Y)


def test_remap_converges_in_space_and_time(oracle_mod):
    """2D Q2: error against the exact nodal values falls with refinement
    (roughly h^3); at fixed mesh the pseudo-time error falls as dt^4."""
    O = oracle_mod
    errs = []
    for n in (4, 8, 16):
        x0 = mg.structured(2, 2, n)
        m = mg.perturb_smooth(mg.structured(2, 2, n), seed=11, amp_smooth=0.6 / n, amp_noise=0.0)
        om = _om(O, m)
        st, eta1, _ = O.remap(om, x0.x, m.x, _smooth(m, x0.x), steps=8, cg_rtol=1e-14, cg_max_it=800)
        assert st == 0
        errs.append(np.abs(eta1 - _smooth(m, m.x)).max())
    assert errs[0] / errs[1] > 5 and errs[1] / errs[2] > 5, errs
    # time: reference with 64 steps on the n = 8 mesh
    x0 = mg.structured(2, 2, 8)
    m = mg.perturb_smooth(mg.structured(2, 2, 8), seed=11, amp_smooth=0.1, amp_noise=0.0)
    om = _om(O, m)
    e0 = _smooth(m, x0.x)
    ref = O.remap(om, x0.x, m.x, e0, steps=64, cg_rtol=1e-15, cg_max_it=2000)[1]
    e = [np.abs(O.remap(om, x0.x, m.x, e0, steps=s, cg_rtol=1e-15, cg_max_it=2000)[1] - ref).max()
         for s in (2, 4)]
    assert 10 < e[0] / e[1] < 24, e                      # 2^4 = 16


def test_discrete_target_constant_field_closed_form(oracle_mod):
    """eta = c, h0 = h on the ideal mesh: T = c^(-1/d) I, mu_55 = (1/c - 1)^2,
    c_q = w_q h^d c, so F = c (1/c - 1)^2; shape metrics give F = 0."""
    O = oracle_mod
    for d, n in ((2, 5), (3, 3)):
        m = mg.structured(d, 2, n)
        for c in (0.5, 1.0, 2.7):
            om = _om(O, m, metric=55, target=O.TARGET_DISCRETE, target_h0=1.0 / n,
                     eta=np.full(m.num_nodes, c))
            st, F, _, _ = O.energy(om, m.x)
            assert st == 0 and abs(F - c * (1 / c - 1) ** 2) < 1e-13
            om2 = _om(O, m, metric=2 if d == 2 else 303, target=O.TARGET_DISCRETE,
                      target_h0=1.0 / n, eta=np.full(m.num_nodes, c))
            assert abs(O.energy(om2, m.x)[1]) < 1e-13
    # non-positive eta at a point: undefined target, reported as inverted
    m = mg.structured(2, 2, 3)
    eta = np.ones(m.num_nodes); eta[m.num_nodes // 2] = -5.0
    om = _om(O, m, metric=55, target=O.TARGET_DISCRETE, target_h0=1 / 3, eta=eta)
    st, F, md, _ = O.energy(om, m.x)
    assert st == O.ERR_INVERTED and F == np.inf and md == -np.inf


def test_discrete_target_approaches_size_target(oracle_mod):
    """eta = nodal interpolant of s(x) = 1 + 0.5 prod sin(2 pi x_k): the
    discrete-target energy converges to the analytic size target's."""
    O = oracle_mod
    diffs = []
    for n in (4, 8):
        m = mg.structured(2, 3, n)
        X, Y = _comp(m, m.x, 0), _comp(m, m.x, 1)
        s = 1 + 0.5 * np.sin(2 * np.pi * X) * np.sin(2 * np.pi * Y)
        Fd = O.energy(_om(O, m, metric=55, target=O.TARGET_DISCRETE, target_h0=1 / n, eta=s),
                      m.x)[1]
        Fs = O.energy(_om(O, m, metric=55, target=O.TARGET_SIZE, target_h0=1 / n), m.x)[1]
        diffs.append(abs(Fd - Fs) / Fs)
    assert diffs[1] < 1e-3 and diffs[0] / diffs[1] > 8, diffs


@pytest.mark.parametrize("d,p,metric", [(2, 2, 2), (3, 2, 30355), (3, 1, 7)])
def test_discrete_target_gradient_hessian_fd(oracle_mod, d, p, metric):
    O = oracle_mod
    n = 3 if d == 3 else 4
    m = _pert(d, p, n, seed=9)
    rng = np.random.default_rng(6)
    eta = rng.uniform(0.7, 1.4, m.num_nodes)
    om = _om(O, m, metric=metric, target=O.TARGET_DISCRETE, target_h0=1.0 / n, eta=eta)
    x0 = m.x
    g = O.gradient(om, x0)
    dlt = 1e-5 * m.h
    for _ in range(2):
        v = rng.standard_normal(m.ndof) * (m.fixed == 0) * m.h
        fd = (O.energy(om, x0 + dlt * v)[1] - O.energy(om, x0 - dlt * v)[1]) / (2 * dlt)
        assert abs(fd - g @ v) < 1e-7 * (np.abs(g) @ np.abs(v))
        fdh = (O.gradient(om, x0 + dlt * v) - O.gradient(om, x0 - dlt * v)) / (2 * dlt)
        hv = O.hessian_apply(om, x0, v)
        free = m.fixed == 0
        assert np.linalg.norm(fdh[free] - hv[free]) < 1e-6 * np.linalg.norm(hv[free])


def test_newton_with_remap_of_constant_field(oracle_mod):
    """A constant field remaps to itself, so Newton with the remap source
    (eta0 = c on x0) takes the same step as Newton with eta = c fixed."""
    O = oracle_mod
    m = _pert(2, 2, 5, seed=4, amp=0.08)
    x0 = mg.structured(2, 2, 5)
    c = np.full(m.num_nodes, 1.3)
    a = _om(O, m, metric=2, target=O.TARGET_DISCRETE, target_h0=0.2, eta=c)
    b = _om(O, m, metric=2, target=O.TARGET_DISCRETE, target_h0=0.2, eta=c,
            remap_x0=x0.x, remap_eta0=c, remap_steps=2)
    xa, xb = m.x.copy(), m.x.copy()
    ra = O.newton_step(a, xa, 1e-10, 200)
    rb = O.newton_step(b, xb, 1e-10, 200)
    assert ra["status"] == 0 and rb["status"] == 0
    np.testing.assert_allclose(xb, xa, rtol=0, atol=1e-13)
