"""Pins for the oracle's mesh functionals: energy, gradient, Hessian action,
diagonal, MINRES and the Newton step (paper Sec. 2.2-2.3, 3.3-3.4).

What fixes each value independently of the oracle's own code:
* the ideal Cartesian mesh has zero energy and zero gradient (mu >= 0 with
  equality on scaled rotations; the paper's stated optimum of the Kershaw
  benchmark is the ideal uniform configuration, Sec. 4.1);
* an affine element has a constant integrand, so F = mu(A) exactly;
* size-target energies of ideal meshes equal an integral computed by scipy;
* F, dF, d2F are equivariant under rotation and scaling of the mesh;
* dF matches central differences of F, d2F v matches central differences
  of dF; the dense Hessian is symmetric and its diagonal is the diagonal;
* MINRES run to full accuracy matches a dense LAPACK solve;
* Newton drives a perturbed mesh back to the uniform mesh.
"""
import numpy as np
import pytest
from scipy import integrate

from paper_2205_12721_b300 import meshgen as mg

SHAPE_CASES = [(2, 1, 2), (2, 2, 2), (2, 3, 2), (2, 4, 2),
               (3, 1, 302), (3, 2, 302), (3, 3, 303), (3, 4, 303), (3, 2, 303), (3, 1, 30355)]


def _om(O, m, metric, nq=None, fixed=True, target=0, h0=1.0):
    return O.Mesh(m.dim, m.order, nq or m.order + 1, m.map, m.num_nodes, metric,
                  m.fixed if fixed else None, target, h0)


@pytest.mark.parametrize("d,p,metric", [c for c in SHAPE_CASES if c[2] != 30355])
def test_ideal_mesh_zero_energy_and_gradient(oracle_mod, d, p, metric):
    n = 3 if d == 3 else 4
    m = mg.structured(d, p, n)
    for nq in (p + 1, p + 2):
        M = _om(oracle_mod, m, metric, nq)
        st, F, md, S = oracle_mod.energy(M, m.x)
        assert st == 0 and abs(F) < 1e-14 * S
        assert abs(md - (1.0 / n) ** d) < 1e-14
        # each term of P is O(1/h) on this mesh, times weights O(1)
        g = oracle_mod.gradient(M, m.x)
        assert np.abs(g).max() < 1e-13 * n
        M2 = _om(oracle_mod, m, metric, nq, fixed=False)
        g2 = oracle_mod.gradient(M2, m.x)
        assert np.abs(g2).max() < 1e-12


@pytest.mark.parametrize("d,metric", [(2, 2), (3, 302), (3, 303), (3, 55), (2, 55),
                                      (2, 7), (3, 7), (2, 9), (3, 9)])
def test_affine_element_energy_is_mu(oracle_mod, d, metric):
    rng = np.random.default_rng(3)
    for order in (1, 2, 3):
        m = mg.structured(d, order, 1)
        B = np.eye(d) + 0.3 * rng.standard_normal((d, d))
        if np.linalg.det(B) < 0:
            B[:, 0] *= -1
        x = mg.rigid_map(m, B, 1.0, shift=rng.standard_normal(d))
        M = _om(oracle_mod, m, metric, order + 2)
        st, F, md, S = oracle_mod.energy(M, x)
        _, mu, _, _ = oracle_mod.metric(metric, B)
        assert st == 0
        assert abs(F - mu) < 1e-13 * max(1, abs(mu))
        assert abs(md - np.linalg.det(B)) < 1e-13


def test_size_target_energy_matches_integral(oracle_mod):
    """W = h0 s(x)^(1/d) I with h0 = h on an ideal mesh gives T = s^(-1/d) I,
    so mu_55 = (1/s - 1)^2 and c_q = w_q h^d s: F = integral of (1-s)^2/s."""
    for d in (2, 3):
        n = 6 if d == 2 else 4
        m = mg.structured(d, 2, n)
        M = _om(oracle_mod, m, 55, nq=10, target=1, h0=1.0 / n)
        st, F, _, _ = oracle_mod.energy(M, m.x)

        def f(*xs):
            s = 0.5
            for t in xs:
                s = s * np.sin(2 * np.pi * t)
            s = 1 + s
            return (1 - s) ** 2 / s
        if d == 2:
            ref = integrate.dblquad(lambda y, x: f(x, y), 0, 1, 0, 1, epsabs=1e-14, epsrel=1e-13)[0]
        else:
            t, w = np.polynomial.legendre.leggauss(60)
            t = (t + 1) / 2; w = w / 2
            X, Y, Z = np.meshgrid(t, t, t, indexing="ij")
            W = w[:, None, None] * w[None, :, None] * w[None, None, :]
            ref = float(np.sum(W * f(X, Y, Z)))
        assert st == 0
        assert abs(F - ref) < 1e-9 * ref
        # shape part of mu_303 + mu_55 vanishes on the ideal mesh
        M3 = _om(oracle_mod, m, 30355, nq=10, target=1, h0=1.0 / n) if d == 3 else None
        if M3 is not None:
            st3, F3, _, _ = oracle_mod.energy(M3, m.x)
            assert abs(F3 - ref) < 1e-9 * ref


@pytest.mark.parametrize("metric", [7, 9])
def test_shape_size_metric_size_target_integral(oracle_mod, metric):
    """Ideal mesh, W = h s^(1/d) I: T = t I with t = s^(-1/d), c_q = w_q h^d s,
    mu_7 = d (t - 1/t)^2 and mu_9 = t^d mu_7, so F = integral of
    s d (t - 1/t)^2 (mu_7) or d (t - 1/t)^2 (mu_9) over the unit cube."""
    for d in (2, 3):
        n = 6 if d == 2 else 4
        m = mg.structured(d, 2, n)
        M = _om(oracle_mod, m, metric, nq=10, target=1, h0=1.0 / n)
        st, F, _, _ = oracle_mod.energy(M, m.x)

        def f(*xs):
            s = 0.5
            for t in xs:
                s = s * np.sin(2 * np.pi * t)
            s = 1 + s
            t = s ** (-1.0 / d)
            v = d * (t - 1 / t) ** 2
            return s * v if metric == 7 else v
        t, w = np.polynomial.legendre.leggauss(60)
        t = (t + 1) / 2; w = w / 2
        G = np.meshgrid(*([t] * d), indexing="ij")
        W = np.ones_like(G[0])
        for k in range(d):
            W = W * w.reshape([-1 if j == k else 1 for j in range(d)])
        ref = float(np.sum(W * f(*G)))
        assert st == 0
        assert abs(F - ref) < 1e-9 * ref


@pytest.mark.parametrize("d,p,metric", [(2, 2, 2), (3, 2, 302), (3, 3, 303)])
def test_rotation_scale_equivariance(oracle_mod, d, p, metric):
    n = 3 if d == 3 else 4
    m = mg.perturb_smooth(mg.structured(d, p, n), seed=5, amp_smooth=0.05, amp_noise=0.025)
    M = _om(oracle_mod, m, metric)
    R = mg.random_rotation(d, 11)
    c = 1.7
    Nx = m.num_nodes
    xr = mg.rigid_map(m, R, c, shift=np.arange(d) * 0.3)
    st, F, _, _ = oracle_mod.energy(M, m.x)
    assert st == 0
    _, Fr, _, _ = oracle_mod.energy(M, xr)
    assert abs(F - Fr) < 1e-12 * F
    rot = lambda v: (R @ v.reshape(d, Nx)).reshape(-1)
    g = oracle_mod.gradient(M, m.x)
    gr = oracle_mod.gradient(M, xr)
    np.testing.assert_allclose(gr, rot(g) / c, rtol=0, atol=1e-12 * np.abs(g).max())
    v = np.random.default_rng(2).standard_normal(m.ndof) * (m.fixed == 0)
    y = oracle_mod.hessian_apply(M, m.x, v)
    yr = oracle_mod.hessian_apply(M, xr, rot(v))
    free = m.fixed == 0
    np.testing.assert_allclose(yr[free], (rot(y) / c ** 2)[free], rtol=0,
                               atol=1e-11 * np.abs(y[free]).max())


@pytest.mark.parametrize("d,p,metric,target", [(2, 2, 2, 0), (2, 3, 2, 0), (3, 1, 302, 0),
                                               (3, 2, 303, 0), (3, 2, 30355, 1), (2, 2, 9, 0),
                                               (3, 2, 7, 1), (3, 1, 9, 1)])
def test_gradient_and_hessian_vs_finite_differences(oracle_mod, d, p, metric, target):
    n = 3 if d == 3 else 4
    m = mg.perturb_smooth(mg.structured(d, p, n), seed=9, amp_smooth=0.05, amp_noise=0.025)
    M = _om(oracle_mod, m, metric, target=target, h0=1.0 / n)
    rng = np.random.default_rng(4)
    x0 = m.x
    g = oracle_mod.gradient(M, x0)
    dlt = 1e-5 * m.h
    for _ in range(3):
        v = rng.standard_normal(m.ndof) * (m.fixed == 0) * m.h
        # targets frozen at x0: the method drops dW/dx (Sec. 3.6)
        Fp = oracle_mod.energy(M, x0 + dlt * v, xw=x0)[1]
        Fm = oracle_mod.energy(M, x0 - dlt * v, xw=x0)[1]
        fd = (Fp - Fm) / (2 * dlt)
        assert abs(fd - g @ v) < 1e-7 * (np.abs(g) @ np.abs(v))
        gp = oracle_mod.gradient(M, x0 + dlt * v, xw=x0)
        gm = oracle_mod.gradient(M, x0 - dlt * v, xw=x0)
        hv = oracle_mod.hessian_apply(M, x0, v)
        fdh = (gp - gm) / (2 * dlt)
        free = m.fixed == 0
        assert np.linalg.norm(fdh[free] - hv[free]) < 1e-6 * np.linalg.norm(hv[free])


@pytest.mark.parametrize("d,p,metric", [(2, 2, 2), (3, 2, 302), (3, 2, 303), (3, 1, 30355),
                                        (2, 2, 7), (3, 1, 9)])
def test_dense_hessian_symmetry_and_diagonal(oracle_mod, d, p, metric):
    shape = (2, 1) if d == 2 else (2, 1, 1)
    m = mg.perturb_uniform(mg.structured(d, p, shape), amp=0.1, seed=3)
    # interior-free perturbation leaves a 2-element mesh undisturbed; move all nodes
    rng = np.random.default_rng(8)
    x = m.x + 0.05 * rng.uniform(-1, 1, m.ndof)
    for fixed in (False, True):
        M = _om(oracle_mod, m, metric, fixed=fixed)
        H = oracle_mod.dense_hessian(M, x)
        np.testing.assert_allclose(H, H.T, rtol=0, atol=1e-12 * np.abs(H).max())
        dg = oracle_mod.hessian_diag(M, x)
        np.testing.assert_allclose(dg, np.diag(H), rtol=0, atol=1e-12 * np.abs(H).max())


def test_minres_matches_dense_solve(oracle_mod):
    m = mg.config_mesh(1, n_e=3)
    M = _om(oracle_mod, m, 2)
    x = m.x
    H = oracle_mod.dense_hessian(M, x)
    b = oracle_mod.gradient(M, x)
    dg = oracle_mod.hessian_diag(M, x)
    st, dx, its, res = oracle_mod.minres(M, x, dg, b, rtol=1e-14, max_it=400)
    ref = np.linalg.solve(H, b)
    assert st == 0 and res <= 1e-14
    assert np.linalg.norm(dx - ref) < 1e-9 * np.linalg.norm(ref)
    # truncated solve: reported preconditioned residual is the true one
    st, dx5, its5, res5 = oracle_mod.minres(M, x, dg, b, rtol=0.0, max_it=5, fixed_its=True)
    minv = 1 / np.abs(dg)
    r = b - H @ dx5
    true = np.sqrt(r @ (minv * r)) / np.sqrt(b @ (minv * b))
    assert its5 == 5 and abs(true - res5) < 1e-10


def test_newton_recovers_uniform_mesh_2d():
    """2D 8x8 Q2 mesh, mu_2, fixed boundary: Newton with Jacobi-MINRES
    (rtol 1e-8) and the 1.2-factor line search returns to the ideal mesh."""
    import oracle as O
    m = mg.config_mesh(1)
    ideal = mg.structured(2, 2, 8)
    M = _om(O, m, 2)
    x = m.x.copy()
    reps = [O.newton_step(M, x, 1e-8, 50) for _ in range(10)]
    assert all(r["status"] == 0 for r in reps)
    assert reps[-1]["grad_norm"] / reps[0]["grad_norm"] < 1e-10
    assert np.abs(x - ideal.x).max() < 1e-10 * m.h
    for r in reps:                               # the accepted step obeys the rules
        assert r["energy_new"] < 1.2 * r["energy"] or r["grad_norm"] == 0
        assert r["min_det"] > 0


def test_newton_3d_decreases_energy(oracle_mod):
    m = mg.config_mesh(2, n_e=3)
    M = _om(oracle_mod, m, 302)
    x = m.x.copy()
    F = []
    for _ in range(6):
        r = oracle_mod.newton_step(M, x, 1e-8, 50)
        assert r["status"] == 0
        F.append(r["energy"])
    assert F[-1] < 1e-6 * F[0]


def test_line_search_rejects_inverting_step(oracle_mod):
    """A mesh one step from inversion: the accepted alpha keeps det A > 0."""
    m = mg.perturb_uniform(mg.structured(2, 1, 3), amp=0.3, seed=12)
    M = _om(oracle_mod, m, 2)
    x = m.x.copy()
    r = oracle_mod.newton_step(M, x, 1e-10, 100)
    assert r["status"] == 0 and r["min_det"] > 0
    st, _, md, _ = oracle_mod.energy(M, x)
    assert st == 0 and md > 0


def test_inverted_mesh_reports_status(oracle_mod):
    m = mg.structured(2, 1, 3)
    x = m.x.copy()
    Nx = m.num_nodes
    c = 5 + 4 * 1   # an interior node; push it across its neighbours
    x[c] += 0.7
    M = _om(oracle_mod, m, 2)
    st, F, md, _ = oracle_mod.energy(M, x)
    assert st == oracle_mod.ERR_INVERTED and F == np.inf and md <= 0
    x2 = x.copy()
    r = oracle_mod.newton_step(M, x2)
    assert r["status"] == oracle_mod.ERR_INVERTED and np.array_equal(x, x2)


@pytest.mark.parametrize("d", [2, 3])
def test_det_affine_and_bilinear(oracle_mod, d):
    """det A at the points (Sec. 2.2, eq. A), pinned by closed forms.
    Affine element x = B xi + c: det A = det B at every point.  Map
    x_1 = xi_1 (1 + alpha xi_2), other coordinates unchanged (degree 1 in each
    reference variable, so Q_p reproduces it exactly): det A = 1 + alpha xi_2
    at the point, with xi_2 the Gauss point of the second direction, which
    fixes the point order q = q1 + nq q2 (+ nq^2 q3) and catches a transposed
    Jacobian (that would give 1 + alpha xi_1)."""
    rng = np.random.default_rng(11)
    for order in (1, 2, 3):
        m = mg.structured(d, order, 1)
        nq = order + 1
        B = np.eye(d) + 0.3 * rng.standard_normal((d, d))
        if np.linalg.det(B) < 0:
            B[:, 0] *= -1
        x = mg.rigid_map(m, B, 1.0, shift=rng.standard_normal(d))
        M = _om(oracle_mod, m, 2 if d == 2 else 303, nq, fixed=False)
        det = oracle_mod.det(M, x)
        assert det.shape == (1, nq ** d)
        np.testing.assert_allclose(det, np.linalg.det(B), rtol=1e-13)
        alpha = 0.4
        xr = m.x.reshape(d, -1).copy()            # the unit element: x = xi
        xb = xr.copy()
        xb[0] = xr[0] * (1.0 + alpha * xr[1])
        det = oracle_mod.det(M, xb.reshape(-1))[0]
        g, _ = oracle_mod.gauss_legendre(nq)
        q = np.arange(nq ** d)
        xi2 = g[(q // nq) % nq]
        np.testing.assert_allclose(det, 1.0 + alpha * xi2, rtol=1e-13)
        assert not np.allclose(det, 1.0 + alpha * g[q % nq])
