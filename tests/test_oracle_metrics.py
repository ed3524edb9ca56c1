"""Pins for the oracle's quality metrics mu(T), dmu/dT, d2mu/dT2
(paper Sec. 2.2 for mu_2, mu_55 and the shape+size metrics
mu_7 = |T - T^-t|^2, mu_9 = tau |T - T^-t|^2; Sec. 4.1 for mu_303; mu_302 from
the benchmark configuration |T|^2 |T^-1|^2 / 9 - 1).

mu is checked against hand values; P against complex-step derivatives of the
definition; K against exact symbolic second derivatives (sympy)."""
import numpy as np
import pytest
import sympy as sp

METRICS = [(2, 2), (302, 3), (303, 3), (55, 2), (55, 3), (30355, 3),
           (7, 2), (7, 3), (9, 2), (9, 3)]


def _mu_def(mid, T):
    """The metric definitions, written so that complex T works (no abs/conj)."""
    I1 = np.sum(T * T)
    tau = np.linalg.det(T)
    if mid == 2:
        return I1 / (2 * tau) - 1
    if mid == 303:
        return I1 / (3 * tau ** (2.0 / 3.0)) - 1
    if mid == 302:
        Ti = np.linalg.inv(T)
        return I1 * np.sum(Ti * Ti) / 9 - 1
    if mid == 55:
        return (tau - 1) ** 2
    if mid == 30355:
        return _mu_def(303, T) + _mu_def(55, T)
    if mid in (7, 9):
        R = T - np.linalg.inv(T).T
        n2 = np.sum(R * R)
        return n2 if mid == 7 else tau * n2
    raise ValueError(mid)


def _random_T(d, rng, n=6):
    out = []
    while len(out) < n:
        T = np.eye(d) + 0.4 * rng.standard_normal((d, d))
        if np.linalg.det(T) > 0.05:
            out.append(T * rng.uniform(0.3, 3.0))
    return out


@pytest.mark.parametrize("mid,d", METRICS)
def test_gradient_complex_step(oracle_mod, mid, d):
    rng = np.random.default_rng(mid + d)
    h = 1e-30
    for T in _random_T(d, rng):
        st, mu, P, _ = oracle_mod.metric(mid, T)
        assert st == 0
        assert abs(mu - _mu_def(mid, T).real) <= 1e-14 * max(1, abs(mu))
        Pcs = np.zeros((d, d))
        for a in range(d):
            for b in range(d):
                Tc = T.astype(complex)
                Tc[a, b] += 1j * h
                Pcs[a, b] = _mu_def(mid, Tc).imag / h
        np.testing.assert_allclose(P, Pcs, rtol=1e-12, atol=1e-13 * np.abs(Pcs).max())


def _sym_mu(mid, d):
    Ts = sp.Matrix(d, d, lambda i, j: sp.Symbol(f"t{i}{j}"))
    I1 = sum(Ts[i, j] ** 2 for i in range(d) for j in range(d))
    tau = Ts.det()
    if mid == 2:
        mu = I1 / (2 * tau) - 1
    elif mid == 303:
        mu = I1 / (3 * tau ** sp.Rational(2, 3)) - 1
    elif mid == 302:
        Ti = Ts.adjugate() / tau
        mu = I1 * sum(Ti[i, j] ** 2 for i in range(d) for j in range(d)) / 9 - 1
    elif mid == 55:
        mu = (tau - 1) ** 2
    elif mid == 30355:
        mu = I1 / (3 * tau ** sp.Rational(2, 3)) - 1 + (tau - 1) ** 2
    elif mid in (7, 9):
        R = Ts - (Ts.adjugate() / tau).T
        mu = sum(R[i, j] ** 2 for i in range(d) for j in range(d))
        if mid == 9:
            mu = tau * mu
    syms = [Ts[i, j] for i in range(d) for j in range(d)]
    return syms, mu


@pytest.mark.parametrize("mid,d", METRICS)
def test_hessian_symbolic(oracle_mod, mid, d):
    syms, mu = _sym_mu(mid, d)
    rng = np.random.default_rng(100 + mid)
    T = _random_T(d, rng, 2)
    for Tn in T:
        sub = {s: sp.Float(v, 30) for s, v in zip(syms, Tn.reshape(-1))}
        _, _, _, K = oracle_mod.metric(mid, Tn)
        dd = d * d
        Kref = np.zeros((dd, dd))
        grads = [sp.diff(mu, s) for s in syms]
        for i in range(dd):
            for j in range(i, dd):
                Kref[i, j] = Kref[j, i] = float(sp.diff(grads[i], syms[j]).evalf(25, subs=sub))
        np.testing.assert_allclose(K, Kref, rtol=1e-11, atol=1e-12 * np.abs(Kref).max())
        np.testing.assert_allclose(K, K.T, rtol=0, atol=1e-13 * np.abs(K).max())


def test_hand_values(oracle_mod):
    for s in (0.1, 0.5, 2.0):
        _, mu, _, _ = oracle_mod.metric(2, np.array([[1.0, s], [0.0, 1.0]]))
        assert abs(mu - s * s / 2) < 1e-15
    for a in (0.5, 1.0, 3.0):
        _, mu, _, _ = oracle_mod.metric(2, np.diag([a, 1.0]))
        assert abs(mu - (a - 1) ** 2 / (2 * a)) < 1e-15
        _, mu, _, _ = oracle_mod.metric(303, np.diag([a, 1.0, 1.0]))
        assert abs(mu - ((a * a + 2) / (3 * a ** (2 / 3)) - 1)) < 1e-15
        _, mu, _, _ = oracle_mod.metric(302, np.diag([a, 1.0, 1.0]))
        assert abs(mu - ((a * a + 2) * (a ** -2 + 2) / 9 - 1)) < 1e-14
        _, mu, _, _ = oracle_mod.metric(55, np.diag([a, 1.0, 1.0]))
        assert abs(mu - (a - 1) ** 2) < 1e-15
        for d in (2, 3):
            # stretch diag(a, 1, ..): T - T^-t = diag(a - 1/a, 0, ..)
            _, mu, _, _ = oracle_mod.metric(7, np.diag([a] + [1.0] * (d - 1)))
            assert abs(mu - (a - 1 / a) ** 2) < 1e-14
            _, mu, _, _ = oracle_mod.metric(9, np.diag([a] + [1.0] * (d - 1)))
            assert abs(mu - a * (a - 1 / a) ** 2) < 1e-14
            # uniform scaling c I: |T - T^-t|^2 = d (c - 1/c)^2
            _, mu, _, _ = oracle_mod.metric(7, a * np.eye(d))
            assert abs(mu - d * (a - 1 / a) ** 2) < 1e-13
            _, mu, _, _ = oracle_mod.metric(9, a * np.eye(d))
            assert abs(mu - a ** d * d * (a - 1 / a) ** 2) < 1e-12


@pytest.mark.parametrize("mid,d", [(7, 2), (7, 3), (9, 2), (9, 3)])
def test_shape_size_metric_invariance_and_minimum(oracle_mod, mid, d):
    """mu_7, mu_9 are >= 0, vanish exactly on rotations (T^T T = I), are
    invariant under T -> R T Q but not under scaling (they see size)."""
    from paper_2205_12721_b300.meshgen import random_rotation
    rng = np.random.default_rng(8)
    for k, T in enumerate(_random_T(d, rng)):
        _, mu, _, _ = oracle_mod.metric(mid, T)
        assert mu >= 0
        R, Q = random_rotation(d, 30 + k), random_rotation(d, 40 + k)
        _, mu2, _, _ = oracle_mod.metric(mid, R @ T @ Q)
        assert abs(mu2 - mu) < 1e-13 * max(1, mu)
        _, mu0, P0, _ = oracle_mod.metric(mid, R)
        assert abs(mu0) < 1e-14 and np.abs(P0).max() < 1e-13
        _, mus, _, _ = oracle_mod.metric(mid, 1.5 * R)
        assert mus > 0.1


@pytest.mark.parametrize("mid,d", [(2, 2), (302, 3), (303, 3)])
def test_shape_metric_invariance_and_minimum(oracle_mod, mid, d):
    """Shape metrics are >= 0, vanish exactly on scaled rotations and are
    invariant under T -> c R T Q (rotations R, Q, scale c > 0)."""
    from paper_2205_12721_b300.meshgen import random_rotation
    rng = np.random.default_rng(7)
    for k, T in enumerate(_random_T(d, rng)):
        _, mu, _, _ = oracle_mod.metric(mid, T)
        assert mu >= -1e-15
        R, Q = random_rotation(d, 10 + k), random_rotation(d, 20 + k)
        _, mu2, _, _ = oracle_mod.metric(mid, 2.7 * R @ T @ Q)
        assert abs(mu2 - mu) < 1e-13 * max(1, mu)
        _, mu0, P0, _ = oracle_mod.metric(mid, 0.8 * R)
        assert abs(mu0) < 1e-14 and np.abs(P0).max() < 1e-13


def test_inverted_and_unknown(oracle_mod):
    assert oracle_mod.metric(2, np.diag([-1.0, 1.0]))[0] == oracle_mod.ERR_INVERTED
    assert oracle_mod.metric(303, np.diag([1.0, 1.0, 0.0]))[0] == oracle_mod.ERR_INVERTED
    assert oracle_mod.metric(2, np.eye(3))[0] == oracle_mod.ERR_ARG
    assert oracle_mod.metric(303, np.eye(2))[0] == oracle_mod.ERR_ARG
