"""Pins for the limiting term xi = |x - x0|^2 / delta^2 of the objective
(paper eq. F_full second term, Sec. 3.5 eq. pa_limiting) in the oracle."""
import numpy as np
import pytest

import oracle as O
from paper_2205_12721_b300 import meshgen as mg


def _mesh(m, metric, delta, x0, target=0, h0=1.0, fixed=True):
    return O.Mesh(m.dim, m.order, m.order + 1, m.map, m.num_nodes, metric,
                  m.fixed if fixed else None, target, h0, delta, x0)


@pytest.mark.parametrize("d,p,metric", [(2, 2, 2), (3, 2, 303), (3, 1, 302)])
def test_rigid_shift_closed_form(oracle_mod, d, p, metric):
    """Ideal mesh (shape energy 0), x0 = x - t: F = E |t|^2 / delta^2."""
    m = mg.structured(d, p, 3)
    t = np.array([0.3, -0.2, 0.1][:d])
    x0 = (m.x.reshape(d, -1) - t[:, None]).reshape(-1)
    delta = 0.7
    st, F, _, _ = oracle_mod.energy(_mesh(m, metric, delta, x0), m.x)
    assert st == 0
    ref = m.num_elems * float(t @ t) / delta ** 2
    assert abs(F - ref) < 1e-12 * ref


@pytest.mark.parametrize("d,p,metric,target", [(2, 2, 2, 0), (3, 2, 303, 0), (3, 1, 30355, 1)])
def test_limiting_derivatives_vs_finite_differences(oracle_mod, d, p, metric, target):
    n = 3
    base = mg.structured(d, p, n)
    m = mg.perturb_smooth(base, seed=3, amp_smooth=0.05, amp_noise=0.025)
    M = _mesh(m, metric, 0.05, base.x, target, 1.0 / n)
    x0 = m.x
    g = oracle_mod.gradient(M, x0)
    rng = np.random.default_rng(1)
    dlt = 1e-5 * m.h
    for _ in range(2):
        v = rng.standard_normal(m.ndof) * (m.fixed == 0) * m.h
        Fp = oracle_mod.energy(M, x0 + dlt * v, xw=x0)[1]
        Fm = oracle_mod.energy(M, x0 - dlt * v, xw=x0)[1]
        assert abs((Fp - Fm) / (2 * dlt) - g @ v) < 1e-7 * (np.abs(g) @ np.abs(v))
        hv = oracle_mod.hessian_apply(M, x0, v)
        fdh = (oracle_mod.gradient(M, x0 + dlt * v, xw=x0) -
               oracle_mod.gradient(M, x0 - dlt * v, xw=x0)) / (2 * dlt)
        free = m.fixed == 0
        assert np.linalg.norm(fdh[free] - hv[free]) < 1e-6 * np.linalg.norm(hv[free])


def test_limiting_dense_hessian_symmetric_and_diag(oracle_mod):
    m = mg.structured(3, 2, (2, 1, 1))
    x = m.x + 0.05 * np.random.default_rng(2).uniform(-1, 1, m.ndof)
    M = _mesh(m, 303, 0.3, m.x, fixed=False)
    H = oracle_mod.dense_hessian(M, x)
    np.testing.assert_allclose(H, H.T, rtol=0, atol=1e-12 * np.abs(H).max())
    np.testing.assert_allclose(oracle_mod.hessian_diag(M, x), np.diag(H), rtol=0,
                               atol=1e-12 * np.abs(H).max())
    # the added term is the mass matrix 2/delta^2 M (positive definite): H_lim - H_0 > 0
    H0 = oracle_mod.dense_hessian(_mesh(m, 303, 0.0, None, fixed=False), x)
    ev = np.linalg.eigvalsh(H - H0)
    assert ev.min() > 0
