"""Pins for the oracle's 1D quadrature and basis (paper Sec. 3.1, eq. B_G_1D)."""
import math
import os

import numpy as np
import pytest
from numpy.polynomial import polynomial as npoly

from paper_2205_12721_b300 import meshgen

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _expr(s):
    return float(eval(s, {"sqrt": math.sqrt}))


def _rows(name):
    with open(os.path.join(GOLD, name)) as f:
        return [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]


def test_gauss_legendre_textbook(oracle_mod):
    rows = _rows("gauss_legendre.txt")
    for n in (1, 2, 3, 4):
        ref = sorted(((_expr(r[1]) + 1) / 2, _expr(r[2]) / 2) for r in rows if int(r[0]) == n)
        x, w = oracle_mod.gauss_legendre(n)
        np.testing.assert_allclose(x, [p for p, _ in ref], rtol=0, atol=2e-16)
        np.testing.assert_allclose(w, [v for _, v in ref], rtol=0, atol=2e-16)


@pytest.mark.parametrize("n", range(1, 11))
def test_gauss_legendre_exactness(oracle_mod, n):
    """An n-point rule integrates t^k exactly on [0,1] for k <= 2n-1; for
    k = 2n its error is the closed form (n!)^4 / ((2n+1) ((2n)!)^2)."""
    x, w = oracle_mod.gauss_legendre(n)
    assert abs(w.sum() - 1.0) < 1e-15
    for k in range(2 * n):
        assert abs(np.dot(w, x ** k) - 1.0 / (k + 1)) < 1e-15
    err = 1.0 / (2 * n + 1) - np.dot(w, x ** (2 * n))
    ref = math.factorial(n) ** 4 / ((2 * n + 1) * math.factorial(2 * n) ** 2)
    assert abs(err - ref) < 1e-14 + 1e-6 * ref


def test_gll_nodes_textbook(oracle_mod):
    rows = _rows("gll_nodes.txt")
    for n in (2, 3, 4, 5):
        ref = [_expr(r[1]) for r in rows if int(r[0]) == n]
        np.testing.assert_allclose(oracle_mod.gll_nodes(n), ref, rtol=0, atol=1e-15)


@pytest.mark.parametrize("n", range(2, 10))
def test_gll_nodes_against_numpy_roots(oracle_mod, n):
    """Newton in long double (oracle) against numpy's eigenvalue root finder."""
    np.testing.assert_allclose(oracle_mod.gll_nodes(n), meshgen.gll_points(n), rtol=0, atol=2e-14)


@pytest.mark.parametrize("p", [1, 2, 3, 4, 6])
def test_lagrange_basis(oracle_mod, p):
    nodes = oracle_mod.gll_nodes(p + 1)
    # cardinality
    for k, t in enumerate(nodes):
        v, _ = oracle_mod.lagrange(nodes, t)
        np.testing.assert_allclose(v, np.eye(p + 1)[k], atol=1e-14)
    rng = np.random.default_rng(1)
    for t in rng.uniform(0, 1, 7):
        v, d = oracle_mod.lagrange(nodes, t)
        assert abs(v.sum() - 1) < 1e-14          # partition of unity
        assert abs(d.sum()) < 1e-12              # derivative of a constant
        # against the interpolating polynomial built from its roots by numpy
        for j in range(p + 1):
            others = np.delete(nodes, j)
            c = npoly.polyfromroots(others) / np.prod(nodes[j] - others)
            tol = 1e-14 * np.abs(c).sum() * (p + 1)     # monomial-basis rounding
            assert abs(npoly.polyval(t, c) - v[j]) < tol
            assert abs(npoly.polyval(t, npoly.polyder(c)) - d[j]) < tol * p


def test_kershaw_dof_counts_pin_dof_definition():
    """The paper's Kershaw table lists unique DOFs d*(24p+1)^3 for 24^3
    elements; the generator's DOF count must match it exactly, and
    24^3 * 9^3 quadrature points split over 36 / 4 ranks gives the listed
    points per core."""
    rows = _rows("kershaw_counts.txt")
    for r in rows:
        if r[0] == "cores":
            assert 24 ** 3 * 9 ** 3 // int(r[1]) == int(r[2])
            continue
        p, dofs = int(r[0]), int(r[1])
        m = meshgen.structured(3, p, 2)   # the count formula, checked on a small mesh
        assert m.ndof == 3 * (2 * p + 1) ** 3
        assert 3 * (24 * p + 1) ** 3 == dofs
