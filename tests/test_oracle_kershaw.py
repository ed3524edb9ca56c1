"""The Kershaw benchmark mesh (paper Sec. 4.1 and appendix): generator
properties, and the paper's statement that optimisation takes the deformed
mesh back to the ideal uniform configuration (checked with the oracle's
Newton solver, boundary nodes sliding in their faces)."""
import numpy as np
import pytest

import oracle as O
from paper_2205_12721_b300 import meshgen as mg


def test_kershaw_map_properties():
    rng = np.random.default_rng(0)
    X = rng.uniform(0, 1, (3, 4000))
    # eps = 1 is the identity
    np.testing.assert_allclose(mg.kershaw_map(X, 1.0, 1.0), X, atol=1e-15)
    Y = mg.kershaw_map(X, 0.3, 0.3)
    assert np.array_equal(Y[0], X[0])                       # x is kept
    # faces of the cube map to themselves
    for k in (1, 2):
        for v in (0.0, 1.0):
            Xb = X.copy()
            Xb[k] = v
            np.testing.assert_allclose(mg.kershaw_map(Xb, 0.3, 0.3)[k], v, atol=1e-15)
    # continuous across the layer boundaries x = j/6
    for j in range(1, 6):
        a, b = X.copy(), X.copy()
        a[0] = j / 6 - 1e-12
        b[0] = j / 6 + 1e-12
        assert np.abs(mg.kershaw_map(a, 0.3, 0.3) - mg.kershaw_map(b, 0.3, 0.3)).max() < 1e-9
    # strictly increasing in y at fixed x (a bijection of each line)
    t = np.linspace(0, 1, 2001)
    for x0 in (0.05, 0.2, 0.4, 0.6, 0.8, 0.95):
        L = mg.kershaw_map(np.vstack([np.full_like(t, x0), t, t]), 0.3, 0.3)
        assert np.all(np.diff(L[1]) > 0) and np.all(np.diff(L[2]) > 0)


def test_kershaw_sizes_and_fixed_components():
    m = mg.kershaw(2, (6, 2, 2))
    assert m.ndof == 3 * (13 * 5 * 5)
    X = mg.structured(3, 2, (6, 2, 2)).x.reshape(3, -1)
    f = m.fixed.reshape(3, -1)
    for a in range(3):
        on = (np.abs(X[a]) < 1e-14) | (np.abs(X[a] - 1) < 1e-14)
        assert np.array_equal(f[a] != 0, on)
    with pytest.raises(ValueError):
        mg.kershaw(1, (5, 2, 2))


@pytest.mark.parametrize("p,nq", [(1, 2), (1, 3), (2, 3)])
def test_kershaw_optimum_is_the_uniform_mesh(oracle_mod, p, nq):
    m = mg.kershaw(p, (6, 2, 2), 0.3, 0.3)
    u = mg.structured(3, p, (6, 2, 2))
    M = O.Mesh(3, p, nq, m.map, m.num_nodes, 303, m.fixed)
    x = m.x.copy()
    g0 = None
    for _ in range(30):
        r = oracle_mod.newton_step(M, x, 1e-10, 200)
        assert r["status"] == 0
        g0 = g0 or r["grad_norm"]
        if r["grad_norm_new"] < 1e-11 * g0:
            break
    assert np.abs(x - u.x).max() < 1e-9 / 6
