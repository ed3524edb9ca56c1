"""Parity at the full benchmark sizes, in the launch configuration the
benchmark uses: 3D 24^3 Q2 (mu_302) and 3D 48^3 Q3 (mu_303).

The energy is compared in full (the oracle needs a few seconds).  Gradient,
Hessian action and diagonal are compared on sampled nodes: the oracle
evaluates only the elements around the sampled nodes, which gives those
nodes' assembled values exactly."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2205_12721_b300 import meshgen as mg

from gpu_common import TOL, assert_vec_close, dev, gpu_mesh, host, oracle_mesh

pytestmark = pytest.mark.gpu


def _sample(m, k, seed):
    rng = np.random.default_rng(seed)
    nodes = rng.choice(m.num_nodes, size=k, replace=False)
    elems = np.unique(np.nonzero(np.isin(m.map, nodes))[0])
    dofs = (np.arange(m.dim)[:, None] * m.num_nodes + nodes[None, :]).reshape(-1)
    return elems, dofs


@pytest.mark.parametrize("cfg", [2, 3])
def test_fullsize_sampled_parity(cfg):
    m = mg.config_mesh(cfg)
    metric = mg.CONFIG_METRIC[cfg]
    om = oracle_mesh(m, metric)
    gm = gpu_mesh(m, metric)
    x = dev(m.x)
    st_o, F_o, md_o, S = O.energy(om, m.x)
    st, F, md = gm.energy(x)
    assert st == 0 and st_o == 0
    assert abs(F - F_o) <= TOL * max(F_o, S)
    assert abs(md - md_o) <= TOL * md_o
    elems, dofs = _sample(m, 60, cfg)
    det = host(gm.det(x))[elems]
    det_o = O.det(om, m.x, elems=elems)
    assert np.all(np.abs(det - det_o) <= TOL * np.abs(det_o)), "det A (sampled elements)"
    g_o, ga = O.gradient(om, m.x, elems=elems, with_abs=True)
    g = host(gm.gradient(x))
    assert_vec_close(g[dofs], g_o[dofs], ga[dofs], what="gradient (sampled)")
    gm.hessian_setup(x)
    v = np.random.default_rng(7).standard_normal(m.ndof)
    y = host(gm.hessian_apply(dev(v)))
    y_o, ya = O.hessian_apply(om, m.x, v, elems=elems, with_abs=True)
    assert_vec_close(y[dofs], y_o[dofs], ya[dofs], what="apply (sampled)")
    dg = host(gm.hessian_diag())
    dg_o, dga = O.hessian_diag(om, m.x, elems=elems, with_abs=True)
    assert_vec_close(dg[dofs], dg_o[dofs], dga[dofs], what="diag (sampled)")
    gm.close()
    if cfg == 3:
        g32 = gpu_mesh(m, metric, precision="fp32")
        g32.hessian_setup(x)
        y32 = host(g32.hessian_apply(dev(v, torch.float32)))
        assert_vec_close(y32[dofs], y_o[dofs], ya[dofs], tol=2e-6, what="fp32 apply (sampled)")
        g32.close()
