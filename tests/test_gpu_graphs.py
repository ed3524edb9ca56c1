"""MINRES iterations as CUDA graphs (tmop_set_graphs): the Newton trajectory
is bitwise the same with and without graphs (the same kernels in the same
order, the iteration index taken from the device counter), with a
tolerance-stopped MINRES (the host test between 4-iteration blocks), fixed
iteration counts that are not a multiple of 4 (the tail runs as separate
launches), FP32 vectors, the limiting term, and a change of kernel variant
between steps (the graphs are captured again)."""
import numpy as np
import pytest
import torch

from gpu_common import dev, host, make_case
from paper_2205_12721_b300 import capi
from paper_2205_12721_b300.mesh_opt import TmopMesh

pytestmark = pytest.mark.gpu


def _run(m, metric, graphs, precision, steps, stream, limit=0.0, variant_switch=False, **opts):
    with torch.cuda.stream(stream):
        gm = TmopMesh(m.dim, m.order, m.map, m.num_nodes, metric, fixed=m.fixed,
                      precision=precision, stream=stream, limit_delta=limit,
                      x0=m.x if limit > 0 else None)
        capi.tmop_set_graphs(gm.ctx, graphs)
        x = dev(m.x)
        n0 = capi.tmop_launch_count()
        reps = []
        for i in range(steps):
            if variant_switch and i == 1:
                capi.tmop_set_apply_variant(m.dim, m.order, m.order + 1,
                                            {"fp64": capi.FP64, "fp32": capi.FP32}[precision], 3)
            reps.append(gm.newton_step(x, **opts))
        stream.synchronize()
        launches = capi.tmop_launch_count() - n0
        out = (host(x), reps, launches, capi.tmop_graph_launches(gm.ctx))
        gm.close()
    if variant_switch:
        capi.tmop_set_apply_variant(m.dim, m.order, m.order + 1,
                                    {"fp64": capi.FP64, "fp32": capi.FP32}[precision], -1)
    return out


@pytest.mark.parametrize("d,p,metric,shape,precision,opts,limit,switch", [
    (3, 2, 302, (4, 3, 3), "fp64", dict(minres_rtol=1e-8, minres_max_it=50), 0.0, False),
    (3, 3, 303, (3, 3, 2), "fp64", dict(minres_rtol=0.0, minres_max_it=22, minres_fixed_its=True), 0.0, True),
    (3, 2, 302, (4, 3, 3), "fp32", dict(minres_rtol=1e-6, minres_max_it=50), 0.0, False),
    (2, 2, 2, (8, 8), "fp64", dict(minres_rtol=1e-8, minres_max_it=50), 0.05, False),
], ids=["3d-p2-rtol", "3d-p3-fixed22-switch", "3d-p2-fp32", "2d-p2-limit"])
def test_graphs_same_trajectory(d, p, metric, shape, precision, opts, limit, switch):
    m = make_case(d, p, shape, seed=70 + p)
    s = torch.cuda.Stream()
    xg, rg, lg, ng = _run(m, metric, True, precision, 3, s, limit, switch, **opts)
    xd, rd, ld, nd = _run(m, metric, False, precision, 3, s, limit, switch, **opts)
    assert ng > 0 and nd == 0
    assert np.array_equal(xg, xd)
    for a, b in zip(rg, rd):
        assert a["status"] == b["status"] == capi.OK
        assert a["minres_iters"] == b["minres_iters"]
        assert a["energy"] == b["energy"] and a["alpha"] == b["alpha"]
    assert lg == ld                  # graph nodes counted as launches


def test_graphs_on_the_legacy_stream():
    """A context on the legacy default stream runs its graph-captured MINRES
    on a stream of its own, ordered by events before and after: the same
    trajectory as with separate launches, and work queued after the step on
    the legacy stream sees the new positions."""
    m = make_case(3, 2, (3, 3, 2), seed=5)
    out = []
    for graphs in (True, False):
        gm = TmopMesh(m.dim, m.order, m.map, m.num_nodes, 302, fixed=m.fixed)
        capi.tmop_set_graphs(gm.ctx, graphs)
        x = dev(m.x)
        reps = [gm.newton_step(x) for _ in range(3)]
        y = x * 2.0
        out.append((host(x), host(y), [r["energy"] for r in reps], capi.tmop_graph_launches(gm.ctx)))
        gm.close()
    assert out[0][3] > 0 and out[1][3] == 0
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    assert np.array_equal(out[0][1], 2.0 * out[0][0])
    assert out[0][2] == out[1][2]


def _batch_run(graphs, precision, join_leave):
    from paper_2205_12721_b300 import meshgen as mg
    from paper_2205_12721_b300.batch import TmopBatch
    meshes = [mg.perturb_smooth(mg.structured(3, 2, s), seed=80 + i, amp_smooth=0.03, amp_noise=0.015)
              for i, s in enumerate([(4, 3, 3), (3, 3, 2), (5, 4, 3), (2, 3, 2)])]
    b = TmopBatch(3, 2, 302, precision=precision, max_meshes=8, minres_rtol=1e-8, minres_max_it=50,
                  graphs=graphs)
    slots = [b.add_structured(m) for m in meshes[:3]]
    states = []
    for step in range(4):
        if join_leave and step == 1:
            slots.append(b.add_structured(meshes[3]))
        if join_leave and step == 2:
            b.remove(slots.pop(1))
        b.step()
        states.append([(b.state(s)["minres_its"], b.state(s)["energy"]) for s in slots])
    xs = [b.positions(s).cpu().numpy() for s in slots]
    ng = capi.tmop_batch_graph_launches(b.handle)
    b.close()
    return xs, states, ng


@pytest.mark.parametrize("precision,join_leave", [("fp64", False), ("fp64", True), ("fp32", True)])
def test_batch_graphs_same_trajectory(precision, join_leave):
    xg, sg, ng = _batch_run(True, precision, join_leave)
    xd, sd, nd = _batch_run(False, precision, join_leave)
    assert ng > 0 and nd == 0
    assert sg == sd
    for a, b in zip(xg, xd):
        assert np.array_equal(a, b)
