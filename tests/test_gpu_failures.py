"""Failure paths of the Newton step (paper Sec. 2.3), on the single-mesh and
batched paths and in the server.  Every failure is made on the host, with no
GPU fault: a line search that cannot succeed (ls_factor = 0: F(x+) < 0 F(x)
never holds for a shape metric, F >= 0), a MINRES breakdown reported by the
library's host-side fault hook after a normal solve, and an inverted input
mesh.  The caller must get the failure status with x unchanged, and in a
batch or the server the other meshes' results must be those of a run
without the failure, bitwise."""
import numpy as np
import pytest
import torch

from paper_2205_12721_b300 import capi, meshgen as mg
from paper_2205_12721_b300.batch import TmopBatch
from paper_2205_12721_b300.serve import Server

from gpu_common import dev, gpu_mesh, host

pytestmark = pytest.mark.gpu


def _meshes():
    return [mg.perturb_smooth(mg.structured(3, 2, s), seed=70 + i, amp_smooth=0.03, amp_noise=0.015)
            for i, s in enumerate([(3, 3, 2), (4, 3, 2), (2, 3, 3)])]


def test_linesearch_exhaustion_single_mesh():
    m = mg.config_mesh(1)
    gm = gpu_mesh(m, 2)
    x = dev(m.x)
    x0 = x.clone()
    r = gm.newton_step(x, ls_factor=0.0, ls_max_halvings=3)
    assert r["status"] == capi.ERR_LINESEARCH and r["alpha"] == 0.0
    assert torch.equal(x, x0)
    r = gm.newton_step(x)                        # the context stays usable
    assert r["status"] == capi.OK and not torch.equal(x, x0)
    gm.close()


def test_linesearch_exhaustion_batch():
    ms = _meshes()
    b = TmopBatch(3, 2, 302, max_meshes=4, ls_factor=0.0, ls_max_halvings=2)
    slots = [b.add_structured(m) for m in ms]
    b.step()
    for s, m in zip(slots, ms):
        st = b.state(s)
        assert st["status"] == capi.ERR_LINESEARCH and st["done"]
        assert np.array_equal(b.positions(s).cpu().numpy(), m.x)
    b.close()


def test_minres_breakdown_single_mesh():
    m = mg.perturb_uniform(mg.structured(2, 2, 8), 0.08, 20260102)
    gm = gpu_mesh(m, 2)
    x = dev(m.x)
    x0 = x.clone()
    capi.tmop_inject_fault(gm.ctx, capi.FAULT_MINRES_BREAKDOWN)
    r = gm.newton_step(x)
    assert r["status"] == capi.ERR_MINRES and r["minres_iters"] > 0
    assert torch.equal(x, x0)
    assert "breakdown" in capi.last_error()
    r = gm.newton_step(x)                        # applies once
    assert r["status"] == capi.OK
    with pytest.raises(capi.TmopError):
        capi.tmop_inject_fault(gm.ctx, 99)
    gm.close()


def test_minres_breakdown_batch_mesh_retired_others_unchanged():
    ms = _meshes()

    def run(inject):
        b = TmopBatch(3, 2, 302, max_meshes=4, minres_max_it=30)
        slots = [b.add_structured(m) for m in ms]
        if inject:
            capi.tmop_batch_inject_fault(b.handle, slots[1], capi.FAULT_MINRES_BREAKDOWN)
        out = []
        for _ in range(2):
            b.step()
        for s in slots:
            out.append((b.state(s), b.positions(s).cpu().numpy()))
        b.close()
        return out

    ref = run(False)
    got = run(True)
    st1, x1 = got[1]
    assert st1["status"] == capi.ERR_MINRES and st1["done"] and st1["newton_its"] == 0
    assert np.array_equal(x1, ms[1].x)
    for k in (0, 2):
        assert got[k][0]["status"] == capi.OK and got[k][0]["newton_its"] == ref[k][0]["newton_its"]
        assert np.array_equal(got[k][1], ref[k][1])


def test_served_failing_request_is_retired_alone():
    jobs = mg.serving_workload(6, rate=2000.0, seed=9, n2=(4, 8), n3=(2, 3), orders=(1, 2))
    bad = jobs[2]["id"]

    def build(job):
        m = mg.serving_mesh(job)
        if job["id"] == bad:                     # fold one interior node over its neighbours
            m = m.copy()
            interior = np.flatnonzero(m.fixed[:m.num_nodes] == 0)
            m.x[interior[len(interior) // 2]] += 3.0 * m.h
        return m

    srv = Server(8 << 30, newton_rtol=1e-6, newton_max_it=20, minres_max_it=40)
    done = {r["job"]["id"]: r for r in srv.run(jobs, build=build, keep_positions=True)}
    srv.close()
    assert len(done) == len(jobs)
    assert done[bad]["status"] == capi.ERR_INVERTED and done[bad]["newton_its"] == 0
    for j in jobs:
        if j["id"] == bad:
            continue
        a = Server(8 << 30, newton_rtol=1e-6, newton_max_it=20, minres_max_it=40)
        (ra,) = a.run([dict(j, arrival=0.0)], keep_positions=True)
        a.close()
        assert done[j["id"]]["status"] == capi.OK == ra["status"]
        assert np.array_equal(done[j["id"]]["x"], ra["x"])
