"""The element-partitioned Newton step (dist.py) with the library as every
rank's local operator, against the single-mesh tmop_newton_step on the same
mesh (paper Sec. 2.3, Sec. 3 P operator): one rank, and two ranks that are
threads of one process sharing this GPU (each with its own context and
stream; they meet only on the host, in the communicator, so no kernel waits
for another).  Iterates to 1e-10 h, equal MINRES counts and halvings."""
import threading

import numpy as np
import pytest
import torch

from paper_2205_12721_b300 import capi, dist, meshgen as mg

from gpu_common import dev, gpu_mesh, host

pytestmark = pytest.mark.gpu


def _mesh():
    return mg.perturb_smooth(mg.structured(3, 2, (4, 3, 3)), seed=5, amp_smooth=0.03, amp_noise=0.015)


def _single(m, metric, steps):
    gm = gpu_mesh(m, metric)
    x = dev(m.x)
    reps = [gm.newton_step(x, 1e-8, 200) for _ in range(steps)]
    gm.close()
    return host(x), reps


def _split(m, metric, steps, world):
    comms = dist.ThreadComm.group(world)
    out, errs = [None] * world, []

    def run(r):
        try:
            s = torch.cuda.Stream()
            with torch.cuda.stream(s):
                part = dist.partition(m.map, m.num_nodes, m.dim, m.fixed, world, r)
                be = dist.LibraryBackend(part, m.order, metric, stream=s)
                dn = dist.DistNewton(be, comms[r])
                x = be.from_host(part.to_local(m.x, m.num_nodes))
                reps = [dn.newton_step(x, 1e-8, 200) for _ in range(steps)]
                s.synchronize()
                out[r] = (part, be.to_host(x), reps)
                be.close()
        except BaseException as ex:                # noqa: BLE001
            errs.append(ex)

    ts = [threading.Thread(target=run, args=(r,)) for r in range(world)]
    for t in ts:
        t.start()
    for t in ts:
        t.join(timeout=300)
    assert not errs, errs
    return out


@pytest.mark.parametrize("world", [1, 2])
def test_split_newton_matches_single_mesh(world):
    m, metric, steps = _mesh(), 302, 2
    xref, rref = _single(m, metric, steps)
    for part, x, reps in _split(m, metric, steps, world):
        assert np.abs(x - part.to_local(xref, m.num_nodes)).max() <= 1e-10 * m.h
        for r, ro in zip(reps, rref):
            assert r["status"] == 0 and ro["status"] == capi.OK
            assert r["minres_iters"] == ro["minres_iters"] and r["halvings"] == ro["halvings"]
            assert abs(r["energy"] - ro["energy"]) <= 1e-12 * max(abs(ro["energy"]), 1.0)


def test_vector_kernels():
    m = _mesh()
    gm = gpu_mesh(m, 302)
    n = m.ndof
    rng = np.random.default_rng(1)
    a, b, c = (rng.standard_normal(n) for _ in range(3))
    mask = (rng.random(n) < 0.5).astype(np.uint8)
    A, B, C = dev(a), dev(b), dev(c)
    out = torch.empty_like(A)
    capi.tmop_vec_lincomb(gm.ctx, out, 2.0, A, -3.0, B, 0.5, C)
    assert np.allclose(host(out), 2 * a - 3 * b + 0.5 * c, rtol=1e-15, atol=1e-15)
    capi.tmop_vec_mul(gm.ctx, out, A, B)
    assert np.array_equal(host(out), a * b)
    d = capi.tmop_vec_dot(gm.ctx, A, B, torch.from_numpy(mask).cuda())
    assert abs(d - np.dot(a[mask == 1], b[mask == 1])) <= 1e-13 * np.abs(a * b).sum()
    capi.tmop_vec_jacobi(gm.ctx, A, out)
    assert np.allclose(host(out), 1.0 / np.abs(a), rtol=1e-15)
    idx = torch.from_numpy(rng.permutation(n)[:100].astype(np.int32)).cuda()
    g = torch.empty(100, dtype=torch.float64, device="cuda")
    capi.tmop_vec_gather(gm.ctx, idx, A, g)
    assert np.array_equal(host(g), a[idx.cpu().numpy()])
    Bc = B.clone()
    capi.tmop_vec_scatter_add(gm.ctx, idx, g, Bc)
    ref = b.copy()
    ref[idx.cpu().numpy()] += a[idx.cpu().numpy()]
    assert np.array_equal(host(Bc), ref)
    gm.close()
