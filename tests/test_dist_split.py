"""The element-partitioned Newton step (the paper's P operator of Sec. 3 per
rank, interface sums between ranks) on CPU ranks: the partition's
bookkeeping, and full Newton steps (Sec. 2.3) of a split mesh with the FP64
oracle as every rank's local operator, through two communicators: ranks as
threads of one process, and gloo processes of a world of size 2 (127.0.0.1).
The split step must reproduce the single-rank oracle step to 1e-10 h, with
the same MINRES iteration count and line-search halvings."""
import os
import socket
import threading

import numpy as np
import pytest

import oracle as O
from paper_2205_12721_b300 import dist, meshgen as mg

from dist_oracle_backend import OracleBackend

CASES = [  # dim, order, shape, metric, steps
    (3, 2, (4, 3, 3), 302, 2),
    (2, 3, (6, 5), 2, 2),
]


def _mesh(d, p, shape, seed=5):
    return mg.perturb_smooth(mg.structured(d, p, shape), seed=seed, amp_smooth=0.03, amp_noise=0.015)


@pytest.mark.parametrize("world", [2, 3, 4])
def test_partition_bookkeeping(world):
    m = _mesh(3, 2, (5, 3, 3))
    parts = [dist.partition(m.map, m.num_nodes, m.dim, m.fixed, world, r) for r in range(world)]
    elems = np.concatenate([p.elems for p in parts])
    assert np.array_equal(elems, np.arange(m.num_elems))
    # every node is owned by exactly one rank, the lowest that touches it
    own = np.zeros(m.num_nodes, dtype=int)
    for p in parts:
        own[p.nodes[p.owned == 1]] += 1
        assert np.array_equal(p.nodes[p.local_map], m.map[p.elems])
        assert np.array_equal(p.fixed, p.to_local(m.fixed.astype(np.float64), m.num_nodes))
    assert np.all(own == 1)
    for p in parts:
        for r, ids in p.shared.items():
            q = parts[r]
            assert np.array_equal(p.nodes[ids], q.nodes[q.shared[p.rank]])  # same order both sides
            assert np.all(np.diff(p.nodes[ids]) > 0)


def _reference(m, metric, steps):
    om = O.Mesh(m.dim, m.order, m.order + 1, m.map, m.num_nodes, metric, m.fixed)
    x = m.x.copy()
    reps = [O.newton_step(om, x, 1e-8, 200) for _ in range(steps)]
    return x, reps


def _rank_run(m, metric, steps, world, rank, comm):
    part = dist.partition(m.map, m.num_nodes, m.dim, m.fixed, world, rank)
    be = OracleBackend(part, m.order, metric)
    dn = dist.DistNewton(be, comm)
    x = part.to_local(m.x, m.num_nodes)
    reps = [dn.newton_step(x, 1e-8, 200) for _ in range(steps)]
    be.close()
    return part, x, reps


def _check(m, steps, xref, rref, results):
    for part, x, reps in results:
        assert np.abs(x - part.to_local(xref, m.num_nodes)).max() <= 1e-10 * m.h
        for r, ro in zip(reps, rref):
            assert r["status"] == 0 and ro["status"] == 0
            assert r["minres_iters"] == ro["minres_iters"]
            assert r["halvings"] == ro["halvings"]
            assert abs(r["energy"] - ro["energy"]) <= 1e-12 * max(abs(ro["energy"]), 1.0)


@pytest.mark.parametrize("d,p,shape,metric,steps", CASES)
def test_split_newton_threads(d, p, shape, metric, steps):
    m = _mesh(d, p, shape)
    xref, rref = _reference(m, metric, steps)
    world = 2
    comms = dist.ThreadComm.group(world)
    out = [None] * world
    errs = []

    def run(r):
        try:
            out[r] = _rank_run(m, metric, steps, world, r, comms[r])
        except BaseException as ex:                # noqa: BLE001
            errs.append(ex)

    ts = [threading.Thread(target=run, args=(r,)) for r in range(world)]
    for t in ts:
        t.start()
    for t in ts:
        t.join(timeout=300)
    assert not errs, errs
    _check(m, steps, xref, rref, out)


def _gloo_worker(rank, world, port, q):
    import torch.distributed as td
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    td.init_process_group("gloo", rank=rank, world_size=world)
    try:
        d, p, shape, metric, steps = CASES[0]
        m = _mesh(d, p, shape)
        part, x, reps = _rank_run(m, metric, steps, world, rank, dist.TorchComm())
        q.put((rank, x, reps))
    except BaseException as ex:                    # noqa: BLE001
        q.put((rank, None, repr(ex)))
        raise
    finally:
        td.destroy_process_group()


def test_split_newton_gloo_world2():
    import torch.multiprocessing as tmp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = tmp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_gloo_worker, args=(r, 2, port, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    res = {}
    for _ in range(2):
        r, x, reps = q.get(timeout=240)
        assert x is not None, reps
        res[r] = (x, reps)
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    d, p, shape, metric, steps = CASES[0]
    m = _mesh(d, p, shape)
    xref, rref = _reference(m, metric, steps)
    parts = [dist.partition(m.map, m.num_nodes, m.dim, m.fixed, 2, r) for r in range(2)]
    _check(m, steps, xref, rref, [(parts[r], res[r][0], res[r][1]) for r in range(2)])
