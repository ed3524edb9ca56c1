"""Continuous-batching server for mesh-optimisation requests.

Requests arrive over time; each is admitted as soon as the device-memory
budget allows (FIFO), into the batch of its (dim, order, metric) group, where
its positions, stored d2mu/dT2 data and Krylov vectors stay resident.  Every
group is stepped by its own host thread on its own stream: one Newton step of
all of the group's admitted meshes in shared launches, then the meshes that
converged (|dF|/|dF0| <= rtol), hit their step cap or failed are retired at
once (their memory is freed for waiting requests) and the requests admitted
meanwhile join before the next step.  Groups do not wait for each other, so a
group of small meshes is not held back by a group of large ones, and their
launches overlap on the device.  Latency = completion time - arrival time.
"""
from __future__ import annotations

import threading
import time
from collections import deque

import numpy as np

from . import capi, meshgen
from .batch import TmopBatch


class Server:
    def __init__(self, mem_budget_bytes: int, precision: str = "fp64", newton_rtol: float = 1e-6,
                 newton_max_it: int = 50, minres_rtol: float = 1e-8, minres_max_it: int = 50,
                 max_meshes_per_group: int = 512, stream=None, graphs: bool = True):
        self.budget = int(mem_budget_bytes)
        self.kw = dict(precision=precision, newton_rtol=newton_rtol, newton_max_it=newton_max_it,
                       minres_rtol=minres_rtol, minres_max_it=minres_max_it,
                       max_meshes=max_meshes_per_group, stream=stream, graphs=graphs)
        self.groups: dict = {}
        self.used = 0
        self.steps = 0

    def group(self, dim, order, metric) -> TmopBatch:
        key = (dim, order, metric)
        if key not in self.groups:
            self.groups[key] = TmopBatch(dim, order, metric, **self.kw)
        return self.groups[key]

    def close(self):
        for g in self.groups.values():
            g.close()
        self.groups.clear()

    def run(self, jobs, build=meshgen.serving_mesh, keep_positions=False, clock=time.perf_counter):
        """Serve ``jobs`` (dicts with id, arrival, dim, order, metric, ...).
        Returns the completed job records with latency and final state."""
        pending = deque(sorted(jobs, key=lambda j: j["arrival"]))
        waiting: deque = deque()                 # arrived, not admitted (FIFO)
        built: dict = {}                         # job id -> mesh of the head of the queue
        cv = threading.Condition()
        inbox: dict = {}                         # group -> admitted records not yet added
        active: dict = {}                        # group -> {slot: record} (its worker only)
        inflight: dict = {}                      # group -> admitted and not retired
        done = []
        workers: dict = {}
        failure = []
        stop = [False]
        t0 = clock()

        def busy():
            return any(inflight.values())

        def worker(key):
            g = self.groups[key]
            try:
                while True:
                    with cv:
                        while not (inflight[key] or stop[0]):
                            cv.wait(0.05)
                        if stop[0] and not inflight[key]:
                            return
                        joining = list(inbox[key])
                        inbox[key].clear()
                    for rec in joining:
                        m = rec.pop("mesh")
                        slot = g.add_structured(m, h0=1.0 / max(m.n))
                        rec["admitted"] = clock() - t0
                        active[key][slot] = rec
                    if not active[key]:
                        continue
                    g.step()
                    finished = []
                    for slot, rec in list(active[key].items()):
                        st = g.state(slot)
                        if st["done"]:
                            rec.update(st)
                            rec["done_at"] = clock() - t0
                            rec["latency"] = rec["done_at"] - rec["job"]["arrival"]
                            if keep_positions:
                                rec["x"] = g.positions(slot).cpu().numpy()
                            g.remove(slot)
                            del active[key][slot]
                            finished.append(rec)
                    with cv:
                        self.steps += 1
                        for rec in finished:
                            self.used -= rec["bytes"]
                            inflight[key] -= 1
                            done.append(rec)
                        cv.notify_all()
            except BaseException as exc:          # surfaced by run()
                with cv:
                    failure.append(exc)
                    stop[0] = True
                    cv.notify_all()

        try:
            with cv:
                while (pending or waiting or busy()) and not failure:
                    now = clock() - t0
                    while pending and pending[0]["arrival"] <= now:
                        waiting.append(pending.popleft())
                    # FIFO admission by memory budget
                    while waiting:
                        job = waiting[0]
                        if job["id"] not in built:
                            cv.release()                 # build the mesh without the lock
                            try:
                                built[job["id"]] = build(job)
                            finally:
                                cv.acquire()
                        m = built[job["id"]]
                        key = (job["dim"], job["order"], job["metric"])
                        g = self.group(*key)
                        need = g.mesh_bytes(m.num_elems, m.num_nodes)
                        if self.used + need > self.budget and busy():
                            break
                        waiting.popleft()
                        del built[job["id"]]
                        self.used += need
                        if key not in inbox:
                            inbox[key], active[key], inflight[key] = deque(), {}, 0
                        inbox[key].append({"job": job, "bytes": need, "ndof": m.ndof, "mesh": m})
                        inflight[key] += 1
                        if key not in workers:
                            workers[key] = threading.Thread(target=worker, args=(key,), daemon=True)
                            workers[key].start()
                        cv.notify_all()
                    if waiting and not busy():
                        continue                         # admit the head even over budget
                    if pending or waiting or busy():
                        wait = 0.05
                        if pending:
                            wait = min(wait, max(0.0, pending[0]["arrival"] - (clock() - t0)))
                        cv.wait(wait)
                stop[0] = True
                cv.notify_all()
        finally:
            with cv:
                stop[0] = True
                cv.notify_all()
            for t in workers.values():
                t.join()
        if failure:
            raise failure[0]
        return done


def summarize(done):
    lat = np.array([r["latency"] for r in done])
    span = max(r["done_at"] for r in done) - min(r["job"]["arrival"] for r in done)
    ok = sum(1 for r in done if r["status"] == capi.OK)
    return {"jobs": len(done), "ok": ok, "p50_s": float(np.percentile(lat, 50)),
            "p99_s": float(np.percentile(lat, 99)), "mean_s": float(lat.mean()),
            "meshes_per_s": len(done) / span if span > 0 else None,
            "newton_its_mean": float(np.mean([r["newton_its"] for r in done])),
            "dofs_total": int(sum(r["ndof"] for r in done))}
