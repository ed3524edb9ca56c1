"""Continuous-batching server for mesh-optimisation requests.

Requests arrive over time; each is admitted as soon as the device-memory
budget allows (FIFO), into the batch of its (dim, order, metric) group, where
its positions, stored d2mu/dT2 data and Krylov vectors stay resident.  Every
tick advances all admitted meshes of every group by one Newton step in shared
launches; a mesh that converged (|dF|/|dF0| <= rtol), hit its step cap or
failed is retired at once (its slot and memory are freed for waiting
requests).  Latency = completion time - arrival time.
"""
from __future__ import annotations

import time
from collections import deque
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import torch

from . import capi, meshgen
from .batch import TmopBatch, step_all


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
        self.pool = ThreadPoolExecutor(max_workers=16)

    def group(self, dim, order, metric) -> TmopBatch:
        key = (dim, order, metric)
        if key not in self.groups:
            self.groups[key] = TmopBatch(dim, order, metric, **self.kw)
        return self.groups[key]

    def close(self):
        for g in self.groups.values():
            g.close()
        self.groups.clear()
        self.pool.shutdown(wait=True)

    def run(self, jobs, build=meshgen.serving_mesh, keep_positions=False, clock=time.perf_counter):
        """Serve ``jobs`` (dicts with id, arrival, dim, order, metric, ...).
        Returns the completed job records with latency and final state."""
        pending = deque(sorted(jobs, key=lambda j: j["arrival"]))
        waiting: deque = deque()
        active = {}                       # (key, slot) -> record
        done = []
        t0 = clock()
        ticks = 0
        while pending or waiting or active:
            now = clock() - t0
            while pending and pending[0]["arrival"] <= now:
                waiting.append(pending.popleft())
            # FIFO admission by memory budget
            while waiting:
                job = waiting[0]
                m = build(job)
                g = self.group(job["dim"], job["order"], job["metric"])
                need = g.mesh_bytes(m.num_elems, m.num_nodes)
                if self.used + need > self.budget and active:
                    break
                waiting.popleft()
                slot = g.add_structured(m, h0=1.0 / max(m.n))
                self.used += need
                active[((job["dim"], job["order"], job["metric"]), slot)] = {
                    "job": job, "bytes": need, "admitted": clock() - t0, "ndof": m.ndof}
            if not active:
                if pending:
                    time.sleep(max(0.0, min(pending[0]["arrival"] - (clock() - t0), 0.01)))
                continue
            live = {k for k, _ in active}
            step_all([g for key, g in self.groups.items() if key in live], self.pool)
            ticks += 1
            for (key, slot) in list(active):
                g = self.groups[key]
                st = g.state(slot)
                if st["done"]:
                    rec = active.pop((key, slot))
                    rec.update(st)
                    rec["done_at"] = clock() - t0
                    rec["latency"] = rec["done_at"] - rec["job"]["arrival"]
                    if keep_positions:
                        rec["x"] = g.positions(slot).cpu().numpy()
                    g.remove(slot)
                    self.used -= rec["bytes"]
                    done.append(rec)
        self.ticks = ticks
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
