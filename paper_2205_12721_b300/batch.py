"""Many meshes in shared launches: a thin wrapper of the tmop_batch C ABI."""
from __future__ import annotations

import numpy as np
import torch

from . import capi

PRECISIONS = {"fp64": capi.FP64, "fp32": capi.FP32, "fp64-native": capi.FP64_NATIVE}


class TmopBatch:
    """Meshes sharing (dim, order, nq1d, metric, target, precision).

    ``add`` copies a mesh (map, fixed mask, positions) into batch-owned device
    memory and returns its slot; ``step`` runs one Newton step of every active
    mesh; ``state``/``positions`` read a mesh back; ``remove`` frees it."""

    def __init__(self, dim, order, metric, nq1d=None, target=capi.TARGET_IDENTITY,
                 precision="fp64", max_meshes=64, minres_rtol=1e-8, minres_max_it=50,
                 minres_fixed_its=False, ls_factor=1.2, ls_max_halvings=20, newton_rtol=1e-10,
                 newton_max_it=100, stream=None, graphs=True):
        self.dim, self.order = dim, order
        # each batch works on its own stream unless told otherwise, so that
        # batches stepped from different host threads overlap on the GPU
        self.stream = stream if stream is not None else torch.cuda.Stream()
        opts = capi.SolverOpts(minres_rtol, minres_max_it, int(minres_fixed_its), ls_factor,
                               ls_max_halvings)
        self.desc = capi.BatchDesc(dim, order, nq1d or order + 1, metric, target,
                                   PRECISIONS[precision], max_meshes, opts, newton_rtol,
                                   newton_max_it)
        self.handle = capi.tmop_batch_create(self.desc, self.stream)
        capi.tmop_batch_set_graphs(self.handle, graphs)
        self.ndof = {}

    def close(self):
        if getattr(self, "handle", None):
            capi.tmop_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def add(self, emap, num_nodes, x, fixed=None, h0=1.0) -> int:
        with torch.cuda.stream(self.stream):
            emap_d = torch.from_numpy(np.ascontiguousarray(emap, dtype=np.int32)).cuda()
            fixed_d = None if fixed is None else torch.from_numpy(
                np.ascontiguousarray(fixed, dtype=np.uint8)).cuda()
            x_d = x if isinstance(x, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(x)).cuda()
        self.stream.synchronize()
        slot = capi.tmop_batch_add(self.handle, int(emap.shape[0]), int(num_nodes), emap_d, fixed_d,
                                   x_d, h0)
        self.ndof[slot] = self.dim * int(num_nodes)
        return slot

    def add_structured(self, m, h0=1.0) -> int:
        return self.add(m.map, m.num_nodes, m.x, m.fixed, h0)

    def mesh_bytes(self, num_elems, num_nodes) -> int:
        return capi.tmop_batch_mesh_bytes(self.handle, num_elems, num_nodes)

    def device_bytes(self) -> int:
        return capi.tmop_batch_device_bytes(self.handle)

    def step(self) -> int:
        return capi.tmop_batch_step(self.handle)

    def state(self, slot) -> dict:
        return capi.tmop_batch_state(self.handle, slot)

    def positions(self, slot) -> torch.Tensor:
        with torch.cuda.stream(self.stream):
            x = torch.empty(self.ndof[slot], dtype=torch.float64, device="cuda")
        capi.tmop_batch_positions(self.handle, slot, x)
        self.stream.synchronize()
        return x

    def remove(self, slot):
        capi.tmop_batch_remove(self.handle, slot)
        self.ndof.pop(slot, None)

    def solve(self, max_steps=1000):
        """Step until every mesh is done; returns the number of steps."""
        n = 0
        while n < max_steps:
            n += 1
            if self.step() == 0:
                break
        return n


def step_all(batches, pool=None):
    """One Newton step of every batch; with a thread pool the batches run
    from different host threads on their own streams and overlap on the GPU
    (the library calls release the GIL).  Returns the active counts."""
    if pool is None or len(batches) < 2:
        return [b.step() for b in batches]
    return list(pool.map(lambda b: b.step(), batches))
