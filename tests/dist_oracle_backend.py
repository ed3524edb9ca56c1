"""A local-operator backend of the element-partitioned Newton step
(paper_2205_12721_b300.dist) whose element work is the FP64 oracle on the
rank's sub-mesh and whose vectors are numpy arrays: test infrastructure, so
that the partition, the interface sums and the distributed Krylov iteration
run on CPU ranks (gloo) and can be checked against the single-rank oracle."""
from __future__ import annotations

import ctypes

import numpy as np

import oracle as O


class OracleBackend:
    def __init__(self, part, order, metric, nq1d=None, target=0, target_h0=1.0):
        self.part = part
        self.n = part.ndof
        self.om = O.Mesh(part.dim, order, nq1d or order + 1, part.local_map, part.num_nodes, metric,
                         part.fixed, target, target_h0)
        self.owned = part.owned_dofs().astype(bool)
        Nl = part.num_nodes
        self.halo = {r: np.concatenate([a * Nl + ids for a in range(part.dim)])
                     for r, ids in part.shared.items()}
        self.xs = None
        self.H = None

    def empty(self):
        return np.empty(self.n)

    def zeros(self):
        return np.zeros(self.n)

    def lincomb(self, out, a, x, b=0.0, y=None, c=0.0, z=None):
        v = a * x
        if y is not None:
            v = v + b * y
        if z is not None:
            v = v + c * z
        out[:] = v
        return out

    def mul(self, out, x, y):
        out[:] = x * y
        return out

    def dot_owned(self, x, y):
        return float(np.dot(x[self.owned], y[self.owned]))

    def jacobi(self, diag):
        a = np.abs(diag)
        return np.where(a < 1e-300, 1.0, 1.0 / np.where(a < 1e-300, 1.0, a))

    def pack(self, v, r):
        return v[self.halo[r]].copy()

    def unpack_add(self, v, r, vals):
        v[self.halo[r]] += np.asarray(vals)

    def sync(self):
        pass

    def energy(self, x):
        st, F, md, S = O.energy(self.om, x)
        return F, md

    def gradient(self, x, g):
        g[:] = O.gradient(self.om, x)
        return g

    def hessian_setup(self, x):
        self.free()
        self.xs = np.ascontiguousarray(x, dtype=np.float64).copy()
        st = ctypes.c_int(0)
        self.H = O.lib().or_hess_cache_build(self.om.ref(), self.xs.ctypes.data, ctypes.byref(st))

    def hessian_apply(self, v, y):
        v = np.ascontiguousarray(v, dtype=np.float64)
        out = np.zeros(self.n)
        O.lib().or_hessian_apply_cached(self.om.ref(), self.xs.ctypes.data, self.H, v.ctypes.data,
                                        out.ctypes.data)
        y[:] = out
        return y

    def hessian_diag(self, d):
        d[:] = O.hessian_diag(self.om, self.xs)
        return d

    def free(self):
        if self.H:
            O.lib().or_hess_cache_free(self.H)
            self.H = None

    def close(self):
        self.free()
