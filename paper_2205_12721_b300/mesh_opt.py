"""One TMOP problem on one GPU: a context plus its device-resident inputs."""
from __future__ import annotations

import numpy as np
import torch

from . import capi


class TmopMesh:
    """Holds a ``tmop_ctx`` for one mesh.

    ``map`` (E x (p+1)^d int32), ``fixed`` (d*Nx uint8 or None) are copied to
    the device once.  Positions and vectors are torch CUDA tensors of length
    d*Nx in component-major order (float64; float32 for the Hessian action
    of a ``precision="fp32"`` context).  ``precision``: "fp64" (double-float
    contractions on the FP32 units), "fp32" (mixed) or "fp64-native".
    """

    def __init__(self, dim, order, emap, num_nodes, metric, fixed=None, nq1d=None,
                 target=capi.TARGET_IDENTITY, target_h0=1.0, precision="fp64", device="cuda",
                 stream=None, limit_delta=0.0, x0=None):
        self.dim, self.order = dim, order
        self.nq1d = nq1d or order + 1
        self.num_nodes = int(num_nodes)
        self.ndof = dim * self.num_nodes
        self.device = torch.device(device)
        self.prec = {"fp64": capi.FP64, "fp32": capi.FP32, "fp64-native": capi.FP64_NATIVE}[precision]
        self.rdtype = torch.float32 if self.prec == capi.FP32 else torch.float64
        emap = np.ascontiguousarray(emap, dtype=np.int32)
        self.num_elems = int(emap.shape[0])
        self._map = torch.from_numpy(emap).to(self.device)
        self._fixed = None if fixed is None else torch.from_numpy(
            np.ascontiguousarray(fixed, dtype=np.uint8)).to(self.device)
        self.desc = capi.Desc(dim, order, self.nq1d, self.num_elems, self.num_nodes, metric,
                              target, float(target_h0), self.prec, float(limit_delta))
        self.stream = stream
        self.ctx = capi.tmop_setup(self.desc, self._map, self._fixed, stream)
        if limit_delta > 0.0 and x0 is not None:
            self.set_limit_reference(x0)

    def _dev64(self, a):
        t = a if isinstance(a, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(a))
        return t.to(self.device, torch.float64).contiguous()

    def set_target_field(self, eta):
        """Nodal field eta of the discrete target W = h0 eta(x_q)^(1/d) I."""
        self._eta = self._dev64(eta)
        capi.tmop_set_target_field(self.ctx, self._eta)

    def set_remap_source(self, x0, eta0, steps=4, cg_rtol=1e-12, cg_max_it=200):
        """eta0 on positions x0: Newton remaps it to every new position."""
        self._rx0, self._reta0 = self._dev64(x0), self._dev64(eta0)
        capi.tmop_set_remap_source(self.ctx, self._rx0, self._reta0,
                                   capi.RemapOpts(steps, cg_rtol, cg_max_it))

    def remap(self, x0, x1, eta0, steps=4, cg_rtol=1e-12, cg_max_it=200):
        """(eta1 tensor, report dict): eta0 advected from positions x0 to x1."""
        x0, x1, eta0 = self._dev64(x0), self._dev64(x1), self._dev64(eta0)
        eta1 = torch.empty_like(eta0)
        rep = capi.tmop_remap(self.ctx, x0, x1, eta0, eta1, capi.RemapOpts(steps, cg_rtol, cg_max_it))
        return eta1, rep

    def set_limit_reference(self, x0):
        """Reference positions of the limiting term |x - x0|^2 / delta^2."""
        x0d = x0 if isinstance(x0, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(x0))
        self._x0 = x0d.to(self.device, torch.float64)
        capi.tmop_set_limit_reference(self.ctx, self._x0)

    @classmethod
    def from_structured(cls, m, metric, **kw):
        return cls(m.dim, m.order, m.map, m.num_nodes, metric, fixed=m.fixed, **kw)

    def close(self):
        if getattr(self, "ctx", None):
            capi.tmop_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- the seven operations -------------------------------------------------
    def energy(self, x):
        """(status, F, min det A)."""
        return capi.tmop_energy(self.ctx, x)

    def det(self, x, out=None):
        """det(A) at every quadrature point, shape (num_elems, nq1d**dim)."""
        nqd = self.nq1d ** self.dim
        d = out if out is not None else torch.empty(self.num_elems * nqd, dtype=torch.float64,
                                                    device=self.device)
        capi.tmop_det(self.ctx, x, d)
        return d.view(self.num_elems, nqd)

    def gradient(self, x, out=None):
        g = out if out is not None else torch.empty(self.ndof, dtype=torch.float64, device=self.device)
        capi.tmop_gradient(self.ctx, x, g)
        return g

    def hessian_setup(self, x):
        capi.tmop_hessian_setup(self.ctx, x)

    def hessian_apply(self, v, out=None):
        y = out if out is not None else torch.empty(self.ndof, dtype=self.rdtype, device=self.device)
        capi.tmop_hessian_apply(self.ctx, v, y)
        return y

    def hessian_diag(self, out=None):
        d = out if out is not None else torch.empty(self.ndof, dtype=self.rdtype, device=self.device)
        capi.tmop_hessian_diag(self.ctx, d)
        return d

    def newton_step(self, x, minres_rtol=1e-8, minres_max_it=50, minres_fixed_its=False,
                    ls_factor=1.2, ls_max_halvings=20):
        o = capi.SolverOpts(minres_rtol, minres_max_it, int(minres_fixed_its), ls_factor,
                            ls_max_halvings)
        return capi.tmop_newton_step(self.ctx, x, o)

    def solve(self, x, max_newton=100, rtol=1e-10, **kw):
        """Newton iterations until |dF(x)| / |dF(x0)| <= rtol (paper Sec. 2.3)."""
        reps = []
        g0 = None
        for _ in range(max_newton):
            r = self.newton_step(x, **kw)
            reps.append(r)
            if g0 is None:
                g0 = r["grad_norm"]
            if r["status"] != capi.OK:
                break
            if g0 == 0 or r["grad_norm_new"] <= rtol * g0:
                break
        return reps
