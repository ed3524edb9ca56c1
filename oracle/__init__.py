"""TMOP oracle: TEST INFRASTRUCTURE ONLY.

ctypes front end of ``tmop_oracle.c``, the plain FP64 CPU statement of the
TMOP partially assembled Newton step (paper Sec. 2.2-3.4).  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` import
this package; the CUDA library and its Python binding never do.

Arrays are numpy: positions ``x`` have shape ``(dim * num_nodes,)`` in
component-major order (``x[a * Nx + node]``), ``map`` is ``(E, (p+1)**dim)``
int32 in lexicographic local order, ``fixed`` is ``(dim * num_nodes,)`` uint8.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tmop_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

OK, ERR_ARG, ERR_INVERTED, ERR_MINRES, ERR_LINESEARCH = 0, 1, 2, 5, 6
TARGET_IDENTITY, TARGET_SIZE, TARGET_DISCRETE = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, single thread)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Mesh(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int), ("order", ctypes.c_int), ("nq1d", ctypes.c_int),
        ("num_elems", ctypes.c_int64), ("num_nodes", ctypes.c_int64),
        ("metric", ctypes.c_int), ("target", ctypes.c_int), ("target_h0", ctypes.c_double),
        ("map", ctypes.c_void_p), ("fixed", ctypes.c_void_p),
        ("limit_delta", ctypes.c_double), ("x0", ctypes.c_void_p),
        ("eta", ctypes.c_void_p), ("remap_x0", ctypes.c_void_p), ("remap_eta0", ctypes.c_void_p),
        ("remap_steps", ctypes.c_int), ("remap_cg_max_it", ctypes.c_int),
        ("remap_cg_rtol", ctypes.c_double),
    ]


class _Report(ctypes.Structure):
    _fields_ = [
        ("energy", ctypes.c_double), ("grad_norm", ctypes.c_double),
        ("energy_new", ctypes.c_double), ("grad_norm_new", ctypes.c_double),
        ("alpha", ctypes.c_double), ("min_det", ctypes.c_double),
        ("minres_resid", ctypes.c_double), ("minres_iters", ctypes.c_int),
        ("halvings", ctypes.c_int), ("status", ctypes.c_int),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        D, I, I64, P = ctypes.c_double, ctypes.c_int, ctypes.c_int64, ctypes.c_void_p
        sig = {
            "or_gauss_legendre": (I, [I, P, P]),
            "or_gll_nodes": (I, [I, P]),
            "or_lagrange": (None, [I, P, D, P, P]),
            "or_metric": (I, [I, I, P, P, P, P]),
            "or_energy": (I, [P, P, P, P, I64, P, P, P]),
            "or_det": (I, [P, P, P, I64, P]),
            "or_gradient": (I, [P, P, P, P, I64, P, P]),
            "or_hessian_apply": (I, [P, P, P, P, I64, P, P]),
            "or_hessian_diag": (I, [P, P, P, I64, P, P]),
            "or_hess_cache_build": (P, [P, P, P]),
            "or_hess_cache_free": (None, [P]),
            "or_hessian_apply_cached": (I, [P, P, P, P, P]),
            "or_minres": (I, [P, P, P, P, P, D, I, I, P, P, P]),
            "or_newton_step": (I, [P, P, D, I, I, D, I, P]),
            "or_mass_apply": (I, [P, P, P, P]),
            "or_mass_diag": (I, [P, P, P]),
            "or_advect_apply": (I, [P, P, P, P, P]),
            "or_remap": (I, [P, P, P, P, I, D, I, P, P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(_lib, name)
            f.restype = res
            f.argtypes = args
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# ---------------------------------------------------------------- 1D rules
def gauss_legendre(n: int):
    x = np.zeros(n); w = np.zeros(n)
    if lib().or_gauss_legendre(n, _p(x), _p(w)) != OK:
        raise ValueError("bad n")
    return x, w


def gll_nodes(n: int):
    x = np.zeros(n)
    if lib().or_gll_nodes(n, _p(x)) != OK:
        raise ValueError("bad n")
    return x


def lagrange(nodes, t: float):
    nodes = _f64(nodes)
    v = np.zeros(len(nodes)); d = np.zeros(len(nodes))
    lib().or_lagrange(len(nodes), _p(nodes), float(t), _p(v), _p(d))
    return v, d


def metric(mid: int, T):
    """(status, mu, P (d x d), K (d*d x d*d)) for metric id ``mid``."""
    T = _f64(T)
    d = T.shape[0]
    mu = np.zeros(1); P = np.zeros((d, d)); K = np.zeros((d * d, d * d))
    st = lib().or_metric(mid, d, _p(T), _p(mu), _p(P), _p(K))
    return st, float(mu[0]), P, K


# ---------------------------------------------------------------- mesh functionals
@dataclass
class Mesh:
    dim: int
    order: int
    nq1d: int
    map: np.ndarray           # (E, NP) int32
    num_nodes: int
    metric: int
    fixed: np.ndarray | None = None   # (dim*Nx,) uint8
    target: int = TARGET_IDENTITY
    target_h0: float = 1.0
    limit_delta: float = 0.0           # > 0 with x0: limiting term |x - x0|^2 / delta^2
    x0: np.ndarray | None = None
    eta: np.ndarray | None = None      # discrete target: nodal field on the current mesh
    remap_x0: np.ndarray | None = None  # Newton: eta remapped from (remap_x0, remap_eta0)
    remap_eta0: np.ndarray | None = None
    remap_steps: int = 4
    remap_cg_max_it: int = 200
    remap_cg_rtol: float = 1e-12

    def __post_init__(self):
        self.map = np.ascontiguousarray(self.map, dtype=np.int32)
        if self.fixed is not None:
            self.fixed = np.ascontiguousarray(self.fixed, dtype=np.uint8)
        for f in ("x0", "eta", "remap_x0", "remap_eta0"):
            if getattr(self, f) is not None:
                setattr(self, f, np.ascontiguousarray(getattr(self, f), dtype=np.float64))
        self._c = _Mesh(self.dim, self.order, self.nq1d, self.map.shape[0], self.num_nodes,
                        self.metric, self.target, self.target_h0, _p(self.map), _p(self.fixed),
                        self.limit_delta, _p(self.x0), _p(self.eta), _p(self.remap_x0),
                        _p(self.remap_eta0), self.remap_steps, self.remap_cg_max_it,
                        self.remap_cg_rtol)

    def set_eta(self, eta):
        """Replace the discrete target field (nodal values on the current mesh)."""
        self.eta = np.ascontiguousarray(eta, dtype=np.float64)
        self._c.eta = _p(self.eta)

    @property
    def ndof(self):
        return self.dim * self.num_nodes

    @property
    def nqd(self):
        return self.nq1d ** self.dim

    def ref(self):
        return ctypes.byref(self._c)


def _elems(elems):
    if elems is None:
        return None, 0
    e = np.ascontiguousarray(elems, dtype=np.int64)
    return e, len(e)


def energy(m: Mesh, x, xw=None, elems=None):
    """(status, F, min det A, S_F = sum |w_q det W|)."""
    x = _f64(x); xw = None if xw is None else _f64(xw)
    e, ne = _elems(elems)
    F = np.zeros(1); md = np.zeros(1); S = np.zeros(1)
    st = lib().or_energy(m.ref(), _p(x), _p(xw), _p(e), ne, _p(F), _p(md), _p(S))
    return st, float(F[0]), float(md[0]), float(S[0])


def det(m: Mesh, x, elems=None):
    x = _f64(x)
    e, ne = _elems(elems)
    n = m.map.shape[0] if e is None else ne
    out = np.zeros((n, m.nqd))
    st = lib().or_det(m.ref(), _p(x), _p(e), ne, _p(out))
    if st:
        raise RuntimeError(st)
    return out


def gradient(m: Mesh, x, elems=None, with_abs=False, xw=None):
    x = _f64(x); xw = None if xw is None else _f64(xw)
    e, ne = _elems(elems)
    g = np.zeros(m.ndof); a = np.zeros(m.ndof) if with_abs else None
    st = lib().or_gradient(m.ref(), _p(x), _p(xw), _p(e), ne, _p(g), _p(a))
    if st:
        raise RuntimeError(f"oracle gradient status {st}")
    return (g, a) if with_abs else g


def hessian_apply(m: Mesh, x, v, elems=None, with_abs=False):
    x = _f64(x); v = _f64(v)
    e, ne = _elems(elems)
    y = np.zeros(m.ndof); a = np.zeros(m.ndof) if with_abs else None
    st = lib().or_hessian_apply(m.ref(), _p(x), _p(v), _p(e), ne, _p(y), _p(a))
    if st:
        raise RuntimeError(f"oracle hessian_apply status {st}")
    return (y, a) if with_abs else y


def hessian_diag(m: Mesh, x, elems=None, with_abs=False):
    x = _f64(x)
    e, ne = _elems(elems)
    dg = np.zeros(m.ndof); a = np.zeros(m.ndof) if with_abs else None
    st = lib().or_hessian_diag(m.ref(), _p(x), _p(e), ne, _p(dg), _p(a))
    if st:
        raise RuntimeError(f"oracle hessian_diag status {st}")
    return (dg, a) if with_abs else dg


def dense_hessian(m: Mesh, x):
    """Dense d2F (with the fixed-DOF identity rows/columns), one column per
    unit vector through the Hessian action.  Small meshes only."""
    n = m.ndof
    H = np.zeros((n, n))
    for j in range(n):
        u = np.zeros(n); u[j] = 1.0
        H[:, j] = hessian_apply(m, x, u)
    return H


def minres(m: Mesh, x, diag, b, rtol=1e-8, max_it=50, fixed_its=False):
    """(status, dx, iterations, relative preconditioned residual)."""
    x = _f64(x); diag = _f64(diag); b = _f64(b)
    st = ctypes.c_int(0)
    H = lib().or_hess_cache_build(m.ref(), _p(x), ctypes.byref(st))
    try:
        dx = np.zeros(m.ndof)
        it = ctypes.c_int(0); res = ctypes.c_double(0)
        rc = lib().or_minres(m.ref(), _p(x), H, _p(diag), _p(b), rtol, max_it, int(fixed_its),
                             _p(dx), ctypes.byref(it), ctypes.byref(res))
    finally:
        lib().or_hess_cache_free(H)
    return rc, dx, it.value, res.value


def newton_step(m: Mesh, x, minres_rtol=1e-8, minres_max_it=50, minres_fixed_its=False,
                ls_factor=1.2, ls_max_halvings=20):
    """One Newton step in place on ``x`` (float64 array); returns the report dict."""
    assert x.dtype == np.float64 and x.flags.c_contiguous
    r = _Report()
    lib().or_newton_step(m.ref(), _p(x), minres_rtol, minres_max_it, int(minres_fixed_its),
                         ls_factor, ls_max_halvings, ctypes.byref(r))
    return {f: getattr(r, f) for f, _ in _Report._fields_}


# ---------------------------------------------------------------- remap (Sec. 3.6)
def mass_apply(m: Mesh, x, u):
    """(status, M(x) u) for a nodal scalar field u."""
    x = _f64(x); u = _f64(u)
    y = np.zeros(m.num_nodes)
    st = lib().or_mass_apply(m.ref(), _p(x), _p(u), _p(y))
    return st, y


def mass_diag(m: Mesh, x):
    x = _f64(x)
    dg = np.zeros(m.num_nodes)
    st = lib().or_mass_diag(m.ref(), _p(x), _p(dg))
    return st, dg


def advect_apply(m: Mesh, x, vel, u):
    """(status, K(x, vel) u): int w_i vel . grad u over the mesh x."""
    x = _f64(x); vel = _f64(vel); u = _f64(u)
    y = np.zeros(m.num_nodes)
    st = lib().or_advect_apply(m.ref(), _p(x), _p(vel), _p(u), _p(y))
    return st, y


def remap(m: Mesh, x0, x1, eta0, steps=4, cg_rtol=1e-12, cg_max_it=200):
    """(status, eta1, total CG iterations): eta0 on x0 advected to x1."""
    x0 = _f64(x0); x1 = _f64(x1); eta0 = _f64(eta0)
    eta1 = np.zeros(m.num_nodes)
    its = ctypes.c_int(0)
    st = lib().or_remap(m.ref(), _p(x0), _p(x1), _p(eta0), int(steps), float(cg_rtol),
                        int(cg_max_it), _p(eta1), ctypes.byref(its))
    return st, eta1, its.value
