"""Thin ctypes binding of the C ABI in ``include/tmop.h``.

Functions keep the C names (``tmop_setup``, ``tmop_energy``, ...) and only
marshal arguments: device arrays are ``torch`` CUDA tensors (their
``data_ptr()`` is passed), host scalars come back as Python floats.  Every
step of the computation runs in ``libtmop_b300.so``; if the library is missing
the import fails loudly (there is no fallback path).
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtmop_b300.so")

OK, ERR_ARG, ERR_INVERTED, ERR_CUDA, ERR_OOM, ERR_MINRES, ERR_LINESEARCH, ERR_TIMEOUT, \
    ERR_UNSUPPORTED = range(9)
METRIC_2, METRIC_55, METRIC_302, METRIC_303, METRIC_303_55 = 2, 55, 302, 303, 30355
METRIC_7, METRIC_9 = 7, 9
TARGET_IDENTITY, TARGET_SIZE_FIELD, TARGET_DISCRETE = 0, 1, 2
FP64, FP32, FP64_NATIVE = 0, 1, 2
K_ENERGY, K_GRADIENT, K_HSETUP, K_APPLY, K_DIAG, K_ASSEMBLE, K_VECTOR = range(7)
K_REMAP_SETUP, K_MASS, K_ADVECT = 7, 8, 9

# names declared in include/tmop.h (checked by the test-suite)
EXPORTS = ("tmop_setup", "tmop_energy", "tmop_gradient", "tmop_hessian_setup",
           "tmop_hessian_apply", "tmop_hessian_diag", "tmop_newton_step", "tmop_destroy",
           "tmop_status_string", "tmop_last_error", "tmop_launch_count", "tmop_profile_enable",
           "tmop_set_graphs", "tmop_graph_launches", "tmop_step_reuses",
           "tmop_profile_read", "tmop_device_bytes", "tmop_energy_noalloc",
           "tmop_batch_create", "tmop_batch_add", "tmop_batch_step", "tmop_batch_state",
           "tmop_batch_positions", "tmop_batch_remove", "tmop_batch_mesh_bytes",
           "tmop_batch_device_bytes", "tmop_batch_destroy", "tmop_set_limit_reference",
           "tmop_set_target_field", "tmop_set_remap_source", "tmop_remap", "tmop_det",
           "tmop_apply_variants", "tmop_get_apply_variant", "tmop_set_apply_variant",
           "tmop_autotune", "tmop_inject_fault", "tmop_batch_inject_fault",
           "tmop_batch_set_graphs", "tmop_batch_graph_launches",
           "tmop_vec_lincomb", "tmop_vec_mul", "tmop_vec_dot", "tmop_vec_gather",
           "tmop_vec_scatter_add", "tmop_vec_jacobi")


class TmopError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {status_string(status)} ({last_error()})")


class Desc(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("order", ctypes.c_int), ("nq1d", ctypes.c_int),
                ("num_elems", ctypes.c_int64), ("num_nodes", ctypes.c_int64),
                ("metric", ctypes.c_int), ("target", ctypes.c_int),
                ("target_h0", ctypes.c_double), ("hess_precision", ctypes.c_int),
                ("limit_delta", ctypes.c_double)]


class SolverOpts(ctypes.Structure):
    _fields_ = [("minres_rtol", ctypes.c_double), ("minres_max_it", ctypes.c_int),
                ("minres_fixed_its", ctypes.c_int), ("ls_factor", ctypes.c_double),
                ("ls_max_halvings", ctypes.c_int)]


class StepReport(ctypes.Structure):
    _fields_ = [("energy", ctypes.c_double), ("grad_norm", ctypes.c_double),
                ("energy_new", ctypes.c_double), ("grad_norm_new", ctypes.c_double),
                ("alpha", ctypes.c_double), ("min_det", ctypes.c_double),
                ("minres_resid", ctypes.c_double), ("minres_iters", ctypes.c_int),
                ("halvings", ctypes.c_int), ("status", ctypes.c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class RemapOpts(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int), ("cg_rtol", ctypes.c_double), ("cg_max_it", ctypes.c_int)]


class RemapReport(ctypes.Structure):
    _fields_ = [("cg_iters", ctypes.c_int), ("solves", ctypes.c_int), ("min_det", ctypes.c_double),
                ("status", ctypes.c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class BatchDesc(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("order", ctypes.c_int), ("nq1d", ctypes.c_int),
                ("metric", ctypes.c_int), ("target", ctypes.c_int),
                ("hess_precision", ctypes.c_int), ("max_meshes", ctypes.c_int),
                ("solver", SolverOpts), ("newton_rtol", ctypes.c_double),
                ("newton_max_it", ctypes.c_int)]


class MeshState(ctypes.Structure):
    _fields_ = [("done", ctypes.c_int), ("status", ctypes.c_int), ("newton_its", ctypes.c_int),
                ("minres_its", ctypes.c_int), ("energy0", ctypes.c_double),
                ("energy", ctypes.c_double), ("grad_norm0", ctypes.c_double),
                ("grad_norm", ctypes.c_double), ("min_det", ctypes.c_double),
                ("alpha", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_lib = None


def lib():
    """Load the library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: run paper_2205_12721_b300/build.py "
                              "(there is no CPU fallback)")
        L = ctypes.CDLL(LIB_PATH)
        P, I, I64, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
        sig = {
            "tmop_setup": (I, [ctypes.POINTER(Desc), P, P, P, ctypes.POINTER(P)]),
            "tmop_energy": (I, [P, P, ctypes.POINTER(D), ctypes.POINTER(D)]),
            "tmop_gradient": (I, [P, P, P]),
            "tmop_det": (I, [P, P, P]),
            "tmop_apply_variants": (I, [I, I, I]),
            "tmop_get_apply_variant": (I, [I, I, I, I, ctypes.POINTER(I)]),
            "tmop_set_apply_variant": (I, [I, I, I, I, I]),
            "tmop_autotune": (I, [P, I, ctypes.POINTER(I), P]),
            "tmop_inject_fault": (I, [P, I]),
            "tmop_vec_lincomb": (I, [P, I64, D, P, D, P, D, P, P]),
            "tmop_vec_mul": (I, [P, I64, P, P, P]),
            "tmop_vec_dot": (I, [P, I64, P, P, P, ctypes.POINTER(D)]),
            "tmop_vec_gather": (I, [P, I64, P, P, P]),
            "tmop_vec_jacobi": (I, [P, I64, P, P]),
            "tmop_vec_scatter_add": (I, [P, I64, P, P, P]),
            "tmop_batch_inject_fault": (I, [P, I, I]),
            "tmop_batch_set_graphs": (I, [P, I]),
            "tmop_batch_graph_launches": (I64, [P]),
            "tmop_hessian_setup": (I, [P, P]),
            "tmop_hessian_apply": (I, [P, P, P]),
            "tmop_hessian_diag": (I, [P, P]),
            "tmop_newton_step": (I, [P, P, ctypes.POINTER(SolverOpts), ctypes.POINTER(StepReport)]),
            "tmop_destroy": (None, [P]),
            "tmop_status_string": (ctypes.c_char_p, [I]),
            "tmop_last_error": (ctypes.c_char_p, []),
            "tmop_launch_count": (I64, []),
            "tmop_profile_enable": (I, [P, I]),
            "tmop_set_graphs": (I, [P, I]),
            "tmop_graph_launches": (I64, [P]),
            "tmop_step_reuses": (I64, [P]),
            "tmop_profile_read": (I, [P, I, ctypes.POINTER(D), ctypes.POINTER(I64)]),
            "tmop_device_bytes": (I64, [P]),
            "tmop_energy_noalloc": (I, [ctypes.POINTER(Desc), P, P, P, P]),
            "tmop_batch_create": (I, [ctypes.POINTER(BatchDesc), P, ctypes.POINTER(P)]),
            "tmop_batch_add": (I, [P, I64, I64, P, P, P, D, ctypes.POINTER(I)]),
            "tmop_batch_step": (I, [P, ctypes.POINTER(I)]),
            "tmop_batch_state": (I, [P, I, ctypes.POINTER(MeshState)]),
            "tmop_batch_positions": (I, [P, I, P]),
            "tmop_batch_remove": (I, [P, I]),
            "tmop_batch_mesh_bytes": (I64, [P, I64, I64]),
            "tmop_batch_device_bytes": (I64, [P]),
            "tmop_batch_destroy": (None, [P]),
            "tmop_set_limit_reference": (I, [P, P]),
            "tmop_set_target_field": (I, [P, P]),
            "tmop_set_remap_source": (I, [P, P, P, ctypes.POINTER(RemapOpts)]),
            "tmop_remap": (I, [P, P, P, P, P, ctypes.POINTER(RemapOpts), ctypes.POINTER(RemapReport)]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return t.data_ptr()


def _check(st: int, where: str):
    if st != OK:
        raise TmopError(st, where)


def status_string(st: int) -> str:
    return lib().tmop_status_string(st).decode()


def last_error() -> str:
    return lib().tmop_last_error().decode()


def tmop_launch_count() -> int:
    return lib().tmop_launch_count()


def tmop_setup(desc: Desc, elem_to_node, fixed=None, stream=None) -> int:
    """Returns the context handle (an int).  ``stream``: a torch.cuda.Stream,
    a raw cudaStream_t int, or None for the current torch stream."""
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    elif not isinstance(stream, int):
        stream = stream.cuda_stream
    out = ctypes.c_void_p()
    _check(lib().tmop_setup(ctypes.byref(desc), _ptr(elem_to_node), _ptr(fixed), stream,
                            ctypes.byref(out)), "tmop_setup")
    return out.value


def tmop_energy(ctx: int, x, check: bool = True):
    """(status, F, min det A)."""
    F = ctypes.c_double(); md = ctypes.c_double()
    st = lib().tmop_energy(ctx, _ptr(x), ctypes.byref(F), ctypes.byref(md))
    if check and st not in (OK, ERR_INVERTED):
        _check(st, "tmop_energy")
    return st, F.value, md.value


def tmop_apply_variants(dim: int, order: int, nq1d: int) -> int:
    return int(lib().tmop_apply_variants(dim, order, nq1d))


def tmop_get_apply_variant(dim: int, order: int, nq1d: int, precision: int) -> int:
    v = ctypes.c_int(0)
    _check(lib().tmop_get_apply_variant(dim, order, nq1d, precision, ctypes.byref(v)),
           "tmop_get_apply_variant")
    return v.value


def tmop_set_apply_variant(dim: int, order: int, nq1d: int, precision: int, variant: int):
    _check(lib().tmop_set_apply_variant(dim, order, nq1d, precision, variant),
           "tmop_set_apply_variant")


def tmop_autotune(ctx: int, reps: int = 10):
    """(chosen variant, [ms per launch of variant 0, 1, ...])."""
    v = ctypes.c_int(0)
    ms = (ctypes.c_double * 32)(*([float("nan")] * 32))
    _check(lib().tmop_autotune(ctx, reps, ctypes.byref(v), ms), "tmop_autotune")
    times = [float(t) for t in ms]
    while times and times[-1] != times[-1]:      # drop the unused (NaN) slots
        times.pop()
    return v.value, times


def tmop_vec_lincomb(ctx: int, out, a, x, b=0.0, y=None, c=0.0, z=None):
    """out = a x + b y + c z on device FP64 tensors (y, z optional)."""
    _check(lib().tmop_vec_lincomb(ctx, out.numel(), float(a), _ptr(x), float(b), _ptr(y), float(c),
                                  _ptr(z), _ptr(out)), "tmop_vec_lincomb")


def tmop_vec_mul(ctx: int, out, x, y):
    _check(lib().tmop_vec_mul(ctx, out.numel(), _ptr(x), _ptr(y), _ptr(out)), "tmop_vec_mul")


def tmop_vec_dot(ctx: int, x, y, mask=None) -> float:
    out = ctypes.c_double(0.0)
    _check(lib().tmop_vec_dot(ctx, x.numel(), _ptr(x), _ptr(y), _ptr(mask), ctypes.byref(out)),
           "tmop_vec_dot")
    return out.value


def tmop_vec_jacobi(ctx: int, diag, minv):
    """minv = 1/|diag| (1 where |diag| < 1e-300)."""
    _check(lib().tmop_vec_jacobi(ctx, diag.numel(), _ptr(diag), _ptr(minv)), "tmop_vec_jacobi")


def tmop_vec_gather(ctx: int, idx, src, dst):
    """dst[k] = src[idx[k]] (idx: device int32 tensor)."""
    _check(lib().tmop_vec_gather(ctx, idx.numel(), _ptr(idx), _ptr(src), _ptr(dst)), "tmop_vec_gather")


def tmop_vec_scatter_add(ctx: int, idx, vals, dst):
    """dst[idx[k]] += vals[k] (distinct indices)."""
    _check(lib().tmop_vec_scatter_add(ctx, idx.numel(), _ptr(idx), _ptr(vals), _ptr(dst)),
           "tmop_vec_scatter_add")


FAULT_NONE, FAULT_MINRES_BREAKDOWN = 0, 1


def tmop_inject_fault(ctx: int, fault: int):
    _check(lib().tmop_inject_fault(ctx, fault), "tmop_inject_fault")


def tmop_batch_inject_fault(b: int, slot: int, fault: int):
    _check(lib().tmop_batch_inject_fault(b, slot, fault), "tmop_batch_inject_fault")


def tmop_batch_set_graphs(b: int, on: bool = True):
    _check(lib().tmop_batch_set_graphs(b, int(on)), "tmop_batch_set_graphs")


def tmop_batch_graph_launches(b: int) -> int:
    return int(lib().tmop_batch_graph_launches(b))


def tmop_det(ctx: int, x, det):
    """det(A) at every quadrature point into det (device FP64, E * nq1d^dim)."""
    _check(lib().tmop_det(ctx, _ptr(x), _ptr(det)), "tmop_det")


def tmop_gradient(ctx: int, x, g):
    _check(lib().tmop_gradient(ctx, _ptr(x), _ptr(g)), "tmop_gradient")


def tmop_hessian_setup(ctx: int, x):
    _check(lib().tmop_hessian_setup(ctx, _ptr(x)), "tmop_hessian_setup")


def tmop_hessian_apply(ctx: int, v, y):
    _check(lib().tmop_hessian_apply(ctx, _ptr(v), _ptr(y)), "tmop_hessian_apply")


def tmop_hessian_diag(ctx: int, diag):
    _check(lib().tmop_hessian_diag(ctx, _ptr(diag)), "tmop_hessian_diag")


def tmop_newton_step(ctx: int, x, opts: SolverOpts | None = None) -> dict:
    rep = StepReport()
    st = lib().tmop_newton_step(ctx, _ptr(x), ctypes.byref(opts) if opts is not None else None,
                                ctypes.byref(rep))
    d = rep.as_dict()
    d["status"] = st
    return d


def tmop_set_limit_reference(ctx: int, x0):
    _check(lib().tmop_set_limit_reference(ctx, _ptr(x0)), "tmop_set_limit_reference")


def tmop_set_target_field(ctx: int, eta):
    _check(lib().tmop_set_target_field(ctx, _ptr(eta)), "tmop_set_target_field")


def tmop_set_remap_source(ctx: int, x0, eta0, opts: RemapOpts | None = None):
    _check(lib().tmop_set_remap_source(ctx, _ptr(x0), _ptr(eta0),
                                       ctypes.byref(opts) if opts is not None else None),
           "tmop_set_remap_source")


def tmop_remap(ctx: int, x0, x1, eta0, eta1, opts: RemapOpts | None = None) -> dict:
    """Status in the returned dict (TMOP_ERR_INVERTED is reported, not raised)."""
    rep = RemapReport()
    st = lib().tmop_remap(ctx, _ptr(x0), _ptr(x1), _ptr(eta0), _ptr(eta1),
                          ctypes.byref(opts) if opts is not None else None, ctypes.byref(rep))
    if st not in (OK, ERR_INVERTED):
        _check(st, "tmop_remap")
    d = rep.as_dict()
    d["status"] = st
    return d


def tmop_destroy(ctx: int):
    lib().tmop_destroy(ctx)


def tmop_profile_enable(ctx: int, on: bool = True):
    _check(lib().tmop_profile_enable(ctx, int(on)), "tmop_profile_enable")


def tmop_set_graphs(ctx: int, on: bool = True):
    _check(lib().tmop_set_graphs(ctx, int(on)), "tmop_set_graphs")


def tmop_graph_launches(ctx: int) -> int:
    return int(lib().tmop_graph_launches(ctx))


def tmop_step_reuses(ctx: int) -> int:
    return int(lib().tmop_step_reuses(ctx))


def tmop_profile_read(ctx: int, kernel_class: int):
    ms = ctypes.c_double(); n = ctypes.c_int64()
    _check(lib().tmop_profile_read(ctx, kernel_class, ctypes.byref(ms), ctypes.byref(n)),
           "tmop_profile_read")
    return ms.value, n.value


def tmop_device_bytes(ctx: int) -> int:
    return lib().tmop_device_bytes(ctx)


def tmop_energy_noalloc(desc: Desc, elem_to_node, x, out, stream=None):
    """Energy and min det into the device array ``out`` (2 float64) with no
    allocation by the library.  Returns the status (no exception)."""
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    elif not isinstance(stream, int):
        stream = stream.cuda_stream
    return lib().tmop_energy_noalloc(ctypes.byref(desc), _ptr(elem_to_node), _ptr(x), _ptr(out),
                                     stream)


# ---------------------------------------------------------------- batches
def _stream_handle(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return stream if isinstance(stream, int) else stream.cuda_stream


def tmop_batch_create(desc: BatchDesc, stream=None) -> int:
    out = ctypes.c_void_p()
    _check(lib().tmop_batch_create(ctypes.byref(desc), _stream_handle(stream), ctypes.byref(out)),
           "tmop_batch_create")
    return out.value


def tmop_batch_add(b: int, num_elems: int, num_nodes: int, elem_to_node, fixed, x, h0=1.0) -> int:
    slot = ctypes.c_int()
    _check(lib().tmop_batch_add(b, num_elems, num_nodes, _ptr(elem_to_node), _ptr(fixed), _ptr(x),
                                float(h0), ctypes.byref(slot)), "tmop_batch_add")
    return slot.value


def tmop_batch_step(b: int) -> int:
    n = ctypes.c_int()
    _check(lib().tmop_batch_step(b, ctypes.byref(n)), "tmop_batch_step")
    return n.value


def tmop_batch_state(b: int, slot: int) -> dict:
    st = MeshState()
    _check(lib().tmop_batch_state(b, slot, ctypes.byref(st)), "tmop_batch_state")
    return st.as_dict()


def tmop_batch_positions(b: int, slot: int, x_out):
    _check(lib().tmop_batch_positions(b, slot, _ptr(x_out)), "tmop_batch_positions")


def tmop_batch_remove(b: int, slot: int):
    _check(lib().tmop_batch_remove(b, slot), "tmop_batch_remove")


def tmop_batch_mesh_bytes(b: int, num_elems: int, num_nodes: int) -> int:
    return lib().tmop_batch_mesh_bytes(b, num_elems, num_nodes)


def tmop_batch_device_bytes(b: int) -> int:
    return lib().tmop_batch_device_bytes(b)


def tmop_batch_destroy(b: int):
    lib().tmop_batch_destroy(b)
