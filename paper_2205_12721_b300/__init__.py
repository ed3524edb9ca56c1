"""B300-native (sm_103a) TMOP partial-assembly Newton step.

The computation lives in ``libtmop_b300.so`` (CUDA kernels behind the C ABI of
``include/tmop.h``); ``capi`` is its ctypes binding and ``TmopMesh`` a small
convenience wrapper holding one context.  PyTorch only provides device
memory and streams.  ``meshgen`` builds seeded synthetic input meshes.
"""
from __future__ import annotations

from . import meshgen  # noqa: F401  (geometry only; no method arithmetic)

__all__ = ["TmopMesh", "meshgen", "capi"]


def __getattr__(name):
    import importlib
    if name in ("capi", "mesh_opt", "build"):
        return importlib.import_module(f".{name}", __name__)
    if name == "TmopMesh":
        return importlib.import_module(".mesh_opt", __name__).TmopMesh
    raise AttributeError(name)
