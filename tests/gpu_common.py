"""Helpers shared by the GPU parity tests: build a case, run both sides,
compare with the condition-aware tolerances of the parity contract."""
from __future__ import annotations

import numpy as np
import torch

import oracle as O
from paper_2205_12721_b300 import meshgen as mg
from paper_2205_12721_b300.mesh_opt import TmopMesh

TOL = 1e-12          # FP64 GPU path vs FP64 oracle (relative, condition-aware)


def make_case(d, p, shape, seed=1, amp=0.05):
    m = mg.structured(d, p, shape)
    return mg.perturb_smooth(m, seed=seed, amp_smooth=amp, amp_noise=amp / 2)


def oracle_mesh(m, metric, nq=None, target=0, h0=1.0, fixed=True):
    return O.Mesh(m.dim, m.order, nq or m.order + 1, m.map, m.num_nodes, metric,
                  m.fixed if fixed else None, target, h0)


def gpu_mesh(m, metric, nq=None, target=0, h0=1.0, precision="fp64", fixed=True):
    return TmopMesh(m.dim, m.order, m.map, m.num_nodes, metric, fixed=m.fixed if fixed else None,
                    nq1d=nq or m.order + 1, target=target, target_h0=h0, precision=precision)


def dev(a, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dtype)


def host(t):
    return t.detach().double().cpu().numpy()


def assert_vec_close(gpu, ref, scale, tol=TOL, what=""):
    """Entry by entry, |gpu_i - ref_i| <= tol * max(|ref_i|, |scale_i|) + floor
    (scale_i: the same sum evaluated with absolute values, so an entry formed by
    cancellation is judged against the size of its terms; floor = tol * 1e-3 *
    max|scale|, below the rounding of any entry of that size); and the l2 form
    ||gpu - ref||_2 <= tol * max(||ref||_2, ||scale||_2)."""
    gpu, ref, scale = (np.asarray(a, dtype=np.float64) for a in (gpu, ref, scale))
    err = np.linalg.norm(gpu - ref)
    bound = tol * max(np.linalg.norm(ref), np.linalg.norm(scale), 1e-300)
    assert err <= bound, f"{what}: |diff| = {err:.3e} > {bound:.3e} (|ref| = {np.linalg.norm(ref):.3e})"
    floor = tol * 1e-3 * max(float(np.abs(scale).max(initial=0.0)), 1e-300)
    ent = np.abs(gpu - ref)
    lim = tol * np.maximum(np.abs(ref), np.abs(scale)) + floor
    bad = np.flatnonzero(ent > lim)
    assert bad.size == 0, (f"{what}: {bad.size} entries off, worst i={bad[np.argmax(ent[bad] / lim[bad])]}"
                           f" diff {ent[bad].max():.3e}, limit there {lim[bad][np.argmax(ent[bad])]:.3e}")
