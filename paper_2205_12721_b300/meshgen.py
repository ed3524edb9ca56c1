"""Seeded synthetic meshes: the inputs shared by the CUDA path, the oracle, the
tests and the benchmark.

This module builds geometry only.  It holds none of the TMOP arithmetic (no
basis evaluation, Jacobian, metric or quadrature), so both sides of a parity
test receive identical inputs without sharing any of the method's code.

Meshes are structured Q_p quadrilateral / hexahedral meshes of [0,1]^d
(paper Sec. 2.1).  Within an element, nodes sit at the tensor product of the
Gauss-Lobatto-Legendre points of degree p; node and element numbering is
lexicographic, matching the local ordering of paper Sec. 3.1:

* global node (I_1, .., I_d) -> I_1 + M_1 (I_2 + M_2 I_3), M_k = p n_k + 1;
* element (e_1, .., e_d) -> e_1 + n_1 (e_2 + n_2 e_3);
* ``map[e, i]`` = global node of local node i = i_1 + (p+1) i_2 + (p+1)^2 i_3.

Positions are component-major: ``x[a * Nx + node]``.  Boundary nodes of the
cube are fixed in every component (the fixed-boundary reading of the
benchmark configurations).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
from numpy.polynomial import legendre as _leg

BASE_SEED = 20260101


def gll_points(n: int) -> np.ndarray:
    """n Gauss-Lobatto-Legendre points on [0,1] (end points plus the roots of
    P'_{n-1}), from numpy's Legendre-series root finder."""
    if n < 2:
        raise ValueError("need at least 2 points")
    c = np.zeros(n)
    c[-1] = 1.0
    inner = np.sort(np.real(_leg.legroots(_leg.legder(c)))) if n > 2 else np.zeros(0)
    z = np.concatenate([[-1.0], inner, [1.0]])
    return (z + 1.0) / 2.0


@dataclass
class StructuredMesh:
    dim: int
    order: int
    n: tuple                     # elements per side
    x: np.ndarray                # (dim * Nx,) float64, component-major
    map: np.ndarray              # (E, (p+1)^dim) int32
    fixed: np.ndarray            # (dim * Nx,) uint8
    grid: tuple = field(default=())   # nodes per side M_k

    @property
    def num_nodes(self) -> int:
        return int(np.prod(self.grid))

    @property
    def num_elems(self) -> int:
        return int(self.map.shape[0])

    @property
    def ndof(self) -> int:
        return self.dim * self.num_nodes

    @property
    def h(self) -> float:
        return 1.0 / max(self.n)

    def copy(self) -> "StructuredMesh":
        return StructuredMesh(self.dim, self.order, self.n, self.x.copy(), self.map, self.fixed,
                              self.grid)


def structured(dim: int, order: int, n_e, ) -> StructuredMesh:
    """Uniform Cartesian Q_order mesh of [0,1]^dim with n_e elements per side
    (an int, or one count per axis)."""
    if dim not in (2, 3) or order < 1:
        raise ValueError("dim must be 2 or 3 and order >= 1")
    ns = tuple([int(n_e)] * dim) if np.isscalar(n_e) else tuple(int(v) for v in n_e)
    ni = order + 1
    M = tuple(order * n + 1 for n in ns)
    g = gll_points(ni)
    coords = []
    for k in range(dim):
        c = np.empty(M[k])
        for e in range(ns[k]):
            c[order * e: order * e + ni] = (e + g) / ns[k]
        c[-1] = 1.0
        coords.append(c)
    Nx = int(np.prod(M))
    # node grid (I_1 fastest)
    idx = np.indices(M[::-1])[::-1]          # idx[k] has shape M reversed, I_k values
    x = np.empty(dim * Nx)
    for a in range(dim):
        x[a * Nx:(a + 1) * Nx] = coords[a][idx[a].reshape(-1)]
    # element map
    eidx = np.indices(ns[::-1])[::-1]        # element multi-indices, e_1 fastest
    lidx = np.indices((ni,) * dim)[::-1]     # local multi-indices, i_1 fastest
    E = int(np.prod(ns))
    NP = ni ** dim
    gi = [(order * eidx[k].reshape(E, 1) + lidx[k].reshape(1, NP)) for k in range(dim)]
    node = gi[0].astype(np.int64)
    stride = 1
    for k in range(1, dim):
        stride *= M[k - 1]
        node = node + stride * gi[k]
    emap = node.astype(np.int32)
    # boundary nodes fixed in all components
    on_bnd = np.zeros(Nx, dtype=bool)
    for k in range(dim):
        Ik = idx[k].reshape(-1)
        on_bnd |= (Ik == 0) | (Ik == M[k] - 1)
    fixed = np.tile(on_bnd.astype(np.uint8), dim)
    return StructuredMesh(dim, order, ns, x, emap, fixed, M)


def perturb_uniform(mesh: StructuredMesh, amp: float = 0.15, seed: int = BASE_SEED) -> StructuredMesh:
    """Interior nodes displaced by U[-amp h, amp h] per component
    (the 2D 8x8 Q2 configuration uses amp = 0.15)."""
    rng = np.random.default_rng(seed)
    out = mesh.copy()
    h = mesh.h
    disp = rng.uniform(-amp * h, amp * h, size=mesh.ndof)
    out.x = mesh.x + np.where(mesh.fixed != 0, 0.0, disp)
    return out


def perturb_smooth(mesh: StructuredMesh, seed: int = BASE_SEED, amp_smooth: float = 0.1,
                   amp_noise: float = 0.05) -> StructuredMesh:
    """Interior nodes displaced by amp_smooth h sin(2 pi k_a . x + phi_a) plus
    U[-amp_noise h, amp_noise h] per component a, with k_a in {1,2,3}^d and
    phi_a in [0, 2 pi) drawn per component; x is the unperturbed node."""
    rng = np.random.default_rng(seed)
    d, Nx, h = mesh.dim, mesh.num_nodes, mesh.h
    X = mesh.x.reshape(d, Nx)
    disp = np.empty((d, Nx))
    for a in range(d):
        k = rng.integers(1, 4, size=d)
        phi = rng.uniform(0.0, 2.0 * np.pi)
        disp[a] = amp_smooth * h * np.sin(2.0 * np.pi * (k @ X) + phi)
    disp += rng.uniform(-amp_noise * h, amp_noise * h, size=(d, Nx))
    out = mesh.copy()
    out.x = mesh.x + np.where(mesh.fixed != 0, 0.0, disp.reshape(-1))
    return out


def rigid_map(mesh: StructuredMesh, R: np.ndarray, scale: float, shift=None) -> np.ndarray:
    """Positions scale * R x + shift (for invariance tests)."""
    d, Nx = mesh.dim, mesh.num_nodes
    X = mesh.x.reshape(d, Nx)
    Y = scale * (R @ X)
    if shift is not None:
        Y = Y + np.asarray(shift).reshape(d, 1)
    return Y.reshape(-1).copy()


def random_rotation(dim: int, seed: int) -> np.ndarray:
    """A random proper rotation (QR of a Gaussian matrix, det +1)."""
    rng = np.random.default_rng(seed)
    Q, R = np.linalg.qr(rng.standard_normal((dim, dim)))
    Q = Q @ np.diag(np.sign(np.diag(R)))
    if np.linalg.det(Q) < 0:
        Q[:, 0] = -Q[:, 0]
    return Q


# ------------------------------------------------------------------ named configurations
def config_mesh(cfg: int, seed: int | None = None, n_e: int | None = None, order: int | None = None):
    """The seeded benchmark meshes.

    1: 2D 8x8 Q2, uniform +-0.15h interior perturbation (metric 2).
    2: 3D 24^3 Q2, smooth + noise perturbation (metric 302).
    3: 3D 48^3 Q3, smooth + noise perturbation (metric 303).
    ``n_e`` / ``order`` override the size for scaled-down cases of the same family.
    """
    s = BASE_SEED + cfg if seed is None else seed
    if cfg == 1:
        m = structured(2, order or 2, n_e or 8)
        return perturb_uniform(m, 0.15, s)
    if cfg == 2:
        return perturb_smooth(structured(3, order or 2, n_e or 24), s)
    if cfg == 3:
        return perturb_smooth(structured(3, order or 3, n_e or 48), s)
    raise ValueError(cfg)


CONFIG_METRIC = {1: 2, 2: 302, 3: 303}


# ------------------------------------------------------------------ many-mesh workloads
def batched_workload(n_meshes: int = 512, seed: int = BASE_SEED + 4, n_range=(4, 20),
                     orders=(1, 2, 3, 4), amp=0.05):
    """Independent 3D hex meshes of uneven size: elements per side uniform in
    n_range (inclusive), order uniform in ``orders``; seeded smooth + noise
    perturbation (amplitude ``amp`` h, noise amp/2 h).  Returns a list of
    (mesh, h0) with h0 = 1/n_e the size-target scale."""
    rng = np.random.default_rng(seed)
    out = []
    for j in range(n_meshes):
        n = int(rng.integers(n_range[0], n_range[1] + 1))
        p = int(rng.choice(orders))
        m = perturb_smooth(structured(3, p, n), seed=seed * 1000 + j, amp_smooth=amp,
                           amp_noise=amp / 2)
        out.append((m, 1.0 / n))
    return out


def serving_workload(n_jobs: int = 2000, rate: float = 100.0, seed: int = BASE_SEED + 5,
                     n2=(8, 128), n3=(4, 40), orders=(1, 2, 3, 4), amp=0.05):
    """A Poisson stream of mesh-optimisation requests: exponential
    inter-arrival times at ``rate`` per second; each request is a 2D quad mesh
    (elements per side uniform in n2, metric mu_2) or a 3D hex mesh (n3,
    mu_302), order uniform in ``orders``, seeded perturbation.  Returns a list
    of dicts {id, arrival, dim, order, metric, n, seed}; the mesh is built by
    ``serving_mesh`` so the list itself stays small."""
    rng = np.random.default_rng(seed)
    t = 0.0
    jobs = []
    for j in range(n_jobs):
        t += float(rng.exponential(1.0 / rate))
        d = int(rng.choice([2, 3]))
        lo, hi = (n2 if d == 2 else n3)
        jobs.append({"id": j, "arrival": t, "dim": d, "order": int(rng.choice(orders)),
                     "metric": 2 if d == 2 else 302, "n": int(rng.integers(lo, hi + 1)),
                     "seed": seed * 10000 + j, "amp": amp})
    return jobs


def serving_mesh(job: dict) -> StructuredMesh:
    m = structured(job["dim"], job["order"], job["n"])
    return perturb_smooth(m, seed=job["seed"], amp_smooth=job["amp"], amp_noise=job["amp"] / 2)


# ------------------------------------------------------------------ Kershaw benchmark mesh
def _kershaw_right(eps, t):
    """1D map of the right end: slope (2 - eps) up to 1/2, slope eps after."""
    return np.where(t <= 0.5, (2.0 - eps) * t, 1.0 + eps * (t - 1.0))


def _kershaw_left(eps, t):
    return 1.0 - _kershaw_right(eps, 1.0 - t)


def _kershaw_blend(a, b, s):
    """a -> b with the quintic smoothstep 10s^3 - 15s^4 + 6s^5, s clamped to [0,1]."""
    s = np.clip(s, 0.0, 1.0)
    w = s * s * s * (10.0 + s * (6.0 * s - 15.0))
    return a + (b - a) * w


def kershaw_map(X, eps_y, eps_z):
    """The Kershaw deformation of [0,1]^3 (paper Sec. 4.1 and its appendix):
    x is kept; the unit x-range is cut into 6 layers; in the first layer y, z
    follow the left-end 1D map, in the last the right-end map, and the middle
    layers blend between them with a quintic smoothstep (layers 1 and 4 go
    left -> right, layers 2-3 go right -> left over two layers).  X has shape
    (3, n); returns the deformed points."""
    x, y, z = X
    layer = np.minimum(np.floor(6.0 * x), 6).astype(int)
    lam = 6.0 * x - layer
    out = np.empty_like(X)
    out[0] = x
    for k, (t, eps) in enumerate(((y, eps_y), (z, eps_z)), start=1):
        L, R = _kershaw_left(eps, t), _kershaw_right(eps, t)
        v = np.where(layer == 0, L, R)                       # layers 0 and >= 5
        v = np.where((layer == 1) | (layer == 4), _kershaw_blend(L, R, lam), v)
        v = np.where(layer == 2, _kershaw_blend(R, L, lam / 2.0), v)
        v = np.where(layer == 3, _kershaw_blend(R, L, (1.0 + lam) / 2.0), v)
        out[k] = v
    return out


def kershaw(order: int, n=(24, 24, 24), eps_y: float = 0.3, eps_z: float = 0.3) -> StructuredMesh:
    """Kershaw mesh: a uniform Q_order mesh of [0,1]^3 (n_x divisible by 6,
    n_y, n_z even) with every node moved by ``kershaw_map``.  Boundary nodes
    keep only their normal component fixed, so they can slide within their
    faces toward the uniform optimum the paper states."""
    if n[0] % 6 or n[1] % 2 or n[2] % 2:
        raise ValueError("n_x must be a multiple of 6 and n_y, n_z even")
    m = structured(3, order, n)
    Nx = m.num_nodes
    X = m.x.reshape(3, Nx)
    m.x = kershaw_map(X, eps_y, eps_z).reshape(-1).copy()
    fixed = np.zeros((3, Nx), dtype=np.uint8)
    for a in range(3):
        fixed[a] = (np.abs(X[a]) < 1e-14) | (np.abs(X[a] - 1.0) < 1e-14)
    m.fixed = fixed.reshape(-1).copy()
    return m
