"""Element-partitioned Newton step of TMOP on several ranks.

The paper's operator decomposition (Sec. 3) writes every global operator as
P^T G^T B^T D B G P, with P the parallel map from the vector of unique DOFs
to the ranks' local DOFs.  Here each rank owns a contiguous range of
elements (a slab of a structured mesh) and the DOFs of the nodes those
elements touch; a node on the interface of several ranks has a copy on each.
Everything element-local (energy, gradient, partial-assembly setup, Hessian
action, diagonal) runs on the rank's own sub-mesh; the only exchange is

* one interface sum per assembled vector (gradient, action, diagonal): each
  rank adds its neighbours' partial values at the shared nodes, so every copy
  holds the full assembled value (P^T then P);
* an allreduce of 2 to 4 scalars per MINRES iteration and per line-search
  trial (dot products over the nodes a rank owns, the energy, min det A).

The Newton step, its Jacobi-preconditioned MINRES and the backtracking line
search (Sec. 2.3) are those of ``tmop_newton_step``: the same MINRES
recurrences (Paige & Saunders) and stop test, the same line-search order,
so a split mesh reproduces the single-rank step up to the summation order of
the interface sums and dot products.  The vector work runs in the library's
kernels (``tmop_vec_*``) through a local-operator backend; the
communication is a ``Comm``: ``TorchComm`` over ``torch.distributed`` (NCCL
on GPUs, gloo on CPUs) or ``ThreadComm`` for ranks that are threads of one
process.  Identity and size targets are supported (the discrete target's
remap would need a distributed mass solve).
"""
from __future__ import annotations

import math
import threading
from dataclasses import dataclass, field

import numpy as np

OK, ERR_INVERTED, ERR_MINRES, ERR_LINESEARCH = 0, 2, 5, 6


# ---------------------------------------------------------------- partition
@dataclass
class Partition:
    """One rank's share of a mesh: its elements, their local map, the global
    id of each local node, the nodes it owns (lowest rank touching a node),
    and per neighbour rank the local indices of the shared nodes, in
    increasing global node id (the same order on both sides)."""
    rank: int
    world: int
    dim: int
    elems: np.ndarray              # global element ids, increasing
    local_map: np.ndarray          # len(elems) x NP, local node ids
    nodes: np.ndarray              # global node id of each local node
    owned: np.ndarray              # uint8 per local node
    fixed: np.ndarray | None       # uint8 per local DOF (component-major), or None
    shared: dict = field(default_factory=dict)    # neighbour -> local node ids

    @property
    def num_nodes(self) -> int:
        return int(len(self.nodes))

    @property
    def ndof(self) -> int:
        return self.dim * self.num_nodes

    def owned_dofs(self) -> np.ndarray:
        return np.tile(self.owned, self.dim).astype(np.uint8)

    def to_local(self, xg: np.ndarray, num_nodes_global: int) -> np.ndarray:
        """Local DOF vector of a global component-major vector."""
        return np.concatenate([xg[a * num_nodes_global + self.nodes] for a in range(self.dim)])


def element_ranges(num_elems: int, world: int):
    """Contiguous element ranges [e0, e1) of the ranks (sizes differ by at most one)."""
    return [(r * num_elems // world, (r + 1) * num_elems // world) for r in range(world)]


def partition(emap: np.ndarray, num_nodes: int, dim: int, fixed, world: int, rank: int) -> Partition:
    """Partition of the elements into ``world`` contiguous ranges; every rank
    computes the same node ownership from the global map."""
    emap = np.asarray(emap)
    E = emap.shape[0]
    ranges = element_ranges(E, world)
    touch = [np.unique(emap[a:b].reshape(-1)) for a, b in ranges]
    owner = np.full(num_nodes, world, dtype=np.int64)
    for r in range(world - 1, -1, -1):
        owner[touch[r]] = r
    e0, e1 = ranges[rank]
    nodes = touch[rank]
    glob2loc = np.full(num_nodes, -1, dtype=np.int64)
    glob2loc[nodes] = np.arange(len(nodes))
    local_map = glob2loc[emap[e0:e1]].astype(np.int32)
    shared = {}
    for r in range(world):
        if r == rank:
            continue
        common = np.intersect1d(nodes, touch[r], assume_unique=True)
        if len(common):
            shared[r] = glob2loc[common].astype(np.int64)
    fx = None
    if fixed is not None:
        fixed = np.asarray(fixed, dtype=np.uint8)
        fx = np.concatenate([fixed[a * num_nodes + nodes] for a in range(dim)]).astype(np.uint8)
    return Partition(rank, world, dim, np.arange(e0, e1), local_map, nodes,
                     (owner[nodes] == rank).astype(np.uint8), fx, shared)


# ---------------------------------------------------------------- communicators
class TorchComm:
    """Allreduce and neighbour exchange over torch.distributed (the default
    process group unless ``group`` is given); tensors on the backend's device
    (CUDA for NCCL, CPU for gloo)."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self.dist, self.group = dist, group
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)

    def allreduce(self, vals, op: str, like):
        import torch
        t = torch.tensor(np.asarray(vals, dtype=np.float64), dtype=torch.float64, device=like.device)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.SUM if op == "sum" else self.dist.ReduceOp.MIN,
                             group=self.group)
        return t.cpu().numpy()

    def exchange(self, sends: dict):
        """{neighbour: tensor or array} -> {neighbour: the same type and shape}."""
        import torch
        host = {r: not isinstance(t, torch.Tensor) for r, t in sends.items()}
        ts = {r: (torch.from_numpy(np.ascontiguousarray(t, dtype=np.float64)) if host[r]
                  else t.contiguous()) for r, t in sends.items()}
        recvs = {r: torch.empty_like(t) for r, t in ts.items()}
        reqs = []
        for r in sorted(ts):
            reqs.append(self.dist.isend(ts[r], r, group=self.group))
            reqs.append(self.dist.irecv(recvs[r], r, group=self.group))
        for q in reqs:
            q.wait()
        return {r: (recvs[r].numpy() if host[r] else recvs[r]) for r in recvs}


class ThreadComm:
    """Ranks that are threads of one process (e.g. several subdomains on one
    GPU): a shared board and a barrier.  Exchanged values pass through host
    memory; every wait is bounded (``timeout`` seconds, then an error)."""

    class _Shared:
        def __init__(self, world, timeout):
            self.world = world
            self.barrier = threading.Barrier(world, timeout=timeout)
            self.board = {}

    def __init__(self, shared, rank):
        self.s, self.rank, self.world = shared, rank, shared.world

    @classmethod
    def group(cls, world, timeout=60.0):
        sh = cls._Shared(world, timeout)
        return [cls(sh, r) for r in range(world)]

    def allreduce(self, vals, op: str, like=None):
        v = np.asarray(vals, dtype=np.float64)
        self.s.board[("ar", self.rank)] = v
        self.s.barrier.wait()
        parts = [self.s.board[("ar", r)] for r in range(self.world)]
        self.s.barrier.wait()
        out = np.sum(parts, axis=0) if op == "sum" else np.min(parts, axis=0)
        return out

    def exchange(self, sends: dict):
        import torch
        dev = None
        for r, t in sends.items():
            dev = t.device if hasattr(t, "device") else None
            self.s.board[("ex", self.rank, r)] = t.cpu().numpy() if hasattr(t, "cpu") else np.asarray(t)
        self.s.barrier.wait()
        recvs = {}
        for r in sends:
            a = self.s.board[("ex", r, self.rank)]
            recvs[r] = torch.from_numpy(a.copy()).to(dev) if dev is not None else a.copy()
        self.s.barrier.wait()
        return recvs


# ---------------------------------------------------------------- local operator on the GPU
class LibraryBackend:
    """The rank's sub-mesh on its GPU: a ``TmopMesh`` context for the element
    work and the library's vector kernels for everything else.  Local vectors
    are float64 CUDA tensors of length dim * (local nodes).  With a ``stream``,
    run the rank's steps under ``torch.cuda.stream(stream)`` so that the
    tensors it allocates are ordered with the library's launches."""

    def __init__(self, part: Partition, order: int, metric: int, nq1d=None, target=0, target_h0=1.0,
                 device="cuda", stream=None):
        import torch
        from . import capi
        from .mesh_opt import TmopMesh
        self.capi, self.torch = capi, torch
        self.part = part
        self.dev = torch.device(device)
        self.stream = stream
        self.gm = TmopMesh(part.dim, order, part.local_map, part.num_nodes, metric, fixed=part.fixed,
                           nq1d=nq1d, target=target, target_h0=target_h0, precision="fp64",
                           device=device, stream=stream)
        self.ctx = self.gm.ctx
        self.n = part.ndof
        self.owned = torch.from_numpy(part.owned_dofs()).to(self.dev)
        Nl = part.num_nodes
        self.halo = {r: torch.from_numpy(np.concatenate([a * Nl + ids for a in range(part.dim)])
                                         .astype(np.int32)).to(self.dev)
                     for r, ids in part.shared.items()}

    # vectors
    def empty(self):
        return self.torch.empty(self.n, dtype=self.torch.float64, device=self.dev)

    def zeros(self):
        return self.torch.zeros(self.n, dtype=self.torch.float64, device=self.dev)

    def from_host(self, a):
        return self.torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(self.dev)

    def to_host(self, v):
        return v.cpu().numpy()

    def lincomb(self, out, a, x, b=0.0, y=None, c=0.0, z=None):
        self.capi.tmop_vec_lincomb(self.ctx, out, a, x, b, y, c, z)
        return out

    def mul(self, out, x, y):
        self.capi.tmop_vec_mul(self.ctx, out, x, y)
        return out

    def dot_owned(self, x, y):
        return self.capi.tmop_vec_dot(self.ctx, x, y, self.owned)

    def jacobi(self, diag):
        """M^-1 = 1/|diag| (1 where |diag| < 1e-300), the library's rule."""
        minv = self.empty()
        self.capi.tmop_vec_jacobi(self.ctx, diag, minv)
        return minv

    # halo
    def pack(self, v, r):
        out = self.torch.empty(self.halo[r].numel(), dtype=self.torch.float64, device=self.dev)
        self.capi.tmop_vec_gather(self.ctx, self.halo[r], v, out)
        return out

    def unpack_add(self, v, r, vals):
        self.capi.tmop_vec_scatter_add(self.ctx, self.halo[r], vals, v)

    def sync(self):
        if self.stream is not None:
            self.stream.synchronize()
        else:
            self.torch.cuda.synchronize(self.dev)

    # element work
    def energy(self, x):
        st, F, md = self.gm.energy(x)
        return F, md

    def gradient(self, x, g):
        self.gm.gradient(x, out=g)
        return g

    def hessian_setup(self, x):
        self.gm.hessian_setup(x)

    def hessian_apply(self, v, y):
        self.gm.hessian_apply(v, out=y)
        return y

    def hessian_diag(self, d):
        self.gm.hessian_diag(out=d)
        return d

    def close(self):
        self.gm.close()


# ---------------------------------------------------------------- the distributed step
class DistNewton:
    """Newton steps of one rank of an element-partitioned mesh."""

    def __init__(self, backend, comm):
        self.b, self.comm = backend, comm

    def interface_sum(self, v):
        """Add the neighbours' partial values at the shared nodes (P P^T)."""
        b = self.b
        if not getattr(b.part, "shared", None):
            return v
        sends = {r: b.pack(v, r) for r in sorted(b.part.shared)}
        b.sync()
        recvs = self.comm.exchange(sends)
        for r in sorted(recvs):
            b.unpack_add(v, r, recvs[r])
        return v

    def allsum(self, *vals):
        return self.comm.allreduce(list(vals), "sum", like=self._like())

    def allmin(self, *vals):
        return self.comm.allreduce(list(vals), "min", like=self._like())

    def _like(self):
        return self.b.zeros()[:1]

    def energy_grad(self, x, g):
        F, md = self.b.energy(x)
        F = self.allsum(F if np.isfinite(F) else np.inf)[0]
        md = self.allmin(md)[0]
        self.b.gradient(x, g)
        self.interface_sum(g)
        gn = math.sqrt(max(self.allsum(self.b.dot_owned(g, g))[0], 0.0))
        return F, md, gn

    def apply(self, v, y):
        """Assembled Hessian action.  The Krylov vectors are zero on fixed DOFs
        (the right-hand side dF is), where the action is the identity, so
        those entries stay zero, as inside the library's MINRES."""
        self.b.hessian_apply(v, y)
        return self.interface_sum(y)

    def minres(self, rhs, minv, rtol, max_it, fixed_its):
        """Jacobi-preconditioned MINRES (Paige & Saunders 1975) from x0 = 0,
        the recurrences and stop test of the library's device MINRES."""
        b = self.b
        dx, w1, w2 = b.zeros(), b.zeros(), b.zeros()
        r1 = b.lincomb(b.empty(), 1.0, rhs)
        r2 = b.lincomb(b.empty(), 1.0, rhs)
        y = b.mul(b.empty(), minv, rhs)
        bb = self.allsum(b.dot_owned(rhs, y))[0]
        beta1 = math.sqrt(max(bb, 0.0))
        st = dict(beta1=beta1, beta=beta1, beta_old=0.0, alpha=0.0, dbar=0.0, eps=0.0, eps_old=0.0,
                  phibar=beta1, cs=-1.0, sn=0.0, gamma=1.0, delta=0.0, phi=0.0, iters=0, breakdown=0)
        stop = max_it + 1 if beta1 > 0.0 else 0
        v = b.zeros()
        if stop >= 1:
            b.lincomb(v, 1.0 / beta1, y)
        z = b.empty()
        for k in range(1, max_it + 1):
            if stop < k:
                break
            self.apply(v, z)
            c = st["beta"] / st["beta_old"] if k >= 2 else 0.0
            b.lincomb(z, 1.0, z, -c, r1)                      # y = z - (beta/beta_old) r1
            st["alpha"] = self.allsum(b.dot_owned(v, z))[0]
            b.lincomb(z, 1.0, z, -st["alpha"] / st["beta"], r2)
            ynew = b.mul(b.empty(), minv, z)
            bb = self.allsum(b.dot_owned(z, ynew))[0]
            st["iters"] = k
            if not (bb >= 0.0):                               # breakdown
                st["breakdown"] = 1
                stop = k - 1
                break
            st["beta_old"] = st["beta"]
            beta = math.sqrt(bb)
            st["beta"] = beta
            alpha = st["alpha"]
            st["eps_old"] = st["eps"]
            delta = st["cs"] * st["dbar"] + st["sn"] * alpha
            gbar = st["sn"] * st["dbar"] - st["cs"] * alpha
            st["eps"] = st["sn"] * beta
            st["dbar"] = -st["cs"] * beta
            gamma = max(math.sqrt(gbar * gbar + beta * beta), 1e-300)
            st["gamma"], st["delta"] = gamma, delta
            st["cs"], st["sn"] = gbar / gamma, beta / gamma
            st["phi"] = st["cs"] * st["phibar"]
            st["phibar"] = st["sn"] * st["phibar"]
            if (not fixed_its and st["phibar"] <= rtol * st["beta1"]) or beta == 0.0:
                stop = k
            # w_new = (v - eps_old w1 - delta w2) / gamma; dx += phi w_new; v = ynew / beta
            wn = b.lincomb(b.empty(), 1.0 / gamma, v, -st["eps_old"] / gamma, w1, -delta / gamma, w2)
            b.lincomb(dx, 1.0, dx, st["phi"], wn)
            b.lincomb(v, (1.0 / beta) if beta > 0.0 else 0.0, ynew)
            r1, r2, z = r2, z, r1
            w1, w2 = w2, wn
        resid = st["phibar"] / st["beta1"] if st["beta1"] > 0.0 else 0.0
        return dx, st["iters"], resid, st["breakdown"]

    def newton_step(self, x, minres_rtol=1e-8, minres_max_it=50, minres_fixed_its=False,
                    ls_factor=1.2, ls_max_halvings=20):
        """One Newton step in place on the rank's local positions x (Sec. 2.3).
        Returns the report of tmop_newton_step (the same keys)."""
        b = self.b
        rep = dict(energy=0.0, grad_norm=0.0, energy_new=0.0, grad_norm_new=0.0, alpha=0.0,
                   min_det=0.0, minres_resid=0.0, minres_iters=0, halvings=0, status=OK)
        g = b.empty()
        F0, md0, g0 = self.energy_grad(x, g)
        rep.update(energy=F0, min_det=md0, grad_norm=g0)
        if not (md0 > 0.0):
            rep.update(energy=math.inf, status=ERR_INVERTED)
            return rep
        if g0 == 0.0:
            rep.update(energy_new=F0, grad_norm_new=0.0)
            return rep
        b.hessian_setup(x)
        diag = b.hessian_diag(b.empty())
        # (a fixed DOF shared by k ranks sums to k: M^-1 meets only zeros there)
        self.interface_sum(diag)
        minv = b.jacobi(diag)
        dx, its, res, brk = self.minres(g, minv, minres_rtol, minres_max_it, minres_fixed_its)
        rep.update(minres_iters=its, minres_resid=res)
        if brk:
            rep["status"] = ERR_MINRES
            return rep
        alpha = 1.0
        xt, g1v = b.empty(), b.empty()
        for h in range(ls_max_halvings + 1):
            b.lincomb(xt, 1.0, x, -alpha, dx)
            F1, md1, g1 = self.energy_grad(xt, g1v)
            if md1 > 0.0 and F1 < ls_factor * F0 and g1 < ls_factor * g0:
                x.copy_(xt) if hasattr(x, "copy_") else np.copyto(x, xt)
                rep.update(alpha=alpha, halvings=h, energy_new=F1, grad_norm_new=g1, min_det=md1)
                return rep
            alpha *= 0.5
        rep["status"] = ERR_LINESEARCH
        return rep
