"""Benchmark of the TMOP partially assembled Newton step on B300.

Workload (default): 3D hex mesh 48^3 elements, order p = 3, 4^3 Gauss points
per element (3,048,625 nodes, 9,145,875 DOFs), seeded smooth + noise
perturbation, metric mu_303, identity targets, fixed boundary.  One "step"
is one pass of the whole hot path: energy + min det, gradient, partial
assembly of d2mu/dT2, Hessian diagonal, exactly 20 Jacobi-MINRES iterations
(one Hessian action each, the paper's throughput methodology of Sec. 4.1) and
the backtracking line search, starting every step from the same initial
positions.

value = DOF x (Hessian actions per step) / step time, in GDOF/s; the
roofline object reports the Hessian-action kernel alone (CUDA events on the
library's stream).  Inputs (2.5 GB of stored Hessian data) are larger than
the 126 MB L2, so no flush is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp64|fp32]
    python bench.py --impl reference ...     (the FP64 CPU oracle, bounded sample)
Under torchrun every rank runs its own replica (weak scaling, no collective
on the data path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Hessian-apply GDOF/s & %HBM peak (3D hex p=2..4); time-to-converged-mesh, p50/p99"
UNIT = "GDOF/s"
FP64_PEAK_TFLOPS = 1.25      # nominal B300 FP64 rate (profiling recipe table)
MINRES_ITS = 20
# ncu dram__bytes_read.sum + dram__bytes_write.sum of one action launch, captured on the
# 24^3 Q3 case and scaled by elements (x8) to a 48^3 launch; None when the kernel changed
# since the capture.
TRAFFIC_BYTES = {("fp64", 13): 2.692e9, ("fp32", 17): 1.367e9}     # (precision, action variant)
PRECISION_LABEL = {"fp64": "fp64-class (double-float contractions, 48-bit significand)",
                   "fp32": "fp32-mixed (fp32 stored d2mu/dT2, action and MINRES; fp64 residual, "
                           "energy, det and line search)",
                   "fp64-native": "fp64 (every contraction on the FP64 units)"}
APPLY_VARIANT_NAME = {0: "sum-factorised register column", 1: "collocated, register column, 4 warps/CTA",
                      2: "collocated, register column, 2 warps/CTA",
                      3: "collocated, shared-memory column, 4 warps/CTA",
                      4: "collocated, shared-memory column, 2 warps/CTA",
                      5: "collocated, shared-memory column, 8 warps/CTA",
                      6: "collocated, shared-memory column unrolled, 4 warps/CTA",
                      7: "collocated, shared-memory column, 8 warps/CTA, L2 prefetch of the next point",
                      8: "collocated, shared-memory column, 4 warps/CTA, L2 prefetch of the next point",
                      9: "collocated, shared-memory column, 8 warps/CTA, L2 prefetch, chunked register pipeline",
                      10: "collocated, shared-memory column, 4 warps/CTA, chunked register pipeline",
                      11: "collocated, per-warp shared-memory column with aliased buffers, 4 warps/CTA, 20 (FP32 32) warps/SM",
                      12: "collocated, per-warp shared-memory column with aliased buffers, 4 warps/CTA, 24 warps/SM",
                      13: "collocated, per-warp shared-memory column with aliased buffers, 8 warps/CTA, 24 warps/SM, L2 prefetch",
                      14: "collocated, per-warp shared-memory column with aliased buffers, 4 warps/CTA, 20 (FP32 32) warps/SM, L2 prefetch",
                      15: "collocated, per-warp shared-memory column with aliased buffers, 4 warps/CTA, 24 warps/SM, L2 prefetch",
                      16: "collocated, per-warp shared-memory column with aliased buffers, 8 warps/CTA, 24 warps/SM",
                      17: "collocated, per-warp shared-memory column with aliased buffers, 4 warps/CTA, 24 warps/SM, input gathered up front",
                      18: "collocated, per-warp shared-memory column with aliased buffers, 4 warps/CTA, 20 (FP32 32) warps/SM, input gathered up front"}


def flops_apply_per_elem(d, ni, nq, ns, collocated=False):
    """Algorithmic flops of one element of the Hessian action: forward and
    transposed contractions (2 flops per multiply-add) plus the pointwise
    H:dA with the full d^2 x d^2 matrix.  Sum-factorised with B and G
    (the count of the method's statement), or, for the collocated kernels,
    three B contractions to the points and the collocated derivative along
    each direction."""
    if d == 3 and collocated:
        fwd = nq * ni ** 3 + nq ** 2 * ni ** 2 + nq ** 3 * ni + 3 * nq ** 4
        return 2 * (2 * d * fwd) + 2 * (d * d) ** 2 * nq ** 3
    if d == 3:
        fwd = 2 * nq * ni ** 3 + 3 * nq ** 2 * ni ** 2 + 3 * nq ** 3 * ni
        return 2 * (2 * d * fwd) + 2 * (d * d) ** 2 * nq ** 3
    fwd = 2 * nq * ni ** 2 + 2 * nq ** 2 * ni
    return 2 * (2 * d * fwd) + 2 * (d * d) ** 2 * nq ** 2


def bytes_apply(E, ndof, d, ni, nq, ns, rsz):
    """Algorithmic bytes of one Hessian action: the stored quadrature data (ns
    values per point) and the element map of every element, plus the input v
    read and the result y written once per unique DOF (rsz bytes a value)."""
    return E * (ns * nq ** d * rsz + ni ** d * 4) + 2 * ndof * rsz


class Clocks:
    """nvidia-smi sampler over the timed region."""

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile(prefix="clk", suffix=".csv", delete=False)
        self.p = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.p:
            self.p.terminate()
            self.p.wait()
        self.f.close()

    def summary(self):
        rows = []
        try:
            for ln in open(self.f.name):
                parts = [s.strip() for s in ln.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        finally:
            os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for n, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": float(rows[0][2]) if rows[0][2].replace(".", "").isdigit() else None,
                "reasons": sorted(reasons), "samples": len(rows)}


def max_over_ranks(value: float, world: int, device=None) -> float:
    """The slowest rank's time (the contract's max over ranks)."""
    if world <= 1:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def shard(n_units: int, rank: int, world: int):
    """Units (meshes, replicas) of this rank: round robin, no data exchange."""
    return list(range(rank, n_units, world))


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def workload(args):
    from paper_2205_12721_b300 import meshgen
    m = meshgen.config_mesh(3, n_e=args.n_e, order=args.order)
    return m


def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch
    from paper_2205_12721_b300 import capi
    from paper_2205_12721_b300.mesh_opt import TmopMesh

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    m = workload(args)
    d, p, nq = m.dim, m.order, m.order + 1
    ni = p + 1
    ns = (d * d) * (d * d + 1) // 2
    stream = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(stream):
        gm = TmopMesh.from_structured(m, capi.METRIC_303, precision=args.precision,
                                      stream=stream)
        x0 = torch.from_numpy(m.x).to(dev)
        x = x0.clone()
    opts = dict(minres_rtol=0.0, minres_max_it=MINRES_ITS, minres_fixed_its=True)

    def step():
        x.copy_(x0)
        r = gm.newton_step(x, **opts)
        if r["status"] != capi.OK:
            raise RuntimeError(f"newton step failed: {r}")
        return r

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
    stream.synchronize()
    if world > 1:
        torch.distributed.barrier()
    capi.tmop_profile_enable(gm.ctx, True)
    launches0 = capi.tmop_launch_count()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with Clocks(local_rank) as clk:
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            ev0.record(stream)
            reps = [step() for _ in range(args.steps)]
            ev1.record(stream)
        torch.cuda.synchronize()
    launches = capi.tmop_launch_count() - launches0
    ms = ev0.elapsed_time(ev1) / args.steps
    apply_ms, apply_n = capi.tmop_profile_read(gm.ctx, capi.K_APPLY)
    prof = {name: capi.tmop_profile_read(gm.ctx, k) for name, k in
            [("energy", capi.K_ENERGY), ("gradient", capi.K_GRADIENT), ("hsetup", capi.K_HSETUP),
             ("apply", capi.K_APPLY), ("diag", capi.K_DIAG), ("assemble", capi.K_ASSEMBLE)]}
    capi.tmop_profile_enable(gm.ctx, False)
    ms = max_over_ranks(ms, world, dev)
    applies = MINRES_ITS
    value = world * m.ndof * applies / (ms * 1e-3) / 1e9

    # end to end through the C ABI with host buffers (pinned), copies included
    xh = torch.from_numpy(m.x).pin_memory()
    xout = torch.empty_like(xh).pin_memory()
    with torch.cuda.stream(stream):
        for _ in range(2):
            x.copy_(xh, non_blocking=True)
            gm.newton_step(x, **opts)
            xout.copy_(x, non_blocking=True)
        stream.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            x.copy_(xh, non_blocking=True)
            r = gm.newton_step(x, **opts)
            xout.copy_(x, non_blocking=True)
        stream.synchronize()
        e2e_s = (time.perf_counter() - t0) / args.steps
    e2e_s = max_over_ranks(e2e_s, world, dev)
    e2e = {"value": world * m.ndof * applies / e2e_s / 1e9, "unit": UNIT,
           "h2d_bytes_per_step": int(xh.numel() * 8), "d2h_bytes_per_step": int(xout.numel() * 8)}

    # roofline of the Hessian-action kernel
    rsz = 4 if args.precision == "fp32" else 8
    E = m.num_elems
    apply_avg_ms = apply_ms / max(apply_n, 1)
    byts = bytes_apply(E, m.ndof, d, ni, nq, ns, rsz)
    var = capi.tmop_get_apply_variant(d, p, nq, {"fp64": capi.FP64, "fp32": capi.FP32,
                                                 "fp64-native": capi.FP64_NATIVE}[args.precision])
    flops = flops_apply_per_elem(d, ni, nq, ns, collocated=var > 0) * E
    traffic = args.traffic
    if traffic is None and args.n_e == 48 and p == 3 and nq == 4:
        traffic = TRAFFIC_BYTES.get((args.precision, var))
    rc_name = {"fp64": "double,df", "fp32": "float,float", "fp64-native": "double,double"}[args.precision]
    kname = (f"k_apply3c<Cfg<{d},{p},{nq}>,{rc_name},...> variant {var} ({APPLY_VARIANT_NAME[var]})"
             if var > 0 else f"k_apply3<Cfg<{d},{p},{nq}>,{rc_name}> variant 0")
    peaks = measured_peaks()
    hbm = peaks.get("hbm_gbs")
    gbs = byts / (apply_avg_ms * 1e-3) / 1e9
    if args.precision == "fp64-native":
        ach = flops / (apply_avg_ms * 1e-3) / 1e12
        roof = {"bound": "alu", "achieved": ach, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": ach / FP64_PEAK_TFLOPS, "traffic": traffic,
                "peak_source": "nominal FP64 rate of the profiling recipe",
                "kernel": kname, "flops_per_launch": flops,
                "hbm_view": {"achieved_gbs": gbs, "peak_gbs": hbm,
                             "frac": (gbs / hbm) if hbm else None, "bytes_per_launch": byts}}
    else:
        roof = {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s",
                "frac": (gbs / hbm) if hbm else None, "traffic": traffic,
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)",
                "kernel": kname,
                "bytes_per_launch": byts,
                "flops_view": {"fp64_equiv_tflops": flops / (apply_avg_ms * 1e-3) / 1e12}}
    roof["avg_launch_ms"] = apply_avg_ms
    roof["launches"] = apply_n
    roof["apply_gdofs"] = m.ndof / (apply_avg_ms * 1e-3) / 1e9
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {"fp64": "f64 (double-float contractions)", "fp64-native": "f64",
                  "fp32": "f32 (H, MINRES) / f64"}[args.precision],
        "data": "synthetic seeded perturbed Cartesian mesh (no dataset)",
        "config": {"workload": f"3D hex {m.n[0]}^3 Q{p}, {nq}^3 Gauss pts, mu_303, identity target, "
                               f"1 Newton step = energy+grad+PA setup+diag+{MINRES_ITS} MINRES+line search",
                   "dofs": m.ndof, "elements": E, "precision": PRECISION_LABEL[args.precision],
                   "hessian_applies_per_step": applies,
                   "l2": "inputs larger than L2 (stored d2mu/dT2 "
                         f"{ns * nq ** d * E * rsz / 1e9:.2f} GB), no flush",
                   "parallelism": f"replicas x{world} (one mesh per GPU, no collective)"},
        "roofline": roof,
        "e2e": e2e,
        "gpu_launches": launches,
        "kernel_ms": {k: {"total_ms": v[0], "launches": v[1]} for k, v in prof.items()},
        "newton": {"alpha": reps[-1]["alpha"], "minres_iters": reps[-1]["minres_iters"],
                   "energy": reps[-1]["energy"], "energy_new": reps[-1]["energy_new"]},
        "clocks": clk.summary(),
    }
    gm.close()
    if args.variants and rank == 0:
        # the same step in the other precision modes (reported beside the value)
        out["variants"] = {}
        for prec in args.variants:
            if prec == args.precision:
                continue
            sub = argparse.Namespace(**vars(args))
            sub.precision, sub.variants, sub.no_cpu_baseline = prec, [], True
            sub.traffic = None
            v = run_ours(sub, 0, 1, local_rank)
            out["variants"][prec] = {"value": v["value"], "ms_per_step": v["ms_per_step"],
                                     "dtype": v["dtype"], "roofline": v["roofline"],
                                     "kernel_ms": v["kernel_ms"]}
    if rank == 0 and not args.no_ttc and not args.no_cpu_baseline:
        out["time_to_converged"] = time_to_converged(args)
        out["serving_sample"] = serving_sample(args)
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args)
    return out


def _oracle_step(n_s, order, seed):
    """One oracle Newton step (exactly 20 MINRES iterations) on an n_s^3 mesh
    of the benchmark family: (DOFs, seconds, status).  Runs in a worker."""
    import oracle as O
    from paper_2205_12721_b300 import meshgen
    m = meshgen.config_mesh(3, n_e=n_s, order=order, seed=seed)
    om = O.Mesh(3, m.order, m.order + 1, m.map, m.num_nodes, 303, m.fixed)
    x = m.x.copy()
    t0 = time.perf_counter()
    r = O.newton_step(om, x, 0.0, MINRES_ITS, True)
    return m.ndof, time.perf_counter() - t0, r["status"]


def _cpu_model():
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ln.startswith("model name"):
                    return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def cpu_baseline(args, seconds=None):
    """The FP64 oracle as it stands, one Newton step with exactly 20 MINRES
    iterations on a bounded sample of the workload: the same mesh family at
    8^3 elements (1/216 of the 48^3 elements).  Timed single-threaded, and on
    all host cores as one independent oracle process per core, each on the
    same sample (the oracle is single-threaded; the cores share no work);
    value = the all-core throughput.""" 
    import multiprocessing as mp
    n_s, order = args.cpu_sample_n, args.order
    ndof, dt1, st = _oracle_step(n_s, order, None)
    cores = os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        pool.starmap(_oracle_step, [(2, order, 1)] * cores)          # start-up, imports
        t0 = time.perf_counter()
        res = pool.starmap(_oracle_step, [(n_s, order, None)] * cores)
        wall = time.perf_counter() - t0
    tot = sum(r[0] for r in res) * MINRES_ITS
    return {"value": tot / wall / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle",
            "cpu_model": _cpu_model(), "nproc": cores,
            "single_thread": {"value": ndof * MINRES_ITS / dt1 / 1e9, "cores": 1, "seconds": dt1},
            "sample": f"one oracle Newton step (20 MINRES) per core on the {n_s}^3 Q{order} mesh of the "
                      f"same family ({ndof} DOFs), {cores} independent processes, {wall:.2f} s "
                      f"wall; single thread {dt1:.2f} s",
            "status": max([st] + [r[2] for r in res])}


def serving_sample(args, n_jobs=100, rate=50.0):
    """A bounded sample of the serving configuration: the first ``n_jobs``
    requests of the Poisson stream (2D n_e U{8..128} mu_2 / 3D n_e U{4..40}
    mu_302, p U{1..4}, gradient-norm rtol 1e-6) at ``rate`` requests/s,
    continuous batching under a 64 GB budget; p50/p99 from arrival to
    converged mesh and meshes/s."""
    import torch
    from paper_2205_12721_b300 import meshgen
    from paper_2205_12721_b300.serve import Server, summarize
    jobs = meshgen.serving_workload(n_jobs, rate=rate, n2=tuple(args.n2), n3=tuple(args.n3))
    srv = Server(int(args.budget_gb * (1 << 30)), precision="fp64", newton_rtol=1e-6,
                 newton_max_it=50, minres_max_it=50)
    done = srv.run(jobs)
    srv.close()
    torch.cuda.synchronize()
    s = summarize(done)
    s.update({"requests": n_jobs, "rate_per_s": rate, "precision": "fp64-class"})
    return s


def time_to_converged(args, reps=5):
    """Time to converged mesh of the 3D 24^3 Q2 mu_302 configuration (smooth +
    noise perturbation, |dF|/|dF0| <= 1e-10, MINRES rtol 1e-8 / cap 50),
    FP64 class vs FP32 mixed: p50 / p99 over repeated solves from the same
    initial mesh, Newton and MINRES counts, and the final-energy difference."""
    import torch
    from paper_2205_12721_b300 import capi, meshgen
    from paper_2205_12721_b300.mesh_opt import TmopMesh
    m = meshgen.config_mesh(2)
    out = {"workload": "3D hex 24^3 Q2, 3^3 Gauss pts, mu_302, identity target, until "
                       "|dF|/|dF0| <= 1e-10", "dofs": m.ndof, "unit": "s"}
    finals = {}
    for prec in ("fp64", "fp32"):
        times = []
        for rep in range(reps + 1):                       # the first solve warms up
            gm = TmopMesh.from_structured(m, capi.METRIC_302, precision=prec)
            x = torch.from_numpy(m.x).cuda()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            reps_ = gm.solve(x, max_newton=100, rtol=1e-10)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            st, F, _ = gm.energy(x)
            S = float(m.num_elems)                        # sum_q |c_q| for W = I on [0,1]^3
            gm.close()
            if rep:
                times.append(dt)
        finals[prec] = F
        ts = sorted(times)
        out[prec] = {"p50_s": statistics.median(ts), "p99_s": ts[-1], "runs": len(ts),
                     "newton_its": len(reps_), "minres_its": sum(r["minres_iters"] for r in reps_),
                     "status": reps_[-1]["status"], "energy_final": F}
    out["fp32_vs_fp64_final_energy_abs"] = abs(finals["fp32"] - finals["fp64"])
    out["final_energy_tol"] = 1e-8 * S
    return out


def run_reference(args, rank, world):
    if rank != 0:
        return None
    vals = []
    for _ in range(args.warmup):
        cpu_baseline(args)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        vals.append(cpu_baseline(args))
    wall = (time.perf_counter() - t0) / args.steps
    v = statistics.median(c["value"] for c in vals)
    cb = dict(vals[0])
    cb["value"] = v
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": wall * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic seeded perturbed Cartesian mesh (no dataset)",
            "config": {"workload": "3D hex 48^3 Q3, mu_303: each step is the FP64 CPU oracle's "
                                   f"Newton step on a {args.cpu_sample_n}^3 sample of the same family"},
            "cpu_baseline": cb,
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def run_batched(args):
    """512 independent 3D hex meshes (elements per side U{4..20}, order
    U{1..4}), metric mu_303 + mu_55 with the size target, grouped by order;
    time until every mesh has converged (|dF|/|dF0| <= 1e-10 or 40 steps).
    Batched FP32-mixed and FP64 forms, and the single-mesh FP64 path on a
    subset of the same meshes."""
    import torch
    from paper_2205_12721_b300 import capi, meshgen
    from paper_2205_12721_b300.batch import TmopBatch
    from paper_2205_12721_b300.mesh_opt import TmopMesh

    work = meshgen.batched_workload(args.n_meshes)
    out = {"metric": "time-to-converged-mesh (all meshes)", "unit": "s", "higher_is_better": False,
           "config": {"workload": f"{len(work)} 3D hex meshes, n_e U{{4..20}}, p U{{1..4}}, "
                                  "mu_303+mu_55, size target W = h0 s(x)^(1/3) I",
                      "elements": sum(m.num_elems for m, _ in work),
                      "dofs": sum(m.ndof for m, _ in work)}}

    def batched(prec, subset):
        """One batch per order, all batches stepped concurrently and
        independently (host thread and stream per batch); the clock starts
        once every mesh is resident."""
        from concurrent.futures import ThreadPoolExecutor
        groups = {}
        for j in subset:
            m, h0 = work[j]
            groups.setdefault(m.order, []).append(j)
        bs, slots = [], {}
        for p, js in sorted(groups.items()):
            b = TmopBatch(3, p, capi.METRIC_303_55, target=capi.TARGET_SIZE_FIELD, precision=prec,
                          max_meshes=len(js), minres_max_it=50, newton_rtol=1e-10, newton_max_it=40,
                          graphs=not args.no_graphs)
            for j in js:
                slots[j] = (b, b.add_structured(work[j][0], h0=work[j][1]))
            bs.append(b)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        # every order group steps on its own host thread and stream until all
        # of its meshes are done (no group waits for another between steps)
        with ThreadPoolExecutor(max_workers=len(bs)) as pool:
            steps = max(pool.map(lambda b: b.solve(100), bs))
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        states = {j: b.state(s) for j, (b, s) in slots.items()}
        for b in bs:
            b.close()
        return dt, states, steps

    def single(subset):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        states = {}
        for j in subset:
            m, h0 = work[j]
            gm = TmopMesh.from_structured(m, capi.METRIC_303_55, target=capi.TARGET_SIZE_FIELD,
                                          target_h0=h0)
            x = torch.from_numpy(m.x).cuda()
            reps = gm.solve(x, max_newton=40, rtol=1e-10, minres_max_it=50)
            states[j] = reps[-1]
            gm.close()
        torch.cuda.synchronize()
        return time.perf_counter() - t0, states

    allj = list(range(len(work)))
    t32, s32, n32 = batched("fp32", allj)
    t64, s64, n64 = batched("fp64", allj)
    sub = allj[:args.single_subset]
    tsub_single, ssingle = single(sub)
    tsub_b32, _, _ = batched("fp32", sub)
    tsub_b64, _, _ = batched("fp64", sub)
    rel = [abs(s32[j]["energy"] - s64[j]["energy"]) / max(abs(s64[j]["energy"]), 1e-300) for j in allj]
    out.update({"value": t32, "batched_fp32_s": t32, "batched_fp64_s": t64,
                "subset": {"meshes": len(sub), "single_fp64_s": tsub_single,
                           "batched_fp32_s": tsub_b32, "batched_fp64_s": tsub_b64},
                "converged": sum(1 for j in allj if s64[j]["status"] == 0),
                "newton_its_mean": float(sum(s64[j]["newton_its"] for j in allj) / len(allj)),
                "fp32_vs_fp64_final_energy_rel_max": max(rel), "batch_steps": n64})
    return out


def run_sweep(args):
    """Hessian-action throughput versus problem size (the paper's Sec. 4.1
    throughput methodology: one Newton iteration's worth of actions on the
    initial perturbed mesh): 3D, p = 1..4, n_q = p+1 and p+2, n_e in a size
    ladder; FP64-class and FP32.  GDOF/s = DOFs / mean action time, and the
    fraction of the measured HBM bandwidth of the action's algorithmic
    bytes."""
    import torch
    from paper_2205_12721_b300 import capi, meshgen
    from paper_2205_12721_b300.mesh_opt import TmopMesh
    hbm = measured_peaks().get("hbm_gbs")
    rows = []
    for p in (1, 2, 3, 4):
        for n in args.sweep_sizes:
            if (n * p + 1) ** 3 * 3 > 40e6:
                continue
            m = meshgen.config_mesh(3, n_e=n, order=p)
            for dq in (1, 2):
                nq = p + dq
                for prec in args.sweep_precisions:
                    rsz = 4 if prec == "fp32" else 8
                    gm = TmopMesh.from_structured(m, capi.METRIC_303, nq1d=nq, precision=prec)
                    x = torch.from_numpy(m.x).cuda()
                    gm.hessian_setup(x)
                    v = torch.randn(m.ndof, dtype=gm.rdtype, device="cuda")
                    y = torch.empty_like(v)
                    for _ in range(3):
                        gm.hessian_apply(v, y)
                    capi.tmop_profile_enable(gm.ctx, True)
                    reps = 20
                    for _ in range(reps):
                        gm.hessian_apply(v, y)
                    ms, nl = capi.tmop_profile_read(gm.ctx, capi.K_APPLY)
                    ams, _ = capi.tmop_profile_read(gm.ctx, capi.K_ASSEMBLE)
                    gm.close()
                    t = ms / nl
                    byts = bytes_apply(m.num_elems, m.ndof, 3, p + 1, nq, 45, rsz)
                    rows.append({"precision": prec, "p": p, "nq": nq, "n_e": n, "dofs": m.ndof,
                                 "apply_ms": t, "assemble_ms": ams / nl,
                                 "gdofs_kernel": m.ndof / (t * 1e-3) / 1e9,
                                 "gdofs_with_assembly": m.ndof / ((t + ams / nl) * 1e-3) / 1e9,
                                 "hbm_frac": (byts / (t * 1e-3) / 1e9 / hbm) if hbm else None})
                    del x, v, y
                    torch.cuda.empty_cache()
    return {"metric": "Hessian-apply GDOF/s vs size (3D hex, p=1..4)", "unit": "GDOF/s",
            "higher_is_better": True, "value": max(r["gdofs_kernel"] for r in rows), "rows": rows}


def run_solve(args):
    """Time to converged mesh of the single-mesh configurations: 2D 8x8 Q2
    (mu_2, exactly 10 Newton steps, MINRES rtol 1e-8) and 3D 24^3 Q2 (mu_302,
    |dF|/|dF0| <= 1e-10, FP64-class vs FP32-mixed)."""
    import torch
    from paper_2205_12721_b300 import capi, meshgen
    from paper_2205_12721_b300.mesh_opt import TmopMesh
    out = {"metric": "time-to-converged-mesh", "unit": "s", "higher_is_better": False, "runs": {}}
    cases = [("2d_8x8_q2_mu2", 1, capi.METRIC_2, "fp64", dict(max_newton=10, rtol=0.0)),
             ("3d_24cube_q2_mu302_fp64", 2, capi.METRIC_302, "fp64", dict(max_newton=100, rtol=1e-10)),
             ("3d_24cube_q2_mu302_fp32", 2, capi.METRIC_302, "fp32", dict(max_newton=100, rtol=1e-10))]
    for name, cfg, metric, prec, kw in cases:
        m = meshgen.config_mesh(cfg)
        res = []
        for rep in range(2):                              # first run warms up
            gm = TmopMesh.from_structured(m, metric, precision=prec)
            x = torch.from_numpy(m.x).cuda()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            reps = gm.solve(x, **kw)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            st, F, md = gm.energy(x)
            gm.close()
            res = {"seconds": dt, "newton_its": len(reps),
                   "minres_its": sum(r["minres_iters"] for r in reps),
                   "energy0": reps[0]["energy"], "energy": F,
                   "grad_ratio": reps[-1]["grad_norm_new"] / reps[0]["grad_norm"],
                   "status": reps[-1]["status"], "dofs": m.ndof}
        out["runs"][name] = res
    f64 = out["runs"]["3d_24cube_q2_mu302_fp64"]["energy"]
    f32 = out["runs"]["3d_24cube_q2_mu302_fp32"]["energy"]
    out["fp32_vs_fp64_final_energy_rel"] = abs(f32 - f64) / max(abs(f64), 1e-300)
    out["value"] = out["runs"]["3d_24cube_q2_mu302_fp64"]["seconds"]
    return out


def run_kershaw(args):
    """The paper's Kershaw benchmark (Sec. 4.1): 24^3 hexes, eps_y = eps_z =
    0.3, 9^3 quadrature points, mu_303, Jacobi-MINRES with at most 50
    iterations per Newton step, Newton until |dF|/|dF0| <= 1e-10; boundary
    nodes slide in their faces.  Time to solution per order p, FP64 class and
    FP32 mixed, beside the paper's GPU numbers (4 V100, context)."""
    import torch
    from paper_2205_12721_b300 import capi, meshgen
    from paper_2205_12721_b300.mesh_opt import TmopMesh
    paper = {1: 0.4, 2: 0.9, 3: 3.9, 4: 8.5}          # GPU PA + Jacobi, seconds (Sec. 4.1 table)
    rows = []
    for p in args.kershaw_orders:
        m = meshgen.kershaw(p, (args.kershaw_n,) * 3, 0.3, 0.3)
        u = meshgen.structured(3, p, (args.kershaw_n,) * 3)
        for prec in args.kershaw_precisions:
            gm = TmopMesh.from_structured(m, capi.METRIC_303, nq1d=args.kershaw_nq, precision=prec)
            x = torch.from_numpy(m.x).cuda()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            reps = gm.solve(x, max_newton=200, rtol=1e-10, minres_rtol=args.kershaw_minres_rtol,
                            minres_max_it=50)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            gm.close()
            rows.append({"p": p, "precision": prec, "dofs": m.ndof, "seconds": dt,
                         "newton_its": len(reps),
                         "minres_its": sum(r["minres_iters"] for r in reps),
                         "status": reps[-1]["status"],
                         "grad_ratio": reps[-1]["grad_norm_new"] / reps[0]["grad_norm"],
                         "max_dist_to_uniform_over_h":
                             float((x.cpu().numpy() - u.x).__abs__().max() * args.kershaw_n),
                         "paper_gpu_s_4xV100": paper.get(p)})
    return {"metric": "Kershaw time to solution", "unit": "s", "higher_is_better": False,
            "value": rows[0]["seconds"],
            "config": {"workload": f"Kershaw {args.kershaw_n}^3, eps 0.3, {args.kershaw_nq}^3 points, "
                                   f"mu_303, MINRES <= 50 (rtol {args.kershaw_minres_rtol:g}) + Jacobi, "
                                   "Newton to 1e-10"},
            "rows": rows}


def run_remap(args):
    """Advection remap of the discrete target field (Sec. 3.6) on the 48^3 Q3
    mesh: eta0 = 1 + 0.35 sin(2 pi x) cos(pi y) (1 + 0.2 sin(pi z)) given on
    the uniform mesh, remapped to the perturbed positions of the Newton
    workload with RK4 (4 steps) and Jacobi-CG to 1e-12.  Timed with CUDA
    events on the context stream; per-class kernel time from a separate
    profiled run.  The mass action is the dominant kernel; its per-iteration
    time is the class total divided by the CG iterations (launches after
    convergence are no-ops and are charged to the active ones)."""
    import numpy as np
    import torch
    from paper_2205_12721_b300 import capi, meshgen
    from paper_2205_12721_b300.mesh_opt import TmopMesh
    m = workload(args)
    u = meshgen.structured(3, m.order, m.n)
    N = m.num_nodes
    X = [u.x[a * N:(a + 1) * N] for a in range(3)]
    eta0 = 1.0 + 0.35 * np.sin(2 * np.pi * X[0]) * np.cos(np.pi * X[1]) * (1.0 + 0.2 * np.sin(np.pi * X[2]))
    stream = torch.cuda.Stream()
    out = {"metric": "advection remap time (Sec. 3.6)", "unit": "ms", "higher_is_better": False,
           "config": {"workload": f"3D hex {m.n[0]}^3 Q{m.order}, {m.order + 1}^3 points, eta remapped "
                                  "from the uniform to the perturbed mesh, RK4 4 steps, Jacobi-CG 1e-12",
                      "dofs_scalar_field": N, "elements": m.num_elems},
           "data": "synthetic seeded perturbed Cartesian mesh (no dataset)", "rows": []}
    peaks = measured_peaks()
    for prec in args.remap_precisions:
        with torch.cuda.stream(stream):
            gm = TmopMesh.from_structured(m, capi.METRIC_303, precision=prec, stream=stream)
            x0 = torch.from_numpy(u.x).cuda()
            x1 = torch.from_numpy(m.x).cuda()
            e0 = torch.from_numpy(eta0).cuda()
            e1 = torch.empty_like(e0)
        opts = capi.RemapOpts(4, 1e-12, 200)
        for _ in range(max(args.warmup, 1)):
            rep = capi.tmop_remap(gm.ctx, x0, x1, e0, e1, opts)
        times = []
        for _ in range(args.steps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            rep = capi.tmop_remap(gm.ctx, x0, x1, e0, e1, opts)
            b.record(stream)
            b.synchronize()
            times.append(a.elapsed_time(b))
        capi.tmop_profile_enable(gm.ctx, True)
        capi.tmop_remap(gm.ctx, x0, x1, e0, e1, opts)
        cls = {n: capi.tmop_profile_read(gm.ctx, k) for n, k in
               [("setup", capi.K_REMAP_SETUP), ("mass", capi.K_MASS), ("advect", capi.K_ADVECT)]}
        capi.tmop_profile_enable(gm.ctx, False)
        E, NQD, NP = m.num_elems, (m.order + 1) ** 3, (m.order + 1) ** 3
        mass_bytes = E * NQD * 8 + E * NP * 4 + N * 8 + E * NP * 8
        mass_ms = cls["mass"][0] / max(rep["cg_iters"], 1)
        ach = mass_bytes / (mass_ms * 1e-3) / 1e9
        hbm = peaks.get("hbm_gbs", 6400.0)
        out["rows"].append({"precision": prec, "ms_per_remap": float(np.median(times)),
                            "cg_iters": rep["cg_iters"], "solves": rep["solves"],
                            "class_ms": {k: {"total_ms": v[0], "launches": v[1]} for k, v in cls.items()},
                            "mass_ms_per_iter": mass_ms, "mass_bytes": mass_bytes,
                            "mass_gbs": ach, "mass_frac_hbm": ach / hbm})
        gm.close()
    out["value"] = out["rows"][0]["ms_per_remap"]
    return out


def run_serving(args):
    """Poisson stream of mesh-optimisation requests (2D n_e U{8..128} mu_2 or
    3D n_e U{4..40} mu_302, p U{1..4}); continuous batching under a device
    memory budget; p50/p99 time from arrival to converged mesh (rtol 1e-6)."""
    import torch
    from paper_2205_12721_b300 import meshgen
    from paper_2205_12721_b300.serve import Server, summarize

    res = {}
    for rate in args.rates:
        jobs = meshgen.serving_workload(args.n_jobs, rate=rate, n2=tuple(args.n2), n3=tuple(args.n3))
        srv = Server(int(args.budget_gb * (1 << 30)), precision=args.precision, newton_rtol=1e-6,
                     newton_max_it=50, minres_max_it=50, graphs=not args.no_graphs)
        done = srv.run(jobs)
        srv.close()
        torch.cuda.synchronize()
        res[str(rate)] = summarize(done)
    first = res[str(args.rates[0])]
    return {"metric": "time-to-converged-mesh p50/p99 under a Poisson request stream", "unit": "s",
            "higher_is_better": False, "value": first["p50_s"],
            "config": {"workload": f"{args.n_jobs} requests, 2D n_e U{tuple(args.n2)} mu_2 / "
                                   f"3D n_e U{tuple(args.n3)} mu_302, p U{{1..4}}, rtol 1e-6",
                       "budget_gb": args.budget_gb, "precision": args.precision},
            "by_rate": res}


def run_split(args, rank, world, local_rank):
    """The element-partitioned Newton step (dist.py) of the benchmark mesh over
    the ranks (strong scaling: the mesh is fixed, each rank owns a slab of
    elements, one interface sum per gradient / action / diagonal and
    allreduced scalars over NCCL).  With one rank it measures the
    host-driven distributed MINRES against the device MINRES of the default
    bench line."""
    import torch
    from paper_2205_12721_b300 import capi, dist
    torch.cuda.set_device(local_rank)
    m = workload(args)
    comm = dist.TorchComm() if world > 1 else dist.ThreadComm.group(1)[0]
    part = dist.partition(m.map, m.num_nodes, 3, m.fixed, world, rank)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        be = dist.LibraryBackend(part, m.order, capi.METRIC_303, stream=s)
        dn = dist.DistNewton(be, comm)
        x0 = be.from_host(part.to_local(m.x, m.num_nodes))
        x = x0.clone()
        for _ in range(args.warmup):
            x.copy_(x0)
            dn.newton_step(x, 0.0, MINRES_ITS, True)
        s.synchronize()
        if world > 1:
            torch.distributed.barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            x.copy_(x0)
            r = dn.newton_step(x, 0.0, MINRES_ITS, True)
        s.synchronize()
        dt = (time.perf_counter() - t0) / args.steps
    be.close()
    dt = max_over_ranks(dt, world, torch.device("cuda", local_rank))
    return {"metric": METRIC, "value": m.ndof * MINRES_ITS / dt / 1e9, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3,
            "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
            "dtype": "f64 (double-float contractions)",
            "data": "synthetic seeded perturbed Cartesian mesh (no dataset)",
            "config": {"workload": f"3D hex {m.n[0]}^3 Q{m.order}, mu_303, 1 element-partitioned Newton "
                                   f"step with {MINRES_ITS} MINRES", "dofs": m.ndof,
                       "parallelism": f"element partition x{world} (slabs), interface sums + allreduce"},
            "newton": {"status": r["status"], "alpha": r["alpha"], "minres_iters": r["minres_iters"]}}


def run_autotune(args):
    """The autotuner over the Hessian-action kernel variants: for every
    configuration with more than one variant (3D, p = 1..4, n_q = p+1 and p+2
    with n_q^2 <= 32; or those of --autotune-configs) and every precision, a
    mesh of the benchmark family whose stored data exceeds L2 (~1.2 GB, or
    --autotune-n-e elements per side), tmop_autotune (CUDA events, 10 launches
    per variant) repeated --autotune-passes times, the per-variant minimum of
    the passes; prints the measured times and the chosen variant per
    configuration, the rows of autotune_table.json."""
    import torch
    from paper_2205_12721_b300 import capi, meshgen
    from paper_2205_12721_b300.mesh_opt import TmopMesh
    hbm = measured_peaks().get("hbm_gbs")
    precs = {"fp64": capi.FP64, "fp32": capi.FP32, "fp64-native": capi.FP64_NATIVE}
    rows = []
    sel = [tuple(int(v) for v in c.split(":")) for c in args.autotune_configs]
    for p in (1, 2, 3, 4):
        for nq in (p + 1, p + 2):
            if capi.tmop_apply_variants(3, p, nq) <= 1 or (sel and (p, nq) not in sel):
                continue
            for name in args.autotune_precisions:
                rsz = 4 if name == "fp32" else 8
                per_el = 45 * nq ** 3 * rsz
                n = args.autotune_n_e or max(8, int(round((args.autotune_bytes / per_el) ** (1.0 / 3.0))))
                m = meshgen.config_mesh(3, n_e=n, order=p)
                gm = TmopMesh.from_structured(m, capi.METRIC_303, nq1d=nq, precision=name)
                x = torch.from_numpy(m.x).cuda()
                gm.hessian_setup(x)
                ms = None
                for _ in range(args.autotune_passes):
                    _, t = capi.tmop_autotune(gm.ctx, 10)
                    ms = t if ms is None else [min(a, b) for a, b in zip(ms, t)]
                best = min(range(len(ms)), key=lambda i: ms[i])
                capi.tmop_set_apply_variant(3, p, nq, precs[name], best)
                gm.close()
                byts = bytes_apply(m.num_elems, m.ndof, 3, p + 1, nq, 45, rsz)
                rows.append({"d": 3, "p": p, "nq": nq, "precision": name, "prec": precs[name],
                             "n_e": n, "dofs": m.ndof, "variant": best,
                             "ms": [round(t, 5) for t in ms],
                             "hbm_frac_best": (byts / (min(ms) * 1e-3) / 1e9 / hbm) if hbm else None,
                             "gdofs_best": m.ndof / (min(ms) * 1e-3) / 1e9})
                del x
                torch.cuda.empty_cache()
    return {"metric": "Hessian-action kernel variant per configuration (autotuner)",
            "unit": "ms", "higher_is_better": False, "rows": rows}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32", "fp64-native"])
    ap.add_argument("--n-e", dest="n_e", type=int, default=48)
    ap.add_argument("--order", type=int, default=3)
    ap.add_argument("--cpu-sample-n", dest="cpu_sample_n", type=int, default=8)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-ttc", action="store_true", help="skip the 24^3 Q2 time-to-converged leg")
    ap.add_argument("--variants", nargs="*", default=["fp32", "fp64-native"],
                    help="other precisions timed after the main run (rank 0)")
    ap.add_argument("--workload", default="newton",
                    choices=["newton", "batched", "serving", "sweep", "solve", "kershaw", "remap",
                             "autotune", "split"])
    ap.add_argument("--kershaw-orders", dest="kershaw_orders", type=int, nargs="+", default=[1, 2, 3, 4])
    ap.add_argument("--kershaw-precisions", dest="kershaw_precisions", nargs="+",
                    default=["fp64", "fp32"])
    ap.add_argument("--kershaw-n", dest="kershaw_n", type=int, default=24)
    ap.add_argument("--kershaw-nq", dest="kershaw_nq", type=int, default=9)
    ap.add_argument("--kershaw-minres-rtol", dest="kershaw_minres_rtol", type=float, default=1e-12)
    ap.add_argument("--sweep-sizes", dest="sweep_sizes", type=int, nargs="+",
                    default=[4, 8, 16, 24, 32, 48])
    ap.add_argument("--sweep-precisions", dest="sweep_precisions", nargs="+", default=["fp64", "fp32"])
    ap.add_argument("--remap-precisions", dest="remap_precisions", nargs="+",
                    default=["fp64", "fp64-native"])
    ap.add_argument("--n-meshes", dest="n_meshes", type=int, default=512)
    ap.add_argument("--no-graphs", dest="no_graphs", action="store_true",
                    help="batched / serving workloads: MINRES without CUDA graphs")
    ap.add_argument("--single-subset", dest="single_subset", type=int, default=32)
    ap.add_argument("--n-jobs", dest="n_jobs", type=int, default=2000)
    ap.add_argument("--rates", type=float, nargs="+", default=[10, 50, 200])
    ap.add_argument("--n2", type=int, nargs=2, default=[8, 128])
    ap.add_argument("--n3", type=int, nargs=2, default=[4, 40])
    ap.add_argument("--budget-gb", dest="budget_gb", type=float, default=64.0)
    ap.add_argument("--autotune-precisions", dest="autotune_precisions", nargs="+",
                    default=["fp64", "fp32", "fp64-native"])
    ap.add_argument("--autotune-bytes", dest="autotune_bytes", type=float, default=1.2e9)
    ap.add_argument("--autotune-n-e", dest="autotune_n_e", type=int, default=0,
                    help="elements per side of the autotuner's meshes (default: from --autotune-bytes)")
    ap.add_argument("--autotune-configs", dest="autotune_configs", nargs="*", default=[],
                    help="p:nq pairs to tune (default: all with more than one variant)")
    ap.add_argument("--autotune-passes", dest="autotune_passes", type=int, default=1)
    ap.add_argument("--traffic", type=float, default=None,
                    help="override the ncu dram bytes per launch of the apply kernel")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    if args.workload == "split":
        if world > 1:
            import torch
            torch.cuda.set_device(local_rank)
            torch.distributed.init_process_group("nccl")
        out = run_split(args, rank, world, local_rank)
        if world > 1:
            import torch
            torch.distributed.destroy_process_group()
        if rank == 0:
            print(json.dumps(out))
        return
    if args.workload != "newton":
        out = {"batched": run_batched, "serving": run_serving, "sweep": run_sweep,
               "solve": run_solve, "kershaw": run_kershaw, "remap": run_remap,
               "autotune": run_autotune}[args.workload](args)
        if rank == 0:
            print(json.dumps(out))
        return
    if args.impl == "reference":
        out = run_reference(args, rank, world)
    else:
        if world > 1:
            import torch
            torch.distributed.init_process_group("nccl")
        out = run_ours(args, rank, world, local_rank)
        if world > 1:
            import torch
            torch.distributed.destroy_process_group()
    if rank == 0 and out is not None:
        print(json.dumps(out))


if __name__ == "__main__":
    main()
