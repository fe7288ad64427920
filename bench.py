#!/usr/bin/env python
"""Benchmark of the FDPB Jacobi-PCG hot path on GB300.

One step = one MD-like snapshot of the workload: grid setup on the device
(dielectric map, charges, Debye-Hueckel boundary), the FP32 + FP64-refined
Jacobi-PCG solve to a 1e-6 true relative residual, and the energy read back to
the host.  Prints one JSON line (rank 0).  Multi-GPU runs are independent
replicas (each rank solves its own snapshots; no collective on the data path).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload globule129]
    python bench.py --impl reference ...   # the FP64 CPU oracle on the host cores
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_1704_02745_gb300 import inputs  # noqa: E402

METRIC = "solves/s, p50/p99 @1e-6 rel resid: served FP32+refine vs plain FP64 PCG"
WORKLOADS = {
    "globule33": inputs.small_33,
    "globule129": inputs.globule_129,
    "globule257": inputs.globule_257,
}
# Algorithmic HBM bytes per grid node of one launch of each phase kernel
# (FP32 inner solve, packed one-byte coefficients):
#   stencil pass: read r, p_old, d (4 B each) and the code byte; write p, Ap, d
#   update pass:  read r, Ap and the code byte; write r
BYTES_PER_NODE = {"stencil": 4 + 4 + 4 + 1 + 4 + 4 + 4, "update": 4 + 4 + 1 + 4}
# DRAM bytes per node per stencil-pass launch from the ncu capture summarised in
# profiles/ (None until a capture of the current kernel exists).
NCU_TRAFFIC_PER_NODE = {"stencil": None}
SNAPSHOT_SIGMA = 0.2  # A, per-coordinate perturbation between snapshots


def env_rank():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def snapshots(problem, count, seed):
    rng = np.random.default_rng([seed, 31])
    out = []
    for _ in range(count):
        a = problem.atoms.copy()
        a.xyz = a.xyz + rng.normal(0.0, SNAPSHOT_SIGMA, size=a.xyz.shape)
        out.append(a)
    return out


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                smax.append(float(f[1]))
            except ValueError:
                continue
            for nm, v in zip(names, f[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def pct(v, q):
    return float(np.percentile(np.asarray(v), q)) if v else None


def run_loop(g, phi, snaps, steps, warmup, stream, flush, solve_kw, ctx=None, marks=None):
    import torch
    dev_ms, wall_ms, iters, energies = [], [], [], []
    for i in range(warmup + steps):
        if i == warmup and marks is not None:
            torch.cuda.synchronize()
            marks.append(ctx.stats())
        a = snaps[i % len(snaps)]
        flush.zero_()  # write > L2 between steps
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        e0.record(stream)
        g.update_atoms(a)
        info = g.solve(phi, **solve_kw)
        en = g.energy(phi)
        e1.record(stream)
        e1.synchronize()
        t1 = time.perf_counter()
        if i >= warmup:
            dev_ms.append(e0.elapsed_time(e1))
            wall_ms.append((t1 - t0) * 1e3)
            iters.append(info.iterations)
            energies.append(en)
    if marks is not None:
        torch.cuda.synchronize()
        marks.append(ctx.stats())
    return dev_ms, wall_ms, iters, energies


def run_ours(args):
    import torch
    from paper_1704_02745_gb300 import pb
    from paper_1704_02745_gb300 import build as pbbuild

    rank, world, local = env_rank()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    pbbuild.build()
    torch.cuda.set_device(local)
    stream = torch.cuda.Stream()
    problem = WORKLOADS[args.workload]()
    spec = problem.grid.replace(coef=args.coef, dh=args.dh)
    n_nodes = spec.n
    snaps = snapshots(problem, 8, seed=100 + rank)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    solve_kw = dict(precision="f32_refine", tol=args.tol, inner_tol=args.inner_tol)
    with torch.cuda.stream(stream):
        ctx = pb.Context(local, stream=stream.cuda_stream)
        g = pb.Grid(ctx, spec, snaps[0])
        phi = torch.zeros(spec.shape, dtype=torch.float64, device="cuda")
        # warm-up and timed region
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        clocks = ClockSampler(local)
        clocks.start()
        marks = []
        dev_ms, wall_ms, iters, energies = run_loop(g, phi, snaps, args.steps, args.warmup, stream,
                                                    flush, solve_kw, ctx, marks)
        clk = clocks.stop()
        st0, st1 = marks
        # launches and copies of the timed steps (counted by the library)
        launches = int(st1[0] - st0[0])
        h2d = (st1[1] - st0[1]) / float(args.steps)
        d2h = (st1[2] - st0[2]) / float(args.steps)
        total_dev_s = sum(dev_ms) / 1e3
        total_wall_s = sum(wall_ms) / 1e3
        if world > 1:
            t = torch.tensor([total_dev_s, total_wall_s], dtype=torch.float64, device="cuda")
            torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
            total_dev_s, total_wall_s = float(t[0]), float(t[1])
        if args.quick:  # profiling runs: the timed loop only
            if rank == 0:
                print(json.dumps({"quick": True, "ms_per_step": sum(dev_ms) / len(dev_ms),
                                  "iterations_mean": float(np.mean(iters))}), flush=True)
            return
        # plain FP64 PCG, one solve at a time, on the same snapshots and setup
        k64 = max(3, args.steps // 2)
        d64, w64, it64, _ = run_loop(g, phi, snaps, k64, 1, stream, flush,
                                     dict(precision="f64", tol=args.tol))
        # per-kernel device time of one solve (kernels launched one by one between events)
        g.update_atoms(snaps[0])
        prof = g.solve(phi, profile=True, **solve_kw)
    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    hbm, peak_kind = peaks()
    t_st = prof.ms_stencil / max(prof.n_stencil, 1) / 1e3
    t_up = prof.ms_update / max(prof.n_update, 1) / 1e3
    ach_st = BYTES_PER_NODE["stencil"] * n_nodes / t_st / 1e9
    ach_up = BYTES_PER_NODE["update"] * n_nodes / t_up / 1e9
    trf = NCU_TRAFFIC_PER_NODE["stencil"]
    out = {
        "metric": METRIC,
        "value": world * args.steps / total_dev_s,
        "unit": "solves/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": total_dev_s * 1e3 / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32+f64",
        "data": "synthetic",
        "config": {"workload": problem.name, "grid": f"{spec.nx}x{spec.ny}x{spec.nz}",
                   "atoms": problem.atoms.n, "h": spec.h, "tol": args.tol,
                   "solver": "jacobi-pcg fp32 inner + fp64 refinement",
                   "inner_tol": args.inner_tol, "coef": args.coef,
                   "debye_hueckel_sum": args.dh,
                   "snapshot_sigma_A": SNAPSHOT_SIGMA,
                   "l2": "256 MB buffer written between timed steps",
                   "parallelism": f"replicas x{world}"},
        "latency_ms": {"p50": pct(dev_ms, 50), "p99": pct(dev_ms, 99)},
        "iterations_mean": float(np.mean(iters)),
        "grid_point_iters_per_s": float(np.mean(iters)) * n_nodes * world * args.steps / total_dev_s,
        "fp64_plain": {"value": k64 / (sum(d64) / 1e3), "unit": "solves/s",
                       "latency_ms": {"p50": pct(d64, 50), "p99": pct(d64, 99)},
                       "iterations_mean": float(np.mean(it64)), "steps": k64},
        "roofline": {"bound": "hbm", "kernel": "k_stencil<float,packed> (CG stencil pass)",
                     "achieved": ach_st, "peak": hbm, "unit": "GB/s", "frac": ach_st / hbm,
                     "peak_kind": peak_kind,
                     "traffic": None if trf is None else trf * n_nodes,
                     "bytes_per_node": BYTES_PER_NODE["stencil"], "launch_ms": t_st * 1e3,
                     "update_pass": {"achieved": ach_up, "frac": ach_up / hbm,
                                     "bytes_per_node": BYTES_PER_NODE["update"],
                                     "launch_ms": t_up * 1e3},
                     "resid_pass_ms": prof.ms_resid / max(prof.n_resid, 1)},
        "e2e": {"value": world * args.steps / total_wall_s, "unit": "solves/s",
                "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                "latency_ms": {"p50": pct(wall_ms, 50), "p99": pct(wall_ms, 99)}},
        "gpu_launches": launches,
        "clocks": clk,
    }
    if not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(problem, snaps[0], float(np.mean(iters)), args)
    print(json.dumps(out), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def oracle_solve_sample(problem, atoms, tol, max_sample_iters):
    """Time the oracle's setup and a bounded number of PCG iterations."""
    import oracle
    t0 = time.perf_counter()
    s = oracle.setup(problem.grid, atoms)
    t1 = time.perf_counter()
    r = oracle.pcg(s, tol=tol, max_iter=max_sample_iters)
    t2 = time.perf_counter()
    oracle.energy(s, r.phi)
    t3 = time.perf_counter()
    return (t1 - t0) + (t3 - t2), (t2 - t1) / max(r.iters, 1), r


def cpu_baseline(problem, atoms, gpu_iters, args):
    """The FP64 oracle (single thread) on the host: setup + a bounded number of
    PCG iterations, scaled to a full solve with the iteration count of a full
    FP64 solve (estimated from the GPU run's iterations)."""
    import oracle
    oracle.build()
    n_iter = max(20, int(args.cpu_sample_iters))
    t_fixed, t_iter, r = oracle_solve_sample(problem, atoms, args.tol, n_iter)
    full_iters = r.iters if r.status == 0 else gpu_iters
    t_solve = t_fixed + t_iter * full_iters
    return {"value": 1.0 / t_solve, "unit": "solves/s", "cores": 1, "kind": "oracle",
            "sample": (f"one {problem.name} snapshot: oracle setup + {min(r.iters, n_iter)} FP64 "
                       f"Jacobi-PCG iterations timed, scaled to {full_iters:.0f} iterations"),
            "cpu": platform_cpu()}


def platform_cpu():
    import platform
    try:
        for ln in open("/proc/cpuinfo"):
            if ln.lower().startswith(("model name", "cpu part")):
                return platform.machine() + " " + ln.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.machine()


def run_reference(args):
    """The FP64 CPU oracle as the reference arm (rank 0 only)."""
    rank, world, _ = env_rank()
    if rank != 0:
        return
    import oracle
    oracle.build()
    problem = WORKLOADS[args.workload]()
    snaps = snapshots(problem, 8, seed=100)
    # calibrate the full iteration count once (untimed)
    s = oracle.setup(problem.grid, snaps[0])
    full = oracle.pcg(s, tol=args.tol, max_iter=args.cpu_sample_iters if problem.grid.n > 5e6 else 100000)
    full_iters = full.iters
    times = []
    for i in range(args.warmup + args.steps):
        t_fixed, t_iter, _ = oracle_solve_sample(problem, snaps[i % len(snaps)], args.tol,
                                                 args.cpu_sample_iters)
        if i >= args.warmup:
            times.append(t_fixed + t_iter * full_iters)
    total = sum(times)
    val = args.steps / total
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": val, "unit": "solves/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": problem.name, "grid": f"{problem.grid.nx}^3",
                   "atoms": problem.atoms.n, "tol": args.tol, "solver": "oracle FP64 Jacobi-PCG"},
        "latency_ms": {"p50": pct([t * 1e3 for t in times], 50),
                       "p99": pct([t * 1e3 for t in times], 99)},
        "cpu_baseline": {"value": val, "unit": "solves/s", "cores": 1, "kind": "oracle",
                         "sample": (f"per step: oracle setup + {args.cpu_sample_iters} FP64 "
                                    f"Jacobi-PCG iterations, scaled to {full_iters} iterations"),
                         "cpu": platform_cpu()},
        "e2e": {"value": val, "unit": "solves/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="globule129", choices=sorted(WORKLOADS))
    ap.add_argument("--coef", default="packed", choices=["packed", "f32", "bf16"])
    ap.add_argument("--tol", type=float, default=1e-6)
    ap.add_argument("--inner-tol", type=float, default=1e-3)
    ap.add_argument("--cpu-sample-iters", type=int, default=40)
    ap.add_argument("--dh", default="f32", choices=["f32", "f64"],
                    help="precision of the Debye-Hueckel boundary sum in the grid setup")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--quick", action="store_true",
                    help="timed loop only (no FP64 comparator, profiled solve or CPU baseline)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
