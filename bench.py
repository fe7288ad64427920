#!/usr/bin/env python
"""Benchmark of the FDPB Jacobi-PCG hot path on GB300.

Default workload ("serving"): 16 MD-like trajectories (300-8,000 atoms, grids
33^3-193^3 at fill ratio 1.5, snapshots a 0.2 A random walk).  One step = a
batch of 64 snapshot requests to the continuous-batching server (steady state:
step k+1 is queued while step k completes) (grid setup, FP32 Jacobi-PCG with FP64 iterative refinement to a 1e-6
true relative residual, warm start along each trajectory, energy back to the
host).  The same requests are also solved one at a time with plain FP64 PCG,
and a Poisson request stream at 0.8x the measured plain-FP64 capacity gives
p50/p99 latency for both.

Single-grid workloads (globule33/129/257): one step = one snapshot solved with
pb_pcg_solve (setup, FP32 + FP64 refinement to 1e-6, energy).

Prints one JSON line (rank 0).  Multi-GPU runs are independent replicas (each
rank solves its own requests; no collective on the data path).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload serving]
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
from types import SimpleNamespace

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_1704_02745_gb300 import inputs  # noqa: E402

METRIC = "solves/s, p50/p99 @1e-6 rel resid: served FP32+refine vs plain FP64 PCG"
BATCH_METRIC = "solves/s @1e-6 rel resid: batch of 256 snapshots, FP32+refine"
SERVING = "serving"
BATCH = "batch256"
SOLVATION = "solvation129"
SOLVATION_METRIC = "solvation energies/s @1e-6 rel resid (two solves each), FP32+refine"
WORKLOADS = {
    SERVING: None,
    BATCH: None,
    SOLVATION: inputs.globule_129,
    "globule33": inputs.small_33,
    "globule129": inputs.globule_129,
    "globule257": inputs.globule_257,
}
# Algorithmic HBM bytes per grid node of one launch of each phase kernel
# (FP32 inner solve, packed one-byte coefficients).  Grids of a server batch:
#   stencil pass: read z = M^-1 r, p_old, d (4 B each) and the code byte; write p, d
#   update pass (over the stencil tiles): read p (Ap is formed again from it), z
#   and the code byte; write z
BYTES_PER_NODE = {"stencil": 4 + 4 + 4 + 1 + 4 + 4, "update": 4 + 4 + 1 + 4}
# A single grid: the stencil pass also writes Ap, which the update pass (over
# row chunks) reads in place of p.
BYTES_PER_NODE_GRID = {"stencil": 4 + 4 + 4 + 1 + 4 + 4 + 4, "update": 4 + 4 + 1 + 4}


def bytes_per_node(coef):
    """Algorithmic bytes per node of the two passes of a single-grid solve for a
    coefficient storage: the packed code byte, or explicit eps_x, eps_y, eps_z
    (4 or 2 B) and an FP32 diagonal in place of it (the update pass then reads
    the diagonal)."""
    if coef == "packed":
        return dict(BYTES_PER_NODE_GRID)
    c = 2 if coef == "bf16" else 4
    return {"stencil": 4 + 4 + 4 + 3 * c + 4 + 4 + 4 + 4, "update": 4 + 4 + 4 + 4}
# DRAM bytes (read + write) per grid node of one stencil-pass launch, from
# bounded ncu captures (one kernel, at most three launches, a few GB on the
# device) summarised in profiles/: (bytes per node, the summary it comes from).
# None where no such capture of the current kernel exists.
NCU_TRAFFIC_PER_NODE = {
    # k_stencil<float, packed, batch, fast>, launches 40-41 of the batch256 kernel-profile window:
    # (3.2555 + 1.7578 + 3.2563 + 1.7551) GB / (2 x 214,261,784 nodes)
    "stencil_batch": (10.024756736e9 / 428523568, "profiles/k_stencil_batch256.md"),
    # k_stencil<float, packed, single grid, fast> on 257^3, one launch: 405.05 MB / 16,974,593 nodes
    "stencil_grid": (405.05472e6 / 16974593, "profiles/k_stencil_globule257.md"),
}
# FP64 operations per grid node of the residual pass: x + d (1), the operator
# diag x - sum of six eps x_nb (1 multiply, 6 multiply-adds), b - A x (1).
RESID_FP64_OPS_PER_NODE = 9
SNAPSHOT_SIGMA = 0.2  # A, per-coordinate perturbation between snapshots


def cg_iteration_in_graph(solve_ms, resid_steps, iters, prof, n_nodes, bpn, hbm, precond):
    """One CG iteration of the timed solves as they run (device graphs, launches
    overlapping through programmatic dependent launch): each solve's device time
    less its residual passes (their profiled launch time), per iteration."""
    if precond == "gmg" or not solve_ms or sum(iters) == 0:
        return None
    t_res = prof.ms_resid / max(prof.n_resid, 1)
    cg_ms = sum(s - r * t_res for s, r in zip(solve_ms, resid_steps)) / sum(iters)
    b = (bpn["stencil"] + bpn["update"]) * n_nodes
    return {"ms": cg_ms, "bytes_per_node": bpn["stencil"] + bpn["update"],
            "achieved": b / (cg_ms * 1e-3) / 1e9, "frac": b / (cg_ms * 1e-3) / 1e9 / hbm,
            "note": ("timed solves' device time less their residual passes (profiled launch time), "
                     "per CG iteration")}


def resid_roofline(kp, alu):
    """The FP64 residual pass against the device's measured FP64 rate: it is
    bound by FP64 arithmetic, not by its 37 B per node."""
    nodes = kp.bytes_resid / 37.0
    sec = kp.ms_resid / 1e3
    out = {"bound": "alu", "launch_ms": kp.ms_resid / max(kp.launches_resid, 1),
           "launches": kp.launches_resid, "bytes_per_node": 37,
           "achieved_gbs": kp.bytes_resid / max(sec, 1e-15) / 1e9,
           "fp64_ops_per_node": RESID_FP64_OPS_PER_NODE}
    if alu is not None and sec > 0:
        ach = RESID_FP64_OPS_PER_NODE * nodes / sec
        out.update({"achieved": ach / 1e12, "peak": alu["fp64_fma_per_s"] / 1e12, "unit": "T FP64 op/s",
                    "frac": ach / alu["fp64_fma_per_s"],
                    "peak_kind": "measured (pb_measure_alu: FP64 FMA loop, this run)"})
    return out


def max_over_ranks(values, world):
    """Element-wise maximum of per-rank timings over the process group (the
    slowest rank sets the job's time); identity on one rank."""
    if world <= 1:
        return list(values)
    import torch
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    t = torch.tensor(list(values), dtype=torch.float64, device=dev)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return [float(v) for v in t.cpu()]


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


def run_loop(g, phi, snaps, steps, warmup, stream, flush, solve_kw, ctx=None, marks=None,
             prange=False):
    import torch
    dev_ms, wall_ms, iters, energies = [], [], [], []
    solve_ms, resid_steps = [], []
    for i in range(warmup + steps):
        if i == warmup and marks is not None:
            torch.cuda.synchronize()
            marks.append(ctx.stats())
        if i == warmup and prange:
            torch.cuda.profiler.start()
        a = snaps[i % len(snaps)]
        flush.zero_()  # write > L2 between steps
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        es0 = torch.cuda.Event(enable_timing=True)
        es1 = torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        e0.record(stream)
        g.update_atoms(a)
        es0.record(stream)
        info = g.solve(phi, **solve_kw)
        es1.record(stream)
        en = g.energy(phi)
        e1.record(stream)
        e1.synchronize()
        t1 = time.perf_counter()
        if i >= warmup:
            dev_ms.append(e0.elapsed_time(e1))
            wall_ms.append((t1 - t0) * 1e3)
            iters.append(info.iterations)
            energies.append(en)
            solve_ms.append(es0.elapsed_time(es1))
            resid_steps.append(info.outer_steps + 1)
    if prange:
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
    if marks is not None:
        torch.cuda.synchronize()
        marks.append(ctx.stats())
    run_loop.solve_ms, run_loop.resid_steps = solve_ms, resid_steps
    return dev_ms, wall_ms, iters, energies


# --------------------------------------------------------------------------- serving

class Stream:
    """Snapshot requests of the serving workload: request i is the next
    snapshot of a random trajectory (seeded)."""

    def __init__(self, seed=5, n_traj=16, sigma=0.2, req_seed=99):
        self.trajs = inputs.trajectories(seed=seed, count=n_traj, sigma=sigma)
        self.rng = np.random.default_rng([seed, req_seed])
        self.cur = [t.base.copy() for t in self.trajs]
        self.walk = [np.random.default_rng([seed, 1000 + k]) for k in range(n_traj)]

    def next(self):
        k = int(self.rng.integers(0, len(self.trajs)))
        a = self.cur[k].copy()
        a.xyz = a.xyz + self.walk[k].normal(0.0, self.trajs[k].sigma, a.xyz.shape)
        self.cur[k] = a
        return k, self.trajs[k].grid, a

    def take(self, n):
        return [self.next() for _ in range(n)]


def serve_batch(srv, reqs, want_phi=False):
    """Submit all requests, wait for all; (wall seconds, latencies s, results)."""
    t0 = time.perf_counter()
    tickets = [srv.submit(k, g, a, want_phi=want_phi) for k, g, a in reqs]
    res = []
    for t in tickets:
        r, _ = srv.poll(t, 600000)
        res.append(r)
    return time.perf_counter() - t0, [r.seconds for r in res], res


def prewarm_pinned(pb, batches):
    """Page-locked phi buffers, allocated once before the timed region (as a
    client would hold them), then back in the pool: for each size class,
    three times the most any step asks for (two steps in flight, one being
    collected)."""
    from collections import Counter
    need = Counter()
    for b in batches:
        c = Counter(pb.PinnedPool.size_class(8 * int(np.prod(g.shape))) for _, g, _ in b)
        for k, v in c.items():
            need[k] = max(need[k], 3 * v)
    bufs = [pb.pinned_empty((k // 8,)) for k, v in need.items() for _ in range(v)]
    del bufs


def serve_steps(srv, batches, want_phi=False):
    """Steady state: step k+1's requests are queued before step k's results are
    collected, so the server always has work.  Returns (wall seconds, latencies
    s (submit -> ready), results)."""
    t0 = time.perf_counter()
    pend = [srv.submit(k, g, a, want_phi=want_phi) for k, g, a in batches[0]]
    lats, res = [], []
    for i in range(len(batches)):
        nxt = ([srv.submit(k, g, a, want_phi=want_phi) for k, g, a in batches[i + 1]]
               if i + 1 < len(batches) else [])
        for t in pend:
            r, _ = srv.poll(t, 600000)
            res.append(r)
            lats.append(r.seconds)
        pend = nxt
    return time.perf_counter() - t0, lats, res


class PlainFP64:
    """One request at a time: per-trajectory grid, setup, FP64 Jacobi-PCG from
    phi0 = 0, energy (pb_pcg_solve)."""

    def __init__(self, pb, ctx, torch):
        self.pb, self.ctx, self.torch = pb, ctx, torch
        self.grids, self.phis = {}, {}

    def solve(self, k, g, a, tol):
        if k not in self.grids:
            self.grids[k] = self.pb.Grid(self.ctx, g.replace(dh="f32"), a)
            self.phis[k] = self.torch.zeros(g.shape, dtype=self.torch.float64, device="cuda")
        else:
            self.grids[k].update_atoms(a)
        info = self.grids[k].solve(self.phis[k], precision="f64", tol=tol)
        return self.grids[k].energy(self.phis[k]), info

    def close(self):
        for gr in self.grids.values():
            gr.close()


def poisson_run(submit_fn, reqs, rate, seed=17):
    """Open-loop stream: request i arrives at its Poisson time; returns
    (makespan s, latencies s = completion - arrival)."""
    rng = np.random.default_rng(seed)
    arrivals = np.cumsum(rng.exponential(1.0 / rate, len(reqs)))
    arrivals -= arrivals[0]
    return submit_fn(reqs, arrivals)


def run_serving(args):
    import torch
    from paper_1704_02745_gb300 import pb
    from paper_1704_02745_gb300 import build as pbbuild

    rank, world, local = env_rank()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    pbbuild.build()
    torch.cuda.set_device(local)
    stream = Stream(seed=5, req_seed=99 + 1000 * rank)
    per_step = args.batch
    ctx = pb.Context(local)
    alu = ctx.measure_alu().as_dict()  # the FP64 roofline of the residual pass
    budget = int(args.budget_gb * (1 << 30))
    srv = pb.Server(ctx, budget, precision="f32_refine", tol=args.tol, inner_tol=args.inner_tol,
                    warm_start=True)
    if args.plan:
        srv.set_plan(*[int(v) for v in args.plan.split(",")])
        args.no_autotune = True
    # warm-up steps (the batch's tile plan is tuned on the first), then the timed steps
    tune = None
    for w in range(args.warmup):
        reqs = [(k, g.replace(dh="f32"), a) for k, g, a in stream.take(per_step)]
        if w == 0 and not args.no_autotune:
            tickets = [srv.submit(k, g, a) for k, g, a in reqs]
            tune = srv.autotune(600000).as_dict()
            for t in tickets:
                srv.poll(t, 600000)
        else:
            serve_batch(srv, reqs)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    st0 = ctx.stats()
    clocks = ClockSampler(local)
    clocks.start()
    batches = [[(k, g.replace(dh="f32"), a) for k, g, a in stream.take(per_step)]
               for _ in range(args.steps)]
    if args.profile_range:
        torch.cuda.profiler.start()
    total, lats, res = serve_steps(srv, batches)
    if args.profile_range:
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
    iters = [r.info.iterations for r in res]
    # grid nodes x CG iterations of the timed steps: each iteration is one
    # stencil pass over the grid (the denominator of the ncu DRAM traffic)
    node_passes = int(sum(int(np.prod(g.shape)) * r.info.iterations
                          for (_, g, _), r in zip([x for b in batches for x in b], res)))
    bad = [r.status for r in res if r.status != 0]
    if bad:
        raise RuntimeError(f"served requests failed: {bad[:5]}")
    clk = clocks.stop()
    torch.cuda.synchronize()
    st1 = ctx.stats()
    total = max_over_ranks([total], world)[0]
    if args.quick:  # sweeps: the closed-loop rate only
        if rank == 0:
            print(json.dumps({"quick": True, "workload": "serving", "plan": args.plan, "tune": tune,
                              "solves_per_s": world * args.steps * per_step / total,
                              "iterations_mean": float(np.mean(iters)), "clocks": clk}), flush=True)
        srv.close()
        ctx.close()
        return
    # end to end: the same steady state with phi copied back to the host per request,
    # as many steps as the timed phase (the requests differ; fewer steps sample grid
    # sizes too unevenly to compare)
    e2e_steps = max(2, args.steps)
    e2e_batches = [[(k, g.replace(dh="f32"), a) for k, g, a in stream.take(per_step)]
                   for _ in range(e2e_steps)]
    prewarm_pinned(pb, e2e_batches)
    e2e0 = ctx.stats()
    e2e_wall, _, _ = serve_steps(srv, e2e_batches, want_phi=True)
    e2e1 = ctx.stats()
    # plain FP64, one at a time: its capacity, measured on the first requests
    # of the Poisson stream's request list (after one untimed solve of each
    # trajectory's grid, so that grid creation is not timed)
    pois_reqs = Stream(seed=5, req_seed=77 + rank).take(max(args.stream_requests, per_step))
    plain = PlainFP64(pb, ctx, torch)
    seen = set()
    for k, g, a in pois_reqs:
        if k not in seen:
            seen.add(k)
            plain.solve(k, g, a, args.tol)
    p_lat = []
    n_plain = min(len(pois_reqs), max(8, per_step))
    t0 = time.perf_counter()
    for k, g, a in pois_reqs[:n_plain]:
        t1 = time.perf_counter()
        plain.solve(k, g, a, args.tol)
        p_lat.append(time.perf_counter() - t1)
    plain_rate = n_plain / (time.perf_counter() - t0)
    # Open-loop Poisson streams (configs: 4,000 requests).  One sequence of
    # unit-mean exponential gaps (seeded) and one list of requests serve every
    # run: run at rate R, request i arrives at gap_sum[i] / R.  The served arm
    # runs at 0.5x, 0.8x and 1.0x its own closed-loop capacity; both arms run the
    # whole stream at 1.5x the plain-FP64 capacity (the shared comparison: the
    # plain arm saturates there) and its first --stream-requests-low requests at
    # 0.8x the plain capacity (a load the plain arm sustains).
    n_pois = args.stream_requests
    n_low = min(args.stream_requests_low, n_pois)
    served_cap = args.steps * per_step / total  # this rank's closed-loop rate
    gaps = np.random.default_rng([17, rank]).exponential(1.0, max(n_pois, 1))
    gap_sum = np.cumsum(gaps) - gaps[0]

    def served_stream_lat(reqs, arrivals):
        """Latency = result ready - scheduled arrival (a late submit counts)."""
        t_start = time.perf_counter()
        tickets = []
        for (k, g, a), ta in zip(reqs, arrivals):
            d = t_start + ta - time.perf_counter()
            if d > 0:
                time.sleep(d)
            lag = time.perf_counter() - t_start - ta
            tickets.append((srv.submit(k, g.replace(dh="f32"), a), lag))
        lat = []
        for t, lag in tickets:
            r, _ = srv.poll(t, 600000)
            if r.status != 0:
                raise RuntimeError(f"served stream request failed: {r.status}")
            lat.append(r.seconds + lag)
        return time.perf_counter() - t_start, lat

    def plain_stream(reqs, arrivals):
        t_start = time.perf_counter()
        lat = []
        for (k, g, a), ta in zip(reqs, arrivals):
            now = time.perf_counter() - t_start
            if now < ta:
                time.sleep(ta - now)
            plain.solve(k, g, a, args.tol)
            lat.append(time.perf_counter() - t_start - ta)  # queueing + service
        return time.perf_counter() - t_start, lat

    def stream_stats(n, make, lat):
        ms = [1e3 * x for x in lat]
        return {"solves_per_s": n / make, "p50_ms": pct(ms, 50), "p99_ms": pct(ms, 99),
                "max_ms": max(ms)}

    runs = []
    for label, rate, n, both in () if n_pois == 0 else (("0.5x served capacity", 0.5 * served_cap, n_pois, False),
                                 ("0.8x served capacity", 0.8 * served_cap, n_pois, False),
                                 ("1.0x served capacity", 1.0 * served_cap, n_pois, False),
                                 ("1.5x plain capacity", 1.5 * plain_rate, n_pois, True),
                                 ("0.8x plain capacity", 0.8 * plain_rate, n_low, True)):
        arr = gap_sum[:n] / rate
        sm, sl = served_stream_lat(pois_reqs[:n], arr)
        run = {"load": label, "rate_per_s": rate, "requests": n,
               "served": stream_stats(n, sm, sl), "fp64_plain": None}
        if both:
            pm, pl = plain_stream(pois_reqs[:n], arr)
            run["fp64_plain"] = stream_stats(n, pm, pl)
        runs.append(run)
    plain.close()
    # per-kernel device time on the served workload: one step with every
    # phase kernel launched on its own between CUDA events
    # kernel profile in the timed loop's steady state: three steps, each queued
    # before the previous one's results are collected
    srv.profile_begin()
    serve_steps(srv, [[(k, g.replace(dh="f32"), a) for k, g, a in stream.take(per_step)]
                      for _ in range(3)])
    kp = srv.profile_end()
    srv.close()
    if rank != 0:
        ctx.close()
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    n_req = args.steps * per_step
    hbm, peak_kind = peaks()
    t_st = kp.ms_stencil / max(kp.launches_stencil, 1) / 1e3
    t_up = kp.ms_update / max(kp.launches_update, 1) / 1e3
    ach_st = kp.bytes_stencil / max(kp.ms_stencil, 1e-12) / 1e6
    ach_up = kp.bytes_update / max(kp.ms_update, 1e-12) / 1e6
    trf = NCU_TRAFFIC_PER_NODE["stencil_batch"]
    out = {
        "metric": METRIC,
        "value": world * n_req / total,
        "unit": "solves/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": total * 1e3 / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32+f64",
        "data": "synthetic",
        "config": {"workload": "serving stream: 16 trajectories, 300-8000 atoms, grids 33^3-193^3",
                   "requests_per_step": per_step, "tol": args.tol,
                   "solver": "continuous-batching FP32 Jacobi-PCG + FP64 refinement, warm start",
                   "inner_tol": args.inner_tol, "budget_gb": args.budget_gb,
                   "debye_hueckel_sum": "f32", "snapshot_sigma_A": 0.2,
                   "l2": "inputs larger than L2 (2.1 M nodes mean per request, 64 per step)",
                   "parallelism": f"replicas x{world}",
                   "batch_plan": tune if tune is not None else (args.plan or "default {min_planes 32, height 100%, 3 CTAs/SM}")},
        "latency_ms": {"p50": pct([1e3 * x for x in lats], 50), "p99": pct([1e3 * x for x in lats], 99),
                       "note": "steady state: 64 requests per step, the next step queued while "
                               "this one completes; submit -> result"},
        "iterations_mean": float(np.mean(iters)),
        "stencil_node_passes": node_passes,
        "fp64_plain": {"value": plain_rate, "unit": "solves/s",
                       "latency_ms": {"p50": pct([1e3 * x for x in p_lat], 50),
                                      "p99": pct([1e3 * x for x in p_lat], 99)},
                       "requests": n_plain,
                       "note": "one at a time, phi0 = 0, the first requests of the Poisson stream's list"},
        "poisson_stream": {"requests": n_pois, "capacity_per_s": {"served": served_cap,
                                                                   "fp64_plain": plain_rate},
                           "arrivals": ("one seeded sequence of unit-mean exponential gaps and one "
                                        "request list, scaled to each rate; latency = result ready - "
                                        "scheduled arrival"),
                           "sweep": runs},
        "roofline": {"bound": "hbm",
                     "kernel": "k_stencil<float,packed>: batched stencil pass over the active grids",
                     "achieved": ach_st, "peak": hbm, "unit": "GB/s", "frac": ach_st / hbm,
                     "peak_kind": peak_kind,
                     "traffic": None if trf is None else trf[0] * kp.bytes_stencil / BYTES_PER_NODE["stencil"] /
                     max(kp.launches_stencil, 1),
                     "traffic_source": None if trf is None else (
                         f"scaled from {trf[1]}: DRAM bytes per node of two bounded captures on the "
                         f"256-snapshot batch, times the nodes of this run's launches"),
                     "bytes_per_launch": kp.bytes_stencil / max(kp.launches_stencil, 1),
                     "bytes_per_node": BYTES_PER_NODE["stencil"], "launch_ms": t_st * 1e3,
                     "launches": kp.launches_stencil,
                     "measured": "three serving steps in steady state, each kernel between CUDA events",
                     "update_pass": {"achieved": ach_up, "frac": ach_up / hbm,
                                     "bytes_per_node": BYTES_PER_NODE["update"],
                                     "launch_ms": t_up * 1e3, "launches": kp.launches_update},
                     "resid_pass": resid_roofline(kp, alu)},
        "e2e": {"value": world * e2e_steps * per_step / e2e_wall, "unit": "solves/s",
                "h2d_bytes_per_step": int((e2e1[1] - e2e0[1]) / e2e_steps),
                "d2h_bytes_per_step": int((e2e1[2] - e2e0[2]) / e2e_steps),
                "note": "same steps with phi copied to host memory per request"},
        "gpu_launches": int(st1[0] - st0[0]),
        "clocks": clk,
        "alu_rates": alu,
    }
    if not args.no_cpu_baseline:
        sample = [(g, a) for k, g, a in batches[0][:args.cpu_sample]]
        out["cpu_baseline"] = cpu_baseline(sample, "the first requests of the timed serving steps",
                                           args)
    print(json.dumps(out), flush=True)
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()


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
    spec = problem.grid.replace(coef=args.coef, dh=args.dh, periodic=args.periodic,
                                eps_model=args.eps_model)
    if args.eps_model == "harmonic" and args.coef == "packed":
        spec = spec.replace(coef="f32")  # non-binary edges need explicit coefficients
    n_nodes = spec.n
    snaps = snapshots(problem, 8, seed=100 + rank)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    solve_kw = dict(precision="f32_refine", tol=args.tol, inner_tol=args.inner_tol)
    if args.precond == "gmg":  # FP64 CG with an FP32 multigrid V-cycle
        solve_kw = dict(precision="f64", precond="gmg", tol=args.tol)
    with torch.cuda.stream(stream):
        ctx = pb.Context(local, stream=stream.cuda_stream)
        alu = ctx.measure_alu().as_dict()
        g = pb.Grid(ctx, spec, snaps[0])
        # the library's tile-plan autotuner (opt-in: the default plan is the one
        # the committed ncu traffic figure was taken on)
        tune = g.autotune(solve_kw["precision"]).as_dict() if args.autotune else None
        phi = torch.zeros(spec.shape, dtype=torch.float64, device="cuda")
        # warm-up and timed region
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        clocks = ClockSampler(local)
        clocks.start()
        marks = []
        dev_ms, wall_ms, iters, energies = run_loop(g, phi, snaps, args.steps, args.warmup, stream,
                                                    flush, solve_kw, ctx, marks, args.profile_range)
        solve_ms, resid_steps = run_loop.solve_ms, run_loop.resid_steps
        clk = clocks.stop()
        st0, st1 = marks
        # launches and copies of the timed steps (counted by the library)
        launches = int(st1[0] - st0[0])
        h2d = (st1[1] - st0[1]) / float(args.steps)
        d2h = (st1[2] - st0[2]) / float(args.steps)
        total_dev_s = sum(dev_ms) / 1e3
        total_wall_s = sum(wall_ms) / 1e3
        total_dev_s, total_wall_s = max_over_ranks([total_dev_s, total_wall_s], world)
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
        # the multigrid path has no kernel profile: its roofline is that of the
        # Jacobi-PCG passes on the same grid, measured the same way
        prof = g.solve(phi, profile=True, **(solve_kw if args.precond != "gmg" else
                                             dict(precision="f32_refine", tol=args.tol,
                                                  inner_tol=args.inner_tol)))
    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    hbm, peak_kind = peaks()
    t_st = prof.ms_stencil / max(prof.n_stencil, 1) / 1e3
    t_up = prof.ms_update / max(prof.n_update, 1) / 1e3
    bpn = bytes_per_node(spec.coef)
    ach_st = bpn["stencil"] * n_nodes / t_st / 1e9
    ach_up = bpn["update"] * n_nodes / t_up / 1e9
    trf = NCU_TRAFFIC_PER_NODE["stencil_grid"]
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
                   "solver": ("gmg-pcg: fp64 cg, fp32 multigrid v-cycle" if args.precond == "gmg"
                              else "jacobi-pcg fp32 inner + fp64 refinement"),
                   "inner_tol": args.inner_tol, "coef": args.coef,
                   "boundary": "periodic" if args.periodic else "Debye-Hueckel",
                   "eps_model": args.eps_model, "coef_storage": spec.coef,
                   "debye_hueckel_sum": args.dh,
                   "snapshot_sigma_A": SNAPSHOT_SIGMA,
                   "l2": "256 MB buffer written between timed steps",
                   "parallelism": f"replicas x{world}",
                   "tile_autotune": tune},
        "latency_ms": {"p50": pct(dev_ms, 50), "p99": pct(dev_ms, 99)},
        "iterations_mean": float(np.mean(iters)),
        "grid_point_iters_per_s": float(np.mean(iters)) * n_nodes * world * args.steps / total_dev_s,
        "fp64_plain": {"value": k64 / (sum(d64) / 1e3), "unit": "solves/s",
                       "latency_ms": {"p50": pct(d64, 50), "p99": pct(d64, 99)},
                       "iterations_mean": float(np.mean(it64)), "steps": k64},
        "roofline": {"bound": "hbm", "kernel": f"k_stencil<float,{spec.coef}> (CG stencil pass)",
                     "measured_on": ("the Jacobi-PCG passes of the same grid (the multigrid solve has no "
                                     "kernel profile)" if args.precond == "gmg" else "the timed solver"),
                     "achieved": ach_st, "peak": hbm, "unit": "GB/s", "frac": ach_st / hbm,
                     "peak_kind": peak_kind,
                     "traffic": (None if trf is None or spec.coef != "packed" or spec.periodic or tune
                                 or spec.nx != 257 else trf[0] * n_nodes),
                     "traffic_source": (None if trf is None or spec.coef != "packed" or spec.periodic or tune
                                        or spec.nx != 257 else trf[1]),
                     "bytes_per_node": bpn["stencil"], "launch_ms": t_st * 1e3,
                     "update_pass": {"achieved": ach_up, "frac": ach_up / hbm,
                                     "bytes_per_node": bpn["update"],
                                     "launch_ms": t_up * 1e3},
                     "cg_iteration_in_graph": cg_iteration_in_graph(
                         solve_ms, resid_steps, iters, prof, n_nodes, bpn, hbm, args.precond),
                     "resid_pass": resid_roofline(SimpleNamespace(
                         ms_resid=prof.ms_resid, launches_resid=prof.n_resid,
                         bytes_resid=37.0 * n_nodes * prof.n_resid), alu)},
        "e2e": {"value": world * args.steps / total_wall_s, "unit": "solves/s",
                "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                "latency_ms": {"p50": pct(wall_ms, 50), "p99": pct(wall_ms, 99)}},
        "gpu_launches": launches,
        "clocks": clk,
    }
    if not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline([(problem.grid, snaps[0])], f"one {problem.name} snapshot",
                                           args)
    print(json.dumps(out), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def oracle_pool_run(jobs, tol, procs, warmup_jobs=()):
    """Complete FP64 oracle solves (setup with the full Debye-Hueckel sum,
    Jacobi-PCG from phi0 = 0 to `tol`, energy) of independent (grid, atoms)
    jobs, run side by side in `procs` spawned worker processes (the oracle's
    arithmetic stays single-threaded).  The warm-up jobs run first, untimed.
    Returns (wall seconds of the timed jobs, their per-job results)."""
    from oracle import pool as opool
    import multiprocessing as mp
    with mp.get_context("spawn").Pool(procs) as p:
        p.map(_noop, range(procs))  # workers started and imported before any timing
        if warmup_jobs:
            p.map(opool._solve_one, [(g, a, tol, False, None) for g, a in warmup_jobs], chunksize=1)
        t0 = time.perf_counter()
        res = p.map(opool._solve_one, [(g, a, tol, False, None) for g, a in jobs], chunksize=1)
        wall = time.perf_counter() - t0
    bad = [r["status"] for r in res if r["status"] != 0]
    if bad:
        raise RuntimeError(f"oracle solves failed: {bad[:5]}")
    return wall, res


def _noop(i):
    import oracle  # noqa: F401  (the worker's import, outside the timed region)
    return i


def cpu_baseline(jobs, label, args):
    """The FP64 oracle on the host cores: complete solves of a bounded sample
    of the workload's requests, one per worker process; value = solves / wall."""
    from oracle import pool as opool
    import oracle
    oracle.build()
    procs = max(1, min(opool.host_cores(), len(jobs)))
    wall, res = oracle_pool_run(jobs, args.tol, procs)
    return {"value": len(jobs) / wall, "unit": "solves/s", "cores": procs, "kind": "oracle",
            "sample": (f"{len(jobs)} complete FP64 oracle solves ({label}; full setup with the "
                       f"Debye-Hueckel sum, Jacobi-PCG from phi0 = 0 to {args.tol:g}, energy), one "
                       f"per worker process on {procs} host cores, {wall:.1f} s wall"),
            "solve_seconds": [round(r["seconds"], 3) for r in res],
            "iterations": [r["iters"] for r in res],
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


def reference_jobs(args, n):
    """The first n steps of the workload as lists of (grid, atoms) oracle jobs
    (the oracle's Debye-Hueckel sum is FP64 whatever the GPU arm's setting)."""
    if args.workload == SERVING:  # the serving stream's first requests, in order
        return "serving stream: 16 trajectories, 300-8000 atoms, grids 33^3-193^3", \
            [[(g, a)] for _, g, a in Stream(seed=5, req_seed=99).take(n)]
    if args.workload == BATCH:
        return ("batch of 256 snapshots: 1,000-atom cluster, sigma 0.3 A, grids 49^3-97^3, "
                "one snapshot per step"), [[(p.grid, p.atoms)] for p in inputs.snapshot_batch()[:n]]
    problem = WORKLOADS[args.workload]()
    import oracle
    if args.workload == SOLVATION:  # the solvated and the reference system of a snapshot
        ref_grid = oracle.reference_grid(problem.grid)
        return "solvation energy of 129^3 globule snapshots (2,500 atoms)", \
            [[(problem.grid, a), (ref_grid, a)] for a in snapshots(problem, n, seed=100)]
    return problem.name, [[(problem.grid, a)] for a in snapshots(problem, n, seed=100)]


def run_reference(args):
    """The FP64 CPU oracle as the reference arm (rank 0 only): each step is one
    request of the workload (two solves for a solvation energy), solved
    completely; the steps run side by side in spawned worker processes on the
    host cores.  value = timed steps / wall time of the timed steps."""
    rank, world, _ = env_rank()
    if rank != 0:
        return
    import oracle
    from oracle import pool as opool
    oracle.build()
    name, steps = reference_jobs(args, args.warmup + args.steps)
    warm = [j for st in steps[:args.warmup] for j in st]
    timed = steps[args.warmup:]
    jobs = [j for st in timed for j in st]
    procs = max(1, min(opool.host_cores(), len(jobs)))
    wall, res = oracle_pool_run(jobs, args.tol, procs, warmup_jobs=warm)
    per_step, k = [], 0
    for st in timed:
        per_step.append(sum(r["seconds"] for r in res[k:k + len(st)]))
        k += len(st)
    val = args.steps / wall
    unit = "energies/s" if args.workload == SOLVATION else "solves/s"
    print(json.dumps({
        "impl": "reference",
        "metric": {BATCH: BATCH_METRIC, SOLVATION: SOLVATION_METRIC}.get(args.workload, METRIC),
        "value": val, "unit": unit, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": wall * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": name, "tol": args.tol,
                   "solver": "oracle FP64 Jacobi-PCG from phi0 = 0 (complete solves)"},
        "latency_ms": {"p50": pct([t * 1e3 for t in per_step], 50),
                       "p99": pct([t * 1e3 for t in per_step], 99),
                       "note": "one request's solve time in its worker"},
        "iterations_mean": float(np.mean([r["iters"] for r in res])),
        "cpu_baseline": {"value": val, "unit": unit, "cores": procs, "kind": "oracle",
                         "sample": (f"{args.steps} steps of the workload, each solved completely by "
                                    f"the oracle (full setup with the Debye-Hueckel sum, Jacobi-PCG to "
                                    f"{args.tol:g}, energy), side by side in {procs} worker processes "
                                    f"(after {args.warmup} untimed steps); {wall:.1f} s wall"),
                         "cpu": platform_cpu()},
        "e2e": {"value": val, "unit": unit, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }), flush=True)


# --------------------------------------------------------------------------- solvation energy

def run_solvation(args):
    """The solvation-energy pipeline (pb_solvation_energy) on snapshots of the
    129^3 globule: per step, setup + solve + energy of the solvated system and
    of the reference system (eps_in everywhere, no salt), one grid at a time."""
    import torch
    from paper_1704_02745_gb300 import pb
    from paper_1704_02745_gb300 import build as pbbuild

    rank, world, local = env_rank()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    pbbuild.build()
    torch.cuda.set_device(local)
    problem = inputs.globule_129()
    spec = problem.grid.replace(dh=args.dh)
    snaps = snapshots(problem, 8, seed=100 + rank)
    ctx = pb.Context(local)
    phi = torch.zeros(spec.shape, dtype=torch.float64, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    kw = dict(precision="f32_refine", tol=args.tol, inner_tol=args.inner_tol)
    times, outs = [], []
    for i in range(args.warmup + args.steps):
        if i == args.warmup:
            if world > 1:
                torch.distributed.barrier()
            st0 = ctx.stats()
            clocks = ClockSampler(local)
            clocks.start()
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = ctx.solvation(spec, snaps[i % len(snaps)], phi, **kw)
        torch.cuda.synchronize()
        if i >= args.warmup:
            times.append(time.perf_counter() - t0)
            outs.append(out)
    clk = clocks.stop()
    st1 = ctx.stats()
    total = sum(times)
    total = max_over_ranks([total], world)[0]
    if rank == 0:
        print(json.dumps({
            "metric": SOLVATION_METRIC, "value": world * args.steps / total, "unit": "energies/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": total * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": "solvation energy of 129^3 globule snapshots (2,500 atoms)",
                       "tol": args.tol, "inner_tol": args.inner_tol, "debye_hueckel_sum": args.dh,
                       "l2": "256 MB buffer written between timed steps",
                       "parallelism": f"replicas x{world}"},
            "dG_kcal": [o.dG for o in outs[:3]],
            "iterations_mean": {"solvated": float(np.mean([o.solv.iterations for o in outs])),
                                "reference": float(np.mean([o.ref.iterations for o in outs]))},
            "e2e": {"value": world * args.steps / total, "unit": "energies/s",
                    "h2d_bytes_per_step": int((st1[1] - st0[1]) / args.steps),
                    "d2h_bytes_per_step": int((st1[2] - st0[2]) / args.steps),
                    "note": "host atoms in, energies out: the call is end to end"},
            "gpu_launches": int(st1[0] - st0[0]), "clocks": clk,
        }), flush=True)
    ctx.close()


# --------------------------------------------------------------------------- batch of snapshots

def run_batch(args):
    """256 snapshots of one 1,000-atom cluster (sigma 0.3 A), grids 49^3-97^3,
    all submitted to one server at once: a step is the whole batch, cold
    started (phi0 = 0), FP32 Jacobi-PCG + FP64 refinement to the tolerance."""
    import torch
    from paper_1704_02745_gb300 import pb
    from paper_1704_02745_gb300 import build as pbbuild

    rank, world, local = env_rank()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    pbbuild.build()
    torch.cuda.set_device(local)
    snaps = inputs.snapshot_batch(seed=4 + 1000 * rank)
    reqs = [(s, p.grid.replace(dh="f32"), p.atoms) for s, p in enumerate(snaps)]
    ctx = pb.Context(local)
    srv = pb.Server(ctx, int(args.budget_gb * (1 << 30)), precision="f32_refine", tol=args.tol,
                    inner_tol=args.inner_tol, warm_start=False)
    if args.plan:
        srv.set_plan(*[int(v) for v in args.plan.split(",")])
    for _ in range(args.warmup):
        serve_batch(srv, reqs)
    tune, default_rate = None, None
    if args.autotune:  # the default plan timed, then the batch tuned on a live step
        if world > 1:
            torch.distributed.barrier()
        t_def, _, _ = serve_steps(srv, [reqs] * args.steps)
        default_rate = len(reqs) * args.steps / max_over_ranks([t_def], world)[0]
        tickets = [srv.submit(k, g, a) for k, g, a in reqs]
        tune = srv.autotune(600000).as_dict()
        for t in tickets:
            srv.poll(t, 600000)
        serve_batch(srv, reqs)  # one more warm-up step under the kept plan
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    st0 = ctx.stats()
    clocks = ClockSampler(local)
    clocks.start()
    if args.profile_range:
        torch.cuda.profiler.start()
    total, lats, res = serve_steps(srv, [reqs] * args.steps)
    if args.profile_range:
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
    clk = clocks.stop()
    st1 = ctx.stats()
    bad = [r.status for r in res if r.status != 0]
    if bad:
        raise RuntimeError(f"batch requests failed: {bad[:5]}")
    total = max_over_ranks([total], world)[0]
    prewarm_pinned(pb, [reqs])
    e0 = ctx.stats()
    e2e_wall, _, _ = serve_steps(srv, [reqs] * max(1, args.steps // 2), want_phi=True)
    e1 = ctx.stats()
    e2e_steps = max(1, args.steps // 2)
    torch.cuda.synchronize()
    if args.ncu_window:  # the server is idle: the first stencil launches inside are profiled ones
        torch.cuda.profiler.start()
    srv.profile_begin()
    serve_steps(srv, [reqs] * 3)  # steady state, as in the timed loop
    kp = srv.profile_end()
    if args.ncu_window:
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
    srv.close()
    if rank != 0:
        ctx.close()
        return
    hbm, peak_kind = peaks()
    nodes = sum(p.grid.n for p in snaps)
    iters = [r.info.iterations for r in res]
    ach_st = kp.bytes_stencil / max(kp.ms_stencil, 1e-12) / 1e6
    ach_up = kp.bytes_update / max(kp.ms_update, 1e-12) / 1e6
    out = {
        "metric": BATCH_METRIC,
        "value": world * len(reqs) * args.steps / total, "unit": "solves/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
        "data": "synthetic",
        "config": {"workload": "batch of 256 snapshots: 1,000-atom cluster, sigma 0.3 A, "
                               "grids 49^3-97^3, one server batch",
                   "nodes_per_step": nodes, "tol": args.tol, "inner_tol": args.inner_tol,
                   "debye_hueckel_sum": "f32", "l2": f"inputs larger than L2 ({nodes / 1e6:.0f} M nodes)",
                   "parallelism": f"replicas x{world}",
                   "batch_plan": tune if tune is not None else (args.plan or "default {min_planes 32, height 100%, 3 CTAs/SM}")},
        "default_plan_solves_per_s": None if default_rate is None else world * default_rate,
        "iterations_mean": float(np.mean(iters)),
        "grid_point_iters_per_s": world * args.steps * sum(
            p.grid.n * r.info.iterations for p, r in zip(snaps * args.steps, res)) / args.steps / total,
        "roofline": {"bound": "hbm", "kernel": "k_stencil<float,packed>: batched stencil pass",
                     "achieved": ach_st, "peak": hbm, "unit": "GB/s", "frac": ach_st / hbm,
                     "peak_kind": peak_kind,
                     "traffic": (None if NCU_TRAFFIC_PER_NODE["stencil_batch"] is None else
                                 NCU_TRAFFIC_PER_NODE["stencil_batch"][0] * kp.bytes_stencil /
                                 BYTES_PER_NODE["stencil"] / max(kp.launches_stencil, 1)),
                     "traffic_source": (None if NCU_TRAFFIC_PER_NODE["stencil_batch"] is None else
                                        f"scaled from {NCU_TRAFFIC_PER_NODE['stencil_batch'][1]} "
                                        f"(bounded captures of this workload's kernel)"),
                     "bytes_per_node": BYTES_PER_NODE["stencil"],
                     "launch_ms": kp.ms_stencil / max(kp.launches_stencil, 1),
                     "launches": kp.launches_stencil,
                     "update_pass": {"achieved": ach_up, "frac": ach_up / hbm,
                                     "launch_ms": kp.ms_update / max(kp.launches_update, 1),
                                     "launches": kp.launches_update},
                     "resid_pass": {"launch_ms": kp.ms_resid / max(kp.launches_resid, 1),
                                    "launches": kp.launches_resid},
                     "capture_window": {
                         "first_bytes_stencil": list(kp.first_bytes_stencil)[:kp.first_stencil],
                         "first_bytes_update": list(kp.first_bytes_update)[:kp.first_update],
                         "note": ("algorithmic bytes of the first stencil / update launches of the "
                                  "profiled steps (--ncu-window brackets them for a counter capture)")}},
        "e2e": {"value": world * len(reqs) * e2e_steps / e2e_wall, "unit": "solves/s",
                "h2d_bytes_per_step": int((e1[1] - e0[1]) / e2e_steps),
                "d2h_bytes_per_step": int((e1[2] - e0[2]) / e2e_steps),
                "note": "same steps with phi copied to host memory per request"},
        "gpu_launches": int(st1[0] - st0[0]),
        "clocks": clk,
    }
    print(json.dumps(out), flush=True)
    ctx.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=SERVING, choices=sorted(WORKLOADS))
    ap.add_argument("--batch", type=int, default=64, help="serving: requests per step")
    ap.add_argument("--budget-gb", type=float, default=120.0, help="serving: device-memory budget")
    ap.add_argument("--stream-requests", type=int, default=4000,
                    help="serving: requests of the open-loop Poisson stream")
    ap.add_argument("--stream-requests-low", type=int, default=1000,
                    help="serving: requests of the stream at 0.8x the plain-FP64 capacity (both arms)")
    ap.add_argument("--coef", default="packed", choices=["packed", "f32", "bf16"])
    ap.add_argument("--tol", type=float, default=1e-6)
    ap.add_argument("--inner-tol", type=float, default=None,
                    help="inner FP32 tolerance of the refinement (default: 1e-4 for the warm-started "
                         "serving stream and the batch, 1e-3 for cold single grids)")
    ap.add_argument("--cpu-sample", type=int, default=8,
                    help="serving: requests the oracle solves completely for cpu_baseline")
    ap.add_argument("--dh", default="f32", choices=["f32", "f64"],
                    help="precision of the Debye-Hueckel boundary sum in the grid setup")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--precond", default="jacobi", choices=["jacobi", "gmg"],
                    help="single-grid workloads: Jacobi-PCG with refinement, or multigrid PCG")
    ap.add_argument("--eps-model", default="midpoint", choices=["midpoint", "harmonic"],
                    help="single-grid workloads: boundary dielectric (harmonic: weighted harmonic average)")
    ap.add_argument("--periodic", action="store_true",
                    help="single-grid workloads: periodic boundary instead of Debye-Hueckel")
    ap.add_argument("--ncu-window", action="store_true",
                    help="batch256: bracket the kernel-profile steps with cudaProfilerStart/Stop "
                         "(for a bounded counter capture of their first launches)")
    ap.add_argument("--profile-range", action="store_true",
                    help="bracket the timed steps with cudaProfilerStart/Stop "
                         "(for ncu --profile-from-start off)")
    ap.add_argument("--autotune", action="store_true",
                    help="single grids: run the library's tile-plan autotuner before timing; batch256: "
                         "time the default plan, tune the batch, then time the tuned plan")
    ap.add_argument("--no-autotune", action="store_true",
                    help="serving: keep the default batch plan (no tuning during the warm-up)")
    ap.add_argument("--plan", default=None,
                    help="serving/batch256: fixed batch plan 'min_planes,height_pct,occupancy' "
                         "(skips the tuning)")
    ap.add_argument("--quick", action="store_true",
                    help="timed loop only (no FP64 comparator, profiled solve or CPU baseline)")
    args = ap.parse_args()
    if args.inner_tol is None:
        args.inner_tol = 1e-4 if args.workload in (SERVING, BATCH) else 1e-3
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == SERVING:
        run_serving(args)
    elif args.workload == BATCH:
        run_batch(args)
    elif args.workload == SOLVATION:
        run_solvation(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
