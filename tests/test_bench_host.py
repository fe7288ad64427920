"""Host-side arithmetic of bench.py (CPU): the FP64 residual pass's ALU
roofline, the in-graph CG iteration, and the reference arm's job lists."""
import os
import sys
from types import SimpleNamespace

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_resid_roofline_against_the_measured_fp64_rate():
    # 10 launches of 37e9 algorithmic bytes (1e9 nodes each) in 100 ms in all
    kp = SimpleNamespace(bytes_resid=37e9 * 10, ms_resid=100.0, launches_resid=10)
    r = bench.resid_roofline(kp, {"fp64_fma_per_s": 0.6e12})
    assert r["bound"] == "alu" and r["launch_ms"] == pytest.approx(10.0)
    nodes = 1e10
    assert r["achieved"] == pytest.approx(bench.RESID_FP64_OPS_PER_NODE * nodes / 0.1 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / 0.6)
    assert r["achieved_gbs"] == pytest.approx(37e10 / 0.1 / 1e9)
    # without a measured rate there is no fraction
    assert "frac" not in bench.resid_roofline(kp, None)


def test_cg_iteration_in_graph_subtracts_the_residual_passes():
    prof = SimpleNamespace(ms_resid=3.0, n_resid=3)  # 1 ms a residual pass
    bpn = {"stencil": 25, "update": 13}
    out = bench.cg_iteration_in_graph([42.0, 44.0], [4, 4], [300, 320], prof, 1_000_000, bpn, 6000.0,
                                      "jacobi")
    ms = ((42.0 - 4.0) + (44.0 - 4.0)) / 620
    assert out["ms"] == pytest.approx(ms)
    assert out["bytes_per_node"] == 38
    assert out["achieved"] == pytest.approx(38e6 / (ms * 1e-3) / 1e9)
    assert out["frac"] == pytest.approx(out["achieved"] / 6000.0)
    assert bench.cg_iteration_in_graph([1.0], [1], [10], prof, 1, bpn, 1.0, "gmg") is None
    assert bench.cg_iteration_in_graph([], [], [], prof, 1, bpn, 1.0, "jacobi") is None


def test_reference_jobs_follow_the_workload():
    args = SimpleNamespace(workload="globule33", tol=1e-6)
    name, steps = bench.reference_jobs(args, 3)
    assert len(steps) == 3 and all(len(s) == 1 for s in steps)
    g0, a0 = steps[0][0]
    assert (g0.nx, g0.ny, g0.nz) == (33, 33, 33) and a0.n == 200
    # steps are distinct snapshots of the same problem
    assert (steps[0][0][1].xyz != steps[1][0][1].xyz).any()
    args = SimpleNamespace(workload="solvation129", tol=1e-6)
    _, steps = bench.reference_jobs(args, 2)
    assert all(len(s) == 2 for s in steps)  # the solvated and the reference system
    solv, ref = steps[0]
    assert ref[0].eps_out == ref[0].eps_in and ref[0].ionic_strength == 0.0
    assert solv[1] is ref[1]
    args = SimpleNamespace(workload="serving", tol=1e-6)
    name, steps = bench.reference_jobs(args, 4)
    # the serving stream's first requests, in the GPU arm's order
    want = bench.Stream(seed=5, req_seed=99).take(4)
    for st, (_, g, a) in zip(steps, want):
        assert st[0][0] == g and (st[0][1].xyz == a.xyz).all()
