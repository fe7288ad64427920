"""Failure paths on the GPU, made to happen on purpose without faulting,
trapping or hanging anything.

A separately built copy of the library (-DPB_FAULT_TEST; the product library
has no such hooks) adds two test switches:

* pb_test_abandon_waits(n): the next n first-plane TMA stage waits give up at
  once, exactly as a wait that ran out of its ~50 ms clock budget would.  The
  copies are issued and land as usual, and the kernel's exit path waits for
  every one of them before the CTA leaves.  Expected: the solve (or served
  request) reports PB_ERR_TIMEOUT, and the next solve on the same context,
  grid or server is clean and matches the oracle.
* pb_test_fail_allocs(n): the next n device allocations fail.  Expected: a
  served request whose grid cannot be allocated fails with PB_ERR_OOM, and the
  server goes on serving.

The copy runs in a process of its own (PB_LIBRARY names it), so the product
library of this process is never mixed with it.
"""
import json
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r'''
import ctypes, json, sys
import numpy as np
import torch
sys.path.insert(0, sys.argv[1])
import oracle
from paper_1704_02745_gb300 import inputs, pb

lib = pb.load()
lib.pb_test_abandon_waits.argtypes = [ctypes.c_int]
lib.pb_test_fail_allocs.argtypes = [ctypes.c_int]
p = inputs.small_33()
s = oracle.setup(p.grid, p.atoms)
ref = oracle.pcg(s, tol=1e-10)
e_ref = oracle.energy(s, ref.phi)
q = inputs.random_small(12, 29, 23, 19, n_atoms=30)
sq = oracle.setup(q.grid, q.atoms)
eq_ref = oracle.energy(sq, oracle.pcg(sq, tol=1e-10).phi)
out = {}
rel = lambda e, r: abs(e - r) / abs(r)
torch.cuda.set_device(0)
with pb.Context(0) as ctx, pb.Grid(ctx, p.grid, p.atoms) as g:
    for prec in ("f32_refine", "f64"):
        phi = torch.zeros(p.grid.shape, dtype=torch.float64, device="cuda")
        lib.pb_test_abandon_waits(1)
        info = g.solve(phi, check=False, precision=prec, tol=1e-9)
        out[prec + "_fault"] = info.status
        lib.pb_test_abandon_waits(0)
        phi.zero_()
        info = g.solve(phi, check=False, precision=prec, tol=1e-9)
        out[prec + "_clean"] = [info.status, rel(g.energy(phi), e_ref)]
    with pb.Server(ctx, 1 << 30, tol=1e-9, inner_tol=1e-4, warm_start=False) as srv:
        r, _ = srv.poll(srv.submit(0, p.grid, p.atoms), 60000)
        out["served_first"] = [r.status, rel(r.energy, e_ref)]
        lib.pb_test_abandon_waits(1)
        r, _ = srv.poll(srv.submit(0, p.grid, p.atoms), 60000)
        out["served_fault"] = r.status
        lib.pb_test_abandon_waits(0)
        r, _ = srv.poll(srv.submit(0, p.grid, p.atoms), 60000)
        out["served_after_fault"] = [r.status, rel(r.energy, e_ref)]
        lib.pb_test_fail_allocs(1000)
        r, _ = srv.poll(srv.submit(7, q.grid, q.atoms), 60000)
        out["served_oom"] = r.status
        lib.pb_test_fail_allocs(0)
        r, _ = srv.poll(srv.submit(7, q.grid, q.atoms), 60000)
        out["served_after_oom"] = [r.status, rel(r.energy, eq_ref)]
        r, _ = srv.poll(srv.submit(0, p.grid, p.atoms), 60000)
        out["served_last"] = [r.status, rel(r.energy, e_ref)]
print("RESULT " + json.dumps(out))
'''


def test_timeouts_and_allocation_failures_report_and_recover():
    from paper_1704_02745_gb300 import build
    lib = build.build_fault_test()
    env = dict(os.environ, PB_LIBRARY=lib)
    r = subprocess.run([sys.executable, "-c", SCRIPT, ROOT], env=env, capture_output=True,
                       text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    line = [ln for ln in r.stdout.splitlines() if ln.startswith("RESULT ")][-1]
    out = json.loads(line[len("RESULT "):])
    TIMEOUT, OOM = 7, 2
    for prec in ("f32_refine", "f64"):
        assert out[prec + "_fault"] == TIMEOUT, out
        st, err = out[prec + "_clean"]
        assert st == 0 and err <= 1e-7, out
    assert out["served_first"][0] == 0 and out["served_first"][1] <= 1e-7, out
    assert out["served_fault"] == TIMEOUT, out
    for k in ("served_after_fault", "served_after_oom", "served_last"):
        assert out[k][0] == 0 and out[k][1] <= 1e-7, (k, out)
    assert out["served_oom"] == OOM, out
