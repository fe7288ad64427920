"""The continuous-batching server (pb_server_* / pb_batch_*) on the GPU:
results against the FP64 oracle, the same result alone and in a mix (bitwise),
warm start along a trajectory, admission under a memory budget, errors."""
import numpy as np
import pytest

import oracle
from paper_1704_02745_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pbm():
    from paper_1704_02745_gb300 import build, pb
    build.build()
    pb.load()
    return pb


@pytest.fixture(scope="module")
def ctx(pbm):
    c = pbm.Context(0)
    yield c
    c.close()


GB = 1 << 30


def mixed_requests(n=10, seed=3):
    rng = np.random.default_rng(seed)
    out = []
    for t in range(n):
        nx, ny, nz = (int(v) for v in rng.integers(17, 61, 3))
        out.append(inputs.random_small(100 + t, nx, ny, nz, n_atoms=int(rng.integers(5, 60))))
    return out


def run_all(srv, items):
    tickets = [srv.submit(tid, p.grid, p.atoms, want_phi=True) for tid, p in items]
    return [srv.poll(t, 60000) for t in tickets]


def test_results_match_oracle(pbm, ctx):
    probs = [inputs.small_33(seed=s) for s in (1, 2)] + mixed_requests(3)
    with pbm.Server(ctx, 8 * GB, tol=1e-9, inner_tol=1e-4, warm_start=False) as srv:
        res = run_all(srv, list(enumerate(probs)))
    for p, (r, phi) in zip(probs, res):
        assert r.status == 0, r.info.as_dict()
        s = oracle.setup(p.grid, p.atoms)
        ref = oracle.pcg(s, tol=1e-11)
        e_ref = oracle.energy(s, ref.phi)
        assert abs(r.energy - e_ref) <= 1e-7 * abs(e_ref)
        assert np.max(np.abs(phi - ref.phi)) <= 1e-7 * np.max(np.abs(ref.phi))
        assert r.info.relres_true < 1e-9


def test_same_result_alone_and_in_a_mix(pbm, ctx):
    probe = inputs.random_small(55, 41, 37, 29, n_atoms=30)
    with pbm.Server(ctx, 8 * GB, warm_start=False) as srv:
        alone, _ = srv.poll(srv.submit(0, probe.grid, probe.atoms), 60000)
    others = mixed_requests(12, seed=9)
    with pbm.Server(ctx, 8 * GB, warm_start=False) as srv:
        items = [(i + 1, p) for i, p in enumerate(others[:6])] + [(0, probe)] + \
                [(i + 20, p) for i, p in enumerate(others[6:])]
        res = run_all(srv, items)
    mixed = res[6][0]
    assert alone.status == 0 and mixed.status == 0
    assert mixed.energy == alone.energy  # bitwise
    assert mixed.info.iterations == alone.info.iterations
    assert mixed.info.relres_true == alone.info.relres_true


def test_warm_start_along_a_trajectory(pbm, ctx):
    base = inputs.small_33()
    rng = np.random.default_rng(4)
    snaps = []
    a = base.atoms.copy()
    for _ in range(4):
        a = a.copy()
        a.xyz = a.xyz + rng.normal(0, 0.05, a.xyz.shape)
        snaps.append(a)
    with pbm.Server(ctx, 8 * GB, tol=1e-6) as srv:
        res = []
        for sn in snaps:  # one at a time: each snapshot starts from the last solution
            res.append(srv.poll(srv.submit(42, base.grid, sn), 60000)[0])
    with pbm.Server(ctx, 8 * GB, tol=1e-6, warm_start=False) as srv:
        cold = [srv.poll(srv.submit(43, base.grid, sn), 60000)[0] for sn in snaps]
    assert [r.warm_started for r in res] == [0, 1, 1, 1]
    assert [r.warm_started for r in cold] == [0, 0, 0, 0]
    for sn, r in zip(snaps, res):
        s = oracle.setup(base.grid, sn)
        e_ref = oracle.energy(s, oracle.pcg(s, tol=1e-10).phi)
        assert r.status == 0 and abs(r.energy - e_ref) <= 1e-6 * abs(e_ref)
        assert r.info.relres_true < 1e-6
    assert sum(r.info.iterations for r in res[1:]) < sum(r.info.iterations for r in cold[1:])


def test_budget_admission_and_eviction(pbm, ctx):
    probs = mixed_requests(6, seed=11)
    need = max(pbm.pb_grid_bytes(pbm.grid_desc(p.grid)) for p in probs)
    with pbm.Server(ctx, need + (1 << 20), warm_start=False) as srv:
        res = run_all(srv, list(enumerate(probs)))
        st = srv.stats()
    assert all(r.status == 0 for r, _ in res)
    assert st["resident"] <= 2 and st["bytes"] <= need + (1 << 20)
    assert st["completed"] == len(probs)


def test_request_errors(pbm, ctx):
    p = inputs.random_small(3, 12, 12, 12, n_atoms=4)
    bad = p.atoms.copy()
    bad.xyz[0, 1] = p.grid.origin[1] + 20.0  # trilinear cell outside: found on the device
    nan = p.atoms.copy()
    nan.r[1] = np.nan  # rejected on the host at submit
    with pbm.Server(ctx, 4 * GB) as srv:
        r, _ = srv.poll(srv.submit(1, p.grid, bad), 60000)
        assert r.status == pbm.PB_ERR_ARG
        with pytest.raises(pbm.PbError) as ei:
            srv.submit(2, p.grid, nan)
        assert ei.value.status == pbm.PB_ERR_ARG
        st, _ = pbm.pb_batch_poll(srv.handle, 987654, 0)
        assert st == pbm.PB_ERR_NOT_FOUND
        ok, _ = srv.poll(srv.submit(3, p.grid, p.atoms), 60000)
        assert ok.status == 0
        st, _ = pbm.pb_batch_poll(srv.handle, 987654, 10)
        assert st == pbm.PB_ERR_NOT_FOUND
    with pytest.raises(pbm.PbError):
        with pbm.Server(ctx, 1 << 20) as small:  # a grid larger than the budget
            small.submit(1, inputs.small_33().grid, inputs.small_33().atoms)


def test_fp64_server(pbm, ctx):
    p = inputs.small_33()
    s = oracle.setup(p.grid, p.atoms)
    ref = oracle.pcg(s, tol=1e-10)
    with pbm.Server(ctx, 4 * GB, precision="f64", tol=1e-10, warm_start=False) as srv:
        r, phi = srv.poll(srv.submit(1, p.grid, p.atoms, want_phi=True), 60000)
    assert r.status == 0
    assert np.max(np.abs(phi - ref.phi)) <= 1e-8 * np.max(np.abs(ref.phi))
    assert abs(r.info.iterations - ref.iters) <= max(1, 0.02 * ref.iters)


def test_kernel_profile(pbm, ctx):
    probs = mixed_requests(4, seed=21)
    with pbm.Server(ctx, 8 * GB, warm_start=False) as srv:
        srv.profile_begin()
        res = run_all(srv, list(enumerate(probs)))
        kp = srv.profile_end()
    assert all(r.status == 0 for r, _ in res)
    assert kp.launches_stencil > 0 and kp.launches_update > 0
    assert kp.bytes_stencil > 0 and kp.ms_stencil > 0 and kp.ms_update > 0
    assert kp.launches_resid > 0 and kp.ms_resid > 0 and kp.bytes_resid > 0
    # every update launch covers at most all grids, each at 13 B per node
    total_nodes = sum(p.grid.n for p in probs)
    assert kp.bytes_update <= kp.launches_update * 13 * total_nodes


def test_zero_charge_request(pbm, ctx):
    p = inputs.random_small(7, 21, 19, 17, n_atoms=6)
    a = p.atoms.copy()
    a.q = np.zeros_like(a.q)  # b = 0: the solution is phi = 0
    phi = np.ones(p.grid.shape)
    with pbm.Server(ctx, 4 * GB) as srv:
        r, _ = srv.poll(srv.submit(5, p.grid, a, phi_out=phi), 60000)
        ok, phi2 = srv.poll(srv.submit(5, p.grid, p.atoms, want_phi=True), 60000)
    assert r.status == 0 and r.energy == 0.0 and r.info.iterations == 0
    assert not phi.any()
    assert ok.status == 0 and np.abs(phi2).max() > 0


def test_phi_into_pageable_and_pinned_memory(pbm, ctx):
    """phi_out in pageable memory (pinned staging, host copy) and in page-locked
    memory (direct device copy on the copy stream) receive the same phi, bit
    for bit, whichever finishes in which round."""
    probs = mixed_requests(6, seed=21)
    with pbm.Server(ctx, 8 * GB, warm_start=False) as srv:
        outs, tickets = [], []
        for i, p in enumerate(probs):
            for pinned in (False, True):
                out = pbm.pinned_empty(tuple(p.grid.shape)) if pinned else \
                    np.empty(p.grid.shape, dtype=np.float64)
                out.fill(np.nan)
                tickets.append(srv.submit(2 * i + int(pinned), p.grid, p.atoms, phi_out=out))
                outs.append(out)
        res = [srv.poll(t, 60000) for t in tickets]
    for i in range(len(probs)):
        (r0, phi0), (r1, phi1) = res[2 * i], res[2 * i + 1]
        assert r0.status == 0 and r1.status == 0
        assert phi0 is outs[2 * i] and phi1 is outs[2 * i + 1]
        assert np.isfinite(phi0).all()
        assert np.array_equal(phi0, phi1)
        assert r0.energy == r1.energy


def test_steady_stream_every_result_is_its_own(pbm, ctx):
    """Bursts of snapshots from a few trajectories, each burst submitted before
    the previous one is collected (the bench's steady state): slots finish, are
    re-admitted while the graph runs, and wait for their setups.  Every result
    is the solve of its own snapshot (energy against the oracle), none is lost
    or handed out twice."""
    base = [inputs.random_small(500 + t, 29 + 4 * t, 25, 27, n_atoms=20) for t in range(3)]
    rng = np.random.default_rng(8)
    bursts = []
    for _ in range(5):
        burst = []
        for t, p in enumerate(base):
            for _ in range(3):
                a = p.atoms.copy()
                a.xyz = a.xyz + rng.normal(0, 0.05, a.xyz.shape)
                burst.append((t, p, a))
        bursts.append(burst)
    got = []
    with pbm.Server(ctx, 8 * GB, tol=1e-6) as srv:
        pend = [(srv.submit(t, p.grid, a), p, a) for t, p, a in bursts[0]]
        for i in range(len(bursts)):
            nxt = [(srv.submit(t, p.grid, a), p, a) for t, p, a in bursts[i + 1]] \
                if i + 1 < len(bursts) else []
            for tk, p, a in pend:
                out = srv.poll(tk, 60000)
                assert out is not None, "a result never arrived"
                got.append((out[0], p, a))
            pend = nxt
        assert srv.stats()["completed"] == sum(len(b) for b in bursts)
    for r, p, a in got:
        assert r.status == 0, r.info.as_dict()
        s = oracle.setup(p.grid, a)
        e_ref = oracle.energy(s, oracle.pcg(s, tol=1e-10).phi)
        assert abs(r.energy - e_ref) <= 1e-6 * abs(e_ref)
        assert r.info.iterations > 0 and r.info.relres_true < 1e-6
