"""The 256-snapshot batch at full size: one 1,000-atom cluster with Gaussian
coordinate perturbations (sigma 0.3 A), cubic grids drawn from 49^3-97^3,
FP32 Jacobi-PCG with FP64 refinement to 1e-6, all 256 in one server batch
(one persistent launch of each phase kernel per tick, graph captured).

Every solve must reach the tolerance; three sampled snapshots (the smallest
grid, the largest, one between) are checked against the FP64 oracle, and one
of them is solved again alone and must give the same result bit for bit."""
import numpy as np
import pytest

import oracle
from paper_1704_02745_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GB = 1 << 30
TOL = 1e-6


@pytest.fixture(scope="module")
def pbm():
    from paper_1704_02745_gb300 import build, pb
    build.build()
    pb.load()
    return pb


def test_batch_of_256_snapshots(pbm):
    snaps = inputs.snapshot_batch()
    assert len(snaps) == 256
    sizes = [p.grid.nx for p in snaps]
    order = np.argsort(sizes, kind="stable")
    sample = [int(order[0]), int(order[len(order) // 2]), int(order[-1])]
    with pbm.Context(0) as ctx:
        opts = dict(precision="f32_refine", tol=TOL, inner_tol=1e-3, warm_start=False)
        with pbm.Server(ctx, 120 * GB, **opts) as srv:
            tickets = [srv.submit(s, p.grid, p.atoms, want_phi=s in sample)
                       for s, p in enumerate(snaps)]
            res = [srv.poll(t, 600000) for t in tickets]
        with pbm.Server(ctx, 8 * GB, **opts) as srv:
            k = sample[1]
            alone, _ = srv.poll(srv.submit(k, snaps[k].grid, snaps[k].atoms), 600000)
    for s, (r, _) in enumerate(res):
        assert r.status == 0, (s, r.info.as_dict())
        assert r.info.relres_true < TOL
    k = sample[1]
    assert alone.status == 0
    assert alone.energy == res[k][0].energy  # bitwise: the mix changes nothing
    assert alone.info.iterations == res[k][0].info.iterations
    for s in sample:
        p = snaps[s]
        st = oracle.setup(p.grid, p.atoms)
        ref = oracle.pcg(st, tol=1e-10)
        e_ref = oracle.energy(st, ref.phi)
        r, phi = res[s]
        assert abs(r.energy - e_ref) <= 1e-6 * abs(e_ref), (s, r.energy, e_ref)
        assert np.max(np.abs(phi - ref.phi)) <= 1e-5 * np.max(np.abs(ref.phi))
