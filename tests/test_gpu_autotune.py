"""The tile-plan autotuners on the GPU.  pb_grid_autotune (one grid) times
candidate plans, keeps one no slower than the analytic default, and the
grid's solves afterwards still match the oracle.  pb_server_autotune (a
server's batch) times candidate batch plans on the live batch and keeps the
fastest; pb_server_set_plan sets one by hand; results match the oracle under
every plan."""
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


@pytest.mark.parametrize("shape", [(61, 45, 37), (97, 33, 41)])
def test_autotuned_plan_keeps_parity(pbm, ctx, shape):
    p = inputs.random_small(70 + shape[0], *shape, n_atoms=40)
    s = oracle.setup(p.grid, p.atoms)
    ref = oracle.pcg(s, tol=1e-11)
    e_ref = oracle.energy(s, ref.phi)
    with pbm.Grid(ctx, p.grid, p.atoms) as g:
        for prec, tol, etol in (("f32_refine", 1e-9, 1e-7), ("f64", 1e-10, 1e-8)):
            info = g.autotune(prec)
            assert info.candidates >= 2
            assert info.W % 4 == 0 and 0 < info.W <= 64 and 0 < info.H <= 24
            assert 1 <= info.tz <= shape[2] and info.n_tiles >= 1
            assert 0 < info.us_best <= info.us_default
            phi = torch.zeros(p.grid.shape, dtype=torch.float64, device="cuda")
            r = g.solve(phi, precision=prec, tol=tol)
            assert r.status == 0
            e = g.energy(phi)
            assert abs(e - e_ref) <= etol * abs(e_ref)
            dphi = np.max(np.abs(phi.cpu().numpy() - ref.phi)) / np.max(np.abs(ref.phi))
            assert dphi <= 10 * etol


def test_autotune_errors(pbm, ctx):
    p = inputs.random_small(5, 20, 20, 20, n_atoms=5)
    with pbm.Grid(ctx, p.grid, p.atoms) as g:
        st = pbm.load().pb_grid_autotune(pbm._P(g.handle), 7, None)
        assert st == pbm.PB_ERR_ARG
    assert pbm.load().pb_grid_autotune(None, 0, None) == pbm.PB_ERR_ARG


def test_server_plan_and_batch_autotune(pbm, ctx):
    """A server's batch under a plan set by hand, then tuned on the live batch:
    every result against the oracle, and the same energies before and after
    (the plan changes only the order of the partial sums)."""
    from oracle import pool as opool
    snaps = inputs.snapshot_batch(count=24)
    refs = opool.solve_many([(p.grid, p.atoms) for p in snaps], tol=1e-11)
    with pbm.Server(ctx, 16 << 30, precision="f32_refine", tol=1e-9, inner_tol=1e-4,
                    warm_start=False) as srv:
        srv.set_plan(min_planes=128, height_pct=67, occupancy=2)
        first = [srv.poll(t, 600000)[0] for t in
                 [srv.submit(k, p.grid, p.atoms) for k, p in enumerate(snaps)]]
        tickets = [srv.submit(k, p.grid, p.atoms) for k, p in enumerate(snaps)]
        info = srv.autotune(600000)
        second = [srv.poll(t, 600000)[0] for t in tickets]
        third = [srv.poll(t, 600000)[0] for t in
                 [srv.submit(k, p.grid, p.atoms) for k, p in enumerate(snaps)]]
        with pytest.raises(pbm.PbError):
            srv.set_plan(min_planes=0)
    assert info.candidates == 20
    assert info.gbs_best >= info.gbs_default > 0
    assert info.plan.occupancy in (2, 3) and 1 <= info.plan.height_pct <= 100
    for batch in (first, second, third):
        for r, ref in zip(batch, refs):
            assert r.status == 0 and r.info.relres_true < 1e-9
            assert abs(r.energy - ref["energy"]) <= 1e-7 * abs(ref["energy"])
    for a, b in zip(first, third):
        assert abs(a.energy - b.energy) <= 1e-8 * abs(a.energy)
