"""The tile-plan autotuner (pb_grid_autotune) on the GPU: it times candidate
plans, keeps one no slower than the analytic default, and the grid's solves
afterwards still match the oracle."""
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
