"""Geometric-multigrid preconditioned CG (PB_PRECOND_GMG) on the GPU against the
oracle's (oracle/gmg.py): the same solution of A phi = b (phi and E to 1e-8 at
1e-10), iteration counts close to the oracle's (the GPU V-cycle runs in FP32,
the oracle's in FP64), far fewer iterations than Jacobi-PCG, on the midpoint and
the harmonic-average dielectric, and the argument errors."""
import numpy as np
import pytest

import oracle
import oracle.gmg as G
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


def rel_max(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / max(np.max(np.abs(np.asarray(b))), 1e-300))


CASES = [lambda: (inputs.small_33(), "midpoint", "packed"),
         lambda: (inputs.random_small(6, 37, 29, 45, n_atoms=120), "midpoint", "packed"),
         lambda: (inputs.random_small(7, 24, 31, 18, n_atoms=60), "harmonic", "f32")]


@pytest.mark.parametrize("case", CASES)
def test_gmg_matches_oracle(pbm, ctx, case):
    p, model, coef = case()
    spec = p.grid.replace(eps_model=model, coef=coef)
    s = oracle.setup(spec, p.atoms)
    ref = G.gmg_pcg(s, tol=1e-10)
    e_ref = oracle.energy(s, ref.phi)
    phi = torch.zeros(spec.shape, dtype=torch.float64, device="cuda")
    with pbm.Grid(ctx, spec, p.atoms) as g:
        info = g.solve(phi, precision="f64", precond="gmg", tol=1e-10)
        e = g.energy(phi)
        assert info.status == 0
        assert rel_max(phi.cpu().numpy(), ref.phi) <= 1e-8
        assert abs(e - e_ref) <= 1e-8 * abs(e_ref)
        assert abs(info.iterations - ref.iters) <= max(2, 0.15 * ref.iters)
        assert info.relres_true < 2e-10
        # warm start from the solution: nothing left to do
        info2 = g.solve(phi, precision="f64", precond="gmg", tol=1e-10, warm_start=True)
        assert info2.status == 0 and info2.iterations <= 1


def test_gmg_needs_far_fewer_iterations(pbm, ctx):
    p = inputs.globule_129()
    phi = torch.zeros(p.grid.shape, dtype=torch.float64, device="cuda")
    with pbm.Grid(ctx, p.grid, p.atoms) as g:
        jac = g.solve(phi, precision="f64", precond="jacobi", tol=1e-8)
        phi.zero_()
        mg = g.solve(phi, precision="f64", precond="gmg", tol=1e-8)
    assert jac.status == 0 and mg.status == 0
    assert mg.iterations * 3 < jac.iterations


def test_gmg_iteration_cap_and_repeat(pbm, ctx):
    """The outer iterations run as graphs of several iterations with the CG
    scalars on the device: a cap that is not a multiple of the graph's length
    stops exactly there, and a second solve (the graph reused) repeats the
    first bit for bit."""
    p = inputs.random_small(5, 41, 37, 33, n_atoms=90)
    phi = torch.zeros(p.grid.shape, dtype=torch.float64, device="cuda")
    with pbm.Grid(ctx, p.grid, p.atoms) as g:
        for cap in (1, 4, 5):
            phi.zero_()
            info = g.solve(phi, check=False, precision="f64", precond="gmg", tol=1e-14, max_iter=cap)
            assert info.status == pbm.PB_ERR_NOT_CONVERGED and info.iterations == cap
        phi.zero_()
        a = g.solve(phi, precision="f64", precond="gmg", tol=1e-9)
        first = phi.clone()
        phi.zero_()
        b = g.solve(phi, precision="f64", precond="gmg", tol=1e-9)
        assert a.status == 0 and b.status == 0 and a.iterations == b.iterations
        assert torch.equal(first, phi)


def test_gmg_argument_errors(pbm, ctx):
    p = inputs.random_small(3, 12, 12, 12, n_atoms=4)
    phi = torch.zeros(p.grid.shape, dtype=torch.float64, device="cuda")
    with pbm.Grid(ctx, p.grid.replace(periodic=True), p.atoms) as g:
        with pytest.raises(pbm.PbError) as ei:
            g.solve(phi, precision="f64", precond="gmg", tol=1e-8)
        assert ei.value.status == pbm.PB_ERR_ARG
    with pytest.raises(pbm.PbError) as ei:
        pbm.Server(ctx, 1 << 30, precond="gmg")
    assert ei.value.status == pbm.PB_ERR_ARG
