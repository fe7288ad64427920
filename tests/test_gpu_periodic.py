"""Periodic boundary (the paper's Fig. 2 runs) on the GPU against the FP64 oracle:
every axis periodic with period n*h, atoms anywhere in the cell (spheres and
charge cells wrap around), no boundary sum.  Same tolerances as the free-space
parity tests: setup bit-exact (b to 1e-13), operator to 1e-13 (FP64), PCG to
1e-10 within 1e-8 in phi and E with iterations within 2%, refinement to 1e-9
within 1e-7 in E; the last tiles overhang the grid (ragged sizes)."""
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


def dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype).cuda()


def rel_max(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / max(np.max(np.abs(np.asarray(b))), 1e-300))


def periodic_problem(seed, nx, ny, nz, n_atoms, h=0.5, radii=(1.5, 2.0)):
    """Atoms uniform over the whole periodic cell, so many spheres and charge
    cells cross a face."""
    rng = np.random.default_rng(seed)
    origin = (-0.5 * h * nx, -0.5 * h * ny, -0.5 * h * nz)
    grid = inputs.GridSpec(nx, ny, nz, h, origin, periodic=True)
    lo = np.array(origin) - 0.5 * h
    span = h * np.array([nx, ny, nz])
    xyz = lo + rng.uniform(0, 1, (n_atoms, 3)) * span
    atoms = inputs.Atoms(xyz, rng.uniform(-1, 1, n_atoms), rng.uniform(*radii, n_atoms))
    return inputs.Problem(f"periodic{nx}x{ny}x{nz}", grid, atoms)


# atoms per cell volume leave nodes outside every atom: with lambda = 0 on
# every node the periodic operator has no salt term and is singular
SIZES = [(7, 9, 11, 4), (37, 29, 23, 150), (33, 33, 33, 200), (3, 4, 5, 1), (61, 13, 9, 30)]


@pytest.mark.parametrize("dims", SIZES)
def test_setup_arrays(pbm, ctx, dims):
    p = periodic_problem(1, *dims, radii=(0.8, 1.2) if dims[0] < 5 else (1.5, 2.0))
    s = oracle.setup(p.grid, p.atoms)
    with pbm.Grid(ctx, p.grid, p.atoms) as g:
        assert np.array_equal(g.export("eps_x"), s.ex)
        assert np.array_equal(g.export("eps_y"), s.ey)
        assert np.array_equal(g.export("eps_z"), s.ez)
        assert np.array_equal(g.export("lambda"), s.lam)
        assert rel_max(g.export("b"), s.b) < 1e-13
    assert (s.ex[:, :, 0] == p.grid.eps_in).any() or dims[0] < 5  # something wraps


@pytest.mark.parametrize("dims", SIZES)
def test_apply(pbm, ctx, dims):
    p = periodic_problem(2, *dims, radii=(0.8, 1.2) if dims[0] < 5 else (1.5, 2.0))
    s = oracle.setup(p.grid, p.atoms)
    u = np.random.default_rng(3).normal(size=p.grid.shape)
    want = oracle.apply(s, u)
    for coef in ("packed", "f64"):
        with pbm.Grid(ctx, p.grid.replace(coef=coef), p.atoms) as g:
            du = dev(u)
            dau = torch.empty_like(du)
            g.apply(du, dau, pbm.PB_F64)
            assert rel_max(dau.cpu().numpy(), want) < 1e-13
    with pbm.Grid(ctx, p.grid, p.atoms) as g:
        du = dev(u, torch.float32)
        dau = torch.empty_like(du)
        g.apply(du, dau, pbm.PB_F32)
        assert rel_max(dau.cpu().numpy(), want) < 2e-6


@pytest.mark.parametrize("dims", [(7, 9, 11, 4), (37, 29, 23, 150), (61, 13, 9, 30)])
def test_pcg_f64_parity(pbm, ctx, dims):
    p = periodic_problem(4, *dims)
    s = oracle.setup(p.grid, p.atoms)
    ref = oracle.pcg(s, tol=1e-10)
    e_ref = oracle.energy(s, ref.phi)
    phi = torch.zeros(p.grid.shape, dtype=torch.float64, device="cuda")
    with pbm.Grid(ctx, p.grid, p.atoms) as g:
        info = g.solve(phi, precision="f64", tol=1e-10)
        e = g.energy(phi)
    assert info.status == 0
    assert rel_max(phi.cpu().numpy(), ref.phi) <= 1e-8
    assert abs(e - e_ref) <= 1e-8 * abs(e_ref)
    assert abs(info.iterations - ref.iters) <= max(1, 0.02 * ref.iters)


@pytest.mark.parametrize("coef", ["packed", "bf16"])
def test_refinement_parity(pbm, ctx, coef):
    p = periodic_problem(5, 37, 29, 23, 150)
    s = oracle.setup(p.grid, p.atoms)
    ref = oracle.pcg(s, tol=1e-11)
    e_ref = oracle.energy(s, ref.phi)
    phi = torch.zeros(p.grid.shape, dtype=torch.float64, device="cuda")
    with pbm.Grid(ctx, p.grid.replace(coef=coef), p.atoms) as g:
        info = g.solve(phi, precision="f32_refine", tol=1e-9, inner_tol=1e-3)
        e = g.energy(phi)
    assert info.status == 0 and info.relres_true < 1e-9
    assert abs(e - e_ref) <= 1e-7 * abs(e_ref)


def test_served_periodic_request(pbm, ctx):
    p = periodic_problem(6, 41, 37, 33, 120)
    s = oracle.setup(p.grid, p.atoms)
    e_ref = oracle.energy(s, oracle.pcg(s, tol=1e-11).phi)
    with pbm.Server(ctx, 4 << 30, tol=1e-8, warm_start=False) as srv:
        r, phi = srv.poll(srv.submit(1, p.grid, p.atoms, want_phi=True), 60000)
    assert r.status == 0
    assert abs(r.energy - e_ref) <= 1e-6 * abs(e_ref)


def test_periodic_argument_errors(pbm, ctx):
    p = periodic_problem(7, 9, 9, 9, 5)
    with pytest.raises(pbm.PbError) as ei:
        pbm.Grid(ctx, p.grid.replace(ionic_strength=0.0), p.atoms)  # singular without salt
    assert ei.value.status == pbm.PB_ERR_ARG
    with pytest.raises(pbm.PbError) as ei:
        pbm.Grid(ctx, p.grid.replace(nx=2), p.atoms)
    assert ei.value.status == pbm.PB_ERR_ARG
