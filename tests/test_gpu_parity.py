"""GPU parity: libpb's CUDA path (through the C ABI) against the FP64 CPU oracle.

Tolerances:
* dielectric edges and lambda: bit-exact (a binary decision per edge/node);
* b: 1e-13 of max|b| (fixed-point charge accumulation, exp/sqrt rounding);
* FP64 operator: 1e-13 of max|Au| (summation order and FMA contraction only);
* FP32 operator: 2e-6 of max|Au| (FP32 rounding of a 7-term sum);
* FP64 PCG to 1e-10: max|dphi|/max|phi| <= 1e-8, |dE|/|E| <= 1e-8, iterations
  within 2% of the oracle's;
* FP32 PCG to 1e-6 on 129^3: |dE|/|E| <= 1e-4; FP32+FP64 refinement to 1e-9:
  |dE|/|E| <= 1e-7.
"""
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


SMALL = [lambda: inputs.random_small(5, 7, 9, 11, n_atoms=40),
         lambda: inputs.random_small(6, 37, 29, 45, n_atoms=120),
         lambda: inputs.small_33(),
         lambda: inputs.random_small(8, 2, 9, 3, n_atoms=3)]


# --------------------------------------------------------------------------- setup

@pytest.mark.parametrize("maker", SMALL)
@pytest.mark.parametrize("mask", [True, False])
def test_setup_arrays(pbm, ctx, maker, mask):
    p = maker()
    spec = p.grid.replace(kappa_mask=mask)
    s = oracle.setup(spec, p.atoms)
    with pbm.Grid(ctx, spec, p.atoms) as g:
        assert np.array_equal(g.export("eps_x"), s.ex)
        assert np.array_equal(g.export("eps_y"), s.ey)
        assert np.array_equal(g.export("eps_z"), s.ez)
        assert np.array_equal(g.export("lambda"), s.lam)
        assert rel_max(g.export("ghost"), s.ghost) < 1e-13
        assert rel_max(g.export("b"), s.b) < 1e-13


def test_setup_surface_ties(pbm, ctx):
    # radii equal (to the last bit, or one ulp either side) to the distance of
    # a chosen edge midpoint or node: the exact FP64 rule decides those cases
    rng = np.random.default_rng(77)
    g = inputs.GridSpec(20, 18, 16, 0.45, (-4.1, -3.7, -3.3))
    ox, oy, oz = g.origin
    xyz, q, r = [], [], []
    for t in range(60):
        a = np.array([ox, oy, oz]) + rng.uniform(2.0, 5.5, 3)
        i, j, k = rng.integers(2, 12, 3)
        kind = t % 4
        mx = ox + ((i + 0.5) if kind == 1 else i) * g.h
        my = oy + ((j + 0.5) if kind == 2 else j) * g.h
        mz = oz + ((k + 0.5) if kind == 3 else k) * g.h
        dx, dy, dz = mx - a[0], my - a[1], mz - a[2]
        d2 = dx * dx + dy * dy
        d2 = d2 + dz * dz
        rad = float(np.sqrt(d2))
        rad = [rad, np.nextafter(rad, 0.0), np.nextafter(rad, 9.0)][t % 3]
        xyz.append(a); q.append(rng.uniform(-1, 1)); r.append(rad)
    atoms = inputs.Atoms(np.array(xyz), np.array(q), np.array(r))
    s = oracle.setup(g, atoms)
    with pbm.Grid(ctx, g, atoms) as grid:
        for name, want in (("eps_x", s.ex), ("eps_y", s.ey), ("eps_z", s.ez), ("lambda", s.lam)):
            assert np.array_equal(grid.export(name), want), name


def test_setup_dh_f32(pbm, ctx):
    p = inputs.small_33()
    s = oracle.setup(p.grid, p.atoms)
    with pbm.Grid(ctx, p.grid.replace(dh="f32"), p.atoms) as g:
        assert rel_max(g.export("ghost"), s.ghost) < 3e-6
        assert rel_max(g.export("b"), s.b) < 1e-6


def test_setup_deterministic_and_update_atoms(pbm, ctx):
    p = inputs.small_33()
    q = inputs.small_33(seed=9)
    with pbm.Grid(ctx, p.grid, p.atoms) as g1, pbm.Grid(ctx, p.grid, p.atoms) as g2:
        b1 = g1.export("b")
        assert np.array_equal(b1, g2.export("b"))
        g2.update_atoms(q.atoms)
        s = oracle.setup(p.grid, q.atoms)
        assert np.array_equal(g2.export("eps_y"), s.ey)
        assert rel_max(g2.export("b"), s.b) < 1e-13
        g2.update_atoms(p.atoms)
        assert np.array_equal(g2.export("b"), b1)


def test_setup_argument_errors(pbm, ctx):
    p = inputs.random_small(3, 8, 8, 8, n_atoms=4)
    bad = p.atoms.copy()
    bad.xyz[1, 0] = p.grid.origin[0] - 0.1  # cell leaves the grid
    with pytest.raises(pbm.PbError) as ei:
        pbm.Grid(ctx, p.grid, bad)
    assert ei.value.status == pbm.PB_ERR_ARG
    bad = p.atoms.copy()
    bad.q[2] = np.nan  # injected non-finite charge
    with pytest.raises(pbm.PbError) as ei:
        pbm.Grid(ctx, p.grid, bad)
    assert ei.value.status == pbm.PB_ERR_ARG
    with pytest.raises(pbm.PbError):
        pbm.Grid(ctx, p.grid.replace(nx=0), p.atoms)
    with pytest.raises(pbm.PbError):
        pbm.Grid(ctx, p.grid.replace(h=-0.5), p.atoms)


# --------------------------------------------------------------------------- operator

@pytest.mark.parametrize("maker", SMALL[:3])
def test_apply_f64(pbm, ctx, maker):
    p = maker()
    s = oracle.setup(p.grid, p.atoms)
    u = np.random.default_rng(1).normal(size=p.grid.shape)
    want = oracle.apply(s, u)
    for coef in ("packed", "f64"):
        with pbm.Grid(ctx, p.grid.replace(coef=coef), p.atoms) as g:
            du = dev(u)
            dau = torch.empty_like(du)
            g.apply(du, dau, pbm.PB_F64)
            assert rel_max(dau.cpu().numpy(), want) < 1e-13


@pytest.mark.parametrize("coef", ["packed", "f32", "bf16"])
def test_apply_f32(pbm, ctx, coef):
    p = inputs.random_small(6, 37, 29, 45, n_atoms=120)
    s = oracle.setup(p.grid, p.atoms)
    u = np.random.default_rng(2).normal(size=p.grid.shape)
    want = oracle.apply(s, u)
    with pbm.Grid(ctx, p.grid.replace(coef=coef), p.atoms) as g:
        du = dev(u, torch.float32)
        dau = torch.empty_like(du)
        g.apply(du, dau, pbm.PB_F32)
        assert rel_max(dau.cpu().double().numpy(), want) < 2e-6


# --------------------------------------------------------------------------- solves

def solve(pbm, g, spec, **kw):
    phi = torch.zeros(spec.shape, dtype=torch.float64, device="cuda")
    info = g.solve(phi, **kw)
    return phi.cpu().numpy(), info


@pytest.mark.parametrize("maker", SMALL[:3])
@pytest.mark.parametrize("precond", ["jacobi", "none"])
def test_pcg_f64_parity(pbm, ctx, maker, precond):
    p = maker()
    s = oracle.setup(p.grid, p.atoms)
    ref = oracle.pcg(s, tol=1e-10, precond=precond == "jacobi")
    e_ref = oracle.energy(s, ref.phi)
    with pbm.Grid(ctx, p.grid, p.atoms) as g:
        phi, info = solve(pbm, g, p.grid, precision="f64", tol=1e-10, precond=precond)
        assert info.status == 0
        assert rel_max(phi, ref.phi) <= 1e-8
        e = g.energy(dev(phi))
        assert abs(e - e_ref) <= 1e-8 * abs(e_ref)
        assert abs(info.iterations - ref.iters) <= max(1, 0.02 * ref.iters)
        assert info.relres < 1e-10
        assert oracle.relres(s, phi) < 2e-10


def test_energy_matches_oracle_definition(pbm, ctx):
    p = inputs.small_33()
    s = oracle.setup(p.grid, p.atoms)
    phi = np.random.default_rng(3).normal(size=p.grid.shape)
    with pbm.Grid(ctx, p.grid, p.atoms) as g:
        e = g.energy(dev(phi))
    want = oracle.energy(s, phi)
    assert abs(e - want) <= 1e-12 * np.sum(np.abs(s.q_node * phi)) * 166.0


@pytest.fixture(scope="module")
def globule129():
    p = inputs.globule_129()
    s = oracle.setup(p.grid, p.atoms)
    ref = oracle.pcg(s, tol=1e-10)
    return p, s, ref, oracle.energy(s, ref.phi)


def test_pcg_f64_parity_129(pbm, ctx, globule129):
    p, s, ref, e_ref = globule129
    with pbm.Grid(ctx, p.grid, p.atoms) as g:
        phi, info = solve(pbm, g, p.grid, precision="f64", tol=1e-10)
        assert info.status == 0
        assert rel_max(phi, ref.phi) <= 1e-8
        assert abs(g.energy(dev(phi)) - e_ref) <= 1e-8 * abs(e_ref)
        assert abs(info.iterations - ref.iters) <= max(1, 0.02 * ref.iters)


def test_pcg_f64_parity_129_fp32_boundary(pbm, ctx, globule129):
    # the FP32 Debye-Hueckel sum moves phi and E far less than the FP64 tolerances
    p, s, ref, e_ref = globule129
    spec = p.grid.replace(dh="f32")
    with pbm.Grid(ctx, spec, p.atoms) as g:
        phi, info = solve(pbm, g, spec, precision="f64", tol=1e-10)
        assert info.status == 0
        assert rel_max(phi, ref.phi) <= 1e-8
        assert abs(g.energy(dev(phi)) - e_ref) <= 1e-8 * abs(e_ref)
        assert abs(info.iterations - ref.iters) <= max(1, 0.02 * ref.iters)


@pytest.mark.parametrize("coef", ["packed", "f32", "bf16"])
def test_fp32_and_refinement_129(pbm, ctx, globule129, coef):
    p, s, ref, e_ref = globule129
    spec = p.grid.replace(coef=coef)
    with pbm.Grid(ctx, spec, p.atoms) as g:
        phi, info = solve(pbm, g, spec, precision="f32", tol=1e-6)
        assert info.status == 0, info.as_dict()
        e = g.energy(dev(phi))
        assert abs(e - e_ref) <= 1e-4 * abs(e_ref)
        phi, info = solve(pbm, g, spec, precision="f32_refine", tol=1e-9, inner_tol=1e-4)
        assert info.status == 0, info.as_dict()
        assert info.relres_true < 1e-9
        e = g.energy(dev(phi))
        assert abs(e - e_ref) <= 1e-7 * abs(e_ref)
        assert oracle.relres(s, phi) < 1e-9


def test_refinement_to_1e6_matches_oracle(pbm, ctx, globule129):
    p, s, ref, e_ref = globule129
    with pbm.Grid(ctx, p.grid, p.atoms) as g:
        phi, info = solve(pbm, g, p.grid, precision="f32_refine", tol=1e-6, inner_tol=1e-3)
        assert info.status == 0
        assert oracle.relres(s, phi) < 1e-6
        assert abs(g.energy(dev(phi)) - e_ref) <= 1e-5 * abs(e_ref)


# --------------------------------------------------------------------------- edge cases

def test_solve_edge_cases(pbm, ctx):
    p = inputs.random_small(22, 5, 5, 6)
    s = oracle.setup(p.grid, p.atoms)
    with pbm.Grid(ctx, p.grid, p.atoms) as g:
        exact, info = solve(pbm, g, p.grid, precision="f64", tol=1e-13)
        # warm start from the solution: zero iterations
        phi = dev(exact)
        info = g.solve(phi, precision="f64", tol=1e-6, warm_start=True)
        assert info.iterations == 0 and info.status == 0
        # iteration cap
        phi = torch.zeros_like(phi)
        info = g.solve(phi, check=False, precision="f64", tol=1e-14, max_iter=3)
        assert info.status == pbm.PB_ERR_NOT_CONVERGED and info.iterations == 3
        # the profiled path gives the same answer and counts its launches
        phi2 = torch.zeros_like(phi)
        info = g.solve(phi2, precision="f32_refine", tol=1e-9, profile=True)
        assert info.status == 0 and info.n_stencil == info.iterations
        assert info.n_update == info.iterations and info.n_resid == info.outer_steps + 1
        assert rel_max(phi2.cpu().numpy(), exact) < 1e-8
    # no atoms: b = 0, phi = 0
    none = inputs.Atoms(np.zeros((0, 3)), np.zeros(0), np.zeros(0))
    with pbm.Grid(ctx, p.grid, none) as g:
        phi = torch.ones(p.grid.shape, dtype=torch.float64, device="cuda")
        info = g.solve(phi, precision="f64", tol=1e-6)
        assert info.iterations == 0 and float(phi.abs().max()) == 0.0
    # a one-node grid with no atoms
    g1 = inputs.GridSpec(1, 1, 1, 0.5, (0.0, 0.0, 0.0))
    with pbm.Grid(ctx, g1, none) as g:
        phi = torch.zeros((1, 1, 1), dtype=torch.float64, device="cuda")
        assert g.solve(phi, precision="f32_refine", tol=1e-6).status == 0


# (159, ...) and (175, ...): the last x tile reaches whole NV-groups past the
# row pitch (pitch = nx + 1), which must store nothing
@pytest.mark.parametrize("dims", [(2, 9, 9), (33, 2, 5), (64, 8, 17), (65, 9, 16), (159, 7, 6),
                                  (175, 5, 9), (261, 4, 3)])
def test_ragged_tiles(pbm, ctx, dims):
    p = inputs.random_small(40, *dims, n_atoms=6)
    s = oracle.setup(p.grid, p.atoms)
    ref = oracle.pcg(s, tol=1e-11)
    with pbm.Grid(ctx, p.grid, p.atoms) as g:
        phi, info = solve(pbm, g, p.grid, precision="f64", tol=1e-11)
        assert rel_max(phi, ref.phi) < 1e-8
        phi, info = solve(pbm, g, p.grid, precision="f32_refine", tol=1e-10)
        assert info.status == 0 and rel_max(phi, ref.phi) < 1e-8


def test_energy_atoms_on_and_off_the_grid(pbm, ctx):
    """Trilinear interpolation at the last node reads only nodes of the grid;
    an atom whose cell leaves the grid reads nothing and gives NaN."""
    spec = inputs.random_small(8, 9, 7, 6, n_atoms=3).grid
    rng = np.random.default_rng(11)
    phi = rng.normal(size=spec.shape)
    last = np.array(spec.origin) + spec.h * (np.array([spec.nx, spec.ny, spec.nz]) - 1)
    out = torch.zeros(1, dtype=torch.float64, device="cuda")

    def energy_of(xyz, q):
        xyzq = torch.as_tensor(np.concatenate([xyz, q[:, None]], 1)).cuda().contiguous()
        pbm.pb_energy_noalloc(xyzq, spec, dev(phi), out, torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        return float(out.item())

    e = energy_of(last[None, :], np.array([1.5]))
    assert e == pytest.approx(0.5 * 332.0637 * 1.5 * phi[-1, -1, -1], rel=1e-14)
    for off in ([spec.h * 0.25, 0, 0], [0, spec.h * 0.5, 0], [0, 0, 1e-3]):
        assert np.isnan(energy_of((last + np.array(off))[None, :], np.array([1.0])))
    assert np.isnan(energy_of(np.array(spec.origin)[None, :] - 0.1, np.array([1.0])))
