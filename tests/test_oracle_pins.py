"""Pins of the FP64 CPU oracle against closed forms, special cases and brute force.

Each test fixes a value that the paper or the mathematics determines without
reference to the oracle's own code, chosen so that a dropped term, a wrong sign
or a transposed index in ``oracle/pb_oracle.c`` fails at least one of them.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_1704_02745_gb300 import inputs

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "closed_forms.json")))


def const_grid(nx, ny, nz, eps=2.0, h=0.5, ionic=0.0, mask=False):
    return inputs.GridSpec(nx, ny, nz, h, (0.0, 0.0, 0.0), eps_in=eps, eps_out=eps,
                           ionic_strength=ionic, kappa_mask=mask)


def const_setup(nx, ny, nz, eps=2.0, **kw):
    g = const_grid(nx, ny, nz, eps=eps, **kw)
    ex = np.full((nz, ny, nx + 1), eps)
    ey = np.full((nz, ny + 1, nx), eps)
    ez = np.full((nz + 1, ny, nx), eps)
    lam = np.ones((nz, ny, nx), dtype=np.uint8)
    return oracle.operator_from(g, ex, ey, ez, lam)


def random_setup(rng, nx, ny, nz, ionic=0.15):
    g = inputs.GridSpec(nx, ny, nz, 0.5, (0.0, 0.0, 0.0), ionic_strength=ionic)
    ex = rng.uniform(1.0, 80.0, (nz, ny, nx + 1))
    ey = rng.uniform(1.0, 80.0, (nz, ny + 1, nx))
    ez = rng.uniform(1.0, 80.0, (nz + 1, ny, nx))
    lam = rng.integers(0, 2, (nz, ny, nx)).astype(np.uint8)
    return oracle.operator_from(g, ex, ey, ez, lam)


def mode(nx, ny, nz):
    i = np.arange(nx); j = np.arange(ny); k = np.arange(nz)
    vx = np.sin(np.pi * (i + 1) / (nx + 1))
    vy = np.sin(np.pi * (j + 1) / (ny + 1))
    vz = np.sin(np.pi * (k + 1) / (nz + 1))
    return vz[:, None, None] * vy[None, :, None] * vx[None, None, :]


def mode_eigenvalue(nx, ny, nz, eps):
    return eps * sum(4.0 * math.sin(math.pi / (2 * (n + 1))) ** 2 for n in (nx, ny, nz))


# --------------------------------------------------------------------------- constants

def test_coulomb_constant_from_codata():
    e, eps0, na = 1.602176634e-19, 8.8541878128e-12, 6.02214076e23
    val = e * e / (4 * math.pi * eps0 * 1e-10) * na / 4184.0
    assert abs(val - oracle.COULOMB_KCAL) / val < 1e-6


def test_debye_length_textbook():
    # 1:1 salt in water at 25 C: Debye length 0.304/sqrt(I) nm (eps 78.54).
    ref = GOLDEN["debye_length_nm_sqrtM_25C_water"]["value"] / math.sqrt(0.15) * 10.0
    k2 = oracle.kappa_debye2(0.15, 298.15, 78.54)
    assert abs(1.0 / math.sqrt(k2) - ref) / ref < 3e-3
    # kappa^2 proportional to I, inversely to T and eps
    assert math.isclose(oracle.kappa_debye2(0.3, 300, 80), 2 * oracle.kappa_debye2(0.15, 300, 80),
                        rel_tol=1e-14)
    assert math.isclose(oracle.kappa_debye2(0.15, 600, 80), 0.5 * oracle.kappa_debye2(0.15, 300, 80),
                        rel_tol=1e-14)
    assert math.isclose(oracle.kappa_debye2(0.15, 300, 40), 2 * oracle.kappa_debye2(0.15, 300, 80),
                        rel_tol=1e-14)
    assert oracle.kappa_debye2(0.0, 300, 80) == 0.0


# --------------------------------------------------------------------------- operator (O2)

def test_eigenmode_8cubed():
    s = const_setup(8, 8, 8, eps=3.0)
    v = mode(8, 8, 8)
    lam = GOLDEN["eigenvalue_8cubed_per_eps"]["value"] * 3.0
    assert abs(mode_eigenvalue(8, 8, 8, 3.0) - lam) < 1e-6
    av = oracle.apply(s, v)
    assert np.max(np.abs(av - lam * v)) < 1e-5 * np.max(np.abs(v))
    assert np.max(np.abs(av - mode_eigenvalue(8, 8, 8, 3.0) * v)) < 1e-13


@pytest.mark.parametrize("dims", [(5, 7, 9), (1, 4, 6), (12, 3, 2)])
def test_eigenmode_noncubic_with_salt(dims):
    nx, ny, nz = dims
    s = const_setup(nx, ny, nz, eps=1.7, ionic=0.1, mask=False)
    v = mode(nx, ny, nz)
    lam = mode_eigenvalue(nx, ny, nz, 1.7) + s.kbar2_h2
    assert s.kbar2_h2 > 0
    av = oracle.apply(s, v)
    assert np.max(np.abs(av - lam * v)) < 1e-13 * lam


def test_symmetric_positive_definite():
    rng = np.random.default_rng(11)
    s = random_setup(rng, 6, 7, 8)
    for _ in range(3):
        u = rng.normal(size=s.grid.shape)
        v = rng.normal(size=s.grid.shape)
        a = np.vdot(oracle.apply(s, u), v)
        b = np.vdot(u, oracle.apply(s, v))
        assert abs(a - b) <= 1e-13 * max(abs(a), 1.0) * 10
        assert np.vdot(u, oracle.apply(s, u)) > 0


def test_row_sums_are_ghost_edges():
    # A annihilates constants in the interior; a row's sum is the eps of its
    # ghost edges plus the Boltzmann term.
    rng = np.random.default_rng(12)
    s = random_setup(rng, 5, 6, 7)
    nz, ny, nx = s.grid.shape
    want = s.kbar2_h2 * s.lam.astype(float)
    want[:, :, 0] += s.ex[:, :, 0]
    want[:, :, -1] += s.ex[:, :, nx]
    want[:, 0, :] += s.ey[:, 0, :]
    want[:, -1, :] += s.ey[:, ny, :]
    want[0, :, :] += s.ez[0, :, :]
    want[-1, :, :] += s.ez[nz, :, :]
    got = oracle.apply(s, np.ones(s.grid.shape))
    assert np.max(np.abs(got - want)) < 1e-12 * np.max(want)


def test_single_off_diagonal_entry():
    # A e_c has -eps_edge at the six neighbours of c: check the x+ neighbour
    # against the edge between c and c+x (a transposed edge index fails here).
    rng = np.random.default_rng(13)
    s = random_setup(rng, 4, 5, 6)
    u = np.zeros(s.grid.shape)
    k, j, i = 2, 3, 1
    u[k, j, i] = 1.0
    au = oracle.apply(s, u)
    assert au[k, j, i + 1] == -s.ex[k, j, i + 1]
    assert au[k, j, i - 1] == -s.ex[k, j, i]
    assert au[k, j + 1, i] == -s.ey[k, j + 1, i]
    assert au[k, j - 1, i] == -s.ey[k, j, i]
    assert au[k + 1, j, i] == -s.ez[k + 1, j, i]
    assert au[k - 1, j, i] == -s.ez[k, j, i]
    assert au[k, j, i] == s.diag[k, j, i]
    assert np.count_nonzero(au) == 7


# --------------------------------------------------------------------------- solvers (O3/O4/O6)

def columns_matrix(s):
    n = s.grid.n
    A = np.empty((n, n))
    for c in range(n):
        e = np.zeros(n)
        e[c] = 1.0
        A[:, c] = oracle.apply(s, e).ravel()
    return A


@pytest.mark.parametrize("ionic,mask", [(0.0, True), (0.15, True), (0.15, False)])
def test_pcg_matches_dense_solve(ionic, mask):
    p = inputs.random_small(21, 6, 7, 8, ionic_strength=ionic, kappa_mask=mask)
    s = oracle.setup(p.grid, p.atoms)
    A = columns_matrix(s)
    x_ref = np.linalg.solve(A, s.b.ravel())
    for precond in (True, False):
        r = oracle.pcg(s, tol=1e-13, precond=precond)
        assert r.status == oracle.OK
        err = np.max(np.abs(r.phi.ravel() - x_ref)) / np.max(np.abs(x_ref))
        assert err < 1e-10, (precond, err)
        assert r.iters <= s.grid.n
    # the oracle's explicit matrix and dense Cholesky agree with numpy
    D = oracle.dense_matrix(s)
    assert np.array_equal(D, A)
    x_ch = oracle.cholesky_solve(D, s.b.ravel())
    assert np.max(np.abs(x_ch - x_ref)) / np.max(np.abs(x_ref)) < 1e-12


def test_pcg_eigenmode_one_iteration():
    # constant eps, no salt: diag(A) = 6 eps I, so Jacobi-PCG is CG, and an
    # eigenvector right-hand side converges in exactly one step to v / lambda.
    s = const_setup(7, 8, 9, eps=5.0)
    v = mode(7, 8, 9)
    lam = mode_eigenvalue(7, 8, 9, 5.0)
    for precond in (True, False):
        r = oracle.pcg(s, b=v, tol=1e-12, precond=precond)
        assert r.iters == 1
        assert np.max(np.abs(r.phi - v / lam)) < 1e-14 * np.max(np.abs(v / lam)) * 10


def test_cg_finite_termination():
    # 3x3x3 constant eps has at most 10 distinct eigenvalues: exact CG ends in <= 10 steps
    s = const_setup(3, 3, 3, eps=1.0)
    b = np.random.default_rng(3).normal(size=s.grid.shape)
    r = oracle.pcg(s, b=b, tol=1e-10, precond=False)
    assert r.status == oracle.OK and r.iters <= 11


def test_stopping_rule_and_edge_cases():
    p = inputs.random_small(22, 5, 5, 6)
    s = oracle.setup(p.grid, p.atoms)
    exact = np.linalg.solve(columns_matrix(s), s.b.ravel()).reshape(s.grid.shape)
    r = oracle.pcg(s, tol=1e-6, phi0=exact)
    assert r.iters == 0 and r.relres < 1e-6
    z = oracle.pcg(s, b=np.zeros(s.grid.shape), tol=1e-6, phi0=np.ones(s.grid.shape))
    assert z.iters == 0 and np.all(z.phi == 0)
    nc = oracle.pcg(s, tol=1e-14, max_iter=3)
    assert nc.status == oracle.NOT_CONVERGED and nc.iters == 3
    ok = oracle.pcg(s, tol=1e-6)
    assert ok.relres < 1e-6
    # the check is strict and at the recursive residual; the true residual agrees
    assert oracle.relres(s, ok.phi) < 2e-6


def test_cg_and_pcg_agree_33():
    p = inputs.small_33()
    s = oracle.setup(p.grid, p.atoms)
    a = oracle.pcg(s, tol=1e-10, precond=True)
    b = oracle.pcg(s, tol=1e-10, precond=False)
    assert a.iters < b.iters
    assert np.max(np.abs(a.phi - b.phi)) / np.max(np.abs(a.phi)) < 1e-8


# --------------------------------------------------------------------------- setup (O1)

def brute_force_dielectric(grid, atoms):
    """All atoms against every midpoint, in the same rounding as the definition."""
    nx, ny, nz, h = grid.nx, grid.ny, grid.nz, grid.h
    ox, oy, oz = grid.origin

    def any_inside(mx, my, mz):
        ins = np.zeros(mx.shape, dtype=bool)
        for a in range(atoms.n):
            dx = mx - atoms.xyz[a, 0]; dy = my - atoms.xyz[a, 1]; dz = mz - atoms.xyz[a, 2]
            d2 = dx * dx + dy * dy
            d2 = d2 + dz * dz
            ins |= d2 < atoms.r[a] * atoms.r[a]
        return ins

    K, J, I = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(-1, nx), indexing="ij")
    ex = np.where(any_inside(ox + (I + 0.5) * h, oy + J * h, oz + K * h), grid.eps_in, grid.eps_out)
    K, J, I = np.meshgrid(np.arange(nz), np.arange(-1, ny), np.arange(nx), indexing="ij")
    ey = np.where(any_inside(ox + I * h, oy + (J + 0.5) * h, oz + K * h), grid.eps_in, grid.eps_out)
    K, J, I = np.meshgrid(np.arange(-1, nz), np.arange(ny), np.arange(nx), indexing="ij")
    ez = np.where(any_inside(ox + I * h, oy + J * h, oz + (K + 0.5) * h), grid.eps_in, grid.eps_out)
    K, J, I = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    lam = np.where(any_inside(ox + I * h, oy + J * h, oz + K * h), 0, 1).astype(np.uint8)
    return ex, ey, ez, lam


@pytest.mark.parametrize("maker", [lambda: inputs.random_small(5, 7, 9, 11, n_atoms=40),
                                   lambda: inputs.small_33()])
def test_dielectric_equals_brute_force(maker):
    p = maker()
    got = oracle.dielectric(p.grid, p.atoms)
    want = brute_force_dielectric(p.grid, p.atoms)
    for g, w in zip(got, want):
        assert g.shape == w.shape
        assert np.array_equal(g, w)


def test_dielectric_single_atom_by_hand():
    h = 0.5
    g = inputs.GridSpec(5, 5, 5, h, (0.0, 0.0, 0.0), eps_in=1.0, eps_out=80.0)
    at = inputs.Atoms(np.array([[2 * h, 2 * h, 2 * h]]), np.array([1.0]), np.array([0.6 * h]))
    ex, ey, ez, lam = oracle.dielectric(g, at)
    # only the six edges touching node (2,2,2) have midpoints within 0.6 h
    assert ex[2, 2, 2] == 1.0 and ex[2, 2, 3] == 1.0 and np.sum(ex == 1.0) == 2
    assert ey[2, 2, 2] == 1.0 and ey[2, 3, 2] == 1.0 and np.sum(ey == 1.0) == 2
    assert ez[2, 2, 2] == 1.0 and ez[3, 2, 2] == 1.0 and np.sum(ez == 1.0) == 2
    assert lam[2, 2, 2] == 0 and np.sum(lam == 0) == 1
    # a radius of exactly h/2 leaves the midpoints on the sphere: outside (strict test)
    at.r[:] = 0.5 * h
    ex, ey, ez, lam = oracle.dielectric(g, at)
    assert np.all(ex == 80.0) and np.all(ey == 80.0) and np.all(ez == 80.0)
    assert np.sum(lam == 0) == 1
    # kappa_mask off: lambda is 1 everywhere
    _, _, _, lam = oracle.dielectric(g.replace(kappa_mask=False), at)
    assert np.all(lam == 1)


def test_charge_spreading_moments():
    p = inputs.random_small(7, 9, 8, 10, n_atoms=50)
    qn = oracle.spread_charge(p.grid, p.atoms)
    scale = np.sum(np.abs(p.atoms.q))
    assert abs(qn.sum() - p.atoms.q.sum()) < 1e-14 * scale * 10
    nz, ny, nx = p.grid.shape
    ox, oy, oz = p.grid.origin
    h = p.grid.h
    K, J, I = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    for ax, coord in ((0, ox + I * h), (1, oy + J * h), (2, oz + K * h)):
        m_grid = np.sum(qn * coord)
        m_atoms = np.sum(p.atoms.q * p.atoms.xyz[:, ax])
        assert abs(m_grid - m_atoms) < 1e-12 * scale * 10


def test_charge_on_node_and_cell_centre():
    h = 0.5
    g = inputs.GridSpec(4, 4, 4, h, (0.0, 0.0, 0.0))
    at = inputs.Atoms(np.array([[h, 2 * h, h]]), np.array([0.7]), np.array([1.0]))
    qn = oracle.spread_charge(g, at)
    assert qn[1, 2, 1] == 0.7 and np.count_nonzero(qn) == 1
    at = inputs.Atoms(np.array([[1.5 * h, 1.5 * h, 1.5 * h]]), np.array([0.8]), np.array([1.0]))
    qn = oracle.spread_charge(g, at)
    assert np.count_nonzero(qn) == 8 and np.allclose(qn[1:3, 1:3, 1:3], 0.1, rtol=0, atol=1e-16)
    for bad in ([-0.01, h, h], [3 * h, h, h], [h, h, 3.2 * h]):
        with pytest.raises(oracle.OracleArgError):
            oracle.spread_charge(g, inputs.Atoms(np.array([bad]), np.array([1.0]), np.array([1.0])))


def test_dh_boundary_closed_forms():
    n, h = 9, 0.5
    g = inputs.centered_grid(n, h, ionic_strength=0.15)
    kd = math.sqrt(oracle.kappa_debye2(0.15, 300.0, 80.0))
    at = inputs.Atoms(np.zeros((1, 3)), np.array([0.9]), np.array([1.5]))
    gh = oracle.dh_ghost(g, at)
    faces = gh.reshape(6, n, n)
    # a centred charge on a cube: all six faces carry the same values
    for f in range(1, 6):
        assert np.max(np.abs(faces[f] - faces[0])) < 1e-15 * np.max(np.abs(faces[0])) * 10
    # face-centre ghost sits (n+1)/2 spacings away: screened Coulomb in eps_out
    d = (n + 1) / 2 * h
    want = 0.9 * math.exp(-kd * d) / (80.0 * d)
    assert abs(faces[0][n // 2, n // 2] - want) < 1e-15 * want * 10
    # salt-free: plain Coulomb at a face corner ghost
    g0 = g.replace(ionic_strength=0.0)
    f0 = oracle.dh_ghost(g0, at).reshape(6, n, n)
    d = math.sqrt(((n + 1) / 2 * h) ** 2 + 2 * ((n - 1) / 2 * h) ** 2)
    assert abs(f0[1][0, 0] - 0.9 / (80.0 * d)) < 1e-15 * 10
    # superposition over atoms
    rng = np.random.default_rng(5)
    a2 = inputs.Atoms(rng.uniform(-1, 1, (3, 3)), rng.uniform(-1, 1, 3), np.ones(3))
    tot = oracle.dh_ghost(g, a2)
    parts = sum(oracle.dh_ghost(g, inputs.Atoms(a2.xyz[i:i + 1], a2.q[i:i + 1], a2.r[i:i + 1]))
                for i in range(3))
    assert np.max(np.abs(tot - parts)) < 1e-14 * np.max(np.abs(tot))


def test_dh_points_match_ghost_faces():
    p = inputs.random_small(12, 6, 7, 8, n_atoms=9)
    pos = oracle.ghost_positions(p.grid)
    assert pos.shape[0] == oracle.ghost_count(p.grid)
    got = oracle.dh_points(p.grid, p.atoms, pos)
    assert np.array_equal(got, oracle.dh_ghost(p.grid, p.atoms))


def test_rhs_fold_reproduces_harmonic_linear_field():
    # A linear field is discrete-harmonic for constant eps: with no charge and
    # ghost values taken from it, the solve must return the field at the nodes.
    nx, ny, nz, h = 6, 7, 8, 0.5
    g = inputs.GridSpec(nx, ny, nz, h, (0.1, -0.2, 0.3), eps_in=3.0, eps_out=3.0,
                        ionic_strength=0.0, kappa_mask=False)
    coef = np.array([0.3, -0.7, 1.1])
    f = lambda x, y, z: 2.0 + coef[0] * x + coef[1] * y + coef[2] * z
    ox, oy, oz = g.origin
    faces = []
    for gi in (-1, nx):
        K, J = np.meshgrid(np.arange(nz), np.arange(ny), indexing="ij")
        faces.append(f(ox + gi * h, oy + J * h, oz + K * h).ravel())
    for gj in (-1, ny):
        K, I = np.meshgrid(np.arange(nz), np.arange(nx), indexing="ij")
        faces.append(f(ox + I * h, oy + gj * h, oz + K * h).ravel())
    for gk in (-1, nz):
        J, I = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
        faces.append(f(ox + I * h, oy + J * h, oz + gk * h).ravel())
    ghost = np.concatenate(faces)
    no_atoms = inputs.Atoms(np.zeros((0, 3)), np.zeros(0), np.zeros(0))
    s = oracle.setup(g, no_atoms, ghost=ghost)
    r = oracle.pcg(s, tol=1e-13)
    K, J, I = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    want = f(ox + I * h, oy + J * h, oz + K * h)
    assert np.max(np.abs(r.phi - want)) < 1e-10


def test_energy_adjoint_of_spreading():
    # sum_nodes q_node phi = sum_atoms q_a * (trilinear interpolation of phi at x_a)
    p = inputs.random_small(9, 6, 7, 8, n_atoms=30)
    s = oracle.setup(p.grid, p.atoms)
    phi = np.random.default_rng(4).normal(size=s.grid.shape)
    e = oracle.energy(s, phi)
    h = p.grid.h
    tot = 0.0
    for a in range(p.atoms.n):
        f = (p.atoms.xyz[a] - np.array(p.grid.origin)) / h
        i0 = np.floor(f).astype(int)
        w = f - i0
        v = 0.0
        for dk in (0, 1):
            for dj in (0, 1):
                for di in (0, 1):
                    wt = (w[0] if di else 1 - w[0]) * (w[1] if dj else 1 - w[1]) * (w[2] if dk else 1 - w[2])
                    v += wt * phi[i0[2] + dk, i0[1] + dj, i0[0] + di]
        tot += p.atoms.q[a] * v
    want = 0.5 * GOLDEN["coulomb_kcal_per_mol"]["value"] * tot
    assert abs(e - want) < 1e-12 * abs(want)


# --------------------------------------------------------------------------- physics

def born_dG(n, h, ionic_strength=0.0):
    p = inputs.single_charge(n, h, ionic_strength=ionic_strength)
    return oracle.solvation_energy(p.grid, p.atoms, tol=1e-9)[0]


def test_born_ion_converges():
    a, ein, eout = 2.0, 1.0, 80.0
    exact = GOLDEN["coulomb_kcal_per_mol"]["value"] / (2 * a) * (1 / eout - 1 / ein)
    assert abs(exact - GOLDEN["born_dG_a2_eps1_80"]["value"]) < 1e-3
    e1 = abs(born_dG(41, 0.5) - exact) / abs(exact)
    e2 = abs(born_dG(81, 0.25) - exact) / abs(exact)
    assert e2 < e1
    assert e1 < 0.06
    assert e2 < 0.02
