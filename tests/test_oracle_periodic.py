"""Pins of the oracle's periodic boundary (the periodic boundary condition of
the paper's Fig. 2): every axis periodic with period n*h, no ghost layer.

Closed forms and symmetries fix it without the oracle's own code: the Fourier
eigenmodes of the constant-coefficient operator, symmetry and definiteness,
a dense solve, and exact translation equivariance of the dielectric map and
the charge spreading across the boundary (dyadic coordinates, so every
rounding is exact)."""
import math

import numpy as np
import pytest

import oracle
from paper_1704_02745_gb300 import inputs


def pgrid(nx, ny, nz, h=0.5, origin=(0.0, 0.0, 0.0), **kw):
    kw.setdefault("ionic_strength", 0.15)
    return inputs.GridSpec(nx, ny, nz, h, origin, periodic=True, **kw)


def const_periodic(nx, ny, nz, eps, ionic):
    g = pgrid(nx, ny, nz, eps_in=eps, eps_out=eps, ionic_strength=ionic, kappa_mask=False)
    ex = np.full((nz, ny, nx + 1), eps)
    ey = np.full((nz, ny + 1, nx), eps)
    ez = np.full((nz + 1, ny, nx), eps)
    return oracle.operator_from(g, ex, ey, ez, np.ones((nz, ny, nx), dtype=np.uint8))


@pytest.mark.parametrize("dims,m", [((6, 7, 9), (1, 2, 3)), ((8, 8, 8), (0, 4, 1)), ((5, 3, 4), (2, 1, 0))])
def test_fourier_eigenmodes(dims, m):
    nx, ny, nz = dims
    eps = 3.5
    s = const_periodic(nx, ny, nz, eps, 0.15)
    i, j, k = np.arange(nx), np.arange(ny), np.arange(nz)
    v = (np.cos(2 * np.pi * m[2] * k / nz)[:, None, None] * np.cos(2 * np.pi * m[1] * j / ny)[None, :, None]
         * np.cos(2 * np.pi * m[0] * i / nx)[None, None, :])
    lam = eps * sum(4 * math.sin(math.pi * md / n) ** 2 for md, n in zip(m, dims)) + s.kbar2_h2
    assert s.kbar2_h2 > 0.05
    np.testing.assert_allclose(oracle.apply(s, v), lam * v, atol=1e-12 * lam)
    # the constant mode: only the salt term remains
    np.testing.assert_allclose(oracle.apply(s, np.ones(s.grid.shape)), s.kbar2_h2, rtol=1e-13)


def test_symmetric_positive_definite_random():
    rng = np.random.default_rng(3)
    nx, ny, nz = 5, 6, 4
    g = pgrid(nx, ny, nz)
    s = oracle.operator_from(g, rng.uniform(1, 80, (nz, ny, nx + 1)), rng.uniform(1, 80, (nz, ny + 1, nx)),
                             rng.uniform(1, 80, (nz + 1, ny, nx)),
                             rng.integers(0, 2, (nz, ny, nx)).astype(np.uint8))
    A = oracle.dense_matrix(s)
    np.testing.assert_array_equal(A, A.T)
    for _ in range(4):
        u, w = rng.normal(size=s.grid.shape), rng.normal(size=s.grid.shape)
        lhs, rhs = np.sum(oracle.apply(s, u) * w), np.sum(u * oracle.apply(s, w))
        assert abs(lhs - rhs) <= 1e-13 * np.sum(np.abs(oracle.apply(s, u) * w))
        assert np.sum(u * oracle.apply(s, u)) > 0
    # every row sums to its salt term: no boundary edge drops out
    np.testing.assert_allclose(A.sum(axis=1), s.kbar2_h2 * s.lam.ravel(), atol=1e-10)


def test_pcg_matches_dense_solve_across_the_boundary():
    rng = np.random.default_rng(8)
    g = pgrid(8, 7, 9, h=0.5, origin=(-1.75, -1.5, -2.0))
    n_at = 5
    # atoms near the faces and corners, so spheres and cells wrap; small radii
    # leave nodes outside every atom, where the salt term keeps A definite
    xyz = np.array([[-1.7, -1.4, -1.9], [1.8, 1.4, 1.9], [-1.5, 0.5, 2.0], [0.2, -1.5, 0.0],
                    [1.9, -1.3, -1.8]])
    atoms = inputs.Atoms(xyz, rng.uniform(-1, 1, n_at), rng.uniform(0.6, 0.9, n_at))
    s = oracle.setup(g, atoms)
    r = oracle.pcg(s, tol=1e-13)
    x = oracle.cholesky_solve(oracle.dense_matrix(s), s.b.ravel())
    np.testing.assert_allclose(r.phi.ravel(), x, atol=1e-10 * np.abs(x).max())
    assert r.status == oracle.OK
    assert abs(s.q_node.sum() - atoms.q.sum()) < 1e-14 * np.abs(atoms.q).sum()


def dyadic_atoms(rng, n):
    xyz = rng.integers(-64, 64, (n, 3)) / 64.0
    r = rng.integers(96, 128, n) / 64.0  # 1.5 .. 2.0 A
    return inputs.Atoms(xyz, rng.integers(-64, 64, n) / 64.0, r)


@pytest.mark.parametrize("shift", [(3, 0, 0), (0, -5, 0), (0, 0, 7), (9, 4, -6)])
def test_translation_equivariance_across_the_boundary(shift):
    """Moving every atom by whole nodes rolls the dielectric map, lambda and the
    grid charges by as many nodes, wrapping around the period."""
    rng = np.random.default_rng(11)
    g = pgrid(12, 10, 14, h=0.5, origin=(-3.0, -2.5, -3.5))
    a = dyadic_atoms(rng, 6)
    b = a.copy()
    b.xyz = a.xyz + np.array(shift) * g.h
    ex0, ey0, ez0, l0 = oracle.dielectric(g, a)
    ex1, ey1, ez1, l1 = oracle.dielectric(g, b)
    sx, sy, sz = shift

    def roll(arr):
        return np.roll(arr, (sz, sy, sx), axis=(0, 1, 2))

    np.testing.assert_array_equal(l1, roll(l0))
    # the edge arrays hold the wrap-around edge twice (entries -1 and n-1):
    # compare the n distinct edges per line
    np.testing.assert_array_equal(ex1[:, :, 1:], roll(ex0[:, :, 1:]))
    np.testing.assert_array_equal(ey1[:, 1:, :], roll(ey0[:, 1:, :]))
    np.testing.assert_array_equal(ez1[1:, :, :], roll(ez0[1:, :, :]))
    np.testing.assert_array_equal(oracle.spread_charge(g, b), roll(oracle.spread_charge(g, a)))
    # something actually wraps in this configuration
    assert (ex0 == g.eps_in).any() and (ex1[:, :, 0] == ex1[:, :, -1]).all()


def test_interior_atoms_give_the_dirichlet_map():
    """Atoms whose spheres stay two spacings away from every face: the periodic
    map equals the Dirichlet one (the boundary edges are eps_out in both)."""
    p = inputs.small_33()
    keep = np.all(np.abs(p.atoms.xyz) + p.atoms.r[:, None] < 6.0, axis=1)
    a = inputs.Atoms(p.atoms.xyz[keep], p.atoms.q[keep], p.atoms.r[keep])
    assert a.n > 20
    d = oracle.dielectric(p.grid, a)
    q = oracle.dielectric(p.grid.replace(periodic=True), a)
    for x, y in zip(d, q):
        np.testing.assert_array_equal(x, y)
