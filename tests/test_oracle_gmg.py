"""Pins of the oracle's geometric-multigrid preconditioned CG (oracle/gmg.py).

The multigrid scheme is a stated reading, not the paper's; what fixes it is
mathematics: the transfer operators are adjoint (restriction = P^T / 2) and
reproduce linear functions, the coarse operator of a constant-coefficient
problem is the same operator rediscretised at 2h, the V-cycle is a symmetric
positive definite operator, and the preconditioned CG reaches the solution of
A phi = b (a dense solve on a small grid; Jacobi-PCG on 33^3) in far fewer
iterations."""
import numpy as np
import pytest

import oracle
import oracle.gmg as G
from paper_1704_02745_gb300 import inputs


def random_problem(seed, nx, ny, nz):
    rng = np.random.default_rng(seed)
    g = inputs.GridSpec(nx, ny, nz, 0.5, (0.0, 0.0, 0.0), ionic_strength=0.15)
    return oracle.operator_from(g, rng.uniform(1, 80, (nz, ny, nx + 1)), rng.uniform(1, 80, (nz, ny + 1, nx)),
                                rng.uniform(1, 80, (nz + 1, ny, nx)),
                                rng.integers(0, 2, (nz, ny, nx)).astype(np.uint8))


@pytest.mark.parametrize("fine,coarse", [((9, 8, 7), (5, 4, 4)), ((12, 13, 6), (6, 7, 3))])
def test_transfer_adjoint_and_linear(fine, coarse):
    rng = np.random.default_rng(1)
    nx, ny, nz = fine
    mx, my, mz = coarse
    assert (G.coarse_size(nx), G.coarse_size(ny), G.coarse_size(nz)) == coarse
    e = rng.normal(size=(mz, my, mx))
    r = rng.normal(size=(nz, ny, nx))
    lhs = np.sum(G.prolong(e, (nz, ny, nx)) * r)
    rhs = 2.0 * np.sum(e * G.restrict(r, (mz, my, mx)))
    assert abs(lhs - rhs) <= 1e-12 * np.sum(np.abs(G.prolong(e, (nz, ny, nx)) * r))
    # a linear function on the coarse nodes interpolates to the same function
    # on fine nodes whose neighbours are not the ghost past the end
    K, J, I = np.meshgrid(np.arange(mz), np.arange(my), np.arange(mx), indexing="ij")
    lin = 0.3 + 2.0 * I - 1.5 * J + 0.7 * K
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    want = 0.3 + 2.0 * (i / 2) - 1.5 * (j / 2) + 0.7 * (k / 2)
    got = G.prolong(lin, (nz, ny, nx))
    inner = (i <= 2 * (mx - 1)) & (j <= 2 * (my - 1)) & (k <= 2 * (mz - 1))
    np.testing.assert_allclose(got[inner], want[inner], atol=1e-12)


def test_constant_coefficient_coarse_operator_is_a_rediscretisation():
    eps = 7.0
    nx, ny, nz = 9, 11, 7
    g = inputs.GridSpec(nx, ny, nz, 0.5, (0.0, 0.0, 0.0), eps_in=eps, eps_out=eps, ionic_strength=0.15,
                        kappa_mask=False)
    s = oracle.operator_from(g, np.full((nz, ny, nx + 1), eps), np.full((nz, ny + 1, nx), eps),
                             np.full((nz + 1, ny, nx), eps), np.ones((nz, ny, nx), dtype=np.uint8))
    c = G.coarsen(s)
    mz, my, mx = c.grid.shape
    want = oracle.operator_from(g.replace(nx=mx, ny=my, nz=mz, h=1.0), np.full((mz, my, mx + 1), eps),
                                np.full((mz, my + 1, mx), eps), np.full((mz + 1, my, mx), eps),
                                np.ones((mz, my, mx), dtype=np.uint8))
    np.testing.assert_allclose(c.ex, want.ex, rtol=1e-15)
    np.testing.assert_allclose(c.diag, want.diag, rtol=1e-15)
    assert abs(c.kbar2_h2 - 4.0 * s.kbar2_h2) <= 1e-15 * s.kbar2_h2


@pytest.mark.parametrize("dims", [(9, 8, 7), (12, 13, 6), (17, 17, 17)])
def test_vcycle_symmetric_positive_definite(dims):
    s = random_problem(2, *dims)
    lv = G.hierarchy(s)
    rng = np.random.default_rng(3)
    for _ in range(3):
        r1, r2 = rng.normal(size=s.grid.shape), rng.normal(size=s.grid.shape)
        v1, v2 = G.vcycle(lv, r1), G.vcycle(lv, r2)
        a, b = np.sum(v1 * r2), np.sum(r1 * v2)
        assert abs(a - b) <= 1e-12 * np.sum(np.abs(v1 * r2))
        assert np.sum(v1 * r1) > 0


def test_gmg_pcg_matches_dense_solve():
    p = inputs.random_small(4, 9, 7, 8, n_atoms=6)
    s = oracle.setup(p.grid, p.atoms)
    r = G.gmg_pcg(s, tol=1e-13)
    x = oracle.cholesky_solve(oracle.dense_matrix(s), s.b.ravel())
    assert r.status == oracle.OK
    np.testing.assert_allclose(r.phi.ravel(), x, atol=1e-10 * np.abs(x).max())


def test_gmg_pcg_matches_jacobi_in_fewer_iterations():
    p = inputs.small_33()
    s = oracle.setup(p.grid, p.atoms)
    g = G.gmg_pcg(s, tol=1e-10)
    j = oracle.pcg(s, tol=1e-10)
    assert g.status == oracle.OK and j.status == oracle.OK
    assert np.abs(g.phi - j.phi).max() <= 1e-8 * np.abs(j.phi).max()
    assert g.iters * 2 < j.iters
