"""The oracle's process pool (oracle/pool.py) changes no arithmetic: the
piecewise boundary sum equals the oracle's own, bit for bit, and pooled solves
equal direct ones."""
import numpy as np

import oracle
from oracle import pool as opool
from paper_1704_02745_gb300 import inputs


def test_pooled_boundary_sum_is_bitwise_the_oracles():
    p = inputs.random_small(31, 13, 11, 9, n_atoms=25)
    assert np.array_equal(opool.dh_ghost(p.grid, p.atoms, procs=3), oracle.dh_ghost(p.grid, p.atoms))


def test_pooled_solves_equal_direct_ones():
    probs = [inputs.random_small(s, 9, 8, 7, n_atoms=12) for s in (1, 2, 3)]
    got = opool.solve_many([(p.grid, p.atoms) for p in probs], tol=1e-9, procs=2, want_phi=True)
    for p, r in zip(probs, got):
        s = oracle.setup(p.grid, p.atoms)
        want = oracle.pcg(s, tol=1e-9)
        assert r["status"] == 0 and r["iters"] == want.iters
        assert np.array_equal(r["phi"], want.phi)
        assert r["energy"] == oracle.energy(s, want.phi)
        assert r["seconds"] > 0


def test_reference_check_reports_deviation_and_residual():
    p = inputs.random_small(4, 8, 9, 10, n_atoms=10)
    s = oracle.setup(p.grid, p.atoms)
    exact = oracle.pcg(s, tol=1e-12).phi
    off = exact.copy()
    off[3, 4, 5] += 1e-3 * np.max(np.abs(exact))
    (r,) = opool.reference_check([(p.grid, p.atoms)], [[exact, off]], tol=1e-12, procs=1)
    assert r["dphi_of"][0] == 0.0
    assert abs(r["dphi_of"][1] - 1e-3) < 1e-12
    assert r["relres_of"][0] < 1e-12 < r["relres_of"][1]
    assert r["energy_of"][0] == r["energy"]
