"""Pins of the oracle's weighted harmonic-average boundary dielectric (Sec. 2.7):
each edge takes 1/(w/eps_in + (1-w)/eps_out), w the fraction of the edge
inside the union of the atom spheres.

Closed forms on dyadic geometry (every rounding exact), a fine sampling of
every edge of a random problem, consistency with the midpoint map where the
edge is wholly inside or outside, and the Born ion."""
import math

import numpy as np
import pytest

import oracle
from paper_1704_02745_gb300 import inputs

EIN, EOUT = 1.0, 80.0


def grid(nx, ny, nz, h=0.5, origin=(0.0, 0.0, 0.0), **kw):
    return inputs.GridSpec(nx, ny, nz, h, origin, eps_in=EIN, eps_out=EOUT, eps_model="harmonic", **kw)


def w_of(eps):
    """Invert the harmonic average: the fraction inside."""
    return (1.0 / eps - 1.0 / EOUT) / (1.0 / EIN - 1.0 / EOUT)


def one_atom(x, y, z, r):
    return inputs.Atoms(np.array([[x, y, z]]), np.array([1.0]), np.array([r]))


def test_half_covered_edge_is_the_harmonic_mean():
    # x-edge from node (2,2,2) at (1,1,1) to (1.5,1,1); a sphere of radius 1/8
    # centred on the edge at (1.25,1,1) covers t in (1/4, 3/4): w = 1/2
    g = grid(6, 5, 5)
    ex, ey, ez, lam = oracle.dielectric(g, one_atom(1.25, 1.0, 1.0, 0.125))
    assert ex[2, 2, 2 + 1] == pytest.approx(2 * EIN * EOUT / (EIN + EOUT), rel=1e-15)  # entry i+1: edge (i, i+1)
    covered = np.argwhere(ex != EOUT)
    assert covered.tolist() == [[2, 2, 3]]
    assert (ey == EOUT).all() and (ez == EOUT).all()


@pytest.mark.parametrize("d", [0.0, 0.0625, 0.09375])
def test_chord_length(d):
    # sphere r = 1/8 centred at t = 1/2 of a y-edge, offset d in x: the chord
    # covers 2 sqrt(r^2 - d^2) / h of the edge (exact for these dyadic values)
    r, h = 0.125, 0.5
    g = grid(5, 6, 5)
    ex, ey, ez, lam = oracle.dielectric(g, one_atom(1.0 + d, 1.25, 1.0, r))
    want = 2 * math.sqrt(r * r - d * d) / h
    assert abs(w_of(ey[2, 2 + 1, 2]) - want) < 1e-14


def test_overlapping_spheres_count_their_union_once():
    # two spheres on a z-edge from z = 1 to 1.5: (1.0625, 1.1875) and
    # (1.125, 1.375) overlap; their union covers (1.0625, 1.375): w = 0.625
    g = grid(5, 5, 6)
    a = inputs.Atoms(np.array([[1.0, 1.0, 1.125], [1.0, 1.0, 1.25]]), np.array([1.0, -1.0]),
                     np.array([0.0625, 0.125]))
    ex, ey, ez, lam = oracle.dielectric(g, a)
    assert abs(w_of(ez[2 + 1, 2, 2]) - 0.625) < 1e-14


def test_fractions_match_fine_sampling():
    p = inputs.random_small(13, 11, 10, 9, n_atoms=25)
    g = p.grid.replace(eps_model="harmonic")
    ex, ey, ez, lam = oracle.dielectric(g, p.atoms)
    xyz, r2 = p.atoms.xyz, p.atoms.r ** 2
    t = (np.arange(4000) + 0.5) / 4000  # midpoint rule: error <= crossings / 4000

    def sampled(start, axis):
        pts = np.repeat(start[None, :], t.size, 0)
        pts[:, axis] += t * g.h
        d2 = ((pts[:, None, :] - xyz[None, :, :]) ** 2).sum(-1)
        return (d2 < r2[None, :]).any(1).mean()

    rng = np.random.default_rng(1)
    o = np.array(g.origin)
    for arr, axis, shape in ((ex, 0, ex.shape), (ey, 1, ey.shape), (ez, 2, ez.shape)):
        idx = np.argwhere(arr != EOUT)
        pick = idx[rng.choice(len(idx), size=min(60, len(idx)), replace=False)]
        for k, j, i in pick:
            node = np.array([i, j, k], dtype=float)
            node[axis] -= 1  # entry 0 along the edge axis is the edge from node -1
            assert abs(w_of(arr[k, j, i]) - sampled(o + node * g.h, axis)) < 2e-3
    assert (ex == EOUT).any() and (ex == EIN).any() and ((ex != EIN) & (ex != EOUT)).any()


def test_consistent_with_the_midpoint_map():
    p = inputs.small_33()
    mid = oracle.dielectric(p.grid, p.atoms)
    har = oracle.dielectric(p.grid.replace(eps_model="harmonic"), p.atoms)
    for m, hv in zip(mid[:3], har[:3]):
        assert (m[hv == EIN] == EIN).all()   # wholly inside: midpoint inside
        assert (m[hv == EOUT] == EOUT).all()  # wholly outside: midpoint outside
        assert ((hv > EIN) & (hv < EOUT))[m == EIN].any()  # partial edges exist
    assert np.array_equal(mid[3], har[3])  # lambda is the node test in both


def test_born_ion_converges_harmonic():
    a = 2.0
    exact = oracle.COULOMB_KCAL / (2 * a) * (1 / EOUT - 1 / EIN)
    errs = []
    for n, h in ((41, 0.5), (81, 0.25)):
        p = inputs.single_charge(n, h, ionic_strength=0.0)
        dG = oracle.solvation_energy(p.grid.replace(eps_model="harmonic"), p.atoms, tol=1e-9)[0]
        errs.append(abs(dG - exact) / abs(exact))
    assert errs[1] < errs[0] < 0.06
    assert errs[1] < 0.02
