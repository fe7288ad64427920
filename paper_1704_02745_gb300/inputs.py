"""Seeded synthetic workload generators for the linear FDPB solve.

This module describes inputs only: atom positions, charges and radii, and the
placement of the uniform grid around them.  It holds none of the solver's
arithmetic (no dielectric map, no charge spreading, no operator), so the CUDA
library and the CPU oracle can both consume the same arrays without sharing
any code of the method.

The shapes follow the paper's workloads (Sec. 2.7): grid spacing 0.5 A, a grid
whose edge is 1.5x the solute's extent, 10^2-10^4 atoms, 10^5-10^7 grid nodes,
solute dielectric 1, solvent 80, potential initialised to zero.  The paper's
573-structure Amber benchmark set, its PDB proteins, Cornell charges and
modified Bondi radii are not available here; uniform random "globules" of
atoms stand in for them:

* positions uniform in a ball of radius R (r = R u^(1/3), isotropic direction),
  overlaps allowed;
* charges uniform in [-1, 1] e;
* radii uniform in [1.5, 2.0] A.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Tuple

import numpy as np

#: Atom number density used to size a globule when only the atom count is given
#: (about 0.04 atoms per cubic Angstrom, as in the 129^3 and 257^3 workloads).
ATOM_DENSITY = 0.04
#: Ratio of the grid edge to the solute extent (Sec. 2.7).
FILL_RATIO = 1.5
#: Largest atom radius drawn by the generators (A).
R_MAX = 2.0


@dataclasses.dataclass
class GridSpec:
    """Uniform grid and physical parameters of one FDPB problem.

    Node (i, j, k) sits at ``origin + (i*h, j*h, k*h)``; unknowns live on all
    ``nx*ny*nz`` nodes and the Dirichlet values on a ghost layer one spacing
    outside the box.  ``coef`` chooses how the CUDA library stores the
    dielectric coefficients ("packed", "f32", "bf16", "f64"); ``dh`` chooses the
    precision of the Debye-Hueckel boundary sum ("f64" or "f32").  ``periodic``
    makes every axis periodic with period n*h (no ghost layer, no boundary sum).
    ``eps_model`` chooses the boundary dielectric: "midpoint" (eps_in when the
    edge midpoint is inside an atom) or "harmonic" (the weighted harmonic
    average over the fraction of the edge inside the atoms).
    """

    nx: int
    ny: int
    nz: int
    h: float
    origin: Tuple[float, float, float]
    eps_in: float = 1.0
    eps_out: float = 80.0
    ionic_strength: float = 0.15  # mol/L
    temperature: float = 300.0  # K
    kappa_mask: bool = True  # lambda = 0 inside atoms (ion exclusion)
    coef: str = "packed"
    dh: str = "f64"
    periodic: bool = False
    eps_model: str = "midpoint"

    @property
    def n(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def shape(self) -> Tuple[int, int, int]:
        """Array shape (nz, ny, nx) of node arrays, x fastest."""
        return (self.nz, self.ny, self.nx)

    def replace(self, **kw) -> "GridSpec":
        return dataclasses.replace(self, **kw)


@dataclasses.dataclass
class Atoms:
    xyz: np.ndarray  # (N, 3) float64, Angstrom
    q: np.ndarray  # (N,) float64, e
    r: np.ndarray  # (N,) float64, Angstrom

    @property
    def n(self) -> int:
        return int(self.q.shape[0])

    def copy(self) -> "Atoms":
        return Atoms(self.xyz.copy(), self.q.copy(), self.r.copy())


@dataclasses.dataclass
class Problem:
    name: str
    grid: GridSpec
    atoms: Atoms


def ball_atoms(rng: np.random.Generator, n_atoms: int, radius: float,
               center=(0.0, 0.0, 0.0)) -> Atoms:
    """n_atoms uniform in a ball; charges U[-1,1] e; radii U[1.5,2.0] A."""
    u = rng.random(n_atoms)
    rad = radius * np.cbrt(u)
    v = rng.normal(size=(n_atoms, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    xyz = np.asarray(center, dtype=np.float64)[None, :] + rad[:, None] * v
    q = rng.uniform(-1.0, 1.0, n_atoms)
    r = rng.uniform(1.5, R_MAX, n_atoms)
    return Atoms(np.ascontiguousarray(xyz, dtype=np.float64),
                 np.ascontiguousarray(q, dtype=np.float64),
                 np.ascontiguousarray(r, dtype=np.float64))


def centered_grid(n: int, h: float, center=(0.0, 0.0, 0.0), **kw) -> GridSpec:
    """Cubic n^3 grid of spacing h whose middle node sits at `center`."""
    half = h * (n - 1) / 2.0
    origin = tuple(float(c) - half for c in center)
    return GridSpec(n, n, n, float(h), origin, **kw)


def globule_radius(n_atoms: int, density: float = ATOM_DENSITY) -> float:
    return (3.0 * n_atoms / (4.0 * math.pi * density)) ** (1.0 / 3.0)


def fill_spacing(n: int, radius: float) -> float:
    """Spacing that makes an n^3 grid 1.5x the solute's extent (2R + 2*rmax)."""
    return FILL_RATIO * (2.0 * radius + 2.0 * R_MAX) / (n - 1)


# ---------------------------------------------------------------------------
# The five workloads
# ---------------------------------------------------------------------------

def small_33(seed: int = 1, **kw) -> Problem:
    """33^3 grid, h = 0.5 A, 200 atoms in a 7 A ball (35,937 unknowns)."""
    rng = np.random.default_rng(seed)
    atoms = ball_atoms(rng, 200, 7.0)
    return Problem("globule33_200atoms", centered_grid(33, 0.5, **kw), atoms)


def globule_129(seed: int = 2, **kw) -> Problem:
    """129^3 grid, h = 0.5 A, 2,500 atoms in a 24 A ball."""
    rng = np.random.default_rng(seed)
    atoms = ball_atoms(rng, 2500, 24.0)
    return Problem("globule129_2500atoms", centered_grid(129, 0.5, **kw), atoms)


def globule_257(seed: int = 3, **kw) -> Problem:
    """257^3 grid (16,974,593 unknowns), h = 0.5 A, 20,000 atoms in a 50 A ball."""
    rng = np.random.default_rng(seed)
    atoms = ball_atoms(rng, 20000, 50.0)
    return Problem("globule257_20000atoms", centered_grid(257, 0.5, **kw), atoms)


def snapshot_batch(seed: int = 4, count: int = 256, n_atoms: int = 1000,
                   radius: float = 18.0, sigma: float = 0.3,
                   n_lo: int = 49, n_hi: int = 97, **kw) -> List[Problem]:
    """Snapshots of one cluster: base + N(0, sigma^2) per coordinate.

    Each snapshot gets a cubic grid with N drawn uniformly from [n_lo, n_hi]
    and the spacing that keeps the fill ratio at 1.5.
    """
    rng = np.random.default_rng(seed)
    base = ball_atoms(rng, n_atoms, radius)
    ns = rng.integers(n_lo, n_hi + 1, size=count)
    out = []
    for s in range(count):
        a = base.copy()
        a.xyz = a.xyz + rng.normal(0.0, sigma, size=a.xyz.shape)
        n = int(ns[s])
        out.append(Problem(f"snap{s}_{n}", centered_grid(n, fill_spacing(n, radius), **kw), a))
    return out


@dataclasses.dataclass
class Trajectory:
    grid: GridSpec
    base: Atoms
    sigma: float
    seed: int

    def snapshot(self, k: int) -> Atoms:
        """Snapshot k of a random walk x_k = x_{k-1} + N(0, sigma^2)."""
        rng = np.random.default_rng([self.seed, 7919])
        a = self.base.copy()
        for _ in range(k):
            a.xyz = a.xyz + rng.normal(0.0, self.sigma, size=a.xyz.shape)
        return a


def trajectories(seed: int = 5, count: int = 16, atoms_lo: int = 300, atoms_hi: int = 8000,
                 n_lo: int = 33, n_hi: int = 193, sigma: float = 0.2, **kw) -> List[Trajectory]:
    """Trajectories with log-uniform atom counts paired (sorted) with odd grid sizes."""
    rng = np.random.default_rng(seed)
    counts = np.sort(np.exp(rng.uniform(math.log(atoms_lo), math.log(atoms_hi), count)).astype(int))
    odd = np.arange(n_lo | 1, n_hi + 1, 2)
    ns = np.sort(rng.choice(odd, size=count, replace=True))
    out = []
    for t in range(count):
        rad = globule_radius(int(counts[t]))
        base = ball_atoms(rng, int(counts[t]), rad)
        n = int(ns[t])
        out.append(Trajectory(centered_grid(n, fill_spacing(n, rad), **kw), base, sigma,
                              seed * 1000 + t))
    return out


def request_stream(trajs: List[Trajectory], n_requests: int, rate_hz: float,
                   seed: int = 5) -> List[Tuple[float, int, int]]:
    """Poisson arrivals: (arrival time s, trajectory id, snapshot index)."""
    rng = np.random.default_rng([seed, 17])
    gaps = rng.exponential(1.0 / rate_hz, n_requests)
    t = np.cumsum(gaps) - gaps[0]
    tid = rng.integers(0, len(trajs), n_requests)
    nxt = [0] * len(trajs)
    out = []
    for a, k in zip(t, tid):
        out.append((float(a), int(k), nxt[k]))
        nxt[k] += 1
    return out


def single_charge(n: int, h: float, q: float = 1.0, radius: float = 2.0, **kw) -> Problem:
    """One charge on the middle node of an n^3 grid (Born ion)."""
    g = centered_grid(n, h, **kw)
    atoms = Atoms(np.zeros((1, 3)), np.array([q], dtype=np.float64),
                  np.array([radius], dtype=np.float64))
    return Problem(f"born{n}", g, atoms)


def random_small(seed: int, nx: int, ny: int, nz: int, h: float = 0.5, n_atoms: int = 20,
                 **kw) -> Problem:
    """Small non-cubic grid with atoms scattered inside its interior."""
    rng = np.random.default_rng(seed)
    ext = np.array([nx - 1, ny - 1, nz - 1], dtype=np.float64) * h
    origin = -ext / 2.0
    lo = origin + 1.01 * h
    hi = origin + ext - 1.01 * h
    xyz = lo + rng.random((n_atoms, 3)) * (hi - lo)
    q = rng.uniform(-1.0, 1.0, n_atoms)
    r = rng.uniform(0.6, 1.4, n_atoms) * h * 2.0
    g = GridSpec(nx, ny, nz, h, tuple(float(v) for v in origin), **kw)
    return Problem(f"rand{nx}x{ny}x{nz}", g, Atoms(xyz, q, r))
