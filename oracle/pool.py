"""Process pool around the FP64 oracle (test infrastructure, like the rest of
``oracle/``).

The oracle itself stays single-threaded; this module only runs independent
oracle calls side by side in worker processes, so that the large reference
solves of the parity tests and the timed CPU arm of the benchmark finish in
reasonable wall time on a many-core host:

* ``solve_many``  -- complete solves (setup with the full Debye-Hueckel sum,
  Jacobi-PCG, energy) of independent problems, one per worker;
* ``dh_ghost``    -- the Debye-Hueckel boundary values of one grid, the ghost
  nodes split into contiguous pieces (the same per-point sum as
  ``oracle.dh_points``, which the CPU tests pin against ``oracle.dh_ghost``).

Workers are started with the ``spawn`` method: a process forked after the
parent has made a CUDA call can hang, and spawn never inherits that state.
"""
from __future__ import annotations

import multiprocessing as mp
import os
import time
from typing import List, Optional, Sequence

import numpy as np


def host_cores() -> int:
    """Cores this process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover - non-Linux
        return os.cpu_count() or 1


def _pool(procs: int):
    return mp.get_context("spawn").Pool(processes=procs)


def _solve_one(args):
    """One complete oracle solve.  Returns a dict with the energy, the
    iteration count, the status, the wall seconds of setup / solve / energy
    and (when asked) the potential."""
    grid, atoms, tol, want_phi, ghost = args
    import oracle
    t0 = time.perf_counter()
    s = oracle.setup(grid, atoms, ghost=ghost)
    t1 = time.perf_counter()
    r = oracle.pcg(s, tol=tol)
    t2 = time.perf_counter()
    e = oracle.energy(s, r.phi)
    t3 = time.perf_counter()
    out = {"energy": e, "iters": r.iters, "status": r.status, "relres": r.relres,
           "t_setup": t1 - t0, "t_solve": t2 - t1, "t_energy": t3 - t2, "seconds": t3 - t0}
    if want_phi:
        out["phi"] = r.phi
    return out


def solve_many(problems: Sequence, tol: float, procs: Optional[int] = None, want_phi: bool = False,
               ghosts: Optional[Sequence] = None) -> List[dict]:
    """Complete oracle solves of independent (grid, atoms) pairs, in order.
    ``ghosts[i]`` (optional) supplies problem i's boundary values."""
    items = [(g, a, tol, want_phi, None if ghosts is None else ghosts[i])
             for i, (g, a) in enumerate(problems)]
    if not items:
        return []
    procs = max(1, min(procs or host_cores(), len(items)))
    if procs == 1:
        return [_solve_one(it) for it in items]
    with _pool(procs) as p:
        return p.map(_solve_one, items, chunksize=1)


def _reference_check(args):
    """Reference solve of one problem to `tol`, then, for each candidate
    potential, its true relative residual under the oracle's operator and its
    largest deviation from the reference, relative to max|phi_ref|."""
    grid, atoms, tol, candidates, ghost = args
    import oracle
    s = oracle.setup(grid, atoms, ghost=ghost)
    r = oracle.pcg(s, tol=tol)
    scale = float(np.max(np.abs(r.phi)))
    return {"energy": oracle.energy(s, r.phi), "iters": r.iters, "status": r.status,
            "relres_of": [oracle.relres(s, c) for c in candidates],
            "dphi_of": [float(np.max(np.abs(np.asarray(c).reshape(r.phi.shape) - r.phi))) / scale
                        for c in candidates],
            "energy_of": [oracle.energy(s, c) for c in candidates]}


def reference_check(problems: Sequence, candidates: Sequence[Sequence], tol: float,
                    procs: Optional[int] = None) -> List[dict]:
    """For each (grid, atoms) pair: the oracle's solution to `tol` and how each
    of `candidates[i]` (potentials to be checked) compares with it.  One
    worker per problem."""
    items = [(g, a, tol, list(c), None) for (g, a), c in zip(problems, candidates)]
    procs = max(1, min(procs or host_cores(), len(items)))
    if procs == 1:
        return [_reference_check(it) for it in items]
    with _pool(procs) as p:
        return p.map(_reference_check, items, chunksize=1)


def _dh_piece(args):
    grid, atoms, pts = args
    import oracle
    return oracle.dh_points(grid, atoms, pts)


def dh_ghost(grid, atoms, procs: Optional[int] = None) -> np.ndarray:
    """Ghost-node Debye-Hueckel values of ``grid`` (the order of
    ``oracle.dh_ghost``), computed piecewise in worker processes."""
    import oracle
    pts = oracle.ghost_positions(grid)
    procs = max(1, procs or host_cores())
    if procs == 1:
        return oracle.dh_points(grid, atoms, pts)
    pieces = np.array_split(pts, 4 * procs)
    with _pool(procs) as p:
        vals = p.map(_dh_piece, [(grid, atoms, piece) for piece in pieces], chunksize=1)
    return np.concatenate(vals)
