"""Geometric-multigrid preconditioned CG (oracle).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle``: only the tests, the smoke
check and the benchmark's CPU leg use it.

The paper lists geometric multigrid among the classical PB solvers (Sec. 2) and
names multigrid solvers tailored to the PB problem as the way to further gains
(Sec. 4).  It fixes no scheme, so this module states one (the reading is in the
design notes) and is the reference the GPU version is checked against:

* levels: vertex-centred coarsening, coarse node I at fine node 2I, coarse size
  (n + 1) // 2 per axis, down to 3 nodes on the shortest axis;
* coarse operator: the same h^2-scaled seven-point operator rediscretised at
  spacing 2h; a coarse edge's eps is the series (harmonic) combination of the
  two fine edges it spans on the fine line through the coarse nodes, lambda is
  the fine node's, and kbar^2 (2h)^2 replaces kbar^2 h^2;
* transfer: trilinear prolongation P (coarse ghosts are zero), restriction
  r_c = P^T r / 2 (the Galerkin scaling of a three-dimensional h^2-scaled
  operator);
* V-cycle: NU damped-Jacobi sweeps (weight OMEGA) before and after the coarse
  correction, COARSE_SWEEPS sweeps on the coarsest level, starting from zero --
  a symmetric positive definite preconditioner;
* outer loop: the preconditioned CG of Sec. 2.2 with z = V(r), FP64, the same
  stopping rule as ``pcg``.
"""
from __future__ import annotations

from typing import List, Optional

import numpy as np

from . import BREAKDOWN, NOT_CONVERGED, OK, Setup, SolveResult, apply, operator_from

OMEGA = 0.8
NU = 2
COARSEST = 3
COARSE_SWEEPS = 20


def coarse_size(n: int) -> int:
    return (n + 1) // 2


def _series(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    return 2.0 / (1.0 / a + 1.0 / b)


def coarsen(s: Setup) -> Optional[Setup]:
    """The next coarser level of an operator, or None at the coarsest."""
    g = s.grid
    if min(g.nx, g.ny, g.nz) <= COARSEST:
        return None
    mx, my, mz = coarse_size(g.nx), coarse_size(g.ny), coarse_size(g.nz)
    gc = g.replace(nx=mx, ny=my, nz=mz, h=2.0 * g.h)
    # edge entry e of a line is the edge between nodes e-1 and e (e = 0..n);
    # coarse entry I spans fine entries 2I-1 and 2I, clipped to the line
    def line(n, m):
        a = np.clip(2 * np.arange(m + 1) - 1, 0, n)
        b = np.clip(2 * np.arange(m + 1), 0, n)
        return a, b
    ax_, bx_ = line(g.nx, mx)
    ay_, by_ = line(g.ny, my)
    az_, bz_ = line(g.nz, mz)
    J, K, I = 2 * np.arange(my), 2 * np.arange(mz), 2 * np.arange(mx)
    ex = s.ex[np.ix_(K, J, np.arange(g.nx + 1))]
    ex_c = _series(ex[:, :, ax_], ex[:, :, bx_])
    ey = s.ey[np.ix_(K, np.arange(g.ny + 1), I)]
    ey_c = _series(ey[:, ay_, :], ey[:, by_, :])
    ez = s.ez[np.ix_(np.arange(g.nz + 1), J, I)]
    ez_c = _series(ez[az_, :, :], ez[bz_, :, :])
    lam_c = s.lam[np.ix_(K, J, I)]
    return operator_from(gc, ex_c, ey_c, ez_c, lam_c)


def hierarchy(s: Setup) -> List[Setup]:
    levels = [s]
    while True:
        c = coarsen(levels[-1])
        if c is None:
            return levels
        levels.append(c)


def _prolong_1d(e: np.ndarray, n: int, axis: int) -> np.ndarray:
    """Linear interpolation along one axis from m coarse to n fine nodes
    (coarse node I at fine 2I; the coarse ghost past the end is zero)."""
    m = e.shape[axis]
    ext = np.concatenate([e, np.zeros_like(np.take(e, [0], axis=axis))], axis=axis)  # ghost m
    i = np.arange(n)
    lo, hi = i // 2, (i + 1) // 2
    even = (i % 2 == 0)
    wlo = np.where(even, 1.0, 0.5)
    whi = np.where(even, 0.0, 0.5)
    lo_v = np.take(ext, np.minimum(lo, m), axis=axis)
    hi_v = np.take(ext, np.minimum(hi, m), axis=axis)
    shape = [1, 1, 1]
    shape[axis] = n
    return lo_v * wlo.reshape(shape) + hi_v * whi.reshape(shape)


def prolong(e: np.ndarray, fine_shape) -> np.ndarray:
    nz, ny, nx = fine_shape
    return _prolong_1d(_prolong_1d(_prolong_1d(e, nx, 2), ny, 1), nz, 0)


def restrict(r: np.ndarray, coarse_shape) -> np.ndarray:
    """P^T r / 2: the transpose of the trilinear prolongation, halved."""
    mz, my, mx = coarse_shape
    out = np.zeros(coarse_shape)
    # P^T as the adjoint of prolong: <P e, r> = <e, P^T r>, column by column
    # of the separable 1D operators
    def pt_1d(v: np.ndarray, m: int, axis: int) -> np.ndarray:
        n = v.shape[axis]
        res_shape = list(v.shape)
        res_shape[axis] = m
        res = np.zeros(res_shape)
        for i in range(n):
            vi = np.take(v, [i], axis=axis)
            if i % 2 == 0:
                if i // 2 < m:
                    idx = [slice(None)] * 3
                    idx[axis] = slice(i // 2, i // 2 + 1)
                    res[tuple(idx)] += vi
            else:
                for c in ((i - 1) // 2, (i + 1) // 2):
                    if c < m:
                        idx = [slice(None)] * 3
                        idx[axis] = slice(c, c + 1)
                        res[tuple(idx)] += 0.5 * vi
        return res
    out = pt_1d(pt_1d(pt_1d(r, mx, 2), my, 1), mz, 0)
    return 0.5 * out


def _jacobi(s: Setup, z: np.ndarray, r: np.ndarray, sweeps: int) -> np.ndarray:
    for _ in range(sweeps):
        z = z + OMEGA * (r - apply(s, z)) / s.diag
    return z


def vcycle(levels: List[Setup], r: np.ndarray, level: int = 0) -> np.ndarray:
    s = levels[level]
    z = np.zeros(s.grid.shape)
    if level == len(levels) - 1:
        return _jacobi(s, z, r, COARSE_SWEEPS)
    z = _jacobi(s, z, r, NU)
    rc = restrict(r - apply(s, z), levels[level + 1].grid.shape)
    z = z + prolong(vcycle(levels, rc, level + 1), s.grid.shape)
    return _jacobi(s, z, r, NU)


def gmg_pcg(s: Setup, tol: float = 1e-6, max_iter: int = 1000,
            phi0: Optional[np.ndarray] = None) -> SolveResult:
    """Preconditioned CG (Sec. 2.2) with the V-cycle as the preconditioner."""
    levels = hierarchy(s)
    b = s.b
    x = np.zeros(s.grid.shape) if phi0 is None else np.array(phi0, dtype=np.float64)
    r = b - apply(s, x)
    bn = np.linalg.norm(b)
    if bn == 0.0:
        return SolveResult(np.zeros(s.grid.shape), 0, 0.0, OK)
    it = 0
    rel = np.linalg.norm(r) / bn
    if rel < tol:
        return SolveResult(x, 0, rel, OK)
    z = vcycle(levels, r)
    p = z.copy()
    rz = float(np.sum(r * z))
    while it < max_iter:
        ap = apply(s, p)
        pap = float(np.sum(p * ap))
        if not (pap > 0.0):
            return SolveResult(x, it, rel, BREAKDOWN)
        alpha = rz / pap
        x = x + alpha * p
        r = r - alpha * ap
        it += 1
        rel = np.linalg.norm(r) / bn
        if rel < tol:
            return SolveResult(x, it, rel, OK)
        z = vcycle(levels, r)
        rz_new = float(np.sum(r * z))
        p = z + (rz_new / rz) * p
        rz = rz_new
    return SolveResult(x, it, rel, NOT_CONVERGED)
