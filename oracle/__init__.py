"""FP64 CPU oracle for the linear FDPB Jacobi-PCG solve (arXiv:1704.02745).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's
CPU-baseline leg are the only users.  The product path never imports this
package, and this package never imports the CUDA library.

The arithmetic lives in ``pb_oracle.c`` (plain C, FP64, explicit loops,
-ffp-contract=off); this module builds it with gcc and wraps it with ctypes.
Functions and the passage each follows:

* ``kappa_debye2``   -- the Boltzmann coefficient absorbed into kappa^2 (Eq. 2-3)
* ``setup``          -- O1: edge dielectrics, lambda, grid charges, DH boundary, b (Eq. 3-4)
* ``apply``          -- O2: the seven-point operator of Eq. (3)
* ``pcg``            -- O3/O4: CG and Jacobi-preconditioned CG (Sec. 2.2, 2.4)
* ``energy``         -- O5: 1/2 * 332.0637 * sum q phi (the energies compared in Sec. 3.1)
* ``dense_matrix`` / ``cholesky_solve`` -- O6: explicit A and a dense solve, small grids
* ``dielectric``     -- also the weighted harmonic-average boundary dielectric of Sec. 2.7
  (``eps_model="harmonic"``: each edge from the fraction of it inside the atoms)
* ``solvation_energy`` -- the electrostatic solvation energy of Sec. 3.1 (Figs. 1-2):
  energy of the solvated system minus that of the reference system
* ``gmg``            -- geometric-multigrid preconditioned CG (Sec. 2 lists GMG, Sec. 4 names
  multigrid as the next step), numpy, on top of ``apply`` and ``operator_from``

Every function is pinned by the CPU tests (``tests/test_oracle_*.py``) against
closed forms, special cases and brute force; none is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pb_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

OK, ERR_ARG, NOT_CONVERGED, BREAKDOWN = 0, 1, 5, 6
COULOMB_KCAL = 332.0637


def build(force: bool = False) -> str:
    """Compile pb_oracle.c into liboracle.so (gcc, FP64, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-ffp-contract=off",
                               "-fno-fast-math", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("h", ctypes.c_double), ("ox", ctypes.c_double), ("oy", ctypes.c_double),
                ("oz", ctypes.c_double), ("eps_in", ctypes.c_double),
                ("eps_out", ctypes.c_double), ("kappa_d", ctypes.c_double),
                ("kbar2_h2", ctypes.c_double), ("kappa_mask", ctypes.c_int),
                ("periodic", ctypes.c_int)]


_lib = None
_P = ctypes.c_void_p


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.or_kappa_debye2.restype = ctypes.c_double
        lib.or_kappa_debye2.argtypes = [ctypes.c_double] * 3
        G = ctypes.POINTER(_Grid)
        lib.or_dielectric.argtypes = [G, ctypes.c_int, _P, _P, _P, _P, _P, _P]
        lib.or_dielectric_periodic.argtypes = [G, ctypes.c_int, _P, _P, _P, _P, _P, _P]
        lib.or_dielectric_harmonic.argtypes = [G, ctypes.c_int, _P, _P, _P, _P, _P, _P]
        lib.or_spread_charge.restype = ctypes.c_int
        lib.or_spread_charge.argtypes = [G, ctypes.c_int, _P, _P, _P]
        lib.or_dh_ghost.argtypes = [G, ctypes.c_int, _P, _P, _P]
        lib.or_dh_points.argtypes = [G, ctypes.c_int, _P, _P, ctypes.c_int, _P, _P]
        lib.or_rhs.argtypes = [G, _P, _P, _P, _P, _P, _P]
        lib.or_diag.argtypes = [G, _P, _P, _P, _P, _P]
        lib.or_apply.argtypes = [G, _P, _P, _P, _P, _P, _P]
        lib.or_pcg.restype = ctypes.c_int
        lib.or_pcg.argtypes = [G, _P, _P, _P, _P, _P, _P, ctypes.c_int, ctypes.c_double,
                               ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                               ctypes.POINTER(ctypes.c_double)]
        lib.or_energy.restype = ctypes.c_double
        lib.or_energy.argtypes = [G, _P, _P]
        lib.or_dense_matrix.argtypes = [G, _P, _P, _P, _P, _P]
        lib.or_cholesky_solve.restype = ctypes.c_int
        lib.or_cholesky_solve.argtypes = [ctypes.c_int, _P, _P, _P]
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


def kappa_debye2(ionic_strength: float, temperature: float, eps_out: float) -> float:
    """Inverse Debye length squared (1/A^2) of a 1:1 salt."""
    return float(_load().or_kappa_debye2(ionic_strength, temperature, eps_out))


def _cgrid(g) -> _Grid:
    kd2 = kappa_debye2(g.ionic_strength, g.temperature, g.eps_out)
    return _Grid(g.nx, g.ny, g.nz, g.h, g.origin[0], g.origin[1], g.origin[2], g.eps_in,
                 g.eps_out, float(np.sqrt(kd2)), g.eps_out * kd2 * g.h * g.h,
                 1 if g.kappa_mask else 0, 1 if getattr(g, "periodic", False) else 0)


@dataclass
class Setup:
    """Result of O1 for one grid: dense arrays in the layouts of pb_oracle.c."""
    grid: object
    cg: _Grid
    ex: np.ndarray  # (nz, ny, nx+1)
    ey: np.ndarray  # (nz, ny+1, nx)
    ez: np.ndarray  # (nz+1, ny, nx)
    lam: np.ndarray  # (nz, ny, nx) uint8
    q_node: np.ndarray  # (nz, ny, nx)
    ghost: np.ndarray  # concatenated faces x-, x+, y-, y+, z-, z+
    b: np.ndarray  # (nz, ny, nx)
    diag: np.ndarray  # (nz, ny, nx)

    @property
    def kbar2_h2(self) -> float:
        return self.cg.kbar2_h2


class OracleArgError(ValueError):
    pass


def dielectric(grid, atoms):
    lib = _load()
    g = _cgrid(grid)
    nx, ny, nz = grid.nx, grid.ny, grid.nz
    ex = np.empty((nz, ny, nx + 1)); ey = np.empty((nz, ny + 1, nx)); ez = np.empty((nz + 1, ny, nx))
    lam = np.empty((nz, ny, nx), dtype=np.uint8)
    xyz = np.ascontiguousarray(atoms.xyz, dtype=np.float64)
    r = np.ascontiguousarray(atoms.r, dtype=np.float64)
    harmonic = getattr(grid, "eps_model", "midpoint") == "harmonic"
    if harmonic and g.periodic:
        raise OracleArgError("the harmonic-average dielectric is defined for the free-space boundary")
    fn = (lib.or_dielectric_harmonic if harmonic else
          lib.or_dielectric_periodic if g.periodic else lib.or_dielectric)
    fn(ctypes.byref(g), atoms.n, _ptr(xyz), _ptr(r), _ptr(ex), _ptr(ey), _ptr(ez), _ptr(lam))
    return ex, ey, ez, lam


def spread_charge(grid, atoms) -> np.ndarray:
    lib = _load()
    g = _cgrid(grid)
    qn = np.empty(grid.shape)
    xyz = np.ascontiguousarray(atoms.xyz, dtype=np.float64)
    q = np.ascontiguousarray(atoms.q, dtype=np.float64)
    if lib.or_spread_charge(ctypes.byref(g), atoms.n, _ptr(xyz), _ptr(q), _ptr(qn)) != OK:
        raise OracleArgError("an atom's trilinear cell leaves the grid")
    return qn


def ghost_count(grid) -> int:
    nx, ny, nz = grid.nx, grid.ny, grid.nz
    return 2 * (ny * nz + nx * nz + nx * ny)


def dh_ghost(grid, atoms) -> np.ndarray:
    lib = _load()
    g = _cgrid(grid)
    out = np.empty(ghost_count(grid))
    xyz = np.ascontiguousarray(atoms.xyz, dtype=np.float64)
    q = np.ascontiguousarray(atoms.q, dtype=np.float64)
    lib.or_dh_ghost(ctypes.byref(g), atoms.n, _ptr(xyz), _ptr(q), _ptr(out))
    return out


def ghost_positions(grid) -> np.ndarray:
    """Coordinates (n_ghost x 3) of the ghost nodes in the face order of dh_ghost."""
    nx, ny, nz, h = grid.nx, grid.ny, grid.nz, grid.h
    ox, oy, oz = grid.origin
    out = []
    for gi in (-1, nx):
        K, J = np.meshgrid(np.arange(nz), np.arange(ny), indexing="ij")
        out.append(np.stack([np.full(K.size, ox + gi * h), oy + J.ravel() * h, oz + K.ravel() * h], 1))
    for gj in (-1, ny):
        K, I = np.meshgrid(np.arange(nz), np.arange(nx), indexing="ij")
        out.append(np.stack([ox + I.ravel() * h, np.full(K.size, oy + gj * h), oz + K.ravel() * h], 1))
    for gk in (-1, nz):
        J, I = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
        out.append(np.stack([ox + I.ravel() * h, oy + J.ravel() * h, np.full(J.size, oz + gk * h)], 1))
    return np.ascontiguousarray(np.concatenate(out), dtype=np.float64)


def dh_points(grid, atoms, points: np.ndarray) -> np.ndarray:
    """Debye-Hueckel potential of the atoms at arbitrary points (n x 3)."""
    lib = _load()
    g = _cgrid(grid)
    pts = np.ascontiguousarray(points, dtype=np.float64).reshape(-1, 3)
    out = np.empty(pts.shape[0])
    xyz = np.ascontiguousarray(atoms.xyz, dtype=np.float64)
    q = np.ascontiguousarray(atoms.q, dtype=np.float64)
    lib.or_dh_points(ctypes.byref(g), atoms.n, _ptr(xyz), _ptr(q), pts.shape[0], _ptr(pts), _ptr(out))
    return out


def setup(grid, atoms, ghost: Optional[np.ndarray] = None) -> Setup:
    """O1 for one problem.  `ghost` may be passed to skip the O(atoms x faces) DH sum.
    A periodic grid has no boundary: no ghost values, nothing folded into b."""
    lib = _load()
    g = _cgrid(grid)
    ex, ey, ez, lam = dielectric(grid, atoms)
    qn = spread_charge(grid, atoms)
    if g.periodic:
        ghost = np.zeros(ghost_count(grid))
    elif ghost is None:
        ghost = dh_ghost(grid, atoms)
    b = np.empty(grid.shape)
    lib.or_rhs(ctypes.byref(g), _ptr(qn), _ptr(ghost), _ptr(ex), _ptr(ey), _ptr(ez), _ptr(b))
    diag = np.empty(grid.shape)
    lib.or_diag(ctypes.byref(g), _ptr(ex), _ptr(ey), _ptr(ez), _ptr(lam), _ptr(diag))
    return Setup(grid, g, ex, ey, ez, lam, qn, ghost, b, diag)


def operator_from(grid, ex, ey, ez, lam) -> Setup:
    """A Setup holding only an operator (no charges), e.g. for random coefficients."""
    lib = _load()
    g = _cgrid(grid)
    ex, ey, ez = (np.array(a, dtype=np.float64, order="C") for a in (ex, ey, ez))
    lam = np.ascontiguousarray(lam, dtype=np.uint8)
    if g.periodic:  # the entries at -1 are the wrap-around edges (entries n-1)
        ex[:, :, 0] = ex[:, :, -1]
        ey[:, 0, :] = ey[:, -1, :]
        ez[0, :, :] = ez[-1, :, :]
    diag = np.empty(grid.shape)
    lib.or_diag(ctypes.byref(g), _ptr(ex), _ptr(ey), _ptr(ez), _ptr(lam), _ptr(diag))
    z = np.zeros(grid.shape)
    return Setup(grid, g, ex, ey, ez, lam, z, np.zeros(ghost_count(grid)), z.copy(), diag)


def apply(s: Setup, u: np.ndarray) -> np.ndarray:
    lib = _load()
    u = np.ascontiguousarray(u, dtype=np.float64).reshape(s.grid.shape)
    au = np.empty_like(u)
    lib.or_apply(ctypes.byref(s.cg), _ptr(s.ex), _ptr(s.ey), _ptr(s.ez), _ptr(s.diag), _ptr(u),
                 _ptr(au))
    return au


@dataclass
class SolveResult:
    phi: np.ndarray
    iters: int
    relres: float
    status: int


def pcg(s: Setup, b: Optional[np.ndarray] = None, tol: float = 1e-6, max_iter: int = 100000,
        precond: bool = True, phi0: Optional[np.ndarray] = None) -> SolveResult:
    lib = _load()
    b = s.b if b is None else np.ascontiguousarray(b, dtype=np.float64).reshape(s.grid.shape)
    phi = np.zeros(s.grid.shape) if phi0 is None else np.array(phi0, dtype=np.float64).reshape(
        s.grid.shape)
    it = ctypes.c_int(0)
    rr = ctypes.c_double(0.0)
    st = lib.or_pcg(ctypes.byref(s.cg), _ptr(s.ex), _ptr(s.ey), _ptr(s.ez), _ptr(s.diag), _ptr(b),
                    _ptr(phi), 1 if precond else 0, tol, max_iter, ctypes.byref(it),
                    ctypes.byref(rr))
    return SolveResult(phi, it.value, rr.value, st)


def energy(s: Setup, phi: np.ndarray) -> float:
    lib = _load()
    phi = np.ascontiguousarray(phi, dtype=np.float64).reshape(s.grid.shape)
    return float(lib.or_energy(ctypes.byref(s.cg), _ptr(s.q_node), _ptr(phi)))


def dense_matrix(s: Setup) -> np.ndarray:
    lib = _load()
    n = s.grid.n
    A = np.empty((n, n))
    lib.or_dense_matrix(ctypes.byref(s.cg), _ptr(s.ex), _ptr(s.ey), _ptr(s.ez), _ptr(s.diag),
                        _ptr(A))
    return A


def cholesky_solve(A: np.ndarray, b: np.ndarray) -> np.ndarray:
    lib = _load()
    A = np.array(A, dtype=np.float64, order="C")
    b = np.ascontiguousarray(b, dtype=np.float64).ravel()
    x = np.empty_like(b)
    if lib.or_cholesky_solve(A.shape[0], _ptr(A), _ptr(b), _ptr(x)) != OK:
        raise ArithmeticError("matrix not positive definite")
    return x


def relres(s: Setup, phi: np.ndarray, b: Optional[np.ndarray] = None) -> float:
    """True relative residual ||b - A phi|| / ||b|| with the oracle's operator."""
    b = s.b if b is None else b.reshape(s.grid.shape)
    r = b - apply(s, phi)
    return float(np.linalg.norm(r.ravel()) / np.linalg.norm(b.ravel()))


def reference_grid(grid):
    """The reference system of the solvation energy: eps_in everywhere (the
    solute in a medium of its own dielectric) and no salt."""
    return grid.replace(eps_out=grid.eps_in, ionic_strength=0.0)


def solvation_energy(grid, atoms, tol: float = 1e-10):
    """Electrostatic solvation energy (Sec. 3.1, Figs. 1-2): E of the solvated
    system (grid as given) minus E of the reference system, each from a
    Jacobi-PCG solve to `tol`.  Returns (dG, E_solvated, E_reference)."""
    s1 = setup(grid, atoms)
    e1 = energy(s1, pcg(s1, tol=tol).phi)
    s0 = setup(reference_grid(grid), atoms)
    e0 = energy(s0, pcg(s0, tol=tol).phi)
    return e1 - e0, e1, e0
