"""Thin ctypes binding of libpb (include/pb.h): argument marshalling only.

Every step of the solve runs in libpb's CUDA kernels; this module converts
Python arguments to the C structs and pointers of the C ABI and turns error
codes into exceptions.  There is no fallback: if libpb.so is missing or no GPU
is visible, the calls raise.

Device arrays are passed as anything with a ``data_ptr()`` method (a CUDA
torch.Tensor) or as an integer device address.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# PB_LIBRARY names another build of the same ABI (the failure-path tests load
# the separately built test copy this way, in a process of their own).
LIB_PATH = os.environ.get("PB_LIBRARY") or os.path.join(_HERE, "libpb.so")

PB_OK, PB_ERR_ARG, PB_ERR_OOM, PB_ERR_CUDA = 0, 1, 2, 3
PB_ERR_NOT_CONVERGED, PB_ERR_BREAKDOWN, PB_ERR_TIMEOUT, PB_ERR_BUSY, PB_ERR_NOT_FOUND = 5, 6, 7, 8, 9
PB_ERR_CANCELLED = 10
COEF = {"packed": 0, "f32": 1, "bf16": 2, "f64": 3}
PB_F64, PB_F32 = 0, 1
PREC = {"f64": 0, "f32": 1, "f32_refine": 2}
PRECOND = {"none": 0, "jacobi": 1, "gmg": 2}
EXPORT = {"eps_x": 0, "eps_y": 1, "eps_z": 2, "lambda": 3, "b": 4, "ghost": 5}
STATUS_NAMES = {0: "OK", 1: "ERR_ARG", 2: "ERR_OOM", 3: "ERR_CUDA", 5: "ERR_NOT_CONVERGED",
                6: "ERR_BREAKDOWN", 7: "ERR_TIMEOUT", 8: "ERR_BUSY", 9: "ERR_NOT_FOUND",
                10: "ERR_CANCELLED"}

#: Every symbol include/pb.h declares (checked by the CPU tests).
EXPORTED = ["pb_last_error", "pb_create", "pb_destroy", "pb_ctx_stats", "pb_setup_grid", "pb_free_grid",
            "pb_grid_update_atoms", "pb_apply_operator", "pb_pcg_solve", "pb_energy",
            "pb_grid_export", "pb_grid_bytes", "pb_solvation_energy"]


class PbError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class GridDesc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("h", ctypes.c_double), ("origin", ctypes.c_double * 3),
                ("eps_in", ctypes.c_double), ("eps_out", ctypes.c_double),
                ("ionic_strength", ctypes.c_double), ("temperature", ctypes.c_double),
                ("kappa_mask", ctypes.c_int), ("coef", ctypes.c_int),
                ("dh_precision", ctypes.c_int), ("periodic", ctypes.c_int),
                ("eps_model", ctypes.c_int)]


class SolveOpts(ctypes.Structure):
    _fields_ = [("precond", ctypes.c_int), ("precision", ctypes.c_int),
                ("rel_tol", ctypes.c_double), ("max_iter", ctypes.c_int),
                ("inner_tol", ctypes.c_double), ("max_outer", ctypes.c_int),
                ("warm_start", ctypes.c_int), ("poll_every", ctypes.c_int),
                ("profile", ctypes.c_int)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("iterations", ctypes.c_int),
                ("outer_steps", ctypes.c_int), ("relres", ctypes.c_double),
                ("relres_true", ctypes.c_double), ("ms_stencil", ctypes.c_double),
                ("ms_update", ctypes.c_double), ("ms_resid", ctypes.c_double),
                ("n_stencil", ctypes.c_int), ("n_update", ctypes.c_int), ("n_resid", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class TuneInfo(ctypes.Structure):
    _fields_ = [("W", ctypes.c_int), ("H", ctypes.c_int), ("tz", ctypes.c_int),
                ("n_tiles", ctypes.c_int), ("candidates", ctypes.c_int),
                ("us_default", ctypes.c_double), ("us_best", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Solvation(ctypes.Structure):
    _fields_ = [("dG", ctypes.c_double), ("e_solv", ctypes.c_double), ("e_ref", ctypes.c_double),
                ("solv", SolveInfo), ("ref", SolveInfo)]


class Request(ctypes.Structure):
    _fields_ = [("trajectory_id", ctypes.c_int64), ("desc", GridDesc), ("n_atoms", ctypes.c_int),
                ("xyz", ctypes.c_void_p), ("q", ctypes.c_void_p), ("radius", ctypes.c_void_p),
                ("phi_out", ctypes.c_void_p)]


class Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("energy", ctypes.c_double), ("info", SolveInfo),
                ("seconds", ctypes.c_double), ("warm_started", ctypes.c_int)]


class KernelProfile(ctypes.Structure):
    _fields_ = [("ms_stencil", ctypes.c_double), ("bytes_stencil", ctypes.c_double),
                ("ms_update", ctypes.c_double), ("bytes_update", ctypes.c_double),
                ("launches_stencil", ctypes.c_int), ("launches_update", ctypes.c_int),
                ("ms_resid", ctypes.c_double), ("bytes_resid", ctypes.c_double),
                ("launches_resid", ctypes.c_int),
                ("first_bytes_stencil", ctypes.c_double * 64), ("first_bytes_update", ctypes.c_double * 64),
                ("first_stencil", ctypes.c_int), ("first_update", ctypes.c_int)]

    def as_dict(self):
        d = {}
        for k, _ in self._fields_:
            v = getattr(self, k)
            d[k] = list(v) if isinstance(v, ctypes.Array) else v
        return d


class BatchPlan(ctypes.Structure):
    _fields_ = [("min_planes", ctypes.c_int), ("height_pct", ctypes.c_int), ("occupancy", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ServerTuneInfo(ctypes.Structure):
    _fields_ = [("plan", BatchPlan), ("candidates", ctypes.c_int), ("gbs_default", ctypes.c_double),
                ("gbs_best", ctypes.c_double)]

    def as_dict(self):
        return {"plan": self.plan.as_dict(), "candidates": self.candidates,
                "gbs_default": self.gbs_default, "gbs_best": self.gbs_best}


class AluRates(ctypes.Structure):
    _fields_ = [("fp64_fma_per_s", ctypes.c_double), ("fp32_fma_per_s", ctypes.c_double),
                ("sms", ctypes.c_int), ("sm_max_mhz", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class SlotState(ctypes.Structure):
    _fields_ = [("trajectory_id", ctypes.c_int64), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("nz", ctypes.c_int), ("bytes", ctypes.c_size_t), ("busy", ctypes.c_int),
                ("last_used", ctypes.c_uint64)]


_lib = None
_P = ctypes.c_void_p


def load(path: str = LIB_PATH):
    """Load libpb.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libpb.so not built at {path}: run paper_1704_02745_gb300/build.py")
    lib = ctypes.CDLL(path)
    lib.pb_last_error.restype = ctypes.c_char_p
    lib.pb_last_error.argtypes = []
    lib.pb_create.argtypes = [ctypes.POINTER(_P), ctypes.c_int, _P]
    lib.pb_destroy.argtypes = [_P]
    lib.pb_ctx_stats.argtypes = [_P, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64),
                                 ctypes.POINTER(ctypes.c_uint64)]
    lib.pb_measure_alu.restype = ctypes.c_int
    lib.pb_measure_alu.argtypes = [_P, ctypes.POINTER(AluRates)]
    lib.pb_setup_grid.argtypes = [_P, ctypes.POINTER(GridDesc), ctypes.c_int, _P, _P, _P,
                                  ctypes.POINTER(_P)]
    lib.pb_free_grid.argtypes = [_P]
    lib.pb_grid_update_atoms.argtypes = [_P, ctypes.c_int, _P, _P, _P]
    lib.pb_apply_operator.argtypes = [_P, _P, _P, ctypes.c_int]
    lib.pb_pcg_solve.argtypes = [_P, ctypes.POINTER(SolveOpts), _P, ctypes.POINTER(SolveInfo)]
    lib.pb_grid_autotune.restype = ctypes.c_int
    lib.pb_grid_autotune.argtypes = [_P, ctypes.c_int, ctypes.POINTER(TuneInfo)]
    lib.pb_energy.argtypes = [_P, _P, ctypes.POINTER(ctypes.c_double)]
    lib.pb_solvation_energy.argtypes = [_P, ctypes.POINTER(GridDesc), ctypes.c_int, _P, _P, _P,
                                        ctypes.POINTER(SolveOpts), _P, ctypes.POINTER(Solvation)]
    lib.pb_grid_export.argtypes = [_P, ctypes.c_int, _P, ctypes.c_size_t]
    lib.pb_grid_bytes.restype = ctypes.c_size_t
    lib.pb_grid_bytes.argtypes = [ctypes.POINTER(GridDesc), ctypes.c_int]
    lib.pb_server_create.argtypes = [_P, ctypes.c_size_t, ctypes.POINTER(SolveOpts), ctypes.POINTER(_P)]
    lib.pb_server_destroy.argtypes = [_P]
    lib.pb_batch_submit.argtypes = [_P, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_uint64)]
    lib.pb_batch_poll.argtypes = [_P, ctypes.c_uint64, ctypes.c_int, ctypes.POINTER(Result)]
    lib.pb_server_set_plan.restype = ctypes.c_int
    lib.pb_server_set_plan.argtypes = [_P, ctypes.POINTER(BatchPlan)]
    lib.pb_server_autotune.restype = ctypes.c_int
    lib.pb_server_autotune.argtypes = [_P, ctypes.c_int, ctypes.POINTER(ServerTuneInfo)]
    lib.pb_batch_cancel.restype = ctypes.c_int
    lib.pb_batch_cancel.argtypes = [_P, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int)]
    lib.pb_server_stats.argtypes = [_P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                    ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_size_t),
                                    ctypes.POINTER(ctypes.c_uint64)]
    lib.pb_energy_noalloc.argtypes = [ctypes.c_int, _P, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                      ctypes.c_double, ctypes.POINTER(ctypes.c_double), _P, _P, _P]
    lib.pb_pinned_alloc.restype = ctypes.c_int
    lib.pb_pinned_alloc.argtypes = [ctypes.c_size_t, ctypes.POINTER(_P)]
    lib.pb_pinned_free.restype = ctypes.c_int
    lib.pb_pinned_free.argtypes = [_P]
    lib.pb_server_profile_begin.argtypes = [_P]
    lib.pb_server_profile_end.argtypes = [_P, ctypes.POINTER(KernelProfile)]
    lib.pb_plan_admission.restype = ctypes.c_int
    lib.pb_plan_admission.argtypes = [ctypes.c_size_t, ctypes.POINTER(SlotState), ctypes.c_int,
                                      _P, _P, _P, ctypes.c_int, _P, _P]
    for name in EXPORTED:
        getattr(lib, name).restype = getattr(lib, name).restype if name in (
            "pb_last_error", "pb_grid_bytes", "pb_plan_admission") else ctypes.c_int
    _lib = lib
    return lib


def _check(st: int):
    if st != PB_OK:
        raise PbError(st, load().pb_last_error().decode())


def _dptr(x) -> int:
    if x is None:
        return 0
    if isinstance(x, int):
        return x
    return int(x.data_ptr())


def grid_desc(g) -> GridDesc:
    """GridDesc from an inputs.GridSpec."""
    d = GridDesc()
    d.nx, d.ny, d.nz = g.nx, g.ny, g.nz
    d.h = g.h
    d.origin[:] = list(g.origin)
    d.eps_in, d.eps_out = g.eps_in, g.eps_out
    d.ionic_strength, d.temperature = g.ionic_strength, g.temperature
    d.kappa_mask = 1 if g.kappa_mask else 0
    d.coef = COEF[g.coef]
    d.dh_precision = PB_F32 if g.dh == "f32" else PB_F64
    d.periodic = 1 if getattr(g, "periodic", False) else 0
    d.eps_model = 1 if getattr(g, "eps_model", "midpoint") == "harmonic" else 0
    return d


def solve_opts(precision="f64", tol=1e-6, precond="jacobi", max_iter=100000, inner_tol=1e-4,
               max_outer=20, warm_start=False, poll_every=0, profile=False) -> SolveOpts:
    o = SolveOpts()
    o.precond = PRECOND[precond]
    o.precision = PREC[precision]
    o.rel_tol = tol
    o.max_iter = max_iter
    o.inner_tol = inner_tol
    o.max_outer = max_outer
    o.warm_start = 1 if warm_start else 0
    o.poll_every = poll_every
    o.profile = 1 if profile else 0
    return o


# --- the C ABI, one Python function per entry point -------------------------

def pb_create(device: int = 0, stream=None) -> int:
    h = _P()
    _check(load().pb_create(ctypes.byref(h), device, _P(stream or 0)))
    return h.value


def pb_destroy(ctx: int):
    _check(load().pb_destroy(_P(ctx)))


def pb_ctx_stats(ctx: int):
    """(kernel launches, host->device bytes, device->host bytes) since pb_create."""
    a, b, c = ctypes.c_uint64(0), ctypes.c_uint64(0), ctypes.c_uint64(0)
    _check(load().pb_ctx_stats(_P(ctx), ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
    return a.value, b.value, c.value


def pb_setup_grid(ctx: int, desc: GridDesc, xyz: np.ndarray, q: np.ndarray, r: np.ndarray) -> int:
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    q = np.ascontiguousarray(q, dtype=np.float64)
    r = np.ascontiguousarray(r, dtype=np.float64)
    h = _P()
    _check(load().pb_setup_grid(_P(ctx), ctypes.byref(desc), int(q.shape[0]),
                                xyz.ctypes.data_as(_P), q.ctypes.data_as(_P),
                                r.ctypes.data_as(_P), ctypes.byref(h)))
    return h.value


def pb_free_grid(grid: int):
    _check(load().pb_free_grid(_P(grid)))


def pb_grid_update_atoms(grid: int, xyz: np.ndarray, q: np.ndarray, r: np.ndarray):
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    q = np.ascontiguousarray(q, dtype=np.float64)
    r = np.ascontiguousarray(r, dtype=np.float64)
    _check(load().pb_grid_update_atoms(_P(grid), int(q.shape[0]), xyz.ctypes.data_as(_P),
                                       q.ctypes.data_as(_P), r.ctypes.data_as(_P)))


def pb_apply_operator(grid: int, u, au, dtype: int = PB_F64):
    _check(load().pb_apply_operator(_P(grid), _P(_dptr(u)), _P(_dptr(au)), dtype))


def pb_pcg_solve(grid: int, opts: SolveOpts, phi, check: bool = True) -> SolveInfo:
    info = SolveInfo()
    st = load().pb_pcg_solve(_P(grid), ctypes.byref(opts), _P(_dptr(phi)), ctypes.byref(info))
    if check:
        _check(st)
    return info


def pb_grid_autotune(grid: int, precision: str = "f32_refine") -> TuneInfo:
    info = TuneInfo()
    _check(load().pb_grid_autotune(_P(grid), PREC[precision], ctypes.byref(info)))
    return info


def pb_energy(grid: int, phi) -> float:
    e = ctypes.c_double(0.0)
    _check(load().pb_energy(_P(grid), _P(_dptr(phi)), ctypes.byref(e)))
    return e.value


def pb_solvation_energy(ctx: int, spec, atoms, phi, check: bool = True, **opts) -> Solvation:
    """dG = E(solvated) - E(reference: eps_in everywhere, no salt); phi is the
    device array of the solvated potential (phi0 if warm_start)."""
    d = grid_desc(spec)
    o = solve_opts(**opts)
    xyz = np.ascontiguousarray(atoms.xyz, dtype=np.float64)
    q = np.ascontiguousarray(atoms.q, dtype=np.float64)
    r = np.ascontiguousarray(atoms.r, dtype=np.float64)
    out = Solvation()
    st = load().pb_solvation_energy(_P(ctx), ctypes.byref(d), int(q.shape[0]), xyz.ctypes.data_as(_P),
                                    q.ctypes.data_as(_P), r.ctypes.data_as(_P), ctypes.byref(o),
                                    _P(_dptr(phi)), ctypes.byref(out))
    if check:
        _check(st)
    return out


def pb_energy_noalloc(xyzq, spec, phi, energy, stream=None):
    """Energy without device allocation: xyzq (n x 4 doubles), phi and the
    one-double `energy` output are device arrays; queued on `stream`."""
    n = int(xyzq.shape[0]) if xyzq is not None else 0
    org = (ctypes.c_double * 3)(*spec.origin)
    _check(load().pb_energy_noalloc(n, _P(_dptr(xyzq)), spec.nx, spec.ny, spec.nz, spec.h, org,
                                    _P(_dptr(phi)), _P(_dptr(energy)), _P(stream or 0)))


def pb_grid_export(grid: int, what: str, shape, dtype) -> np.ndarray:
    out = np.empty(shape, dtype=dtype)
    _check(load().pb_grid_export(_P(grid), EXPORT[what], out.ctypes.data_as(_P), out.nbytes))
    return out


def pb_grid_bytes(desc: GridDesc, precision: str = "f32_refine") -> int:
    return int(load().pb_grid_bytes(ctypes.byref(desc), PREC[precision]))


# --- a small object layer over the same calls -------------------------------

class Context:
    def __init__(self, device: int = 0, stream=None):
        self.handle = pb_create(device, stream)

    def stats(self):
        return pb_ctx_stats(self.handle)

    def measure_alu(self) -> AluRates:
        """pb_measure_alu: the device's measured FP64 and FP32 FMA rates."""
        out = AluRates()
        _check(load().pb_measure_alu(_P(self.handle), ctypes.byref(out)))
        return out

    def solvation(self, spec, atoms, phi, check: bool = True, **opts) -> Solvation:
        return pb_solvation_energy(self.handle, spec, atoms, phi, check=check, **opts)

    def close(self):
        if self.handle:
            pb_destroy(self.handle)
            self.handle = 0

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Grid:
    """A set-up grid: pb_setup_grid on construction, pb_free_grid on close()."""

    def __init__(self, ctx: Context, spec, atoms):
        self.spec = spec
        self.ctx = ctx
        self.handle = pb_setup_grid(ctx.handle, grid_desc(spec), atoms.xyz, atoms.q, atoms.r)

    def close(self):
        if self.handle:
            pb_free_grid(self.handle)
            self.handle = 0

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def update_atoms(self, atoms):
        pb_grid_update_atoms(self.handle, atoms.xyz, atoms.q, atoms.r)

    def export(self, what: str) -> np.ndarray:
        g = self.spec
        nx, ny, nz = g.nx, g.ny, g.nz
        shapes = {"eps_x": ((nz, ny, nx + 1), np.float64), "eps_y": ((nz, ny + 1, nx), np.float64),
                  "eps_z": ((nz + 1, ny, nx), np.float64), "lambda": ((nz, ny, nx), np.uint8),
                  "b": ((nz, ny, nx), np.float64),
                  "ghost": ((2 * (ny * nz + nx * nz + nx * ny),), np.float64)}
        shape, dt = shapes[what]
        return pb_grid_export(self.handle, what, shape, dt)

    def apply(self, u, au, dtype: int = PB_F64):
        pb_apply_operator(self.handle, u, au, dtype)

    def solve(self, phi, check: bool = True, **kw) -> SolveInfo:
        return pb_pcg_solve(self.handle, solve_opts(**kw), phi, check=check)

    def autotune(self, precision: str = "f32_refine") -> TuneInfo:
        """pb_grid_autotune: time candidate stencil tile plans, keep the fastest."""
        return pb_grid_autotune(self.handle, precision)

    def energy(self, phi) -> float:
        return pb_energy(self.handle, phi)


# --- continuous-batching server ---------------------------------------------

def pb_server_create(ctx: int, budget_bytes: int, opts: Optional[SolveOpts] = None) -> int:
    h = _P()
    _check(load().pb_server_create(_P(ctx), budget_bytes, ctypes.byref(opts) if opts else None,
                                   ctypes.byref(h)))
    return h.value


def pb_server_destroy(server: int):
    _check(load().pb_server_destroy(_P(server)))


def pb_batch_submit(server: int, trajectory_id: int, spec, atoms, phi_out: Optional[np.ndarray] = None):
    """Queue one snapshot; returns (ticket, keepalive) -- keep `keepalive` (the
    output buffer) alive until the result is polled."""
    r = Request()
    r.trajectory_id = trajectory_id
    r.desc = grid_desc(spec)
    xyz = np.ascontiguousarray(atoms.xyz, dtype=np.float64)
    q = np.ascontiguousarray(atoms.q, dtype=np.float64)
    rad = np.ascontiguousarray(atoms.r, dtype=np.float64)
    r.n_atoms = int(q.shape[0])
    r.xyz, r.q, r.radius = xyz.ctypes.data, q.ctypes.data, rad.ctypes.data
    r.phi_out = phi_out.ctypes.data if phi_out is not None else None
    t = ctypes.c_uint64(0)
    _check(load().pb_batch_submit(_P(server), ctypes.byref(r), ctypes.byref(t)))
    return t.value


def pb_batch_poll(server: int, ticket: int, timeout_ms: int = -1, check: bool = False):
    """(status, Result).  Status PB_ERR_TIMEOUT when not ready."""
    res = Result()
    st = load().pb_batch_poll(_P(server), ticket, timeout_ms, ctypes.byref(res))
    if check:
        _check(st)
    return st, res


def pb_batch_cancel(server: int, ticket: int) -> bool:
    """True: the request was cancelled (its poll reports PB_ERR_CANCELLED);
    False: its result was complete already."""
    c = ctypes.c_int(0)
    _check(load().pb_batch_cancel(_P(server), ticket, ctypes.byref(c)))
    return bool(c.value)


def pb_server_stats(server: int):
    q, a, r = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
    b, c = ctypes.c_size_t(0), ctypes.c_uint64(0)
    _check(load().pb_server_stats(_P(server), ctypes.byref(q), ctypes.byref(a), ctypes.byref(r),
                                  ctypes.byref(b), ctypes.byref(c)))
    return {"queued": q.value, "active": a.value, "resident": r.value, "bytes": b.value,
            "completed": c.value}


def pb_plan_admission(budget: int, slots, reqs):
    """slots: list of dicts (trajectory_id, dims, bytes, busy, last_used);
    reqs: list of (trajectory_id, dims, bytes).  Returns (admit, evict)."""
    ns, nr = len(slots), len(reqs)
    arr = (SlotState * max(ns, 1))()
    for j, sl in enumerate(slots):
        arr[j].trajectory_id = sl["trajectory_id"]
        arr[j].nx, arr[j].ny, arr[j].nz = sl["dims"]
        arr[j].bytes = sl["bytes"]
        arr[j].busy = 1 if sl["busy"] else 0
        arr[j].last_used = sl["last_used"]
    traj = np.array([r[0] for r in reqs] or [0], dtype=np.int64)
    dims = np.array([d for r in reqs for d in r[1]] or [0, 0, 0], dtype=np.int32)
    nbytes = np.array([r[2] for r in reqs] or [0], dtype=np.uint64)
    admit = np.zeros(max(nr, 1), dtype=np.int32)
    evict = np.zeros(max(ns, 1), dtype=np.int32)
    load().pb_plan_admission(budget, arr, ns, traj.ctypes.data, dims.ctypes.data, nbytes.ctypes.data,
                             nr, admit.ctypes.data, evict.ctypes.data)
    return admit[:nr].tolist(), evict[:ns].tolist()


class _PinnedBlock:
    """One pb_pinned_alloc block; back to its pool when no array views it."""

    def __init__(self, pool, nbytes: int, ptr: int):
        self.pool, self.nbytes, self.ptr = pool, nbytes, ptr

    def __del__(self):
        self.pool._release(self.nbytes, self.ptr)


class PinnedPool:
    """Page-locked float64 arrays for phi_out buffers (the server's device
    copies land in them directly).  Blocks are reused by size: allocating
    page-locked memory costs far more than a copy into it."""

    def __init__(self):
        self._free = {}
        self._closed = False

    @staticmethod
    def size_class(nbytes: int) -> int:
        """Blocks come in classes a quarter of a power of two apart, so grids
        of nearby sizes share them (at most 25% of a block unused)."""
        nbytes = max(int(nbytes), 4096)
        step = 1 << max(nbytes.bit_length() - 3, 12)
        return (nbytes + step - 1) // step * step

    def empty(self, shape) -> np.ndarray:
        n = int(np.prod(shape))
        nbytes = self.size_class(8 * n)
        ptrs = self._free.get(nbytes)
        if ptrs:
            ptr = ptrs.pop()
        else:
            p = _P()
            _check(load().pb_pinned_alloc(nbytes, ctypes.byref(p)))
            ptr = p.value
        buf = (ctypes.c_char * nbytes).from_address(ptr)
        buf._block = _PinnedBlock(self, nbytes, ptr)
        return np.frombuffer(buf, dtype=np.float64, count=n).reshape(shape)

    def _release(self, nbytes: int, ptr: int):
        if self._closed or _lib is None:
            return
        self._free.setdefault(nbytes, []).append(ptr)

    def trim(self):
        """Free the blocks no array views."""
        for ptrs in self._free.values():
            for ptr in ptrs:
                load().pb_pinned_free(_P(ptr))
        self._free.clear()


_pinned_pool = PinnedPool()


def pinned_empty(shape) -> np.ndarray:
    """An uninitialised float64 array in page-locked host memory (pooled)."""
    return _pinned_pool.empty(shape)


class Server:
    """pb_server_create / pb_server_destroy around submit and poll."""

    def __init__(self, ctx: Context, budget_bytes: int, **opts):
        o = solve_opts(**{"precision": "f32_refine", "tol": 1e-6, "inner_tol": 1e-3,
                          "warm_start": True, **opts})
        self.handle = pb_server_create(ctx.handle, int(budget_bytes), o)
        self._keep = {}

    def submit(self, trajectory_id: int, spec, atoms, want_phi: bool = False, phi_out=None) -> int:
        """phi_out: a C-contiguous float64 host array of spec.shape that receives
        phi (held until the poll that returns it; page-locked memory, as from
        pinned_empty, takes the device's copy directly); want_phi allocates a
        page-locked one."""
        out = phi_out
        if out is None and want_phi:
            out = pinned_empty(tuple(spec.shape))
        if out is not None and (out.dtype != np.float64 or out.shape != tuple(spec.shape)
                                or not out.flags.c_contiguous):
            raise ValueError("phi_out must be a C-contiguous float64 array of the grid's shape")
        t = pb_batch_submit(self.handle, trajectory_id, spec, atoms, out)
        self._keep[t] = out
        return t

    def poll(self, ticket: int, timeout_ms: int = -1):
        st, res = pb_batch_poll(self.handle, ticket, timeout_ms)
        if st == PB_ERR_TIMEOUT:
            return None
        phi = self._keep.pop(ticket, None)
        return res, phi

    def stats(self):
        return pb_server_stats(self.handle)

    def set_plan(self, min_planes: int = 32, height_pct: int = 100, occupancy: int = 3):
        """pb_server_set_plan: the batch's tile plan from the next round on."""
        p = BatchPlan(min_planes, height_pct, occupancy)
        _check(load().pb_server_set_plan(_P(self.handle), ctypes.byref(p)))

    def autotune(self, timeout_ms: int = -1) -> ServerTuneInfo:
        """pb_server_autotune: tune the batch's tile plan on the live batch
        (waits until solves are active and the tuning has run)."""
        out = ServerTuneInfo()
        _check(load().pb_server_autotune(_P(self.handle), timeout_ms, ctypes.byref(out)))
        return out

    def cancel(self, ticket: int) -> bool:
        """pb_batch_cancel: True if the request was cancelled."""
        return pb_batch_cancel(self.handle, ticket)

    def profile_begin(self):
        _check(load().pb_server_profile_begin(_P(self.handle)))

    def profile_end(self) -> KernelProfile:
        out = KernelProfile()
        _check(load().pb_server_profile_end(_P(self.handle), ctypes.byref(out)))
        return out

    def close(self):
        if self.handle:
            pb_server_destroy(self.handle)
            self.handle = 0

    def __del__(self):  # a server left open stops its worker before the process exits
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
