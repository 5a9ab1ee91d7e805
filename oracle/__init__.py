"""FP64 CPU oracle for ABFT-protected stencil sweeps (arXiv 1909.00709).

TEST INFRASTRUCTURE.  Only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this package; the library under
``paper_1909_00709_gb300`` never does.  The arithmetic lives in ``abft_oracle.c``
(plain C, double precision); this module only marshals numpy arrays through ctypes.

Parity pins: every function is pinned in ``tests/test_oracle_pins.py``; the one
exception ("parity unpinned") is the residual size of the FP32 checksum variants,
which has only an upper bound.
"""
from __future__ import annotations

import ctypes as ct
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "abft_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

CLAMP, PERIODIC, ZERO, CONST = 0, 1, 2, 3
MODE_NONE, MODE_ONLINE, MODE_OFFLINE = 0, 1, 2
EV_CORRECTED, EV_RECOMPUTED, EV_ROLLBACK = 1, 2, 3
TARGET_GRID, TARGET_A, TARGET_B = 0, 1, 2

FLIP = np.dtype([("step", "<i8"), ("grid", "<i4"), ("z", "<i4"), ("y", "<i4"),
                 ("x", "<i4"), ("bit", "<i4"), ("target", "<i4")])
EVENT = np.dtype([("step", "<i8"), ("z", "<i4"), ("y", "<i4"), ("x", "<i4"),
                  ("kind", "<i4"), ("before", "<f8"), ("after", "<f8")])


class _Point(ct.Structure):
    _fields_ = [("dx", ct.c_int32), ("dy", ct.c_int32), ("dz", ct.c_int32), ("w", ct.c_double)]


class _Stencil(ct.Structure):
    _fields_ = [("nx", ct.c_int32), ("ny", ct.c_int32), ("nz", ct.c_int32),
                ("npts", ct.c_int32), ("pts", ct.POINTER(_Point)), ("boundary", ct.c_int32),
                ("bvalue", ct.c_double)]


class _Opts(ct.Structure):
    _fields_ = [("eps", ct.c_double), ("delta", ct.c_int32), ("literal_eq8", ct.c_int32),
                ("band_lo", ct.c_double), ("band_hi", ct.c_double), ("vectors", ct.c_int32)]


class _Out(ct.Structure):
    _fields_ = [("ev", ct.c_void_p), ("ev_cap", ct.c_int64), ("n_ev", ct.c_int64),
                ("marg_step", ct.c_void_p), ("marg_z", ct.c_void_p), ("marg_cap", ct.c_int64),
                ("n_marg", ct.c_int64), ("max_resid", ct.c_double), ("n_rollbacks", ct.c_int64),
                ("n_flips_applied", ct.c_int64)]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, so x86 and Arm agree)."""
    with _lock:
        if not force and os.path.exists(_LIB_PATH) and \
                os.path.getmtime(_LIB_PATH) >= max(os.path.getmtime(_SRC),
                                                   os.path.getmtime(_SRC[:-1] + "h")):
            return _LIB_PATH
        os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-Wall", "-o", tmp, _SRC]
        try:  # OpenMP over the z loops when the toolchain has it
            subprocess.check_call(base + ["-fopenmp", "-lm"], stderr=subprocess.DEVNULL)
        except subprocess.CalledProcessError:
            subprocess.check_call(base + ["-lm"])
        os.replace(tmp, _LIB_PATH)
        return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        lib = ct.CDLL(build())
        P = ct.c_void_p
        lib.orc_set_threads.argtypes = [ct.c_int32]
        lib.orc_max_threads.restype = ct.c_int32
        lib.orc_source_term.argtypes = [ct.c_int64, P, ct.c_float, ct.c_float, ct.c_float, P]
        lib.orc_sweep.argtypes = [ct.POINTER(_Stencil), P, P, P]
        lib.orc_checksums.argtypes = [ct.c_int32, ct.c_int32, ct.c_int32, P, P, P]
        lib.orc_interpolate.argtypes = [ct.POINTER(_Stencil), P, P, P, P, P, P, P]
        lib.orc_interpolate_simple.argtypes = [ct.POINTER(_Stencil), P, P, P, P, P, P]
        lib.orc_interpolate_chain.argtypes = [ct.POINTER(_Stencil), P, P, P, P, P, P, P]
        lib.orc_detect.argtypes = [ct.c_int64, P, P, ct.c_double, P]
        lib.orc_detect.restype = ct.c_int64
        lib.orc_run.argtypes = [ct.POINTER(_Stencil), P, P, ct.c_int64, ct.c_int64, ct.c_int32,
                                P, ct.c_int64, ct.POINTER(_Opts), ct.POINTER(_Out)]
        lib.orc_run.restype = ct.c_int
        lib.orc_splitmix64.argtypes = [ct.c_uint64, ct.c_uint64]
        lib.orc_splitmix64.restype = ct.c_uint64
        lib.orc_schedule.argtypes = [ct.c_uint64, ct.c_double, ct.c_uint32, ct.c_int32, ct.c_int32,
                                     ct.c_int32, ct.c_int32, ct.c_int32, ct.c_int64, ct.c_int64,
                                     P, ct.c_int64]
        lib.orc_schedule.restype = ct.c_int64
        _lib = lib
    return _lib


def set_threads(n: int) -> None:
    """Threads for the oracle's z loops (results do not depend on the count)."""
    _load().orc_set_threads(int(n))


def max_threads() -> int:
    return int(_load().orc_max_threads())


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ct.c_void_p)


def hotspot_points(co: dict):
    """The 7-point set S of the HotSpot-like update: (dx, dy, dz, w)."""
    return [(0, 0, 0, co["cc"]), (-1, 0, 0, co["cw"]), (1, 0, 0, co["ce"]),
            (0, -1, 0, co["cn"]), (0, 1, 0, co["cs"]), (0, 0, -1, co["cb"]), (0, 0, 1, co["ct"])]


class Stencil:
    """Stencil set S on an nx*ny*nz grid with a boundary rule (CONST: every cell outside
    the grid holds `bvalue`)."""

    def __init__(self, shape, points, boundary: int = CLAMP, bvalue: float = 0.0):
        self.nx, self.ny, self.nz = (int(v) for v in shape)
        self.points = [(int(a), int(b), int(c), float(w)) for a, b, c, w in points]
        self._pts = (_Point * len(self.points))(*[_Point(*p) for p in self.points])
        self.c = _Stencil(self.nx, self.ny, self.nz, len(self.points),
                          ct.cast(self._pts, ct.POINTER(_Point)), boundary, float(bvalue))

    @property
    def shape3(self):
        return (self.nz, self.ny, self.nx)


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        assert a.shape == tuple(shape), (a.shape, shape)
    return a


def source_term(power: np.ndarray, co: dict) -> np.ndarray:
    p = np.ascontiguousarray(power, dtype=np.float32)
    C = np.empty(p.shape, dtype=np.float64)
    _load().orc_source_term(p.size, _ptr(p), co["sdc"], co["c_amb"], co["t_amb"], _ptr(C))
    return C


def sweep(st: Stencil, C, u) -> np.ndarray:
    C = _f64(C, st.shape3)
    u = _f64(u, st.shape3)
    out = np.empty_like(u)
    _load().orc_sweep(ct.byref(st.c), _ptr(C), _ptr(u), _ptr(out))
    return out


def checksums(u) -> tuple:
    u = _f64(u)
    nz, ny, nx = u.shape
    a = np.empty((nz, nx))
    b = np.empty((nz, ny))
    _load().orc_checksums(nx, ny, nz, _ptr(u), _ptr(a), _ptr(b))
    return a, b


def interpolate(st: Stencil, cx, cy, a, b, u) -> tuple:
    cx, cy, a, b = (_f64(v) for v in (cx, cy, a, b))
    u = _f64(u, st.shape3)
    ap, bp = np.empty_like(a), np.empty_like(b)
    _load().orc_interpolate(ct.byref(st.c), _ptr(cx), _ptr(cy), _ptr(a), _ptr(b), _ptr(u),
                            _ptr(ap), _ptr(bp))
    return ap, bp


def interpolate_simple(st: Stencil, cx, cy, a, b) -> tuple:
    cx, cy, a, b = (_f64(v) for v in (cx, cy, a, b))
    ap, bp = np.empty_like(a), np.empty_like(b)
    _load().orc_interpolate_simple(ct.byref(st.c), _ptr(cx), _ptr(cy), _ptr(a), _ptr(b),
                                   _ptr(ap), _ptr(bp))
    return ap, bp


def interpolate_chain(st: Stencil, cx, cy, a, b, u) -> tuple:
    """Theorem 1 on predicted vectors a, b with the boundary terms of state u."""
    cx, cy, a, b = (_f64(v) for v in (cx, cy, a, b))
    u = _f64(u, st.shape3)
    ap, bp = np.empty_like(a), np.empty_like(b)
    _load().orc_interpolate_chain(ct.byref(st.c), _ptr(cx), _ptr(cy), _ptr(a), _ptr(b), _ptr(u),
                                  _ptr(ap), _ptr(bp))
    return ap, bp


def detect(pred, comp, eps: float) -> np.ndarray:
    pred, comp = _f64(pred).ravel(), _f64(comp).ravel()
    fail = np.empty(pred.size, dtype=np.int32)
    n = _load().orc_detect(pred.size, _ptr(pred), _ptr(comp), eps, _ptr(fail))
    return fail[:n].copy()


def _as_flips(flips) -> np.ndarray:
    if flips is None or len(flips) == 0:
        return np.zeros(0, dtype=FLIP)
    out = np.zeros(len(flips), dtype=FLIP)
    for name in FLIP.names:
        out[name] = flips[name] if name in flips.dtype.names else 0
    return out


def run(st: Stencil, C, u0, nsteps: int, mode: int, flips=None, *, t0: int = 0,
        eps: float = 1e-5, delta: int = 16, literal_eq8: bool = False,
        band=(0.95, 1.05), vectors: int = 2, ev_cap: int = 1 << 16, marg_cap: int = 1 << 16) -> dict:
    """Run `nsteps` sweeps from u0 (FP64 copy) in the given mode (`vectors`: 2 tests both
    checksum vectors every sweep, 1 tests b and consults a only where b failed).

    Returns the final grid, the event list, the (step, plane) pairs whose residual
    fell inside the guard band, the largest relative residual, rollbacks and flips."""
    C = _f64(C, st.shape3)
    u = _f64(u0, st.shape3).copy()
    fl = _as_flips(flips)
    ev = np.zeros(ev_cap, dtype=EVENT)
    ms = np.zeros(marg_cap, dtype=np.int64)
    mz = np.zeros(marg_cap, dtype=np.int32)
    o = _Opts(eps, delta, int(literal_eq8), band[0], band[1], int(vectors))
    r = _Out(ev.ctypes.data, ev_cap, 0, ms.ctypes.data, mz.ctypes.data, marg_cap, 0, 0.0, 0, 0)
    rc = _load().orc_run(ct.byref(st.c), _ptr(C), _ptr(u), t0, nsteps, mode,
                         _ptr(fl) if len(fl) else None, len(fl), ct.byref(o), ct.byref(r))
    if rc != 0:
        raise RuntimeError(f"orc_run failed with code {rc}")
    n_ev, n_m = min(r.n_ev, ev_cap), min(r.n_marg, marg_cap)
    return dict(u=u, events=ev[:n_ev].copy(), n_events=r.n_ev,
                marginal=set(zip(ms[:n_m].tolist(), mz[:n_m].tolist())),
                max_resid=r.max_resid, n_rollbacks=r.n_rollbacks,
                n_flips_applied=r.n_flips_applied)


def splitmix64(seed: int, counter: int) -> int:
    return int(_load().orc_splitmix64(seed & (2**64 - 1), counter))


def schedule(seed: int, rate: float, bitmask: int, shape, t_begin: int, t_end: int,
             grid: int = 0, n_grids: int = 1, cap: int = 1 << 20) -> np.ndarray:
    nx, ny, nz = shape
    out = np.zeros(cap, dtype=FLIP)
    n = _load().orc_schedule(seed, rate, bitmask, grid, n_grids, nx, ny, nz, t_begin, t_end,
                             _ptr(out), cap)
    return out[:min(n, cap)].copy()
