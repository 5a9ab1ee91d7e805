"""ctypes binding of the C ABI in include/abft.h (argument marshalling only).

Every compute step runs inside libabft.so on the GPU.  PyTorch is used for the
device workspace and the CUDA stream; nothing here computes any part of the
method.  If the library has not been built, ``lib()`` raises: there is no
fallback.
"""
from __future__ import annotations

import ctypes as ct
import os

import numpy as np

from . import build as _build

MODE_NONE, MODE_ONLINE, MODE_OFFLINE = 0, 1, 2
ACC_FP32, ACC_TWOSUM, ACC_FP64 = 0, 1, 2
BC_CLAMP, BC_PERIODIC, BC_ZERO, BC_CONST = 0, 1, 2, 3
MAX_POINTS = 32
EV_CORRECTED, EV_RECOMPUTED, EV_ROLLBACK = 1, 2, 3
KERNEL_KINDS = ("sweep_plain", "sweep_protected", "check_online", "check_offline", "chain", "other",
                "persistent_plain", "persistent_protected")

STATUS = {0: "ABFT_OK", 1: "ABFT_E_INVAL", 2: "ABFT_E_CUDA", 3: "ABFT_E_NOMEM", 4: "ABFT_E_STATE",
          5: "ABFT_E_TIMEOUT", 6: "ABFT_E_UNCORRECTABLE", 7: "ABFT_E_TRUNCATED"}

EXPORTS = ("abft_default_options", "abft_workspace_bytes", "abft_init", "abft_step", "abft_verify",
           "abft_correct", "abft_inject", "abft_inject_list", "abft_schedule", "abft_events",
           "abft_read", "abft_current", "abft_get_counters", "abft_time_kernels",
           "abft_last_error", "abft_status_string", "abft_destroy", "abft_sweep_checksums_static",
           "abft_read_checksums", "abft_selftest_wait", "abft_tune_workspace_bytes", "abft_tune",
           "abft_probe_l2_copy")


class abft_grid(ct.Structure):
    _fields_ = [("nx", ct.c_int32), ("ny", ct.c_int32), ("nz", ct.c_int32)]


class abft_coeffs(ct.Structure):
    _fields_ = [(n, ct.c_float) for n in ("cc", "cw", "ce", "cn", "cs", "cb", "ct", "sdc", "c_amb", "t_amb")]


class abft_options(ct.Structure):
    _fields_ = [("eps", ct.c_double), ("delta", ct.c_int32), ("acc", ct.c_int32),
                ("event_capacity", ct.c_int32), ("graph_steps", ct.c_int32), ("tile_y", ct.c_int32),
                ("max_flips_per_step", ct.c_int32), ("persistent", ct.c_int32), ("shallow", ct.c_int32),
                ("track_residual", ct.c_int32), ("depth", ct.c_int32), ("overlap", ct.c_int32),
                ("batch", ct.c_int32), ("boundary", ct.c_int32), ("vectors", ct.c_int32),
                ("stream", ct.c_void_p), ("stencils", ct.c_void_p), ("boundary_value", ct.c_float)]


class abft_point(ct.Structure):
    _fields_ = [("dx", ct.c_int32), ("dy", ct.c_int32), ("dz", ct.c_int32), ("w", ct.c_float)]


class abft_stencil(ct.Structure):
    _fields_ = [("npts", ct.c_int32), ("pts", abft_point * MAX_POINTS)]


def stencil_array(sets):
    """ctypes array of abft_stencil from per-grid lists of (dx, dy, dz, w)."""
    arr = (abft_stencil * len(sets))()
    for i, pts in enumerate(sets):
        pts = list(pts)
        if not 1 <= len(pts) <= MAX_POINTS:
            raise ValueError(f"a stencil set needs 1..{MAX_POINTS} points")
        arr[i].npts = len(pts)
        for k, (dx, dy, dz, w) in enumerate(pts):
            arr[i].pts[k] = abft_point(int(dx), int(dy), int(dz), float(w))
    return arr


class abft_counters(ct.Structure):
    _fields_ = [("steps_done", ct.c_int64), ("kernel_launches", ct.c_int64), ("events", ct.c_int64),
                ("rollbacks", ct.c_int64), ("flips_scheduled", ct.c_int64), ("max_residual", ct.c_double),
                ("passes_recomputed", ct.c_int64)]


class abft_event(ct.Structure):
    _fields_ = [("step", ct.c_int64), ("grid", ct.c_int32), ("z", ct.c_int32), ("y", ct.c_int32),
                ("x", ct.c_int32), ("kind", ct.c_int32), ("before", ct.c_float), ("after", ct.c_float)]


class abft_flip(ct.Structure):
    _fields_ = [("step", ct.c_int64), ("grid", ct.c_int32), ("z", ct.c_int32), ("y", ct.c_int32),
                ("x", ct.c_int32), ("bit", ct.c_int32), ("target", ct.c_int32)]


# numpy views of the C structs (the C compiler pads abft_event to 40 bytes)
EVENT = np.dtype([("step", "<i8"), ("grid", "<i4"), ("z", "<i4"), ("y", "<i4"), ("x", "<i4"),
                  ("kind", "<i4"), ("before", "<f4"), ("after", "<f4")], align=True)
FLIP = np.dtype([("step", "<i8"), ("grid", "<i4"), ("z", "<i4"), ("y", "<i4"), ("x", "<i4"),
                 ("bit", "<i4"), ("target", "<i4")])

_lib = None


class AbftError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def lib(build_if_missing: bool = False):
    """Load libabft.so (in-tree build).  Raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError(f"CUDA library {path} is not built; call __graft_entry__.build() "
                               "or paper_1909_00709_gb300.build.build()")
        _build.build()
    L = ct.CDLL(path)
    P, I32, I64, U64 = ct.c_void_p, ct.c_int32, ct.c_int64, ct.c_uint64
    L.abft_default_options.argtypes = [ct.POINTER(abft_options)]
    L.abft_default_options.restype = None
    L.abft_workspace_bytes.argtypes = [ct.POINTER(abft_grid), I32, ct.POINTER(abft_options)]
    L.abft_workspace_bytes.restype = ct.c_size_t
    L.abft_init.argtypes = [ct.POINTER(P), ct.POINTER(abft_grid), I32, ct.POINTER(P), ct.POINTER(P),
                            ct.POINTER(abft_coeffs), ct.POINTER(abft_options), P, ct.c_size_t]
    L.abft_step.argtypes = [P, I64, I32]
    L.abft_verify.argtypes = [P, ct.POINTER(I64)]
    L.abft_correct.argtypes = [P, ct.POINTER(I64)]
    L.abft_inject.argtypes = [P, U64, ct.c_double, ct.c_uint32]
    L.abft_inject_list.argtypes = [P, P, I64]
    L.abft_schedule.argtypes = [U64, ct.c_double, ct.c_uint32, I32, I32, I32, I32, I32, I64, I64, P, I64]
    L.abft_schedule.restype = I64
    L.abft_events.argtypes = [P, P, I64, ct.POINTER(I64)]
    L.abft_read.argtypes = [P, I32, P]
    L.abft_current.argtypes = [P, I32, ct.POINTER(P), ct.POINTER(I64)]
    L.abft_read_checksums.argtypes = [P, I32, P, P]
    L.abft_selftest_wait.argtypes = [I32, I64, P, ct.POINTER(ct.c_double)]
    L.abft_tune_workspace_bytes.argtypes = [ct.POINTER(abft_grid), I32, ct.POINTER(abft_options)]
    L.abft_tune_workspace_bytes.restype = ct.c_size_t
    L.abft_tune.argtypes = [ct.POINTER(abft_grid), I32, ct.POINTER(P), ct.POINTER(P), ct.POINTER(abft_coeffs),
                            ct.POINTER(abft_options), I32, I32, P, ct.c_size_t, ct.POINTER(abft_options),
                            ct.POINTER(ct.c_double)]
    L.abft_probe_l2_copy.argtypes = [P, P, ct.c_size_t, I32, P, ct.POINTER(ct.c_double)]
    L.abft_get_counters.argtypes = [P, ct.POINTER(abft_counters)]
    L.abft_time_kernels.argtypes = [P, I64, I32, P, P]
    L.abft_last_error.argtypes = [P]
    L.abft_last_error.restype = ct.c_char_p
    L.abft_status_string.argtypes = [ct.c_int]
    L.abft_status_string.restype = ct.c_char_p
    L.abft_destroy.argtypes = [P]
    L.abft_destroy.restype = None
    for name in ("abft_init", "abft_step", "abft_verify", "abft_correct", "abft_inject", "abft_inject_list",
                 "abft_events", "abft_read", "abft_current", "abft_get_counters", "abft_time_kernels",
                 "abft_read_checksums", "abft_selftest_wait", "abft_tune", "abft_probe_l2_copy"):
        getattr(L, name).restype = ct.c_int
    _lib = L
    return L


# ------------------------------------------------------------ plain wrappers

def abft_default_options(**kw) -> abft_options:
    o = abft_options()
    lib().abft_default_options(ct.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def _grids(shapes):
    arr = (abft_grid * len(shapes))()
    for i, (nx, ny, nz) in enumerate(shapes):
        arr[i] = abft_grid(nx, ny, nz)
    return arr


def abft_workspace_bytes(shapes, opt: abft_options) -> int:
    return int(lib().abft_workspace_bytes(_grids(shapes), len(shapes), ct.byref(opt)))


def abft_schedule(seed: int, rate: float, bitmask: int, shape, t_begin: int, t_end: int,
                  grid: int = 0, n_grids: int = 1, cap: int = 1 << 20) -> np.ndarray:
    nx, ny, nz = shape
    out = np.zeros(cap, dtype=FLIP)
    n = lib().abft_schedule(seed & (2**64 - 1), rate, bitmask, grid, n_grids, nx, ny, nz, t_begin, t_end,
                            out.ctypes.data, cap)
    if n < 0:
        raise AbftError(1, "abft_schedule: invalid arguments")
    return out[:min(n, cap)].copy()


def abft_sweep_checksums_static(u_in: int, C: int, u_out: int, a_out: int, b_out: int, shape, pitch: int,
                                co: dict, stream: int = 0) -> int:
    """One protected sweep plus the checksums of its result, with no allocation
    (device pointers in, device pointers out).  Returns the abft_status code."""
    L = lib()
    f = L.abft_sweep_checksums_static
    if f.argtypes is None:
        P = ct.c_void_p
        f.argtypes = [P, P, P, P, P, ct.c_int32, ct.c_int32, ct.c_int32, ct.c_int64,
                      ct.POINTER(abft_coeffs), P]
        f.restype = ct.c_int
    nx, ny, nz = shape
    c = _coeffs(co)
    return f(u_in, C, u_out, a_out, b_out, nx, ny, nz, pitch, ct.byref(c), stream)


def abft_selftest_wait(which: int, limit_us: int, stream: int = 0):
    """Make one bounded device wait run out (0: grid barrier, 1: mbarrier); returns
    (status, elapsed_ms)."""
    ms = ct.c_double()
    st = lib().abft_selftest_wait(which, limit_us, ct.c_void_p(stream), ct.byref(ms))
    return st, ms.value


def probe_l2_copy(nbytes: int = 8 << 20, passes: int = 400, *, device=None, stream=None) -> float:
    """Sustained L2 copy bandwidth in GB/s (abft_probe_l2_copy on two torch-allocated
    buffers of nbytes each; 2 * nbytes * passes bytes moved)."""
    import torch
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    st = stream if stream is not None else torch.cuda.current_stream(dev)
    src = torch.ones(nbytes // 4, dtype=torch.float32, device=dev)
    dst = torch.empty_like(src)
    ms = ct.c_double()
    with torch.cuda.device(dev):
        r = lib().abft_probe_l2_copy(ct.c_void_p(src.data_ptr()), ct.c_void_p(dst.data_ptr()), nbytes, passes,
                                     ct.c_void_p(st.cuda_stream), ct.byref(ms))
    if r != 0:
        raise AbftError(r, "abft_probe_l2_copy failed")
    return 2.0 * nbytes * passes / (ms.value / 1e3) / 1e9


def abft_tune_workspace_bytes(shapes, opt: abft_options) -> int:
    return lib().abft_tune_workspace_bytes(_grids(shapes), len(shapes), ct.byref(opt))


OPTION_KEYS = ("tile_y", "shallow", "persistent", "batch", "depth")


def autotune(shapes, temps, powers, coeffs, mode: int, sweeps: int = 20, *, device=None, stream=None, **opt_kw):
    """abft_tune on device buffers allocated here: returns (options dict for Context,
    microseconds per sweep of the winner)."""
    import torch
    shapes = [tuple(int(v) for v in s) for s in shapes]
    n = len(shapes)
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    st = stream if stream is not None else torch.cuda.current_stream(dev)
    base = abft_default_options(**opt_kw)
    base.stream = st.cuda_stream
    nbytes = abft_tune_workspace_bytes(shapes, base)
    if nbytes == 0:
        raise AbftError(1, "invalid grid shapes or options")
    ws = torch.empty(nbytes, dtype=torch.uint8, device=dev)

    def ptr(a):  # device tensors are used in place, anything else through host memory
        if isinstance(a, torch.Tensor):
            assert a.dtype == torch.float32 and a.is_contiguous()
            return a, a.data_ptr()
        a = np.ascontiguousarray(a, dtype=np.float32)
        return a, a.ctypes.data
    keep = [ptr(a) for a in list(temps) + list(powers)]
    tp = (ct.c_void_p * n)(*[keep[i][1] for i in range(n)])
    pp = (ct.c_void_p * n)(*[keep[n + i][1] for i in range(n)])
    cos = (abft_coeffs * n)(*[_coeffs(c) for c in coeffs])
    best = abft_options()
    us = ct.c_double()
    with torch.cuda.device(dev):
        r = lib().abft_tune(_grids(shapes), n, tp, pp, cos, ct.byref(base), mode, sweeps,
                            ct.c_void_p(ws.data_ptr()), nbytes, ct.byref(best), ct.byref(us))
    if r != 0:
        raise AbftError(r, "abft_tune failed")
    return {k: getattr(best, k) for k in OPTION_KEYS}, us.value


def abft_status_string(s: int) -> str:
    return lib().abft_status_string(s).decode()


def _coeffs(co: dict) -> abft_coeffs:
    return abft_coeffs(*[co[n] for n in ("cc", "cw", "ce", "cn", "cs", "cb", "ct", "sdc", "c_amb", "t_amb")])


class Context:
    """One abft_ctx plus the torch-allocated device workspace it borrows.

    Methods are named after the C calls they wrap (abft_step -> step, ...)."""

    def __init__(self, shapes, temps, powers, coeffs, *, device=None, stream=None, stencils=None, **opt_kw):
        """stencils: None (each grid's 7-point set from its coefficients) or one list of
        (dx, dy, dz, w) per grid (a general set S of Eq. 1, offsets within -2..2)."""
        import torch
        self._torch = torch
        self.shapes = [tuple(int(v) for v in s) for s in shapes]
        n = len(self.shapes)
        if device is None:
            device = torch.device("cuda", torch.cuda.current_device())
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        opt = abft_default_options(**opt_kw)
        opt.stream = self.stream.cuda_stream
        sarr = None
        if stencils is not None:
            if len(stencils) != n:
                raise ValueError("one stencil set per grid")
            sarr = stencil_array(stencils)
            opt.stencils = ct.cast(sarr, ct.c_void_p)
        self.opt = opt
        nbytes = abft_workspace_bytes(self.shapes, opt)
        if nbytes == 0:
            raise AbftError(1, "invalid grid shapes or options")
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self._keep = []
        tp = (ct.c_void_p * n)()
        pp = (ct.c_void_p * n)()
        for i in range(n):
            tp[i] = self._ptr(temps[i])
            pp[i] = self._ptr(powers[i])
        cos = (abft_coeffs * n)(*[_coeffs(c) for c in coeffs])
        h = ct.c_void_p()
        with torch.cuda.device(self.device):
            st = lib().abft_init(ct.byref(h), _grids(self.shapes), n, tp, pp, cos, ct.byref(opt),
                                 ct.c_void_p(self.workspace.data_ptr()), nbytes)
        if st != 0:
            raise AbftError(st, "abft_init failed")
        self._keep.clear()
        del sarr  # abft_init copied the sets
        opt.stencils = None
        self.h = h

    def _ptr(self, a):
        torch = self._torch
        if isinstance(a, torch.Tensor):
            assert a.dtype == torch.float32 and a.is_contiguous()
            self._keep.append(a)
            return a.data_ptr()
        a = np.ascontiguousarray(a, dtype=np.float32)
        self._keep.append(a)
        return a.ctypes.data

    def _check(self, st: int, what: str, ok=(0,)):
        if st not in ok:
            raise AbftError(st, f"{what}: {lib().abft_last_error(self.h).decode()}")
        return st

    def step(self, n: int, mode: int) -> int:
        return self._check(lib().abft_step(self.h, n, mode), "abft_step", ok=(0, 7))

    def verify(self) -> int:
        v = ct.c_int64()
        self._check(lib().abft_verify(self.h, ct.byref(v)), "abft_verify")
        return v.value

    def correct(self) -> int:
        v = ct.c_int64()
        self._check(lib().abft_correct(self.h, ct.byref(v)), "abft_correct")
        return v.value

    def inject(self, seed: int, rate: float, bitmask: int = 0xFFFFFFFF):
        self._check(lib().abft_inject(self.h, seed & (2**64 - 1), rate, bitmask), "abft_inject")

    def inject_list(self, flips: np.ndarray):
        fl = np.zeros(len(flips), dtype=FLIP)
        for name in FLIP.names:
            fl[name] = flips[name] if name in flips.dtype.names else 0
        self._check(lib().abft_inject_list(self.h, fl.ctypes.data if len(fl) else None, len(fl)),
                    "abft_inject_list")

    def events(self, cap: int = 1 << 16) -> np.ndarray:
        buf = np.zeros(cap, dtype=EVENT)
        n = ct.c_int64()
        self._check(lib().abft_events(self.h, buf.ctypes.data, cap, ct.byref(n)), "abft_events", ok=(0, 7))
        return buf[:min(n.value, cap)].copy()

    def read(self, grid: int = 0, out=None) -> np.ndarray:
        nx, ny, nz = self.shapes[grid]
        if out is None:
            out = np.empty((nz, ny, nx), dtype=np.float32)
        ptr = out.data_ptr() if isinstance(out, self._torch.Tensor) else out.ctypes.data
        self._check(lib().abft_read(self.h, grid, ct.c_void_p(ptr)), "abft_read")
        return out

    def read_checksums(self, grid: int = 0):
        nx, ny, nz = self.shapes[grid]
        a = np.empty((nz, nx), dtype=np.float64)
        b = np.empty((nz, ny), dtype=np.float64)
        self._check(lib().abft_read_checksums(self.h, grid, a.ctypes.data, b.ctypes.data), "abft_read_checksums")
        return a, b

    def current(self, grid: int = 0):
        p = ct.c_void_p()
        pitch = ct.c_int64()
        self._check(lib().abft_current(self.h, grid, ct.byref(p), ct.byref(pitch)), "abft_current")
        return p.value, pitch.value

    def counters(self) -> dict:
        c = abft_counters()
        self._check(lib().abft_get_counters(self.h, ct.byref(c)), "abft_get_counters")
        return {k: getattr(c, k) for k, _ in abft_counters._fields_}

    def time_kernels(self, n: int, mode: int) -> dict:
        nk = len(KERNEL_KINDS)
        ms = (ct.c_double * nk)()
        la = (ct.c_int64 * nk)()
        self._check(lib().abft_time_kernels(self.h, n, mode, ms, la), "abft_time_kernels", ok=(0, 7))
        return {k: (ms[i], la[i]) for i, k in enumerate(KERNEL_KINDS)}

    def close(self):
        if getattr(self, "h", None):
            lib().abft_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
