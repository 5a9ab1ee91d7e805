"""Seeded synthetic inputs for the ABFT-protected HotSpot3D workloads.

This module only *generates inputs*: initial temperatures, power maps, the
stencil coefficients of a HotSpot-like thermal model, explicit bit-flip lists and
the shapes of the uneven batch.  It holds none of the method's arithmetic (no
sweep, checksum, interpolation, detection or correction), so both the CUDA
library and the FP64 oracle can be fed from it.

The paper evaluates on Rodinia's HotSpot3D (Sec. 5), whose data files and chip
constants are not part of the paper.  Stand-ins used here:

* temperatures i.i.d. U[320, 340] K and power i.i.d. U[0, 1e-3] W per cell,
  FP32, from ``numpy.random.default_rng(seed)``;
* coefficients from a textbook explicit (forward-Euler, 7-point) discretisation
  of  rho*c dT/dt = k lap(T) + q - g_amb (T - T_amb)  on a 16 mm x 16 mm x 0.5 mm
  silicon die, with the time step chosen so that the centre weight is 1/2
  (stable, all weights non-negative).  The update is Eq. (1) with
  C = sdc*P + c_amb*T_amb; every opposite pair of weights is equal.
"""
from __future__ import annotations

import numpy as np

T_LOW, T_HIGH = 320.0, 340.0
P_LOW, P_HIGH = 0.0, 1.0e-3

# physical stand-in for the HotSpot3D chip (SI units)
CHIP_W = 0.016          # m
CHIP_H = 0.016          # m
CHIP_T = 0.0005         # m
K_SI = 100.0            # W/(m K), silicon conductivity
CV_SI = 1.75e6          # J/(m^3 K), silicon volumetric heat capacity
G_PACKAGE = 10.0        # W/K, total conductance die -> ambient
T_AMB = 318.15          # K

COEFF_NAMES = ("cc", "cw", "ce", "cn", "cs", "cb", "ct", "sdc", "c_amb", "t_amb")


def hotspot_coeffs(nx: int, ny: int, nz: int) -> dict:
    """FP32 coefficients of the 7-point HotSpot-like update for an nx*ny*nz die.

    Offsets: cw/ce -> x-1/x+1, cn/cs -> y-1/y+1, cb/ct -> z-1/z+1 (Fig. 2 naming).
    Returned values are Python floats that are exactly representable in FP32.
    """
    f32 = lambda v: float(np.float32(v))
    dx, dy, dz = CHIP_W / nx, CHIP_H / ny, CHIP_T / nz
    cap = CV_SI * dx * dy * dz
    gx = K_SI * dy * dz / dx
    gy = K_SI * dx * dz / dy
    gz = K_SI * dx * dy / dz
    g_amb = G_PACKAGE / (nx * ny * nz)
    dt = 0.5 * cap / (2.0 * (gx + gy + gz) + g_amb)
    cw = f32(dt * gx / cap)
    cn = f32(dt * gy / cap)
    cb = f32(dt * gz / cap)
    c_amb = f32(dt * g_amb / cap)
    cc = f32(1.0 - 2.0 * (cw + cn + cb) - c_amb)
    return dict(cc=cc, cw=cw, ce=cw, cn=cn, cs=cn, cb=cb, ct=cb,
                sdc=f32(dt / cap), c_amb=c_amb, t_amb=f32(T_AMB))


def grid_inputs(nx: int, ny: int, nz: int, seed: int):
    """Initial temperature and power of one grid, each float32 [nz, ny, nx]."""
    rng = np.random.default_rng(seed)
    temp = rng.uniform(T_LOW, T_HIGH, size=(nz, ny, nx)).astype(np.float32)
    power = rng.uniform(P_LOW, P_HIGH, size=(nz, ny, nx)).astype(np.float32)
    return temp, power


FLIP_DTYPE = np.dtype([("step", "<i8"), ("grid", "<i4"), ("z", "<i4"),
                       ("y", "<i4"), ("x", "<i4"), ("bit", "<i4"), ("target", "<i4")])
TARGET_GRID, TARGET_A, TARGET_B = 0, 1, 2


def flips_periodic(shape, nsteps: int, period: int, seed: int, grid: int = 0,
                   bits=range(32)) -> np.ndarray:
    """One flip every `period` steps (at steps period-1, 2*period-1, ...): point
    uniform over the grid, bit uniform over `bits` (the paper injects at a random
    point and bit, Sec. 5.1)."""
    nx, ny, nz = shape
    rng = np.random.default_rng(seed)
    steps = np.arange(period - 1, nsteps, period, dtype=np.int64)
    out = np.zeros(len(steps), dtype=FLIP_DTYPE)
    bits = np.asarray(list(bits), dtype=np.int32)
    for i, t in enumerate(steps):
        out[i] = (t, grid, rng.integers(nz), rng.integers(ny), rng.integers(nx),
                  bits[rng.integers(len(bits))], TARGET_GRID)
    return out


def flip_list(entries) -> np.ndarray:
    """Build a flip array from tuples (step, grid, z, y, x, bit[, target])."""
    out = np.zeros(len(entries), dtype=FLIP_DTYPE)
    for i, e in enumerate(entries):
        e = tuple(e) + (TARGET_GRID,) * (7 - len(e))
        out[i] = e
    return out


def batch_shapes(n_grids: int, seed: int, xy=(64, 1024), z=(4, 64)):
    """Shapes (nx, ny, nz) of the uneven batch: x, y ~ U{64..1024}, z ~ U{4..64}."""
    rng = np.random.default_rng(seed)
    return [(int(rng.integers(xy[0], xy[1] + 1)), int(rng.integers(xy[0], xy[1] + 1)),
             int(rng.integers(z[0], z[1] + 1))) for _ in range(n_grids)]


# Named workloads (shapes, lengths, fault model).  `rate` is the expected number of
# bit-flips per step over a whole grid; `period` an explicit one-flip-per-period list.
WORKLOADS = {
    "hotspot3d_64x64x8": dict(shape=(64, 64, 8), steps=100, mode="online", period=10, seed=0),
    "hotspot3d_512x512x8": dict(shape=(512, 512, 8), steps=1000, mode="online", rate=1e-3, seed=1),
    "hotspot3d_512x512x64": dict(shape=(512, 512, 64), steps=500, mode="online", rate=0.0, seed=2),
    "hotspot3d_batch256": dict(n_grids=256, steps=500, mode="online", rate=0.1, seed=3),
    "hotspot3d_1024x1024x256": dict(shape=(1024, 1024, 256), steps=200, mode="offline",
                                    rate_per_point=1e-6, seed=4),
}
