"""Precision variants of the checksum arithmetic (FP32 tile sums, compensated FP32,
FP64) on the 512x512x64 HotSpot3D grid.

Sec. 3.4 sets the detection threshold relative to the checksum's magnitude: it has
to sit above the rounding residual of a fault-free sweep (else false positives) and
it decides which bit flips are still caught (the smaller it is, the lower the bit).
Each variant here
  - runs fault-free online sweeps with the residual tracked: no entry may fail and
    the largest passing residual |a'-a|/|a| is recorded;
  - keeps checksums whose error against the oracle's FP64 sums of the same FP32 grid
    stays within the variant's accumulation bound;
  - with the threshold calibrated to four times its residual, catches every flip whose
    perturbation clears the threshold by the residual's margin and leaves alone every
    flip that stays below it by that margin, locating and correcting the caught ones
    at their true (z, y, x) (Eq. 8).
"""
import numpy as np
import pytest

from paper_1909_00709_gb300 import inputs
from _util import gpu_context

pytestmark = pytest.mark.gpu

ONLINE = 1
SHAPE = (512, 512, 64)
SEED = 11
SWEEPS = 60
ACCS = {0: "fp32", 1: "twosum", 2: "fp64"}
# accumulation bound on |a_gpu - a_exact| / |a_exact|: FP32 sums ty rows in sequence and
# 128 columns pairwise before the FP64 cross-tile sum; the other two are near exact
CHECKSUM_TOL = {0: 4e-6, 1: 1e-11, 2: 1e-11}


@pytest.fixture(scope="module")
def abi():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1909_00709_gb300 import abi, build
    build.build()
    abi.lib()
    return abi


@pytest.fixture(scope="module")
def fault_free(abi, orc):
    """Per variant: the tracked residual, the final grid and its device checksums."""
    out = {}
    for acc in ACCS:
        with gpu_context(abi, [SHAPE], [SEED], acc=acc, track_residual=1) as ctx:
            ctx.step(SWEEPS, ONLINE)
            ev = ctx.events()
            c = ctx.counters()
            u = ctx.read(0)
            a, b = ctx.read_checksums(0)
        out[acc] = dict(events=ev, resid=c["max_residual"], u=u, a=a, b=b)
    return out


@pytest.mark.parametrize("acc", list(ACCS))
def test_no_false_positive_and_residual_recorded(fault_free, acc):
    r = fault_free[acc]
    assert len(r["events"]) == 0, r["events"][:5]
    assert 0.0 < r["resid"] < 1e-5


def test_residual_order(fault_free):
    r32, rts, r64 = (fault_free[a]["resid"] for a in (0, 1, 2))
    # the same FP32 trajectory in all three: compensated and FP64 sums see only the
    # sweep's own rounding, the FP32 tile sums add their own on top
    assert r32 > 1.5 * rts
    assert abs(rts - r64) <= 0.05 * r64


@pytest.mark.parametrize("acc", list(ACCS))
def test_checksums_against_oracle_sums(fault_free, orc, acc):
    r = fault_free[acc]
    a_ref, b_ref = orc.checksums(r["u"])
    ea = np.max(np.abs(r["a"] - a_ref) / np.abs(a_ref))
    eb = np.max(np.abs(r["b"] - b_ref) / np.abs(b_ref))
    assert ea < CHECKSUM_TOL[acc] and eb < CHECKSUM_TOL[acc], (ea, eb)


def _flip_delta(v: np.float32, bit: int) -> float:
    w = np.array([v], dtype=np.float32).view(np.uint32) ^ np.uint32(1 << bit)
    return float(w.view(np.float32)[0]) - float(v)


@pytest.mark.parametrize("acc", list(ACCS))
def test_calibrated_threshold_bit_boundary(abi, fault_free, acc):
    r = fault_free[acc]
    eps = 4.0 * r["resid"]
    rng = np.random.default_rng(100 + acc)
    nx, ny, nz = SHAPE
    entries = []
    for bit in range(32):
        entries.append((2 + 2 * bit, 0, int(rng.integers(1, nz - 1)), int(rng.integers(1, ny - 1)),
                        int(rng.integers(1, nx - 1)), bit))
    flips = inputs.flip_list(entries)
    with gpu_context(abi, [SHAPE], [SEED], acc=acc, eps=eps) as ctx:
        ctx.inject_list(flips)
        ctx.step(2 + 2 * 32, ONLINE)
        ev = ctx.events()
    # the fault-free grid at the end is close enough to the faulted run's values for the
    # size of a flip's perturbation: same binade, same checksum magnitudes to ~1e-6
    u, a, b = r["u"], r["a"], r["b"]
    got = {(int(e["step"]), int(e["z"]), int(e["y"]), int(e["x"])): int(e["kind"]) for e in ev}
    caught = lo_seen = 0
    for (t, _, z, y, x, bit) in entries:
        d = abs(_flip_delta(u[z, y, x], bit))
        big = d / min(abs(a[z, x]), abs(b[z, y]))    # the larger relative perturbation
        small = d / max(abs(a[z, x]), abs(b[z, y]))  # the smaller one
        if not np.isfinite(d) or small > 1.25 * eps:
            assert got.get((t, z, y, x)) == 1, (bit, d, got)
            caught += 1
        elif big < 0.75 * eps:
            assert not any(k[0] == t for k in got), (bit, d, got)
            lo_seen += 1
    assert len(got) <= 32
    assert caught >= 8 and lo_seen >= 1
