"""The paper's accuracy experiment (Sec. 5.2, Eq. 9): 64x64x8 HotSpot3D, 128 sweeps,
one bit-flip at a random sweep, point and bit per run; the arithmetic error is the l2
distance of the final grid from the fault-free run.  The paper states that online ABFT
keeps the median error below 1e-4, that offline ABFT (Delta = 16) cancels the error
completely in most runs (the window is recomputed from its checkpoint), and that the
unprotected code's errors are far larger.

The online error of a corrected point is the error of the interpolated checksum Eq. (8)
subtracts from: with compensated (TwoSum) accumulation that is the sweep's own rounding
and the median stays below 1e-4; with FP32 tile sums the checksums' summation error
(~1e-8 relative, ~2e-4 absolute on a 64-point column of ~330) enters the corrected value
and the median sits at ~1e-4, so that variant is held to 3e-4."""
import numpy as np
import pytest

from paper_1909_00709_gb300 import inputs
from _util import gpu_context

pytestmark = pytest.mark.gpu

SHAPE = (64, 64, 8)
SWEEPS = 128
RUNS = 64
NONE, ONLINE, OFFLINE = 0, 1, 2


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
def errors(abi):
    return _campaign(abi, acc=0)


@pytest.fixture(scope="module")
def errors_twosum(abi):
    return _campaign(abi, acc=1, modes=(ONLINE,))


def _campaign(abi, acc, modes=(NONE, ONLINE, OFFLINE)):
    with gpu_context(abi, [SHAPE], [0]) as ctx:
        ctx.step(SWEEPS, NONE)
        ref = ctx.read(0).astype(np.float64)
    nx, ny, nz = SHAPE
    rng = np.random.default_rng(77)
    flips = [(int(rng.integers(SWEEPS)), 0, int(rng.integers(nz)), int(rng.integers(ny)), int(rng.integers(nx)),
              int(rng.integers(32))) for _ in range(RUNS)]
    out = {}
    for mode in modes:
        errs = []
        for f in flips:
            with gpu_context(abi, [SHAPE], [0], acc=acc) as ctx:
                ctx.inject_list(inputs.flip_list([f]))
                ctx.step(SWEEPS, mode)
                u = ctx.read(0).astype(np.float64)
            d = u - ref
            errs.append(float(np.sqrt(np.sum(d * d))) if np.all(np.isfinite(u)) else float("inf"))
        out[mode] = np.array(errs)
    return out


def test_online_median_error_below_1e4_with_compensated_checksums(errors_twosum):
    assert np.median(errors_twosum[ONLINE]) < 1e-4, np.sort(errors_twosum[ONLINE])


def test_online_median_error_with_fp32_checksums(errors):
    assert np.median(errors[ONLINE]) < 3e-4, np.sort(errors[ONLINE])


def test_offline_cancels_the_error_in_most_runs(errors):
    assert np.mean(errors[OFFLINE] == 0.0) > 0.5, np.sort(errors[OFFLINE])
    assert np.median(errors[OFFLINE]) <= np.median(errors[ONLINE])


def test_unprotected_errors_are_far_larger(errors):
    assert np.median(errors[NONE]) > 100 * max(np.median(errors[ONLINE]), 1e-12)
