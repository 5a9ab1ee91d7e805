"""The launch-configuration autotuner: it returns one of its candidates with a
positive time, caches per shape, and the configuration it picks finds the same
events and computes the same grid (the sweep does not depend on the tiling; a
corrected value may differ in its last bits, since Eq. 8 uses checksums whose
partial sums follow the tiles)."""
import time

import numpy as np
import pytest

from paper_1909_00709_gb300 import inputs
from _util import gpu_context

pytestmark = pytest.mark.gpu

ONLINE = 1


@pytest.fixture(scope="module")
def abi():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1909_00709_gb300 import abi, build
    build.build()
    abi.lib()
    return abi


def _inputs(shapes, seeds):
    tp = [inputs.grid_inputs(*s, seed=k) for s, k in zip(shapes, seeds)]
    return [t for t, _ in tp], [p for _, p in tp], [inputs.hotspot_coeffs(*s) for s in shapes]


@pytest.mark.parametrize("shapes", [[(512, 512, 8)], [(300, 130, 40)], [(200, 37, 5), (64, 64, 8), (129, 17, 30)]])
def test_tuned_configuration_is_valid_and_cached(abi, shapes):
    seeds = list(range(len(shapes)))
    t, p, c = _inputs(shapes, seeds)
    opts, us = abi.autotune(shapes, t, p, c, ONLINE, sweeps=10)
    assert us > 0
    assert opts["tile_y"] in (0, 8, 16, 32) and opts["shallow"] in (0, 1) and opts["persistent"] in (0, 1)
    t0 = time.perf_counter()
    opts2, us2 = abi.autotune(shapes, t, p, c, ONLINE, sweeps=10)
    assert (opts2, us2) == (opts, us)
    assert time.perf_counter() - t0 < 0.5  # served from the cache
    flips = inputs.flip_list([(4, 0, 1, 2, 3, 28), (9, len(shapes) - 1, 0, 1, 1, 25)])
    res = []
    for o in ({}, opts):
        with gpu_context(abi, shapes, seeds, **o) as ctx:
            ctx.inject_list(flips)
            ctx.step(15, ONLINE)
            res.append(([ctx.read(i) for i in range(len(shapes))],
                        sorted((int(e["step"]), int(e["grid"]), int(e["z"]), int(e["y"]), int(e["x"]), int(e["kind"]))
                               for e in ctx.events())))
    for a, b in zip(res[0][0], res[1][0]):
        assert np.max(np.abs(a.astype(np.float64) - b) / np.abs(b)) < 1e-6
    assert res[0][1] == res[1][1] and len(res[0][1]) == 2
