"""Whole-column tiles of 7 rows.  A grid swept alone with the default tile height gets
7-row tiles where they put fewer rows on the busiest SM (512 rows: 73 tiles of 7 rows
and a last one of a single row).  The sweep's arithmetic per point does not depend on
the tiling, so unprotected grids equal those of 8-row tiles bit for bit; checksums are
summed over other tile rows, so online runs are compared through their events (flips
well above the threshold) and with the oracle."""
import numpy as np
import pytest

from paper_1909_00709_gb300 import inputs
from _util import compare_events, gpu_context, oracle_run, rel_err

pytestmark = pytest.mark.gpu

NONE, ONLINE = 0, 1


@pytest.fixture(scope="module")
def abi():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1909_00709_gb300 import abi, build
    build.build()
    abi.lib()
    return abi


@pytest.mark.parametrize("shape", [(512, 512, 8), (256, 256, 8), (200, 37, 5), (130, 71, 16)])
@pytest.mark.parametrize("persistent", [1, 0])
def test_unprotected_grids_equal_8_row_tiles(abi, shape, persistent):
    grids = []
    for tile_y in (0, 8):  # 0: the library's choice (7 rows where it balances the SMs)
        with gpu_context(abi, [shape], [11], tile_y=tile_y, persistent=persistent) as ctx:
            ctx.step(20, NONE)
            grids.append(ctx.read(0))
    assert np.array_equal(grids[0].view(np.uint32), grids[1].view(np.uint32))


@pytest.mark.parametrize("vectors", [1, 2])
@pytest.mark.parametrize("persistent", [1, 0])
def test_online_events_equal_8_row_tiles_and_oracle(abi, orc, vectors, persistent):
    shape, steps = (512, 512, 8), 40
    rng = np.random.default_rng(17)
    flips = [(int(t), 0, int(rng.integers(8)), int(y), int(rng.integers(512)), int(rng.integers(20, 31)))
             for t, y in zip(range(3, steps, 4), (0, 6, 7, 13, 14, 255, 510, 511, 503, 1))]
    fl = inputs.flip_list(flips)
    out = []
    for tile_y in (0, 8):
        with gpu_context(abi, [shape], [5], tile_y=tile_y, persistent=persistent, vectors=vectors) as ctx:
            ctx.inject_list(fl)
            ctx.step(steps, ONLINE)
            out.append((ctx.read(0), ctx.events()))
    ref = oracle_run(orc, shape, 5, steps, orc.MODE_ONLINE, fl, vectors=vectors)
    for got, ev in out:
        g, o = compare_events(ev, ref)
        assert g == o and len(o) >= 8
        assert rel_err(got, ref["u"]) < 1e-5
