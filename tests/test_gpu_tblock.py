"""Temporal blocking: depth-k passes (k = 2, 3, 4) advance k unprotected sweeps at once
on shared-memory levels with recomputed halos.  Every level uses the single sweep's
point update and applies the flips of its own sweep to every point it computes, so
the grids must equal depth-1 runs bit for bit, also across tile edges, ragged tails,
flips in the halo, offline windows (the window's last sweep stays a protected single
sweep) and rollbacks; and the oracle's values."""
import numpy as np
import pytest

from paper_1909_00709_gb300 import inputs
from _util import gpu_context, oracle_run, rel_err

pytestmark = pytest.mark.gpu

NONE, ONLINE, OFFLINE = 0, 1, 2
SHAPES = [(200, 37, 5), (129, 17, 3), (300, 130, 40), (64, 64, 8), (1, 7, 1), (33, 1, 4), (257, 64, 9)]


@pytest.fixture(scope="module")
def abi():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1909_00709_gb300 import abi, build
    build.build()
    abi.lib()
    return abi


def _flips(shape, steps, seed):
    nx, ny, nz = shape
    rng = np.random.default_rng(seed)
    out = []
    for t in range(0, steps, 3):
        # points on tile edges (x = 127/128, y = 7/8) and random ones, all bit positions
        for x, y in ((min(127, nx - 1), min(7, ny - 1)), (min(128, nx - 1), min(8, ny - 1)),
                     (int(rng.integers(nx)), int(rng.integers(ny)))):
            out.append((t, 0, int(rng.integers(nz)), y, x, int(rng.integers(32))))
    return inputs.flip_list(out)


def _run(abi, shape, plan, flips, **opt):
    with gpu_context(abi, [shape], [21], persistent=0, **opt) as ctx:
        ctx.inject_list(flips)
        for n, mode in plan:
            ctx.step(n, mode)
        ev = sorted(map(tuple, ctx.events()[["step", "z", "y", "x", "kind"]].tolist()))
        return ctx.read(0), ev, ctx.counters()["rollbacks"]


@pytest.mark.parametrize("depth", [2, 3, 4])
@pytest.mark.parametrize("shape", SHAPES)
def test_unprotected_depth_k_equals_single_sweeps(abi, shape, depth):
    steps = 13  # not a multiple of k: the remainder runs as single sweeps
    fl = _flips(shape, steps, 4)
    ref, _, _ = _run(abi, shape, [(steps, NONE)], fl, depth=1)
    got, _, _ = _run(abi, shape, [(steps, NONE)], fl, depth=depth)
    np.testing.assert_array_equal(got.view(np.uint32), ref.view(np.uint32))


@pytest.mark.parametrize("depth", [2, 3, 4])
@pytest.mark.parametrize("shape", [(200, 37, 5), (300, 130, 40), (257, 64, 9)])
def test_offline_windows_with_depth_equal_single_sweeps(abi, shape, depth):
    plan = [(37, OFFLINE), (5, NONE), (16, OFFLINE), (3, ONLINE)]
    fl = _flips(shape, 61, 8)
    # one checksum vector: the closing online sweeps (blocked passes with depth >= 2) are
    # bit-identical to single sweeps too
    ref = _run(abi, shape, plan, fl, depth=1, vectors=1)
    got = _run(abi, shape, plan, fl, depth=depth, vectors=1)
    np.testing.assert_array_equal(got[0].view(np.uint32), ref[0].view(np.uint32))
    assert got[1] == ref[1] and got[2] == ref[2]
    assert ref[2] > 0  # some windows were rolled back


@pytest.mark.parametrize("depth", [2, 4])
def test_depth_k_matches_oracle(abi, orc, depth):
    shape, steps = (200, 37, 5), 24
    with gpu_context(abi, [shape], [3], persistent=0, depth=depth) as ctx:
        ctx.step(steps, NONE)
        got = ctx.read(0)
    ref = oracle_run(orc, shape, 3, steps, orc.MODE_NONE)["u"]
    assert rel_err(got, ref) < 1e-5 * max(1.0, steps / 100)


# ------------------------------------------------ online checks with temporal blocking

@pytest.mark.parametrize("vectors", [1, 2])
@pytest.mark.parametrize("depth", [2, 3, 4])
@pytest.mark.parametrize("shape", [(200, 37, 5), (300, 130, 40), (257, 64, 9), (33, 1, 4), (64, 64, 8)])
def test_online_blocked_equals_single_sweeps(abi, shape, depth, vectors):
    """Blocked online passes with the per-level check: the events equal single-sweep
    online checks' and so does the grid, bit for bit with one checksum vector (the b sums
    of a pass equal a single sweep's), with flips on tile edges (passes that fail are
    recomputed sweep by sweep, the pass launched after them discarded), a fault-free
    stretch, and a remainder shorter than a pass.  With two vectors a committed pass
    leaves a summed over 8-row tiles (a single sweep's tiles have 16), so an Eq. (8)
    value computed from it later may differ in the last bit."""
    steps = 23
    fl = _flips(shape, 12, 5)  # flips in the first 12 sweeps, none after
    runs = []
    for d in (1, depth):
        with gpu_context(abi, [shape], [7], depth=d, persistent=0, overlap=0, vectors=vectors) as ctx:
            ctx.inject_list(fl)
            ctx.step(steps, ONLINE)
            runs.append((ctx.read(0), ctx.events(), ctx.counters()))
    (u1, e1, c1), (uk, ek, ck) = runs
    if vectors == 1:
        np.testing.assert_array_equal(uk, u1)
    else:  # a committed pass sums a over 8-row tiles: a later Eq. (8) value may differ in the last bit
        np.testing.assert_allclose(uk, u1, rtol=1e-6, atol=0)
    key = lambda ev: sorted((int(e["step"]), int(e["z"]), int(e["y"]), int(e["x"]), int(e["kind"])) for e in ev)
    assert key(ek) == key(e1)
    assert c1["rollbacks"] == ck["rollbacks"] == 0 and ck["steps_done"] == steps
    if len(e1):
        assert ck["passes_recomputed"] >= 1  # at least one pass was recomputed sweep by sweep


@pytest.mark.parametrize("depth", [2, 4])
def test_online_blocked_fault_free_passes_commit(abi, orc, depth):
    shape, steps = (300, 130, 40), 40
    with gpu_context(abi, [shape], [3], depth=depth, persistent=0, overlap=0, track_residual=1) as ctx:
        ctx.step(steps, ONLINE)
        got = ctx.read(0)
        assert len(ctx.events()) == 0
        c = ctx.counters()
        assert c["passes_recomputed"] == 0 and c["max_residual"] < 1e-6
        # the per-level check leaves the checksums of the committed state (Eq. 2, 3)
        a, b = ctx.read_checksums(0)
    ref = oracle_run(orc, shape, 3, steps, orc.MODE_ONLINE)
    assert rel_err(got, ref["u"]) < 1e-5
    u = got.astype(np.float64)
    assert rel_err(b, u.sum(axis=2)) < 1e-6 and rel_err(a, u.sum(axis=1)) < 1e-6


def test_online_blocked_against_oracle_seeded(abi, orc):
    """Seeded flips at 1.5 per sweep, depth 2 with one checksum vector: events and values
    against the oracle (one vector, the same schedule)."""
    shape, steps = (256, 256, 32), 30
    sched = orc.schedule(21, 1.5, 0xFFFFFFFF, shape, 0, steps)
    with gpu_context(abi, [shape], [8], depth=2, persistent=0, overlap=0, vectors=1) as ctx:
        ctx.inject(21, 1.5, 0xFFFFFFFF)
        ctx.step(steps, ONLINE)
        got = ctx.read(0)
        ev = ctx.events()
    ref = oracle_run(orc, shape, 8, steps, orc.MODE_ONLINE, sched, vectors=1)
    from _util import compare_events
    g, o = compare_events(ev, ref)
    assert g == o and len(o) > 5
    assert rel_err(got, ref["u"]) < 1e-4
