"""Parity of the CUDA path (through the C ABI) with the FP64 oracle on the same seeded
inputs.  Bar: identical sets of detected / located / corrected / recomputed points
and rolled-back windows (outside the oracle's 5 % guard band), zero false positives,
and grid values within 1e-5 relative error per 100 sweeps."""
import numpy as np
import pytest

from paper_1909_00709_gb300 import inputs
from _util import compare_events, gpu_context, oracle_run, rel_err

pytestmark = pytest.mark.gpu

ONLINE, OFFLINE, NONE = 1, 2, 0
# a handful of shapes spanning several tiles and ragged tails in x and y
SHAPES = [(64, 64, 8), (200, 37, 5), (129, 17, 3), (300, 130, 2), (33, 1, 4), (1, 7, 1), (257, 64, 9),
          (150, 40, 20), (64, 33, 37)]


@pytest.fixture(scope="module")
def abi():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1909_00709_gb300 import abi, build
    build.build()
    abi.lib()
    return abi


def value_tol(steps):
    return 1e-5 * max(1.0, steps / 100.0)


@pytest.mark.parametrize("shallow", [0, 1])
@pytest.mark.parametrize("tile_y", [8, 16, 32])
@pytest.mark.parametrize("shape", SHAPES)
def test_one_sweep_matches_eq1(abi, orc, shape, tile_y, shallow):
    with gpu_context(abi, [shape], [3], tile_y=tile_y, shallow=shallow) as ctx:
        ctx.step(1, NONE)
        got = ctx.read(0)
    ref = oracle_run(orc, shape, 3, 1, orc.MODE_NONE)["u"]
    assert rel_err(got, ref) < 1e-6


@pytest.mark.parametrize("shallow", [0, 1])
@pytest.mark.parametrize("persistent", [0, 1])
@pytest.mark.parametrize("acc", [0, 1, 2])
@pytest.mark.parametrize("shape", [(64, 64, 8), (200, 37, 5), (150, 40, 20)])
def test_online_fault_free(abi, orc, shape, acc, persistent, shallow):
    steps = 100
    with gpu_context(abi, [shape], [5], acc=acc, persistent=persistent, shallow=shallow) as ctx:
        ctx.step(steps, ONLINE)
        got = ctx.read(0)
        ev = ctx.events()
    assert len(ev) == 0, ev[:5]
    ref = oracle_run(orc, shape, 5, steps, orc.MODE_ONLINE)
    assert ref["n_events"] == 0
    assert rel_err(got, ref["u"]) < value_tol(steps)


@pytest.mark.parametrize("persistent", [0, 1])
def test_online_one_flip_every_10_steps_64x64x8(abi, orc, persistent):
    """The small workload: 64x64x8, 100 sweeps, one seeded flip every 10 sweeps."""
    shape, steps = (64, 64, 8), 100
    flips = inputs.flips_periodic(shape, steps, 10, seed=0)
    with gpu_context(abi, [shape], [0], persistent=persistent) as ctx:
        ctx.inject_list(flips)
        ctx.step(steps, ONLINE)
        got = ctx.read(0)
        ev = ctx.events()
    ref = oracle_run(orc, shape, 0, steps, orc.MODE_ONLINE, flips)
    g, o = compare_events(ev, ref)
    assert g == o
    assert rel_err(got, ref["u"]) < value_tol(steps)


@pytest.mark.parametrize("bit", list(range(32)))
def test_online_each_bit(abi, orc, bit):
    shape, steps = (64, 64, 8), 12
    flips = inputs.flip_list([(5, 0, 3, 41, 17, bit)])
    with gpu_context(abi, [shape], [1]) as ctx:
        ctx.inject_list(flips)
        ctx.step(steps, ONLINE)
        got = ctx.read(0)
        ev = ctx.events()
    ref = oracle_run(orc, shape, 1, steps, orc.MODE_ONLINE, flips)
    g, o = compare_events(ev, ref)
    assert g == o
    assert (len(o) == 1) == (bit >= 13)
    assert rel_err(got, ref["u"]) < value_tol(steps) + (1e-3 if bit < 13 else 0)


@pytest.mark.parametrize("persistent", [0, 1])
@pytest.mark.parametrize("case", ["two_by_two", "same_row", "same_col", "two_planes"])
def test_online_multi_flip_patterns(abi, orc, case, persistent):
    shape, steps = (200, 37, 5), 8
    e = {"two_by_two": [(3, 0, 2, 5, 7, 30), (3, 0, 2, 20, 150, 28)],
         "same_row": [(3, 0, 2, 5, 7, 30), (3, 0, 2, 5, 150, 28)],
         "same_col": [(3, 0, 2, 5, 7, 30), (3, 0, 2, 30, 7, 28)],
         "two_planes": [(3, 0, 1, 5, 7, 30), (3, 0, 4, 30, 199, 27)]}[case]
    flips = inputs.flip_list(e)
    with gpu_context(abi, [shape], [2], persistent=persistent) as ctx:
        ctx.inject_list(flips)
        ctx.step(steps, ONLINE)
        got = ctx.read(0)
        ev = ctx.events()
    ref = oracle_run(orc, shape, 2, steps, orc.MODE_ONLINE, flips)
    g, o = compare_events(ev, ref)
    assert g == o and len(o) >= 2
    assert rel_err(got, ref["u"]) < value_tol(steps)


@pytest.mark.parametrize("shallow", [0, 1])
@pytest.mark.parametrize("persistent", [0, 1])
@pytest.mark.parametrize("shape", [(64, 64, 8), (200, 37, 5), (140, 70, 19)])
def test_offline_rollback_parity(abi, orc, shape, persistent, shallow):
    steps = 40
    flips = inputs.flip_list([(20, 0, 2, 10, 11, 28), (35, 0, 1, 3, 4, 30), (9, 0, 0, 1, 2, 3)])
    with gpu_context(abi, [shape], [4], persistent=persistent, shallow=shallow) as ctx:
        ctx.inject_list(flips)
        ctx.step(steps, OFFLINE)
        got = ctx.read(0)
        ev = ctx.events()
        cnt = ctx.counters()
    ref = oracle_run(orc, shape, 4, steps, orc.MODE_OFFLINE, flips, delta=16)
    g, o = compare_events(ev, ref)
    assert g == o
    assert cnt["rollbacks"] == ref["n_rollbacks"] == 2
    # rolled-back windows are recomputed without faults; the surviving low-bit flip stays
    assert rel_err(got, ref["u"]) < value_tol(steps)


@pytest.mark.parametrize("shape", [(300, 130, 6), (140, 70, 19)])
@pytest.mark.parametrize("shallow", [0, 1])
@pytest.mark.parametrize("mode", [ONLINE, NONE])
def test_persistent_and_per_launch_paths_agree_bitwise(abi, mode, shallow, shape):
    steps = 37
    flips = inputs.flip_list([(3, 0, 2, 5, 7, 30), (11, 0, 4, 60, 100, 22), (11, 0, 1, 3, 3, 9),
                              (20, 0, 5, 69, 139, 31), (20, 0, 5, 60, 17, 26)])
    out = []
    for persistent in (0, 1):
        with gpu_context(abi, [shape], [12], persistent=persistent, shallow=shallow) as ctx:
            ctx.inject_list(flips)
            ctx.step(steps, mode)
            out.append((ctx.read(0), sorted(map(tuple, ctx.events()[["step", "z", "y", "x", "kind"]].tolist()))))
    np.testing.assert_array_equal(out[0][0], out[1][0])
    assert out[0][1] == out[1][1]


@pytest.mark.parametrize("shape,rate", [((300, 130, 40), 100.0), ((200, 150, 12), 60.0)])
def test_persistent_heavy_flips_recompute_the_speculative_sweep(abi, orc, shape, rate):
    """So many failures in one sweep that repairing the speculative next state point by
    point would exceed a few tiles' work: every CTA recomputes its tiles instead.  The
    result must equal the per-launch path bit for bit and find the oracle's events."""
    steps = 12
    sched = orc.schedule(21, rate, 0xFFFFFFFF, shape, 0, steps)
    assert len(sched) > 400
    out = []
    for persistent in (0, 1):
        with gpu_context(abi, [shape], [13], persistent=persistent, max_flips_per_step=128) as ctx:
            ctx.inject(21, rate, 0xFFFFFFFF)
            ctx.step(steps, ONLINE)
            out.append((ctx.read(0), sorted(map(tuple, ctx.events()[["step", "z", "y", "x", "kind"]].tolist()))))
    np.testing.assert_array_equal(out[0][0].view(np.uint32), out[1][0].view(np.uint32))
    assert out[0][1] == out[1][1]
    ref = oracle_run(orc, shape, 13, steps, orc.MODE_ONLINE, sched)
    marg = ref["marginal"]
    got = {(k[0], k[1], k[2], k[3], k[4]) for k in out[1][1] if (k[0], k[1]) not in marg}
    exp = {(int(e["step"]), int(e["z"]), int(e["y"]), int(e["x"]), int(e["kind"])) for e in ref["events"]
           if (int(e["step"]), int(e["z"])) not in marg}
    assert got == exp
    assert rel_err(out[1][0], ref["u"]) < value_tol(steps)


@pytest.mark.parametrize("rate", [0.0, 0.7, 40.0])
@pytest.mark.parametrize("shape", [(300, 130, 40), (257, 64, 9)])
def test_overlapped_check_matches_sequential(abi, shape, rate):
    """Per-launch online sweeps with each check running beside the next sweep (and the
    conditional recomputation when it corrected something) equal the sequential order
    bit for bit, events included."""
    out = []
    for overlap in (0, 1):
        with gpu_context(abi, [shape], [17], persistent=0, overlap=overlap, max_flips_per_step=64) as ctx:
            if rate:
                ctx.inject(5, rate, 0xFFFFFFFF)
            ctx.step(9, ONLINE)
            ctx.step(14, ONLINE)
            out.append((ctx.read(0), sorted(map(tuple, ctx.events()[["step", "z", "y", "x", "kind"]].tolist()))))
    np.testing.assert_array_equal(out[0][0].view(np.uint32), out[1][0].view(np.uint32))
    assert out[0][1] == out[1][1]
    if rate:
        assert len(out[0][1]) > 0


FIXUP_CASES = {
    # flips in consecutive sweeps at neighbouring points: when sweep 5's flip is
    # corrected, the repaired output of sweep 6 must still carry sweep 6's flip
    "adjacent_sweeps": [(5, 0, 2, 10, 20, 29), (6, 0, 2, 10, 21, 27), (7, 0, 3, 10, 21, 30)],
    "same_point_twice": [(5, 0, 1, 4, 4, 28), (6, 0, 1, 4, 4, 28)],
    "lines_then_neighbour": [(8, 0, 2, 5, 7, 30), (8, 0, 2, 20, 150, 28), (9, 0, 2, 6, 100, 26),
                             (9, 0, 1, 20, 149, 31)],
    "plane_edges": [(4, 0, 0, 0, 0, 29), (4, 0, 5, 129, 299, 30), (5, 0, 0, 1, 0, 27)],
    "last_sweep_of_launch": [(11, 0, 3, 33, 44, 29), (12, 0, 3, 33, 45, 28), (19, 0, 4, 100, 200, 25)],
}


@pytest.mark.parametrize("shallow", [0, 1])
@pytest.mark.parametrize("case", sorted(FIXUP_CASES))
def test_speculative_repair_cases(abi, orc, case, shallow):
    """The persistent online kernel checks sweep s while running sweep s+1 and repairs
    u^{s+1} when sweep s had to be corrected; results must equal checking after every
    sweep (per-launch path, bitwise) and the oracle (events, values)."""
    shape, steps = (300, 130, 6), 20
    flips = inputs.flip_list(FIXUP_CASES[case])
    out = []
    for persistent in (0, 1):
        with gpu_context(abi, [shape], [14], persistent=persistent, shallow=shallow) as ctx:
            ctx.inject_list(flips)
            ctx.step(12, ONLINE)
            ctx.step(steps - 12, ONLINE)  # two launches: the second starts after a trailing check
            out.append((ctx.read(0), ctx.events()))
    np.testing.assert_array_equal(out[0][0], out[1][0])
    key = lambda ev: sorted(map(tuple, ev[["step", "z", "y", "x", "kind"]].tolist()))
    assert key(out[0][1]) == key(out[1][1])
    ref = oracle_run(orc, shape, 14, steps, orc.MODE_ONLINE, flips)
    g, o = compare_events(out[1][1], ref)
    assert g == o and len(o) >= 1
    assert rel_err(out[1][0], ref["u"]) < 1e-5


def test_mixed_modes_continue_consistently(abi, orc):
    """Unprotected, online and offline sweeps interleaved on one context follow the
    same trajectory as the oracle's single run."""
    shape = (130, 70, 5)
    with gpu_context(abi, [shape], [13]) as ctx:
        ctx.step(5, NONE)
        ctx.step(7, ONLINE)
        ctx.step(20, OFFLINE)
        ctx.step(3, NONE)
        ctx.step(4, ONLINE)
        got = ctx.read(0)
        assert len(ctx.events()) == 0
    ref = oracle_run(orc, shape, 13, 39, orc.MODE_NONE)
    assert rel_err(got, ref["u"]) < 1e-5


@pytest.mark.parametrize("persistent", [0, 1])
def test_offline_fault_free_equals_unprotected(abi, persistent):
    shape = (129, 17, 3)
    with gpu_context(abi, [shape], [6], persistent=persistent) as a, gpu_context(abi, [shape], [6]) as b:
        a.step(37, OFFLINE)
        b.step(37, NONE)
        assert len(a.events()) == 0
        np.testing.assert_array_equal(a.read(0), b.read(0))


@pytest.mark.parametrize("delta", [1, 5, 16])
def test_offline_persistent_and_per_launch_agree_bitwise(abi, delta):
    shape, steps = (300, 130, 6), 45
    flips = inputs.flip_list([(3, 0, 2, 5, 7, 30), (11, 0, 4, 60, 100, 22), (12, 0, 1, 3, 3, 9),
                              (33, 0, 5, 129, 299, 31), (44, 0, 0, 0, 0, 26)])
    out = []
    for persistent in (0, 1):
        with gpu_context(abi, [shape], [15], persistent=persistent, delta=delta) as ctx:
            ctx.inject_list(flips)
            ctx.step(20, OFFLINE)
            ctx.step(steps - 20, OFFLINE)
            ev = ctx.events()
            out.append((ctx.read(0), sorted(map(tuple, ev[["step", "kind"]].tolist())), ctx.counters()["rollbacks"]))
    np.testing.assert_array_equal(out[0][0], out[1][0])
    assert out[0][1] == out[1][1] and out[0][2] == out[1][2] >= 1


def test_two_grids_in_one_context(abi, orc):
    shapes = [(64, 64, 8), (200, 37, 5)]
    flips = inputs.flip_list([(4, 0, 3, 10, 20, 29), (6, 1, 2, 30, 100, 25)])
    with gpu_context(abi, shapes, [7, 8]) as ctx:
        ctx.inject_list(flips)
        ctx.step(10, ONLINE)
        ev = ctx.events()
        for gi, (shape, seed) in enumerate(zip(shapes, [7, 8])):
            fl = flips[flips["grid"] == gi]
            ref = oracle_run(orc, shape, seed, 10, orc.MODE_ONLINE, fl)
            g, o = compare_events(ev, ref, grid=gi)
            assert g == o and len(o) == 1
            assert rel_err(ctx.read(gi), ref["u"]) < 1e-5


def test_seeded_schedule_run_matches_oracle(abi, orc):
    shape, steps, seed, rate = (96, 80, 6), 60, 99, 0.3
    with gpu_context(abi, [shape], [9]) as ctx:
        ctx.inject(seed, rate, 0xFFFFFFFF)
        ctx.step(steps, ONLINE)
        got = ctx.read(0)
        ev = ctx.events()
        cnt = ctx.counters()
    sched = orc.schedule(seed, rate, 0xFFFFFFFF, shape, 0, steps)
    assert cnt["flips_scheduled"] == len(sched)
    ref = oracle_run(orc, shape, 9, steps, orc.MODE_ONLINE, sched)
    g, o = compare_events(ev, ref)
    assert g == o
    assert rel_err(got, ref["u"]) < value_tol(steps)


def test_verify_and_correct_point(abi, orc):
    """abft_verify at zero distance after a corrupted online step is not possible; use
    an unprotected sweep with a flip, then verify (chained) and correct (rollback)."""
    shape = (64, 64, 8)
    flips = inputs.flip_list([(2, 0, 3, 4, 5, 29)])
    with gpu_context(abi, [shape], [10]) as ctx:
        ctx.inject_list(flips)
        ctx.step(3, NONE)
        n = ctx.verify()
        assert n >= 2
        fixed = ctx.correct()
        assert fixed == 3
        assert ctx.verify() == 0
        got = ctx.read(0)
    ref = oracle_run(orc, shape, 10, 3, orc.MODE_NONE)
    assert rel_err(got, ref["u"]) < 1e-6


def test_full_size_512x512x8_sampled(abi, orc):
    """512x512x8 in the launch configuration the benchmark times: 1000 online sweeps
    with seeded flips (rate 1e-3 per sweep) and a fault-free run.  The oracle checks
    every scheduled flip (located where it was injected iff its bit is above the
    closed-form detection boundary) and one final sweep point by point."""
    shape, steps = (512, 512, 8), 1000
    ff_events = None
    with gpu_context(abi, [shape], [1]) as ctx:
        ctx.step(steps, ONLINE)
        ff_events = ctx.events()
        ff = ctx.read(0)
    assert len(ff_events) == 0
    seeds = [1, 2, 3]
    located = 0
    for s in seeds:
        sched = orc.schedule(s, 1e-3, 0xFFFFFFFF, shape, 0, steps)
        with gpu_context(abi, [shape], [1]) as ctx:
            ctx.inject(s, 1e-3, 0xFFFFFFFF)
            ctx.step(steps, ONLINE)
            ev = ctx.events()
            got = ctx.read(0)
        expect = {(int(f["step"]), int(f["z"]), int(f["y"]), int(f["x"]), 1) for f in sched if f["bit"] >= 16}
        got_set = {(int(e["step"]), int(e["z"]), int(e["y"]), int(e["x"]), int(e["kind"])) for e in ev}
        assert got_set == expect
        located += len(expect)
        low = [f for f in sched if f["bit"] < 16]
        if not low:
            assert rel_err(got, ff) < 1e-5
    # one more sweep from the GPU's final state against Eq. (1) in FP64
    co = inputs.hotspot_coeffs(*shape)
    _, power = inputs.grid_inputs(*shape, seed=1)
    st = orc.Stencil(shape, orc.hotspot_points(co))
    ref = orc.sweep(st, orc.source_term(power, co), ff.astype(np.float64))
    with abi.Context([shape], [ff], [power], [co]) as c2:  # the final state as a new start
        c2.step(1, NONE)
        one = c2.read(0)
    assert rel_err(one, ref) < 1e-6
