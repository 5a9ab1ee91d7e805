"""One-vector online checks (option vectors = 1, Sec. 3.2): b is summed and tested every
sweep, a is summed from the grid only in planes where b failed, to locate.  Parity with
the FP64 oracle run with the same rule, bitwise agreement of the launch paths, and the
hand-over to offline steps and chained verification (which need a of the verified
state)."""
import numpy as np
import pytest

from paper_1909_00709_gb300 import inputs
from _util import compare_events, gpu_context, oracle_run, rel_err

pytestmark = pytest.mark.gpu

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


def key(ev):
    return sorted(map(tuple, ev[["step", "z", "y", "x", "kind"]].tolist()))


@pytest.mark.parametrize("shallow", [0, 1])
@pytest.mark.parametrize("persistent", [0, 1])
@pytest.mark.parametrize("shape", [(64, 64, 8), (200, 37, 5), (150, 40, 20)])
def test_fault_free(abi, orc, shape, persistent, shallow):
    steps = 80
    with gpu_context(abi, [shape], [5], vectors=1, persistent=persistent, shallow=shallow) as ctx:
        ctx.step(steps, ONLINE)
        got = ctx.read(0)
        assert len(ctx.events()) == 0
    ref = oracle_run(orc, shape, 5, steps, orc.MODE_ONLINE, vectors=1)
    assert ref["n_events"] == 0
    assert rel_err(got, ref["u"]) < 1e-5


@pytest.mark.parametrize("path", ["per_launch", "persistent", "overlapped"])
def test_small_workload_flip_every_10_sweeps(abi, orc, path):
    shape, steps = (64, 64, 8), 100
    flips = inputs.flips_periodic(shape, steps, 10, seed=0)
    opt = {"per_launch": dict(persistent=0, overlap=0), "persistent": dict(persistent=1),
           "overlapped": dict(persistent=0, overlap=1)}[path]
    with gpu_context(abi, [shape], [0], vectors=1, **opt) as ctx:
        ctx.inject_list(flips)
        ctx.step(steps, ONLINE)
        got = ctx.read(0)
        ev = ctx.events()
    ref = oracle_run(orc, shape, 0, steps, orc.MODE_ONLINE, flips, vectors=1)
    g, o = compare_events(ev, ref)
    assert g == o
    assert rel_err(got, ref["u"]) < 1e-5


@pytest.mark.parametrize("persistent", [0, 1])
@pytest.mark.parametrize("bit", [13, 14, 15, 20, 26, 30, 31])
def test_b_threshold_decides(abi, orc, bit, persistent):
    """A non-square plane (nx = 200 > ny = 37): flips that only a's lower threshold would
    see (bits 13, 14 here) pass unseen with one vector, as in the oracle; larger ones are
    located through the on-demand a and corrected."""
    shape, steps = (200, 37, 5), 10
    flips = inputs.flip_list([(6, 0, 2, 20, 150, bit)])
    with gpu_context(abi, [shape], [7], vectors=1, persistent=persistent) as ctx:
        ctx.inject_list(flips)
        ctx.step(steps, ONLINE)
        got = ctx.read(0)
        ev = ctx.events()
    ref = oracle_run(orc, shape, 7, steps, orc.MODE_ONLINE, flips, vectors=1)
    g, o = compare_events(ev, ref)
    assert g == o
    assert (len(o) > 0) == (bit >= 15)
    assert rel_err(got, ref["u"]) < 1e-5 + (1e-3 if bit < 15 else 0)


@pytest.mark.parametrize("persistent", [0, 1])
@pytest.mark.parametrize("case", ["two_by_two", "same_row", "same_col", "two_planes", "faces"])
def test_patterns(abi, orc, case, persistent):
    shape, steps = (200, 37, 5), 8
    e = {"two_by_two": [(3, 0, 2, 5, 7, 30), (3, 0, 2, 20, 150, 28)],
         "same_row": [(3, 0, 2, 5, 7, 30), (3, 0, 2, 5, 150, 28)],
         "same_col": [(3, 0, 2, 5, 7, 30), (3, 0, 2, 30, 7, 28)],
         "two_planes": [(3, 0, 1, 5, 7, 30), (3, 0, 4, 30, 199, 27)],
         "faces": [(2, 0, 0, 0, 0, 29), (4, 0, 4, 36, 199, 30), (5, 0, 0, 36, 0, 28)]}[case]
    flips = inputs.flip_list(e)
    with gpu_context(abi, [shape], [2], vectors=1, persistent=persistent) as ctx:
        ctx.inject_list(flips)
        ctx.step(steps, ONLINE)
        got = ctx.read(0)
        ev = ctx.events()
    ref = oracle_run(orc, shape, 2, steps, orc.MODE_ONLINE, flips, vectors=1)
    g, o = compare_events(ev, ref)
    assert g == o and len(o) >= 2
    assert rel_err(got, ref["u"]) < 1e-5


@pytest.mark.parametrize("rate", [0.7, 30.0])
@pytest.mark.parametrize("shape", [(300, 130, 6), (257, 64, 9), (140, 70, 19)])
def test_paths_agree_bitwise(abi, shape, rate):
    """Per-launch, persistent and overlapped one-vector paths: the same grid and events."""
    out = []
    for opt in (dict(persistent=0, overlap=0), dict(persistent=1), dict(persistent=0, overlap=1)):
        with gpu_context(abi, [shape], [17], vectors=1, max_flips_per_step=64, **opt) as ctx:
            ctx.inject(5, rate, 0xFFFFFFFF)
            ctx.step(9, ONLINE)
            ctx.step(14, ONLINE)
            out.append((ctx.read(0), key(ctx.events())))
    for k in (1, 2):
        np.testing.assert_array_equal(out[0][0].view(np.uint32), out[k][0].view(np.uint32))
        assert out[0][1] == out[k][1]
    assert len(out[0][1]) > 0


@pytest.mark.parametrize("persistent", [0, 1])
def test_square_grid_same_as_two_vectors(abi, persistent):
    """On a square plane one vector finds what two find: the same events, and grids that
    differ only by the rounding of the corrections (a' comes from checksums summed in
    another order, so Eq. (8) can round differently)."""
    shape = (128, 128, 8)
    out = []
    for vec in (2, 1):
        with gpu_context(abi, [shape], [3], vectors=vec, persistent=persistent) as ctx:
            ctx.inject(11, 0.5, 0xFFFFE000)  # bits 13..31
            ctx.step(60, ONLINE)
            out.append((ctx.read(0), key(ctx.events())))
    assert out[0][1] == out[1][1] and len(out[0][1]) > 10
    assert rel_err(out[1][0], out[0][0]) < 1e-6


def test_hand_over_to_offline_and_verify(abi, orc):
    """After one-vector online sweeps a of the state is not held; offline windows,
    chained verification and reading the checksums sum it first."""
    shape = (130, 70, 5)
    with gpu_context(abi, [shape], [13], vectors=1) as ctx:
        ctx.step(7, ONLINE)
        a, b = ctx.read_checksums(0)
        u = ctx.read(0).astype(np.float64)
        np.testing.assert_allclose(a, u.sum(axis=1), rtol=1e-12)
        np.testing.assert_allclose(b, u.sum(axis=2), rtol=1e-12)
        ctx.step(6, ONLINE)
        ctx.step(3, NONE)
        assert ctx.verify() == 0  # chained from the last online state
        ctx.step(20, OFFLINE)
        ctx.step(4, ONLINE)
        assert ctx.verify() == 0
        assert len(ctx.events()) == 0 and ctx.counters()["rollbacks"] == 0
        got = ctx.read(0)
    ref = oracle_run(orc, shape, 13, 40, orc.MODE_NONE)
    assert rel_err(got, ref["u"]) < 1e-5


def test_batched_equals_grid_by_grid(abi):
    shapes = [(200, 37, 5), (64, 64, 8), (129, 17, 3), (150, 40, 20)]
    temps, powers, coeffs = [], [], []
    for i, s in enumerate(shapes):
        t, p = inputs.grid_inputs(*s, seed=40 + i)
        temps.append(t)
        powers.append(p)
        coeffs.append(inputs.hotspot_coeffs(*s))
    flips = inputs.flip_list([(2, 0, 1, 3, 4, 30), (2, 1, 7, 63, 63, 29), (5, 3, 19, 39, 149, 28),
                              (6, 2, 1, 16, 128, 30)])
    out = []
    for batch in (0, 1):
        with abi.Context(shapes, temps, powers, coeffs, vectors=1, batch=batch) as ctx:
            ctx.inject_list(flips)
            ctx.step(9, ONLINE)
            out.append(([ctx.read(i) for i in range(len(shapes))],
                        sorted(map(tuple, ctx.events()[["step", "grid", "z", "y", "x", "kind"]].tolist()))))
    for a, b in zip(out[0][0], out[1][0]):
        np.testing.assert_array_equal(a.view(np.uint32), b.view(np.uint32))
    assert out[0][1] == out[1][1] and len(out[0][1]) == 4


def test_full_size_512x512x8(abi, orc):
    """The benchmark's grid and launch configuration, 1000 sweeps at 1e-3 flips per
    sweep: the located set is the set of scheduled flips above the detection boundary."""
    shape, steps = (512, 512, 8), 1000
    for s in (1, 2):
        sched = orc.schedule(s, 1e-3, 0xFFFFFFFF, shape, 0, steps)
        with gpu_context(abi, [shape], [1], vectors=1) as ctx:
            ctx.inject(s, 1e-3, 0xFFFFFFFF)
            ctx.step(steps, ONLINE)
            ev = ctx.events()
        expect = {(int(f["step"]), int(f["z"]), int(f["y"]), int(f["x"]), 1) for f in sched if f["bit"] >= 16}
        assert {(int(e["step"]), int(e["z"]), int(e["y"]), int(e["x"]), int(e["kind"])) for e in ev} == expect


@pytest.mark.parametrize("persistent", [0, 1])
@pytest.mark.parametrize("acc", [1, 2])
def test_compensated_and_fp64_accumulation(abi, orc, acc, persistent):
    """The TwoSum and FP64 variants with one vector (their kernels still form the column
    partials, which the check ignores): the oracle's events and values."""
    shape, steps = (200, 37, 5), 12
    flips = inputs.flip_list([(3, 0, 2, 5, 7, 30), (5, 0, 0, 0, 0, 28), (8, 0, 4, 36, 199, 27),
                              (8, 0, 1, 20, 150, 29), (8, 0, 1, 3, 10, 30)])
    with gpu_context(abi, [shape], [2], vectors=1, acc=acc, persistent=persistent) as ctx:
        ctx.inject_list(flips)
        ctx.step(steps, ONLINE)
        got = ctx.read(0)
        ev = ctx.events()
    ref = oracle_run(orc, shape, 2, steps, orc.MODE_ONLINE, flips, vectors=1)
    g, o = compare_events(ev, ref)
    assert g == o and len(o) >= 4
    assert rel_err(got, ref["u"]) < 1e-5


@pytest.mark.parametrize("persistent", [0, 1])
def test_offline_windows_in_a_one_vector_context(abi, orc, persistent):
    """Offline windows form both checksum vectors whatever the online option: launched
    window by window (and by the persistent kernel) in a context created with one vector,
    after online sweeps, with a flip to roll back; events and values against the oracle."""
    shape = (200, 37, 5)
    fl = inputs.flip_list([(6, 0, 2, 10, 30, 29), (21, 0, 1, 20, 150, 27)])
    with gpu_context(abi, [shape], [4], vectors=1, persistent=persistent) as ctx:
        ctx.inject_list(fl)
        ctx.step(8, ONLINE)
        ctx.step(32, OFFLINE)
        got = ctx.read(0)
        ev = ctx.events()
        rb = ctx.counters()["rollbacks"]
    ref_on = oracle_run(orc, shape, 4, 8, orc.MODE_ONLINE, fl, vectors=1)
    co = inputs.hotspot_coeffs(*shape)
    _, power = inputs.grid_inputs(*shape, seed=4)
    st = orc.Stencil(shape, orc.hotspot_points(co))
    ref = orc.run(st, orc.source_term(power, co), ref_on["u"], 32, orc.MODE_OFFLINE, fl, t0=8)
    assert rb == ref["n_rollbacks"] == 1
    g = {(int(e["step"]), int(e["z"]), int(e["y"]), int(e["x"]), int(e["kind"])) for e in ev}
    o = {(int(e["step"]), int(e["z"]), int(e["y"]), int(e["x"]), int(e["kind"]))
         for e in list(ref_on["events"]) + list(ref["events"])}
    assert g == o
    assert rel_err(got, ref["u"]) < 1e-5
