"""Batched grids: many independent grids of uneven sizes advanced with one sweep launch
per tile class and one check launch per sweep, CUDA graphs of graph_steps sweeps.

The batched launches run the same tile bodies and check arithmetic as the per-grid
kernels, so the bar is bitwise: final grids, checksums and event logs equal to those
of the same context advanced grid by grid, with and without graphs, through mode
changes; and, per grid, the oracle's events and values."""
import numpy as np
import pytest

from paper_1909_00709_gb300 import inputs
from _util import compare_events, gpu_context, oracle_run, rel_err

pytestmark = pytest.mark.gpu

NONE, ONLINE, OFFLINE = 0, 1, 2
SHAPES = inputs.batch_shapes(10, seed=7, xy=(17, 300), z=(1, 40)) + [(64, 64, 8), (1, 5, 3), (130, 1, 2)]


@pytest.fixture(scope="module")
def abi():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1909_00709_gb300 import abi, build
    build.build()
    abi.lib()
    return abi


def _run(abi, shapes, plan, *, rate=0.0, seed=3, **opt):
    seeds = [100 + i for i in range(len(shapes))]
    with gpu_context(abi, shapes, seeds, **opt) as ctx:
        if rate:
            ctx.inject(seed, rate, 0xFFFFFFFF)
        for n, mode in plan:
            ctx.step(n, mode)
        grids = [ctx.read(i) for i in range(len(shapes))]
        sums = [ctx.read_checksums(i) for i in range(len(shapes))]
        ev = ctx.events()
        cnt = ctx.counters()
    key = sorted((int(e["step"]), int(e["grid"]), int(e["z"]), int(e["y"]), int(e["x"]), int(e["kind"]),
                  float(e["before"]), float(e["after"])) for e in ev)
    return grids, sums, key, cnt


def _same(r1, r2):
    g1, s1, e1, _ = r1
    g2, s2, e2, _ = r2
    for a, b in zip(g1, g2):
        assert np.array_equal(a.view(np.uint32), b.view(np.uint32))
    for (a1, b1), (a2, b2) in zip(s1, s2):
        assert np.array_equal(a1, a2) and np.array_equal(b1, b2)
    assert e1 == e2


@pytest.mark.parametrize("graph_steps", [0, 16])
@pytest.mark.parametrize("acc", [0, 1, 2])
def test_batched_online_bitwise_equals_grid_by_grid(abi, acc, graph_steps):
    plan = [(40, ONLINE)]
    ref = _run(abi, SHAPES, plan, rate=0.3, acc=acc, batch=0)
    got = _run(abi, SHAPES, plan, rate=0.3, acc=acc, batch=1, graph_steps=graph_steps)
    _same(ref, got)
    assert len(ref[2]) > 0  # the flips were seen and corrected


@pytest.mark.parametrize("graph_steps", [0, 5])
def test_batched_mode_changes_bitwise(abi, graph_steps):
    plan = [(7, NONE), (12, ONLINE), (3, NONE), (1, NONE), (11, ONLINE), (4, OFFLINE), (6, ONLINE), (2, NONE)]
    ref = _run(abi, SHAPES, plan, rate=0.2, batch=0)
    got = _run(abi, SHAPES, plan, rate=0.2, batch=1, graph_steps=graph_steps)
    _same(ref, got)


def test_graph_replays_match_eager_and_count_launches(abi):
    plan = [(23, ONLINE), (9, NONE), (23, ONLINE)]
    eager = _run(abi, SHAPES, plan, rate=0.2, batch=1, graph_steps=0)
    graph = _run(abi, SHAPES, plan, rate=0.2, batch=1, graph_steps=10)
    _same(eager, graph)
    assert eager[3]["kernel_launches"] == graph[3]["kernel_launches"]


def test_batched_matches_oracle_per_grid(abi, orc):
    shapes = SHAPES[:4] + [(64, 64, 8)]
    steps = 30
    flips = []
    rng = np.random.default_rng(5)
    for gi, (nx, ny, nz) in enumerate(shapes):
        for t in (3, 11, 20):
            flips.append((t, gi, int(rng.integers(nz)), int(rng.integers(ny)), int(rng.integers(nx)),
                          int(rng.integers(20, 31))))
    fl = inputs.flip_list(flips)
    seeds = [100 + i for i in range(len(shapes))]
    with gpu_context(abi, shapes, seeds, batch=1, graph_steps=8) as ctx:
        ctx.inject_list(fl)
        ctx.step(steps, ONLINE)
        got = [ctx.read(i) for i in range(len(shapes))]
        ev = ctx.events()
    for gi, shape in enumerate(shapes):
        mine = fl[fl["grid"] == gi].copy()
        mine["grid"] = 0
        ref = oracle_run(orc, shape, seeds[gi], steps, orc.MODE_ONLINE, mine)
        g_ev, o_ev = compare_events(ev, ref, grid=gi)
        assert g_ev == o_ev, (gi, shape, g_ev, o_ev)
        assert rel_err(got[gi], ref["u"]) < 1e-5


def test_single_grid_context_ignores_batch_option(abi):
    shapes = [(200, 37, 5)]
    a = _run(abi, shapes, [(20, ONLINE)], rate=0.5, batch=1)
    b = _run(abi, shapes, [(20, ONLINE)], rate=0.5, batch=0)
    _same(a, b)
