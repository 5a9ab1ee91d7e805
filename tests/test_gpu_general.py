"""General stencil sets and the constant boundary (Sec. 3.1, 3.3) on the GPU against the
FP64 oracle with the same set, rule and inputs: one sweep (Eq. 1), fault-free online runs
(zero events), seeded and placed flips (events identical, values), offline windows whose
chains take the boundary terms of Theorem 1 from each sweep's state, and verify/correct.

Sets: a 13-point star with every opposite pair unequal (radius 2), the 27-point box with
asymmetric weights, and the HotSpot 7-point set with asymmetric weights given as a
general set.  Weights sum to 1, so long runs stay near the initial temperatures."""
import numpy as np
import pytest

from paper_1909_00709_gb300 import inputs
from _util import compare_events, rel_err

pytestmark = pytest.mark.gpu

ONLINE, OFFLINE, NONE = 1, 2, 0
CLAMP, PERIODIC, ZERO, CONST = 0, 1, 2, 3
K_OUT = 318.15  # the constant boundary's value (an ambient temperature)


def normalised(pts):
    tot = sum(w for *_, w in pts)
    return [(dx, dy, dz, float(np.float32(w / tot))) for dx, dy, dz, w in pts]


STAR13 = normalised([(0, 0, 0, 0.47), (-1, 0, 0, 0.08), (1, 0, 0, 0.07), (-2, 0, 0, 0.03), (2, 0, 0, 0.02),
                     (0, -1, 0, 0.09), (0, 1, 0, 0.06), (0, -2, 0, 0.025), (0, 2, 0, 0.035),
                     (0, 0, -1, 0.05), (0, 0, 1, 0.04), (0, 0, -2, 0.01), (0, 0, 2, 0.02)])
BOX27 = normalised([(i, j, k, (8.0 if (i, j, k) == (0, 0, 0) else 1.0) * (1 + 0.1 * i + 0.05 * j - 0.07 * k))
                    for k in (-1, 0, 1) for j in (-1, 0, 1) for i in (-1, 0, 1)])
ASYM7 = normalised([(0, 0, 0, 0.5), (-1, 0, 0, 0.06), (1, 0, 0, 0.11), (0, -1, 0, 0.04), (0, 1, 0, 0.13),
                    (0, 0, -1, 0.07), (0, 0, 1, 0.09)])
SETS = {"star13": STAR13, "box27": BOX27, "asym7": ASYM7}
RULES = {"clamp": CLAMP, "periodic": PERIODIC, "zero": ZERO, "const": CONST}


@pytest.fixture(scope="module")
def abi():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1909_00709_gb300 import abi, build
    build.build()
    abi.lib()
    return abi


def make(shape, seed):
    temp, power = inputs.grid_inputs(*shape, seed=seed)
    return temp, power, inputs.hotspot_coeffs(*shape)


def gpu(abi, shape, seed, pts, rule, **opt):
    temp, power, co = make(shape, seed)
    kw = dict(boundary=rule, boundary_value=K_OUT if rule == CONST else 0.0)
    if pts is not None:
        kw["stencils"] = [pts]
    kw.update(opt)
    return abi.Context([shape], [temp], [power], [co], **kw)


def oracle(orc, shape, seed, pts, rule, steps, mode, flips=None, **kw):
    temp, power, co = make(shape, seed)
    st = orc.Stencil(shape, pts if pts is not None else orc.hotspot_points(co), rule,
                     K_OUT if rule == CONST else 0.0)
    return orc.run(st, orc.source_term(power, co), temp, steps, mode, flips, **kw)


SHAPES = [(200, 37, 5), (129, 17, 3), (64, 33, 37), (33, 1, 4), (300, 130, 2), (5, 3, 6)]


@pytest.mark.parametrize("tile_y", [8, 16])
@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("rule", list(RULES.values()), ids=list(RULES))
@pytest.mark.parametrize("sname", list(SETS))
def test_one_sweep_matches_eq1(abi, orc, sname, rule, shape, tile_y):
    pts = SETS[sname]
    with gpu(abi, shape, 3, pts, rule, tile_y=tile_y) as ctx:
        ctx.step(1, NONE)
        got = ctx.read(0)
    ref = oracle(orc, shape, 3, pts, rule, 1, orc.MODE_NONE)["u"]
    assert rel_err(got, ref) < 1e-6


@pytest.mark.parametrize("acc", [0, 1, 2])
@pytest.mark.parametrize("rule", list(RULES.values()), ids=list(RULES))
@pytest.mark.parametrize("sname", list(SETS))
def test_online_fault_free(abi, orc, sname, rule, acc):
    """Theorem 2 with any set and rule: no false positive in 60 online sweeps."""
    shape, steps = (150, 40, 20), 60
    pts = SETS[sname]
    with gpu(abi, shape, 5, pts, rule, acc=acc, track_residual=1) as ctx:
        ctx.step(steps, ONLINE)
        got = ctx.read(0)
        ev = ctx.events()
        resid = ctx.counters()["max_residual"]
    assert len(ev) == 0, ev[:4]
    assert resid < 1e-6
    ref = oracle(orc, shape, 5, pts, rule, steps, orc.MODE_ONLINE)
    assert ref["n_events"] == 0
    assert rel_err(got, ref["u"]) < 1e-5


# flips on faces, edges, corners and inside; detectable bits (>= 20) and undetectable ones
def placed_flips(shape):
    nx, ny, nz = shape
    spots = [(2, 0, 0, 0), (3, nz - 1, ny - 1, nx - 1), (4, nz // 2, 0, nx // 2), (5, 1, ny // 2, nx - 1),
             (6, nz // 2, ny // 2, nx // 2), (6, 0, ny - 2, 1), (7, nz - 2, 1, nx - 2)]
    bits = [30, 26, 22, 28, 24, 23, 31]
    fl = [(t, 0, z, y, x, b) for (t, z, y, x), b in zip(spots, bits)]
    fl += [(8, 0, 1, 3, 5, 4), (9, 0, nz // 2, ny // 3, nx // 3, 27)]  # one below the threshold
    return inputs.flip_list(fl)


@pytest.mark.parametrize("rule", list(RULES.values()), ids=list(RULES))
@pytest.mark.parametrize("sname", list(SETS))
def test_online_placed_flips(abi, orc, sname, rule):
    shape, steps = (150, 40, 20), 12
    pts = SETS[sname]
    fl = placed_flips(shape)
    with gpu(abi, shape, 7, pts, rule) as ctx:
        ctx.inject_list(fl)
        ctx.step(steps, ONLINE)
        got = ctx.read(0)
        ev = ctx.events()
    ref = oracle(orc, shape, 7, pts, rule, steps, orc.MODE_ONLINE, fl)
    g, o = compare_events(ev, ref)
    assert g == o
    assert len(o) >= 7
    assert rel_err(got, ref["u"]) < 1e-5


@pytest.mark.parametrize("rule", list(RULES.values()), ids=list(RULES))
@pytest.mark.parametrize("sname", list(SETS))
def test_online_seeded_flips_many_per_sweep(abi, orc, sname, rule):
    """Several flips per sweep: single intersections corrected, other patterns recomputed
    from the previous state with the general set."""
    shape, steps = (160, 48, 12), 10
    pts = SETS[sname]
    sched = orc.schedule(11, 6.0, 0xFFFFFFFF, shape, 0, steps)
    with gpu(abi, shape, 9, pts, rule) as ctx:
        ctx.inject(11, 6.0, 0xFFFFFFFF)
        ctx.step(steps, ONLINE)
        got = ctx.read(0)
        ev = ctx.events()
    ref = oracle(orc, shape, 9, pts, rule, steps, orc.MODE_ONLINE, sched)
    g, o = compare_events(ev, ref)
    assert g == o
    assert any(e[4] == 2 for e in o) or len(o) > 10
    marg_planes = {z for _, z in ref["marginal"]}
    keep = np.ones(got.shape, dtype=bool)
    for z in marg_planes:
        keep[max(0, z - steps):z + steps + 1] = False
    if keep.any():
        assert rel_err(got[keep], ref["u"][keep]) < 1e-4


# offline windows: general sets (per-step terms unless periodic), and the 7-point kernels
# with asymmetric weights or empty boundaries (per-step terms on the 7-point path)
OFFLINE_CASES = [("star13", CLAMP), ("box27", ZERO), ("box27", PERIODIC), ("asym7", CONST), ("star13", CONST),
                 ("hotspot-asym", CLAMP), ("hotspot", ZERO)]


def offline_points(name, co):
    if name == "hotspot":
        return None, dict(co)
    if name == "hotspot-asym":  # the 7-point kernels with cn != cs and cw != ce
        c = dict(co)
        c["cw"], c["ce"] = float(np.float32(c["cw"] * 0.7)), float(np.float32(c["cw"] * 1.3))
        c["cn"], c["cs"] = float(np.float32(c["cn"] * 1.2)), float(np.float32(c["cn"] * 0.8))
        return None, c
    return SETS[name], dict(co)


@pytest.mark.parametrize("name,rule", OFFLINE_CASES, ids=[f"{n}-{r}" for n, r in OFFLINE_CASES])
def test_offline_windows_with_flips(abi, orc, name, rule):
    shape, steps, delta = (130, 45, 9), 40, 8
    temp, power, co = make(shape, 13)
    pts, c = offline_points(name, co)
    fl = inputs.flip_list([(3, 0, 4, 0, 7, 29), (12, 0, 0, 20, 129, 26), (21, 0, 8, 44, 0, 30),
                           (30, 0, 5, 22, 60, 3)])
    kw = dict(boundary=rule, boundary_value=K_OUT if rule == CONST else 0.0, delta=delta)
    if pts is not None:
        kw["stencils"] = [pts]
    with abi.Context([shape], [temp], [power], [c], **kw) as ctx:
        ctx.inject_list(fl)
        ctx.step(steps, OFFLINE)
        got = ctx.read(0)
        ev = ctx.events()
        rb = ctx.counters()["rollbacks"]
    opts = pts if pts is not None else orc.hotspot_points(c)
    st = orc.Stencil(shape, opts, rule, K_OUT if rule == CONST else 0.0)
    ref = orc.run(st, orc.source_term(power, c), temp, steps, orc.MODE_OFFLINE, fl, delta=delta)
    assert rb == ref["n_rollbacks"] == 3
    g, o = compare_events(ev, ref)
    assert g == o
    assert rel_err(got, ref["u"]) < 1e-5


@pytest.mark.parametrize("name,rule", OFFLINE_CASES, ids=[f"{n}-{r}" for n, r in OFFLINE_CASES])
def test_offline_fault_free_equals_unprotected(abi, orc, name, rule):
    shape, steps = (130, 45, 9), 37
    temp, power, co = make(shape, 14)
    pts, c = offline_points(name, co)
    kw = dict(boundary=rule, boundary_value=K_OUT if rule == CONST else 0.0, delta=8, track_residual=1)
    if pts is not None:
        kw["stencils"] = [pts]
    with abi.Context([shape], [temp], [power], [c], **kw) as ctx:
        ctx.step(steps, OFFLINE)
        off = ctx.read(0)
        assert len(ctx.events()) == 0 and ctx.counters()["rollbacks"] == 0
    with abi.Context([shape], [temp], [power], [c], **kw) as ctx:
        ctx.step(steps, NONE)
        plain = ctx.read(0)
    np.testing.assert_array_equal(off, plain)


def test_hotspot_constant_boundary_online_seeded(abi, orc):
    """The HotSpot 7-point set with a constant outside temperature (through the general
    kernels), seeded flips at 2 per sweep."""
    shape, steps = (256, 96, 16), 40
    sched = orc.schedule(17, 2.0, 0xFFFFFFFF, shape, 0, steps)
    with gpu(abi, shape, 15, None, CONST) as ctx:
        ctx.inject(17, 2.0, 0xFFFFFFFF)
        ctx.step(steps, ONLINE)
        got = ctx.read(0)
        ev = ctx.events()
    ref = oracle(orc, shape, 15, None, CONST, steps, orc.MODE_ONLINE, sched)
    g, o = compare_events(ev, ref)
    assert g == o and len(o) > 10
    marg_planes = {z for _, z in ref["marginal"]}
    keep = np.ones(got.shape, dtype=bool)
    for z in marg_planes:
        keep[max(0, z - steps):z + steps + 1] = False
    if keep.any():
        assert rel_err(got[keep], ref["u"][keep]) < 1e-4


def test_verify_and_correct_general(abi, orc):
    """abft_verify one sweep past the verified state takes the boundary terms of that
    state; two sweeps past it needs vanishing terms (refused for the clamped star)."""
    shape = (100, 40, 6)
    fl = inputs.flip_list([(1, 0, 3, 10, 20, 29)])
    with gpu(abi, shape, 19, STAR13, CLAMP) as ctx:
        ctx.step(1, ONLINE)
        ctx.inject_list(fl)
        ctx.step(1, NONE)
        assert ctx.verify() >= 2
        assert ctx.correct() == 1
        assert ctx.verify() == 0
        got = ctx.read(0)
        ctx.step(2, NONE)
        with pytest.raises(abi.AbftError):
            ctx.verify()
    ref = oracle(orc, shape, 19, STAR13, CLAMP, 2, orc.MODE_NONE)
    assert rel_err(got, ref["u"]) < 1e-6
    with gpu(abi, shape, 19, BOX27, PERIODIC) as ctx:  # terms vanish: any distance
        ctx.step(1, ONLINE)
        ctx.step(3, NONE)
        assert ctx.verify() == 0


def test_invalid_sets_are_refused(abi):
    shape = (32, 16, 4)
    for bad in ([(3, 0, 0, 1.0)], [(0, 0, -3, 1.0)], [(0, 0, 0, float("nan"))]):
        with pytest.raises(abi.AbftError):
            gpu(abi, shape, 1, bad, CLAMP)
