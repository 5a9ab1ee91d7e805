"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: closed forms,
exact identities on integer data, invariants, special cases that reduce to numpy,
and the numbers the paper prints (tests/golden/).  None of them needs a GPU.
"""
import numpy as np
import pytest

from paper_1909_00709_gb300 import inputs

CLAMP, PERIODIC, ZERO, CONST = 0, 1, 2, 3


def seven(cc, cw, ce, cn, cs, cb, ct):
    return [(0, 0, 0, cc), (-1, 0, 0, cw), (1, 0, 0, ce), (0, -1, 0, cn), (0, 1, 0, cs),
            (0, 0, -1, cb), (0, 0, 1, ct)]


def int_grid(shape, seed, hi=1 << 10):
    nx, ny, nz = shape
    return np.random.default_rng(seed).integers(0, hi, size=(nz, ny, nx)).astype(np.float64)


# ----------------------------------------------------------- Eq. (1): sweep

@pytest.mark.parametrize("boundary", [CLAMP, PERIODIC, ZERO])
def test_sweep_identity_stencil(orc, boundary):
    shape = (7, 5, 3)
    u = np.random.default_rng(0).normal(size=shape[::-1])
    st = orc.Stencil(shape, [(0, 0, 0, 1.0)], boundary)
    np.testing.assert_array_equal(orc.sweep(st, np.zeros_like(u), u), u)


def test_sweep_constant_term_only(orc):
    shape = (6, 4, 3)
    C = np.random.default_rng(1).normal(size=shape[::-1])
    st = orc.Stencil(shape, seven(0.5, .1, .1, .1, .1, .05, .05))
    np.testing.assert_array_equal(orc.sweep(st, C, np.zeros_like(C)), C)


def test_sweep_impulse_response(orc):
    """out[p] = sum_d w_d u[p+d]; a unit impulse at q lands weight w_d at q - d.
    Seven distinct dyadic weights pin the direction of every offset and the axis order."""
    shape = (9, 8, 7)
    w = dict(cc=1 / 2, cw=1 / 4, ce=1 / 8, cn=1 / 16, cs=1 / 32, cb=1 / 64, ct=1 / 128)
    st = orc.Stencil(shape, seven(**w))
    u = np.zeros(shape[::-1])
    q = (3, 4, 5)  # (z, y, x)
    u[q] = 1.0
    out = orc.sweep(st, np.zeros_like(u), u)
    expect = np.zeros_like(u)
    z, y, x = q
    expect[z, y, x] = w["cc"]
    expect[z, y, x + 1] = w["cw"]   # west neighbour of x+1 is x
    expect[z, y, x - 1] = w["ce"]
    expect[z, y + 1, x] = w["cn"]   # north = y-1 (Fig. 2: n = c - nx)
    expect[z, y - 1, x] = w["cs"]
    expect[z + 1, y, x] = w["cb"]
    expect[z - 1, y, x] = w["ct"]
    np.testing.assert_array_equal(out, expect)


def test_sweep_clamped_corner(orc):
    """Fig. 2: a neighbour outside the grid is replaced by the centre."""
    shape = (5, 6, 4)
    w = dict(cc=1 / 2, cw=1 / 4, ce=1 / 8, cn=1 / 16, cs=1 / 32, cb=1 / 64, ct=1 / 128)
    st = orc.Stencil(shape, seven(**w), CLAMP)
    u = np.zeros(shape[::-1])
    u[0, 0, 0] = 1.0
    out = orc.sweep(st, np.zeros_like(u), u)
    expect = np.zeros_like(u)
    expect[0, 0, 0] = w["cc"] + w["cw"] + w["cn"] + w["cb"]
    expect[0, 0, 1] = w["cw"]
    expect[0, 1, 0] = w["cn"]
    expect[1, 0, 0] = w["cb"]
    np.testing.assert_array_equal(out, expect)


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_sweep_quadratic_field(orc, axis):
    """u = s^2 along one axis, weights 1/4, 1/2, 1/4 along it: interior -> s^2 + 1/2,
    clamped ends -> 1/4 (first) and (n-1)^2 - (n-1)/2 + 1/4 (last)."""
    shape = (6, 7, 8)  # nx, ny, nz
    nx, ny, nz = shape
    n = (nx, ny, nz)[axis]
    s = np.arange(n, dtype=np.float64) ** 2
    pts = [(0, 0, 0, 0.5)]
    d = [0, 0, 0]
    d[axis] = 1
    pts += [(-d[0], -d[1], -d[2], 0.25), (d[0], d[1], d[2], 0.25)]
    # distractor weights on the other axes act on a constant field
    st = orc.Stencil(shape, pts, CLAMP)
    shp = [1, 1, 1]
    shp[2 - axis] = n
    u = np.broadcast_to(s.reshape(shp), (nz, ny, nx)).copy()
    out = orc.sweep(st, np.zeros_like(u), u)
    line = np.moveaxis(out, 2 - axis, 0)[:, 0, 0]
    expect = s + 0.5
    expect[0] = 0.5 * 0 + 0.25 * (0 + 1)
    last = (n - 1) ** 2
    expect[-1] = 0.5 * last + 0.25 * ((n - 2) ** 2 + last)
    np.testing.assert_array_equal(line, expect)


def test_sweep_conserves_total_when_clamped_symmetric(orc):
    """Clamped boundary + symmetric pairs + weights summing to 1 + C = 0 conserve the sum."""
    shape = (16, 12, 5)
    st = orc.Stencil(shape, seven(1 / 2, 1 / 16, 1 / 16, 1 / 8, 1 / 8, 1 / 16, 1 / 16), CLAMP)
    u = int_grid(shape, 2)
    total = u.sum()
    for _ in range(5):
        u = orc.sweep(st, np.zeros_like(u), u)
        assert u.sum() == total


# ------------------------------------------------ Eq. (2), (3): checksums

def test_checksums_match_numpy_sums(orc):
    u = int_grid((13, 9, 4), 3)
    a, b = orc.checksums(u)
    np.testing.assert_array_equal(a, u.sum(axis=1))  # a[z][x] = sum over y
    np.testing.assert_array_equal(b, u.sum(axis=2))  # b[z][y] = sum over x


# ---------------------------------------------- Theorem 1 and Theorem 2

ASYM = seven(3, 1, 2, 5, 1, 2, 4)  # integer, every opposite pair unequal


@pytest.mark.parametrize("boundary", [CLAMP, PERIODIC, ZERO])
@pytest.mark.parametrize("points", [ASYM, seven(2, 1, 1, 1, 1, 1, 1)], ids=["asym", "sym"])
@pytest.mark.parametrize("shape", [(9, 7, 4), (5, 6, 1)], ids=["3d", "2d"])
def test_theorem1_exact_on_integer_grids(orc, boundary, points, shape):
    """Interpolated checksums equal the recomputed ones exactly (Theorem 1 / 2): integer
    weights and values keep FP64 exact, so any dropped or misplaced boundary term shows."""
    st = orc.Stencil(shape, points, boundary)
    u = int_grid(shape, 4, hi=64)
    C = int_grid(shape, 5, hi=16)
    cx, cy = orc.checksums(C)
    a, b = orc.checksums(u)
    for _ in range(3):
        un = orc.sweep(st, C, u)
        an, bn = orc.checksums(un)
        ap, bp = orc.interpolate(st, cx, cy, a, b, u)
        np.testing.assert_array_equal(ap, an)
        np.testing.assert_array_equal(bp, bn)
        u, a, b = un, an, bn
    assert np.abs(u).max() < 2 ** 52


def test_theorem1_boundary_terms_nonzero_when_asymmetric(orc):
    """With unequal opposite weights the simple form (Eq. 6/7) is wrong by exactly
    (w_{y-1} - w_{y+1}) (u[y=0] - u[y=ny-1]) on a (clamped), and the x analogue on b."""
    shape = (8, 6, 3)
    st = orc.Stencil(shape, ASYM, CLAMP)
    u = int_grid(shape, 6, hi=64)
    C = int_grid(shape, 7, hi=16)
    cx, cy = orc.checksums(C)
    a, b = orc.checksums(u)
    ap, bp = orc.interpolate(st, cx, cy, a, b, u)
    sp_a, sp_b = orc.interpolate_simple(st, cx, cy, a, b)
    cc, cw, ce, cn, cs, cb, ct = [w for *_, w in ASYM]
    np.testing.assert_array_equal(ap - sp_a, (cn - cs) * (u[:, 0, :] - u[:, -1, :]))
    np.testing.assert_array_equal(bp - sp_b, (cw - ce) * (u[:, :, 0] - u[:, :, -1]))


@pytest.mark.parametrize("boundary", [CLAMP, PERIODIC])
def test_simple_form_exact_when_boundary_terms_vanish(orc, boundary):
    shape = (10, 9, 4)
    st = orc.Stencil(shape, seven(2, 1, 1, 3, 3, 1, 1), boundary)
    u = int_grid(shape, 8, hi=64)
    C = int_grid(shape, 9, hi=16)
    cx, cy = orc.checksums(C)
    a, b = orc.checksums(u)
    ap, bp = orc.interpolate_simple(st, cx, cy, a, b)
    an, bn = orc.checksums(orc.sweep(st, C, u))
    np.testing.assert_array_equal(ap, an)
    np.testing.assert_array_equal(bp, bn)


def test_paper_example_stencil_periodic(orc, golden):
    """Sec. 3.1's 4-point average in 2D with periodic boundaries: applying it to the
    checksum vectors gives a'_x = (a_{x-1} + a_{x+1})/4 + a_x/2 (two y-shifts keep a_x)."""
    pts = [(i, j, 0, w) for i, j, w in golden["paper_claims"]["example_stencil_4pt_average"]["value"]]
    # the printed set lists (i, j) = (0,-1), (-1,0), (1,0), (0,1)
    shape = (12, 10, 1)
    st = orc.Stencil(shape, pts, PERIODIC)
    u = int_grid(shape, 10, hi=256)
    a, b = orc.checksums(u)
    zeros = np.zeros_like
    ap, bp = orc.interpolate_simple(st, zeros(a), zeros(b), a, b)
    np.testing.assert_array_equal(ap, (np.roll(a, 1, 1) + np.roll(a, -1, 1)) / 4 + a / 2)
    np.testing.assert_array_equal(bp, (np.roll(b, 1, 1) + np.roll(b, -1, 1)) / 4 + b / 2)


# ------------------------------------------------------- Sec. 3.4: detection

def test_detect_threshold_semantics(orc):
    comp = np.array([1.0, 1.0, 1.0, 1.0, 2.0, 1.0])
    pred = np.array([1.0 + 2e-5, 1.0 + 0.5e-5, np.nan, np.inf, 2.0 - 3e-5, 1.0])
    np.testing.assert_array_equal(orc.detect(pred, comp, 1e-5), [0, 2, 3, 4])


# -------------------------------------------------- online method end to end

def hotspot(orc, shape, seed):
    co = inputs.hotspot_coeffs(*shape)
    temp, power = inputs.grid_inputs(*shape, seed=seed)
    st = orc.Stencil(shape, orc.hotspot_points(co))
    return st, orc.source_term(power, co), temp


@pytest.mark.parametrize("shape,steps", [((64, 64, 8), 128), ((512, 512, 8), 24)])
def test_no_false_positives_at_paper_eps(orc, golden, shape, steps):
    g = golden["paper_claims"]
    assert list(shape) in g["false_positives_at_eps"]["tile_sizes"]
    st, C, temp = hotspot(orc, shape, 0)
    for mode in (orc.MODE_ONLINE, orc.MODE_OFFLINE):
        r = orc.run(st, C, temp, steps, mode, eps=g["eps"]["value"])
        assert r["n_events"] == g["false_positives_at_eps"]["value"]
        assert r["max_resid"] < 1e-12


def test_bit_detectability_matches_paper_64(orc, golden):
    """Online at 64x64x8: flips in bits 0-12 pass unseen, bits 13-31 are located."""
    g = golden["paper_claims"]
    st, C, temp = hotspot(orc, (64, 64, 8), 1)
    rng = np.random.default_rng(11)
    for bit in range(32):
        for trial in range(3):
            z, y, x = int(rng.integers(8)), int(rng.integers(64)), int(rng.integers(64))
            step = int(rng.integers(2, 30))
            fl = inputs.flip_list([(step, 0, z, y, x, bit)])
            r = orc.run(st, C, temp, 32, orc.MODE_ONLINE, fl)
            assert not r["marginal"]
            if bit in g["undetectable_bits_64x64x8"]["value"]:
                assert r["n_events"] == 0, (bit, r["events"])
            else:
                assert bit in g["detectable_bits_64x64x8"]["value"]
                ev = r["events"]
                assert len(ev) == 1 and ev[0]["kind"] == orc.EV_CORRECTED
                assert (ev[0]["step"], ev[0]["z"], ev[0]["y"], ev[0]["x"]) == (step, z, y, x)


@pytest.mark.parametrize("bit", [13, 20, 27, 29, 30, 31])
def test_online_correction_restores_fault_free_state(orc, bit):
    st, C, temp = hotspot(orc, (48, 40, 6), 2)
    ref = orc.run(st, C, temp, 20, orc.MODE_ONLINE)
    fl = inputs.flip_list([(7, 0, 2, 17, 31, bit)])
    r = orc.run(st, C, temp, 20, orc.MODE_ONLINE, fl)
    assert r["n_events"] == 1
    e = r["events"][0]
    assert (e["z"], e["y"], e["x"]) == (2, 17, 31)
    np.testing.assert_allclose(r["u"], ref["u"], rtol=1e-12, atol=0)


def test_literal_eq8_loses_exponent_flips(orc):
    """Evaluating Eq. (8) as a' - (a - u) cancels catastrophically after a high exponent
    flip (the checksum 'overflow' of Sec. 5.3); the rearranged form does not."""
    st, C, temp = hotspot(orc, (48, 40, 6), 2)
    ref = orc.run(st, C, temp, 10, orc.MODE_ONLINE)
    fl = inputs.flip_list([(3, 0, 1, 5, 6, 29)])
    lit = orc.run(st, C, temp, 10, orc.MODE_ONLINE, fl, literal_eq8=True)
    good = orc.run(st, C, temp, 10, orc.MODE_ONLINE, fl)
    assert np.abs(lit["u"] - ref["u"]).max() > 1.0
    assert np.abs(good["u"] - ref["u"]).max() < 1e-9


@pytest.mark.parametrize("target", [inputs.TARGET_A, inputs.TARGET_B])
def test_checksum_corruption_leaves_grid_alone(orc, target):
    """Fig. 4b: a corrupted checksum shows in one vector only; recomputing the flagged
    line from u^t reproduces the same values and refreshes the checksum."""
    st, C, temp = hotspot(orc, (32, 24, 4), 3)
    ref = orc.run(st, C, temp, 8, orc.MODE_ONLINE)
    fl = inputs.flip_list([(4, 0, 1, 9, 13, 27, target)])
    r = orc.run(st, C, temp, 8, orc.MODE_ONLINE, fl)
    np.testing.assert_array_equal(r["u"], ref["u"])
    ev = r["events"]
    assert len(ev) == 1 and ev[0]["kind"] == orc.EV_RECOMPUTED and ev[0]["step"] == 4
    if target == inputs.TARGET_A:
        assert (ev[0]["y"], ev[0]["x"]) == (-1, 13)
    else:
        assert (ev[0]["y"], ev[0]["x"]) == (9, -1)


def test_two_by_two_pattern_is_recomputed_exactly(orc):
    st, C, temp = hotspot(orc, (32, 24, 4), 4)
    ref = orc.run(st, C, temp, 6, orc.MODE_ONLINE)
    fl = inputs.flip_list([(2, 0, 1, 3, 4, 30), (2, 0, 1, 10, 20, 25)])
    r = orc.run(st, C, temp, 6, orc.MODE_ONLINE, fl)
    np.testing.assert_array_equal(r["u"], ref["u"])
    lines = sorted((int(e["y"]), int(e["x"])) for e in r["events"])
    assert lines == [(-1, 4), (-1, 20), (3, -1), (10, -1)]
    assert all(e["kind"] == orc.EV_RECOMPUTED for e in r["events"])


def test_same_row_pair_is_recomputed(orc):
    st, C, temp = hotspot(orc, (32, 24, 4), 4)
    ref = orc.run(st, C, temp, 6, orc.MODE_ONLINE)
    fl = inputs.flip_list([(2, 0, 1, 3, 4, 30), (2, 0, 1, 3, 20, 25)])
    r = orc.run(st, C, temp, 6, orc.MODE_ONLINE, fl)
    np.testing.assert_array_equal(r["u"], ref["u"])


# --------------------------------------------------------------- offline

def test_offline_rollback_erases_detected_flip(orc, golden):
    st, C, temp = hotspot(orc, (64, 64, 8), 5)
    delta = golden["paper_claims"]["offline_period"]["value"]
    ref = orc.run(st, C, temp, 40, orc.MODE_OFFLINE, delta=delta)
    fl = inputs.flip_list([(20, 0, 3, 30, 40, 28)])
    r = orc.run(st, C, temp, 40, orc.MODE_OFFLINE, fl, delta=delta)
    assert r["n_rollbacks"] == 1
    ev = r["events"]
    assert len(ev) == 1 and ev[0]["kind"] == orc.EV_ROLLBACK and ev[0]["step"] == 16
    np.testing.assert_array_equal(r["u"], ref["u"])


def test_offline_matches_unprotected_when_fault_free(orc):
    st, C, temp = hotspot(orc, (20, 18, 5), 6)
    a = orc.run(st, C, temp, 37, orc.MODE_OFFLINE, delta=8)
    b = orc.run(st, C, temp, 37, orc.MODE_NONE)
    np.testing.assert_array_equal(a["u"], b["u"])
    assert a["n_events"] == 0


def dyadic_asym():
    """Clamped-stable weights with every opposite pair unequal, summing to 1, dyadic."""
    return seven(1 / 2, 1 / 16, 1 / 8, 1 / 32, 3 / 32, 1 / 16, 1 / 8)


@pytest.mark.parametrize("rule,bval", [(CLAMP, 0.0), (ZERO, 0.0), (CONST, 300.0)],
                         ids=["clamp-asym", "zero", "const"])
def test_offline_per_step_terms_fault_free(orc, rule, bval):
    """Where the terms of Theorem 1 do not vanish, the chain of Fig. 10 takes them from
    each step's own state: a fault-free offline run has no event and equals the
    unprotected run bit for bit."""
    shape = (20, 18, 5)
    co = inputs.hotspot_coeffs(*shape)
    _, power = inputs.grid_inputs(*shape, seed=6)
    temp, _ = inputs.grid_inputs(*shape, seed=7)
    C = orc.source_term(power, co)
    st = orc.Stencil(shape, dyadic_asym() if rule == CLAMP else orc.hotspot_points(co), rule, bval)
    a = orc.run(st, C, temp, 37, orc.MODE_OFFLINE, delta=8)
    b = orc.run(st, C, temp, 37, orc.MODE_NONE)
    assert a["n_events"] == 0 and a["n_rollbacks"] == 0
    np.testing.assert_array_equal(a["u"], b["u"])
    assert a["max_resid"] < 1e-12


@pytest.mark.parametrize("rule,bval", [(CLAMP, 0.0), (ZERO, 0.0), (CONST, 300.0)],
                         ids=["clamp-asym", "zero", "const"])
@pytest.mark.parametrize("where", ["y0", "ylast", "x0", "corner", "inner"])
def test_offline_per_step_terms_catch_edge_flips(orc, rule, bval, where):
    """A flip on a face row, which also enters the per-step boundary terms of the chain,
    is still detected at the window's end; the rollback restores the fault-free run."""
    shape = (20, 18, 5)
    co = inputs.hotspot_coeffs(*shape)
    _, power = inputs.grid_inputs(*shape, seed=6)
    temp, _ = inputs.grid_inputs(*shape, seed=7)
    C = orc.source_term(power, co)
    st = orc.Stencil(shape, dyadic_asym() if rule == CLAMP else orc.hotspot_points(co), rule, bval)
    zyx = dict(y0=(2, 0, 7), ylast=(2, 17, 7), x0=(3, 9, 0), corner=(0, 0, 19), inner=(2, 9, 9))[where]
    for step in (9, 13, 15):  # early, middle and last sweep of the window 8..15
        fl = inputs.flip_list([(step, 0, *zyx, 27)])
        r = orc.run(st, C, temp, 24, orc.MODE_OFFLINE, fl, delta=8)
        ref = orc.run(st, C, temp, 24, orc.MODE_OFFLINE, delta=8)
        assert r["n_rollbacks"] == 1, (step, zyx)
        assert [int(e["step"]) for e in r["events"]] == [8]
        np.testing.assert_array_equal(r["u"], ref["u"])


def test_clamped_radius_two_terms_do_not_vanish(orc):
    """A symmetric 13-point star under clamped boundaries: the simple form of Eq. (6)/(7)
    misses the terms of Theorem 1 (exact integer arithmetic shows the gap), so the
    offline chain takes the terms from each step's state (per step); periodic boundaries
    need none."""
    pts = [(0, 0, 0, 4.0)] + [(d * s, 0, 0, 1.0) for d in (1, 2) for s in (-1, 1)] + \
          [(0, d * s, 0, 1.0) for d in (1, 2) for s in (-1, 1)] + [(0, 0, s, 1.0) for s in (-1, 1)]
    shape = (9, 7, 3)
    u = int_grid(shape, 4)
    C = np.zeros_like(u)
    st = orc.Stencil(shape, pts, CLAMP)
    out = orc.sweep(st, C, u)
    a_true, b_true = orc.checksums(out)
    a0, b0 = orc.checksums(u)
    ap, bp = orc.interpolate_simple(st, *orc.checksums(C), a0, b0)
    assert np.abs(ap - a_true).max() > 0 and np.abs(bp - b_true).max() > 0
    ap, bp = orc.interpolate(st, *orc.checksums(C), a0, b0, u)
    np.testing.assert_array_equal(ap, a_true)
    np.testing.assert_array_equal(bp, b_true)
    ap, bp = orc.interpolate_chain(st, *orc.checksums(C), a0, b0, u)
    np.testing.assert_array_equal(ap, a_true)
    np.testing.assert_array_equal(bp, b_true)
    assert orc.run(st, C, u, 4, orc.MODE_OFFLINE, delta=2)["n_events"] == 0
    per = orc.Stencil(shape, pts, PERIODIC)
    assert orc.run(per, C, u, 4, orc.MODE_OFFLINE, delta=2)["n_events"] == 0


# ----------------------------------------- general stencil sets and the constant rule

STAR13 = [(0, 0, 0, 4.0)] + [(d * s, 0, 0, float(d + s + 2)) for d in (1, 2) for s in (-1, 1)] + \
         [(0, d * s, 0, float(2 * d - s + 1)) for d in (1, 2) for s in (-1, 1)] + \
         [(0, 0, d * s, float(d)) for d in (1, 2) for s in (-1, 1)]  # integer, asymmetric
BOX27 = [(i, j, k, float(1 + (i + 1) + 2 * (j + 1) + (k + 1) % 2)) for k in (-1, 0, 1) for j in (-1, 0, 1)
         for i in (-1, 0, 1)]  # integer, asymmetric


@pytest.mark.parametrize("rule,bval", [(CLAMP, 0.0), (PERIODIC, 0.0), (ZERO, 0.0), (CONST, 7.0)],
                         ids=["clamp", "periodic", "zero", "const"])
@pytest.mark.parametrize("points", [STAR13, BOX27, ASYM], ids=["star13", "box27", "asym7"])
@pytest.mark.parametrize("shape", [(9, 7, 5), (6, 5, 1), (7, 1, 3), (1, 2, 4)], ids=["3d", "2d", "ny1", "nx1"])
def test_theorem1_exact_for_general_sets(orc, rule, bval, points, shape):
    """Theorem 1 (literal alpha/beta from u) and its chain form (vector entries outside the
    grid by the rule applied to the vector, alpha/beta from u) both equal the recomputed
    checksums exactly on integer data, for radius-2 and 27-point sets, every boundary
    rule, and planes thinner than the stencil (ny = 1, nx = 1)."""
    st = orc.Stencil(shape, points, rule, bval)
    u = int_grid(shape, 11, hi=64)
    C = int_grid(shape, 12, hi=16)
    cx, cy = orc.checksums(C)
    a, b = orc.checksums(u)
    for _ in range(2):
        un = orc.sweep(st, C, u)
        an, bn = orc.checksums(un)
        ap, bp = orc.interpolate(st, cx, cy, a, b, u)
        np.testing.assert_array_equal(ap, an)
        np.testing.assert_array_equal(bp, bn)
        ap, bp = orc.interpolate_chain(st, cx, cy, a, b, u)
        np.testing.assert_array_equal(ap, an)
        np.testing.assert_array_equal(bp, bn)
        u, a, b = un, an, bn
    assert np.abs(u).max() < 2 ** 52


def test_constant_rule_with_zero_value_is_the_empty_rule(orc):
    shape = (11, 9, 4)
    u = int_grid(shape, 13, hi=64)
    C = int_grid(shape, 14, hi=16)
    for pts in (STAR13, BOX27):
        a = orc.sweep(orc.Stencil(shape, pts, CONST, 0.0), C, u)
        b = orc.sweep(orc.Stencil(shape, pts, ZERO), C, u)
        np.testing.assert_array_equal(a, b)


def test_constant_rule_uniform_field_is_a_fixed_point(orc):
    """u = K everywhere, outside cells K, weights summing to 1, no source: every point
    stays K exactly; the empty rule loses mass at the faces instead."""
    shape = (8, 7, 5)
    K = 321.0
    u = np.full(shape[::-1], K)
    w = [(0, 0, 0, 1 / 2)] + [(d, 0, 0, 1 / 16) for d in (-2, -1, 1, 2)] + \
        [(0, d, 0, 1 / 32) for d in (-2, -1, 1, 2)] + [(0, 0, d, 1 / 16) for d in (-1, 1)]
    assert sum(p[3] for p in w) == 1.0
    out = orc.sweep(orc.Stencil(shape, w, CONST, K), np.zeros_like(u), u)
    np.testing.assert_array_equal(out, u)
    assert orc.sweep(orc.Stencil(shape, w, ZERO), np.zeros_like(u), u).min() < K


def test_constant_rule_face_closed_form(orc):
    """u = 0 inside, K outside: a point receives K times the summed weight of its
    neighbours that lie outside (impulse weights pin each offset)."""
    shape = (6, 5, 4)
    K = 2.0
    w = dict(cc=1 / 2, cw=1 / 4, ce=1 / 8, cn=1 / 16, cs=1 / 32, cb=1 / 64, ct=1 / 128)
    st = orc.Stencil(shape, seven(**w), CONST, K)
    u = np.zeros(shape[::-1])
    out = orc.sweep(st, np.zeros_like(u), u)
    nz, ny, nx = u.shape
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                e = (w["cw"] * (x == 0) + w["ce"] * (x == nx - 1) + w["cn"] * (y == 0) + w["cs"] * (y == ny - 1)
                     + w["cb"] * (z == 0) + w["ct"] * (z == nz - 1)) * K
                assert out[z, y, x] == e, (z, y, x)


# ----------------------------------------------------------- flip schedule

def test_splitmix64_published_first_output(orc, golden):
    g = golden["splitmix64"]
    assert orc.splitmix64(g["seed"], 0) == int(g["first_output"], 16)


def test_schedule_statistics(orc):
    shape = (64, 48, 8)
    s = orc.schedule(7, 0.25, 0xFFFFFFFF, shape, 0, 20000)
    assert abs(len(s) / 20000 - 0.25) < 0.02
    assert s["x"].max() < 64 and s["y"].max() < 48 and s["z"].max() < 8
    assert set(np.unique(s["bit"])) == set(range(32))
    assert np.all(np.diff(s["step"]) >= 0)
    many = orc.schedule(7, 3.5, 0x0000F000, shape, 0, 2000)
    assert abs(len(many) / 2000 - 3.5) < 0.1
    assert set(np.unique(many["bit"])) == {12, 13, 14, 15}
    again = orc.schedule(7, 3.5, 0x0000F000, shape, 0, 2000)
    np.testing.assert_array_equal(many, again)
    assert len(orc.schedule(7, 0.0, 0xFFFFFFFF, shape, 0, 100)) == 0
    assert len(orc.schedule(7, 1.0, 0, shape, 0, 100)) == 0


# ------------------------------------------- one-vector detection (Sec. 3.2)

def test_one_vector_square_grid_finds_the_same_events(orc):
    """On a square plane both vectors sum the same number of points, so a flip that moves
    a past its threshold moves b past it too: testing b alone (and a only where b failed)
    finds exactly the events of testing both, for every bit."""
    st, C, temp = hotspot(orc, (64, 64, 8), 1)
    rng = np.random.default_rng(5)
    fl = inputs.flip_list([(2 + k, 0, int(rng.integers(8)), int(rng.integers(64)), int(rng.integers(64)), k)
                           for k in range(32)])
    both = orc.run(st, C, temp, 40, orc.MODE_ONLINE, fl)
    one = orc.run(st, C, temp, 40, orc.MODE_ONLINE, fl, vectors=1)
    key = lambda r: sorted((int(e["step"]), int(e["z"]), int(e["y"]), int(e["x"]), int(e["kind"]))
                           for e in r["events"])
    assert key(both) == key(one) and len(key(one)) == 19  # bits 13..31
    np.testing.assert_array_equal(both["u"], one["u"])


@pytest.mark.parametrize("bit", range(13, 24))  # bit 12 lands inside the guard band of a
def test_one_vector_detects_by_the_b_threshold(orc, bit):
    """A non-square plane (nx = 200, ny = 37): b sums 200 points, a only 37, so b's
    threshold eps |b| is higher.  With one vector a flip of size |delta| is found iff
    |delta| > eps |b[z][y]| (the b entry of its row, from the fault-free grid), whatever
    a would say; with both vectors iff it exceeds eps |a| or eps |b|."""
    shape, t, z, y, x = (200, 37, 5), 6, 2, 20, 150
    st, C, temp = hotspot(orc, shape, 7)
    pre = orc.run(st, C, temp, t, orc.MODE_NONE)["u"]       # u^t
    post = orc.run(st, C, pre, 1, orc.MODE_NONE)["u"]       # u^{t+1}, fault-free
    v = np.float32(post[z, y, x])
    flipped = (np.array([v]).view(np.uint32) ^ np.uint32(1 << bit)).view(np.float32)[0]
    delta = abs(float(flipped) - float(v))
    ta = 1e-5 * abs(post[z, :, x].sum())
    tb = 1e-5 * abs(post[z, y, :].sum())
    assert ta < tb
    margin = lambda d, th: abs(d / th - 1.0) > 0.05  # clear of the guard band
    assert margin(delta, ta) and margin(delta, tb)
    fl = inputs.flip_list([(t, 0, z, y, x, bit)])
    one = orc.run(st, C, temp, t + 2, orc.MODE_ONLINE, fl, vectors=1)
    both = orc.run(st, C, temp, t + 2, orc.MODE_ONLINE, fl)
    assert (one["n_events"] > 0) == (delta > tb)
    assert (both["n_events"] > 0) == (delta > ta)
    if ta < delta <= tb:  # seen by a alone: both vectors recompute its column
        assert [(int(e["y"]), int(e["x"]), int(e["kind"])) for e in both["events"]] == [(-1, x, orc.EV_RECOMPUTED)]


@pytest.mark.parametrize("boundary", [PERIODIC, ZERO])
def test_one_vector_square_grid_under_other_boundaries(orc, boundary):
    """The one-vector rule under periodic and empty boundaries: on a square plane,
    high-bit flips (faces included) give the events of testing both vectors."""
    shape = (48, 48, 4)
    co = inputs.hotspot_coeffs(*shape)
    temp, power = inputs.grid_inputs(*shape, seed=9)
    st = orc.Stencil(shape, orc.hotspot_points(co), boundary)
    C = orc.source_term(power, co)
    fl = inputs.flip_list([(2, 0, 0, 0, 0, 29), (4, 0, 3, 47, 47, 30), (6, 0, 1, 0, 20, 28), (8, 0, 2, 30, 0, 27)])
    both = orc.run(st, C, temp, 12, orc.MODE_ONLINE, fl)
    one = orc.run(st, C, temp, 12, orc.MODE_ONLINE, fl, vectors=1)
    key = lambda r: sorted((int(e["step"]), int(e["z"]), int(e["y"]), int(e["x"]), int(e["kind"]))
                           for e in r["events"])
    assert key(both) == key(one) and len(key(one)) == 4
    assert all(k[4] == orc.EV_CORRECTED for k in key(one))


@pytest.mark.parametrize("bit", [14, 18, 22])  # mantissa bits: residual well below eps = 1
def test_guard_band_logs_flips_near_the_threshold(orc, bit):
    """Sec. 3.4's test compares |a' - a| / |a| with eps; the oracle logs, as marginal, the
    (sweep, plane) pairs whose ratio to eps falls within 5 % of 1.  A flip's own residual r
    (the largest of the run when nothing is caught, eps = 1) placed just inside the band on
    either side of the threshold is logged -- caught at eps = r / 1.03, missed at 1.03 r --
    and placed well outside it (r / 3 caught, 3 r missed) is not."""
    st, C, temp = hotspot(orc, (64, 64, 8), 4)
    z = 3
    fl = inputs.flip_list([(6, 0, z, 20, 30, bit)])
    free = orc.run(st, C, temp, 12, orc.MODE_ONLINE, fl, eps=1.0)
    assert free["n_events"] == 0 and not free["marginal"]
    r = free["max_resid"]
    assert r > 1e-9  # far above the FP64 residual of a fault-free sweep
    caught = orc.run(st, C, temp, 12, orc.MODE_ONLINE, fl, eps=r / 1.03)
    assert caught["n_events"] >= 1
    steps = {int(e["step"]) for e in caught["events"]}
    assert {int(e["z"]) for e in caught["events"]} == {z} and len(steps) == 1
    assert caught["marginal"] == {(steps.pop(), z)}
    missed = orc.run(st, C, temp, 12, orc.MODE_ONLINE, fl, eps=r * 1.03)
    assert missed["n_events"] == 0
    assert missed["marginal"] == caught["marginal"]
    clear_hit = orc.run(st, C, temp, 12, orc.MODE_ONLINE, fl, eps=r / 3)
    assert clear_hit["n_events"] >= 1 and not clear_hit["marginal"]
    clear_miss = orc.run(st, C, temp, 12, orc.MODE_ONLINE, fl, eps=r * 3)
    assert clear_miss["n_events"] == 0 and not clear_miss["marginal"]
