"""Periodic and empty (zero) boundaries (Sec. 3.3, "Dealing with Boundary Conditions")
through the C ABI against the FP64 oracle with the same boundary rule.

Periodic boundaries make the boundary terms of Theorem 1 vanish for any weights (the
simple form, Eq. 6/7); empty ones keep a term made of the edge rows, which online checks
read from the previous state and offline chains from each sweep's input state.
Flips are placed on faces, edges and corners, where the boundary rule decides which
points a correction reaches."""
import numpy as np
import pytest

from paper_1909_00709_gb300 import inputs
from _util import compare_events, rel_err

pytestmark = pytest.mark.gpu

NONE, ONLINE, OFFLINE = 0, 1, 2
PERIODIC, ZERO = 1, 2


@pytest.fixture(scope="module")
def abi():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1909_00709_gb300 import abi, build
    build.build()
    abi.lib()
    return abi


def asym_coeffs(shape):
    """HotSpot weights with opposite pairs made unequal (same total weight)."""
    co = dict(inputs.hotspot_coeffs(*shape))
    f32 = lambda v: float(np.float32(v))
    for m, p, k in (("cw", "ce", 0.3), ("cn", "cs", 0.5), ("cb", "ct", 0.2)):
        w = co[m]
        co[m], co[p] = f32(w * (1 + k)), f32(w * (1 - k))
    return co


def context(abi, shape, seed, bc, coeffs=None, **opt):
    t, p = inputs.grid_inputs(*shape, seed=seed)
    co = coeffs or inputs.hotspot_coeffs(*shape)
    return abi.Context([shape], [t], [p], [co], boundary=bc, **opt)


def oracle(orc, shape, seed, bc, steps, mode, flips=None, coeffs=None, **kw):
    co = coeffs or inputs.hotspot_coeffs(*shape)
    t, p = inputs.grid_inputs(*shape, seed=seed)
    st = orc.Stencil(shape, orc.hotspot_points(co), bc)
    return orc.run(st, orc.source_term(p, co), t, steps, mode, flips, **kw)


def tol(steps):
    return 1e-5 * max(1.0, steps / 100.0)


def face_flips(shape, t0):
    """High-bit flips on faces, edges and corners of the grid, one sweep apart."""
    nx, ny, nz = shape
    pts = [(0, 0, 0), (nz - 1, ny - 1, nx - 1), (0, ny // 2, nx - 1), (nz - 1, 0, nx // 2),
           (nz // 2, ny - 1, 0), (nz // 2, ny // 2, nx // 2)]
    return inputs.flip_list([(t0 + 2 * i, 0, z, y, x, 26 + i % 5) for i, (z, y, x) in enumerate(pts)])


SWEEP_SHAPES = [(64, 64, 8), (200, 37, 5), (129, 17, 3), (33, 1, 4), (1, 7, 1), (257, 64, 9), (150, 40, 20),
                (70, 33, 1)]


@pytest.mark.parametrize("bc", [PERIODIC, ZERO])
@pytest.mark.parametrize("shallow", [0, 1])
@pytest.mark.parametrize("tile_y", [8, 16, 32])
@pytest.mark.parametrize("shape", SWEEP_SHAPES)
def test_one_sweep_matches_eq1(abi, orc, shape, tile_y, shallow, bc):
    with context(abi, shape, 3, bc, tile_y=tile_y, shallow=shallow) as ctx:
        ctx.step(1, NONE)
        got = ctx.read(0)
    assert rel_err(got, oracle(orc, shape, 3, bc, 1, orc.MODE_NONE)["u"]) < 1e-6


@pytest.mark.parametrize("bc", [PERIODIC, ZERO])
@pytest.mark.parametrize("shallow", [0, 1])
@pytest.mark.parametrize("persistent", [0, 1])
@pytest.mark.parametrize("shape", [(64, 64, 8), (200, 37, 5), (150, 40, 20), (70, 33, 1)])
def test_online_fault_free(abi, orc, shape, persistent, shallow, bc):
    """Theorem 1 with the boundary rule's terms predicts every checksum: no event."""
    steps = 60
    with context(abi, shape, 5, bc, coeffs=asym_coeffs(shape), persistent=persistent, shallow=shallow) as ctx:
        ctx.step(steps, ONLINE)
        got = ctx.read(0)
        assert len(ctx.events()) == 0
    ref = oracle(orc, shape, 5, bc, steps, orc.MODE_ONLINE, coeffs=asym_coeffs(shape))
    assert ref["n_events"] == 0
    assert rel_err(got, ref["u"]) < tol(steps)


@pytest.mark.parametrize("bc", [PERIODIC, ZERO])
@pytest.mark.parametrize("path", ["per_launch", "persistent", "overlapped"])
@pytest.mark.parametrize("shape", [(200, 37, 5), (300, 130, 6), (150, 40, 20)])
def test_online_face_flips_parity(abi, orc, shape, path, bc):
    """Flips on faces, edges and corners: the same points located and corrected as the
    oracle, values within tolerance, on every online path."""
    steps = 20
    flips = face_flips(shape, 3)
    opt = {"per_launch": dict(persistent=0, overlap=0), "persistent": dict(persistent=1),
           "overlapped": dict(persistent=0, overlap=1)}[path]
    with context(abi, shape, 7, bc, **opt) as ctx:
        ctx.inject_list(flips)
        ctx.step(11, ONLINE)
        ctx.step(steps - 11, ONLINE)
        got = ctx.read(0)
        ev = ctx.events()
    ref = oracle(orc, shape, 7, bc, steps, orc.MODE_ONLINE, flips)
    g, o = compare_events(ev, ref)
    assert g == o and len(o) == len(flips)
    assert rel_err(got, ref["u"]) < tol(steps)


@pytest.mark.parametrize("bc", [PERIODIC, ZERO])
@pytest.mark.parametrize("shallow", [0, 1])
@pytest.mark.parametrize("shape", [(300, 130, 6), (140, 70, 19)])
def test_online_paths_agree_bitwise(abi, shape, shallow, bc):
    """Per-launch, persistent (speculative sweep repaired after a late correction) and
    overlapped (tiles recomputed after a late correction) online paths give the same
    grid and events bit for bit; a correction on a face reaches the opposite face only
    under periodic boundaries, so the repair must cover it."""
    steps = 24
    nx, ny, nz = shape
    flips = inputs.flip_list([(3, 0, 0, 0, 0, 30), (4, 0, 0, 1, 0, 28), (7, 0, nz - 1, ny - 1, nx - 1, 29),
                              (8, 0, nz - 1, ny - 1, nx - 2, 27), (12, 0, 2, ny - 1, 5, 31), (12, 0, 3, 0, nx - 1, 26),
                              (13, 0, 3, 1, nx - 1, 30), (17, 0, 0, 40, 60, 30), (17, 0, 0, 41, 90, 28)])
    out = []
    for opt in (dict(persistent=0, overlap=0), dict(persistent=1), dict(persistent=0, overlap=1)):
        with context(abi, shape, 9, bc, shallow=shallow, **opt) as ctx:
            ctx.inject_list(flips)
            ctx.step(10, ONLINE)
            ctx.step(steps - 10, ONLINE)
            out.append((ctx.read(0), sorted(map(tuple, ctx.events()[["step", "z", "y", "x", "kind"]].tolist()))))
    for k in (1, 2):
        np.testing.assert_array_equal(out[0][0].view(np.uint32), out[k][0].view(np.uint32))
        assert out[0][1] == out[k][1]
    assert len(out[0][1]) > 0


@pytest.mark.parametrize("shallow", [0, 1])
@pytest.mark.parametrize("persistent", [0, 1])
@pytest.mark.parametrize("shape", [(64, 64, 8), (200, 37, 5), (140, 70, 19)])
def test_offline_periodic_asymmetric_weights(abi, orc, shape, persistent, shallow):
    """Periodic boundaries: the chain of Fig. 10 is exact for unequal opposite weights,
    so windows with a detectable flip are rolled back and recomputed as in the oracle."""
    steps = 40
    co = asym_coeffs(shape)
    flips = inputs.flip_list([(20, 0, 0, 0, 0, 28), (35, 0, shape[2] - 1, 3, shape[0] - 1, 30), (9, 0, 0, 1, 2, 3)])
    with context(abi, shape, 4, PERIODIC, coeffs=co, persistent=persistent, shallow=shallow) as ctx:
        ctx.inject_list(flips)
        ctx.step(steps, OFFLINE)
        got = ctx.read(0)
        ev = ctx.events()
        cnt = ctx.counters()
    ref = oracle(orc, shape, 4, PERIODIC, steps, orc.MODE_OFFLINE, flips, coeffs=co, delta=16)
    g, o = compare_events(ev, ref)
    assert g == o
    assert cnt["rollbacks"] == ref["n_rollbacks"] == 2
    assert rel_err(got, ref["u"]) < tol(steps)


@pytest.mark.parametrize("asym", [True, False], ids=["asym", "sym"])
@pytest.mark.parametrize("bc", [0, PERIODIC, ZERO], ids=["clamp", "periodic", "zero"])
def test_offline_with_any_terms_matches_oracle(abi, orc, bc, asym):
    """Offline windows under every rule and weight choice.  Periodic boundaries, and
    clamped ones with equal opposite weights, chain Eq. (6)/(7) up front; elsewhere (empty
    boundaries, unequal weights under clamping) each link of the chain takes Theorem 1's
    boundary terms from its sweep's input state.  Face and interior flips are rolled back
    as the oracle rolls them back, and the values agree."""
    shape, steps, delta = (64, 64, 8), 48, 16
    co = asym_coeffs(shape) if asym else None
    fl = inputs.flip_list([(2, 0, 0, 0, 10, 28), (20, 0, 7, 63, 63, 27), (37, 0, 3, 30, 0, 30)])
    with context(abi, shape, 1, bc, coeffs=co, delta=delta) as ctx:
        ctx.inject_list(fl)
        ctx.step(steps, OFFLINE)
        got = ctx.read(0)
        ev = ctx.events()
        rb = ctx.counters()["rollbacks"]
    ref = oracle(orc, shape, 1, bc, steps, orc.MODE_OFFLINE, fl, coeffs=co, delta=delta)
    assert rb == ref["n_rollbacks"] == 3
    g, o = compare_events(ev, ref)
    assert g == o
    assert rel_err(got, ref["u"]) < tol(steps)


@pytest.mark.parametrize("bc", [PERIODIC, ZERO])
def test_batched_equals_grid_by_grid(abi, bc):
    """Several uneven grids advanced by batched launches equal advancing them one by one."""
    shapes = [(200, 37, 5), (64, 64, 8), (129, 17, 3), (150, 40, 20), (70, 33, 1)]
    temps, powers, coeffs = [], [], []
    for i, s in enumerate(shapes):
        t, p = inputs.grid_inputs(*s, seed=30 + i)
        temps.append(t)
        powers.append(p)
        coeffs.append(inputs.hotspot_coeffs(*s))
    flips = inputs.flip_list([(2, 0, 0, 0, 0, 30), (2, 1, 7, 63, 63, 29), (5, 3, 19, 39, 149, 28),
                              (6, 4, 0, 32, 0, 30)])
    out = []
    for batch in (0, 1):
        with abi.Context(shapes, temps, powers, coeffs, boundary=bc, batch=batch) as ctx:
            ctx.inject_list(flips)
            ctx.step(9, ONLINE)
            ctx.step(4, NONE)
            out.append(([ctx.read(i) for i in range(len(shapes))],
                        sorted(map(tuple, ctx.events()[["step", "grid", "z", "y", "x", "kind"]].tolist()))))
    for a, b in zip(out[0][0], out[1][0]):
        np.testing.assert_array_equal(a.view(np.uint32), b.view(np.uint32))
    assert out[0][1] == out[1][1] and len(out[0][1]) == 4


def test_periodic_checksums_follow_simple_form(abi, orc):
    """With periodic boundaries the checksums the library holds after a fault-free
    online run equal the oracle's Eq. (2)/(3) sums of its own grid."""
    shape, steps = (150, 40, 20), 30
    with context(abi, shape, 11, PERIODIC, coeffs=asym_coeffs(shape)) as ctx:
        ctx.step(steps, ONLINE)
        a, b = ctx.read_checksums(0)
    ref = oracle(orc, shape, 11, PERIODIC, steps, orc.MODE_ONLINE, coeffs=asym_coeffs(shape))
    u = ref["u"].reshape(shape[2], shape[1], shape[0])
    np.testing.assert_allclose(a.reshape(shape[2], shape[0]), u.sum(axis=1), rtol=1e-5)
    np.testing.assert_allclose(b.reshape(shape[2], shape[1]), u.sum(axis=2), rtol=1e-5)


@pytest.mark.parametrize("bc", [PERIODIC, ZERO])
@pytest.mark.parametrize("path", ["per_launch", "persistent", "overlapped"])
@pytest.mark.parametrize("shape", [(200, 37, 5), (300, 130, 6), (150, 40, 20)])
def test_one_vector_face_flips_parity(abi, orc, shape, path, bc):
    """One checksum vector per sweep (a summed on demand, with the rule's neighbours and
    boundary terms) under periodic and empty boundaries: the oracle's events and values."""
    steps = 20
    flips = face_flips(shape, 3)
    opt = {"per_launch": dict(persistent=0, overlap=0), "persistent": dict(persistent=1),
           "overlapped": dict(persistent=0, overlap=1)}[path]
    co = asym_coeffs(shape)
    with context(abi, shape, 7, bc, coeffs=co, vectors=1, **opt) as ctx:
        ctx.inject_list(flips)
        ctx.step(11, ONLINE)
        ctx.step(steps - 11, ONLINE)
        got = ctx.read(0)
        ev = ctx.events()
    ref = oracle(orc, shape, 7, bc, steps, orc.MODE_ONLINE, flips, coeffs=co, vectors=1)
    g, o = compare_events(ev, ref)
    assert g == o and len(o) > 0
    assert rel_err(got, ref["u"]) < tol(steps)
