"""Host-side checks of the C-ABI library (no GPU needed): it loads, exports every
symbol include/abft.h declares, validates arguments, and its seeded flip schedule
equals the oracle's independent SplitMix64 implementation."""
import ctypes as ct
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="session")
def abi():
    from paper_1909_00709_gb300 import abi, build
    build.build()
    abi.lib()
    return abi


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"^ABFT_API[^(]*?\b(abft_\w+)\s*\(", text, flags=re.M))
    return names


def test_library_exports_every_declared_symbol(abi):
    names = declared_symbols()
    assert len(names) >= 17
    L = abi.lib()
    missing = [n for n in sorted(names) if not hasattr(L, n)]
    assert not missing, missing
    assert set(abi.EXPORTS) <= names


def test_struct_layouts_match_numpy_views(abi):
    assert ct.sizeof(abi.abft_event) == abi.EVENT.itemsize == 40
    assert ct.sizeof(abi.abft_flip) == abi.FLIP.itemsize == 32
    for name, off in abi.EVENT.fields.items():
        assert getattr(abi.abft_event, name).offset == off[1]
    for name, off in abi.FLIP.fields.items():
        assert getattr(abi.abft_flip, name).offset == off[1]


def test_stencil_structs_match_the_header(abi):
    """abft_point is 16 bytes (three int32 offsets and a float weight); abft_stencil holds a
    count and ABFT_MAX_POINTS points; the options end with the stencil pointer and the
    constant boundary value, as include/abft.h declares."""
    assert ct.sizeof(abi.abft_point) == 16
    assert abi.abft_stencil.pts.offset == 4
    assert ct.sizeof(abi.abft_stencil) == 4 + 16 * abi.MAX_POINTS
    hdr = open(os.path.join(ROOT, "include", "abft.h")).read()
    assert f"#define ABFT_MAX_POINTS {abi.MAX_POINTS}" in hdr
    names = [f[0] for f in abi.abft_options._fields_]
    assert names[-3:] == ["stream", "stencils", "boundary_value"]
    arr = abi.stencil_array([[(0, 0, 0, 0.5), (-2, 1, 0, 0.25)]])
    assert arr[0].npts == 2 and arr[0].pts[1].dx == -2 and arr[0].pts[1].dy == 1 and arr[0].pts[1].w == 0.25
    with pytest.raises(ValueError):
        abi.stencil_array([[]])


def test_default_options_follow_table1(abi):
    o = abi.abft_default_options()
    assert o.eps == 1e-5 and o.delta == 16
    assert o.event_capacity > 0 and o.max_flips_per_step > 0


def test_workspace_bytes_validates(abi):
    o = abi.abft_default_options()
    assert abi.abft_workspace_bytes([(64, 64, 8)], o) > 3 * 64 * 64 * 8 * 4
    assert abi.abft_workspace_bytes([(0, 64, 8)], o) == 0
    assert abi.abft_workspace_bytes([(64, 64, 8)], abi.abft_default_options(tile_y=12)) == 0
    assert abi.abft_workspace_bytes([(64, 64, 8)], abi.abft_default_options(eps=-1.0)) == 0
    # boundary rules 0..3 (clamped, periodic, zero, constant); the field sits where the C
    # struct has it
    assert o.boundary == abi.BC_CLAMP
    for bc in (abi.BC_PERIODIC, abi.BC_ZERO, abi.BC_CONST):
        assert abi.abft_workspace_bytes([(64, 64, 8)], abi.abft_default_options(boundary=bc)) > 0
    assert abi.abft_workspace_bytes([(64, 64, 8)], abi.abft_default_options(boundary=4)) == 0
    # the constant boundary's value must be finite (the last field of the C struct)
    assert o.boundary_value == 0.0 and o.stencils is None
    assert abi.abft_workspace_bytes([(64, 64, 8)],
                                    abi.abft_default_options(boundary=abi.BC_CONST, boundary_value=float("nan"))) == 0
    assert abi.abft_workspace_bytes([(64, 64, 8)], abi.abft_default_options(boundary=-1)) == 0
    # checksum vectors of the online check: 2 (default) or 1; the field after `boundary`
    assert o.vectors == 2
    assert abi.abft_workspace_bytes([(64, 64, 8)], abi.abft_default_options(vectors=1)) > 0
    for bad in (0, 3):
        assert abi.abft_workspace_bytes([(64, 64, 8)], abi.abft_default_options(vectors=bad)) == 0
    big = abi.abft_workspace_bytes([(1024, 1024, 256)], o)
    assert big > 4 * 1024 * 1024 * 256 * 4
    two = abi.abft_workspace_bytes([(64, 64, 8), (100, 37, 5)], o)
    assert two > abi.abft_workspace_bytes([(64, 64, 8)], o)


def test_tune_workspace_covers_every_candidate(abi):
    o = abi.abft_default_options()
    for shapes in ([(64, 64, 8)], [(300, 130, 40)], [(64, 64, 8), (200, 37, 30)]):
        need = abi.abft_tune_workspace_bytes(shapes, o)
        for ty in (8, 16, 32):
            for sh in (0, 1):
                assert need >= abi.abft_workspace_bytes(shapes, abi.abft_default_options(tile_y=ty, shallow=sh))
    assert abi.abft_tune_workspace_bytes([(0, 4, 4)], o) == 0
    L = abi.lib()
    best = abi.abft_options()
    us = ct.c_double()
    g = (abi.abft_grid * 1)(abi.abft_grid(8, 8, 2))
    # bad mode / sweep counts are refused before any CUDA call
    assert L.abft_tune(g, 1, None, None, None, ct.byref(o), 0, 10, None, 0, ct.byref(best), ct.byref(us)) == 1
    tp = (ct.c_void_p * 1)(1024)
    co = (abi.abft_coeffs * 1)()
    assert L.abft_tune(g, 1, tp, tp, co, ct.byref(o), 3, 10, ct.c_void_p(0x1000), 1 << 20, ct.byref(best),
                       ct.byref(us)) == 1
    assert L.abft_tune(g, 1, tp, tp, co, ct.byref(o), 1, 0, ct.c_void_p(0x1000), 1 << 20, ct.byref(best),
                       ct.byref(us)) == 1


def test_init_rejects_bad_arguments_without_touching_the_gpu(abi):
    L = abi.lib()
    h = ct.c_void_p()
    g = (abi.abft_grid * 1)(abi.abft_grid(8, 8, 2))
    o = abi.abft_default_options()
    # NULL pointers and misaligned workspaces are refused before any CUDA call
    assert L.abft_init(ct.byref(h), g, 1, None, None, None, ct.byref(o), None, 0) == 1
    tp = (ct.c_void_p * 1)(1024)
    co = (abi.abft_coeffs * 1)()
    assert L.abft_init(ct.byref(h), g, 1, tp, tp, co, ct.byref(o), ct.c_void_p(0x1001), 1 << 30) == 1
    assert L.abft_init(ct.byref(h), g, 1, tp, tp, co, ct.byref(o), ct.c_void_p(0x1000), 16) == 3


@pytest.mark.parametrize("rate,mask,shape,n_grids,grid", [
    (1e-3, 0xFFFFFFFF, (512, 512, 8), 1, 0),
    (0.25, 0xFFFFFFFF, (64, 64, 8), 1, 0),
    (3.7, 0x0000FF00, (100, 37, 5), 4, 2),
    (268.435456, 0xFFFFFFFF, (1024, 1024, 256), 1, 0),
])
def test_schedule_matches_oracle_generator(abi, orc, rate, mask, shape, n_grids, grid):
    steps = 200 if rate > 100 else 2000
    lib_s = abi.abft_schedule(12345, rate, mask, shape, 0, steps, grid=grid, n_grids=n_grids)
    orc_s = orc.schedule(12345, rate, mask, shape, 0, steps, grid=grid, n_grids=n_grids)
    assert len(lib_s) == len(orc_s)
    for f in ("step", "grid", "z", "y", "x", "bit"):
        np.testing.assert_array_equal(lib_s[f], orc_s[f])


def test_schedule_rejects_bad_arguments(abi):
    with pytest.raises(abi.AbftError):
        abi.abft_schedule(1, -1.0, 0xFFFFFFFF, (8, 8, 2), 0, 10)
    with pytest.raises(abi.AbftError):
        abi.abft_schedule(1, 0.5, 0xFFFFFFFF, (8, 8, 2), 5, 2)
    assert len(abi.abft_schedule(1, 0.0, 0xFFFFFFFF, (8, 8, 2), 0, 10)) == 0


def test_status_strings(abi):
    assert abi.abft_status_string(0) == "ok"
    assert "timed out" in abi.abft_status_string(5)


def test_whole_column_tile_height_follows_the_sm_balance(abi):
    """A grid swept alone on whole-column tiles gets 7-row tiles by default where that
    puts fewer rows on the busiest of the GPU's 152 SMs, which shows in the workspace:
    more tile rows mean larger tile-row partial buffers (two sets of nz x ntx x 128 FP32
    values per tile row).  An explicit tile_y = 8, a grid where 7 rows would not balance
    better, and a context of several grids keep 8 rows."""
    d, e8 = abi.abft_default_options(), abi.abft_default_options(tile_y=8)
    # 512 rows: 74 tile rows of 7 against 64 of 8 (296 tiles against 256)
    extra = abi.abft_workspace_bytes([(512, 512, 8)], d) - abi.abft_workspace_bytes([(512, 512, 8)], e8)
    per_tile_row = 2 * 8 * 4 * 128 * 4  # two partial sets, nz = 8, ntx = 4
    assert 10 * per_tile_row <= extra < 10 * per_tile_row + 4096
    # 608 rows: 87 tile rows of 7 would put more than two tiles on some SMs
    assert abi.abft_workspace_bytes([(512, 608, 8)], d) == abi.abft_workspace_bytes([(512, 608, 8)], e8)
    # a batch keeps 8 rows; deep grids use streaming tiles of 16 rows by default
    pair = [(512, 512, 8), (64, 64, 8)]
    assert abi.abft_workspace_bytes(pair, d) == abi.abft_workspace_bytes(pair, e8)
    assert abi.abft_workspace_bytes([(512, 512, 64)], d) == \
        abi.abft_workspace_bytes([(512, 512, 64)], abi.abft_default_options(tile_y=16))
