"""The allocation-free entry point (abft_sweep_checksums_static) against the context
path.  It serves callers that may not allocate device memory, so the test allocates
every buffer itself (with torch) and hands the library only pointers.  Two calls in
a row: the second reuses the library's shared scratch array and must match the
context path's second sweep as well."""
import numpy as np
import pytest

from paper_1909_00709_gb300 import inputs

pytestmark = pytest.mark.gpu


def pitched(torch, a, pitch):
    nz, ny, nx = a.shape
    t = torch.zeros((nz, ny, pitch), dtype=torch.float32, device="cuda")
    t[:, :, :nx] = torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return t


@pytest.mark.parametrize("shape,pitch", [((200, 37, 5), 224),   # two x-tiles, ragged in x and y
                                         ((201, 37, 5), 204)])  # pitch a multiple of 4, not of 32
def test_static_entry_matches_context_path_on_two_calls(shape, pitch):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1909_00709_gb300 import abi, build
    build.build()
    nx, ny, nz = shape
    temp, power = inputs.grid_inputs(*shape, seed=21)
    co = inputs.hotspot_coeffs(*shape)
    with abi.Context([shape], [temp], [power], [co]) as ctx:
        ctx.step(1, abi.MODE_NONE)
        ref1 = ctx.read(0).astype(np.float64)
        ctx.step(1, abi.MODE_NONE)
        ref2 = ctx.read(0).astype(np.float64)

    f32 = np.float32
    C = (f32(co["sdc"]) * power.astype(f32) + f32(co["c_amb"]) * f32(co["t_amb"])).astype(f32)
    dC = pitched(torch, C, pitch)
    u0 = pitched(torch, temp, pitch)
    u1 = torch.zeros_like(u0)
    u2 = torch.zeros_like(u0)
    a = torch.zeros((nz, nx), dtype=torch.float64, device="cuda")
    b = torch.zeros((nz, ny), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream

    # the FP64 oracle's two sweeps (Eq. 1) and checksums (Eq. 2, 3) of the same inputs
    import oracle
    st = oracle.Stencil(shape, oracle.hotspot_points(co))
    Cd = oracle.source_term(power, co)
    o1 = oracle.sweep(st, Cd, temp)
    o2 = oracle.sweep(st, Cd, o1)

    for src, dst, ref, orf in ((u0, u1, ref1, o1), (u1, u2, ref2, o2)):
        st_ = abi.abft_sweep_checksums_static(src.data_ptr(), dC.data_ptr(), dst.data_ptr(), a.data_ptr(),
                                              b.data_ptr(), shape, pitch, co, stream)
        assert st_ == 0, abi.abft_status_string(st_)
        torch.cuda.synchronize()
        got = dst[:, :, :nx].cpu().numpy().astype(np.float64)
        assert np.max(np.abs(got - ref) / np.abs(ref)) < 1e-6
        assert np.max(np.abs(got - orf) / np.abs(orf)) < 1e-6
        # the padding columns past nx are never written
        assert float(dst[:, :, nx:].abs().max().item() if pitch > nx else 0.0) == 0.0
        # the returned checksums are the row and column sums of the returned grid (Eq. 2, 3)
        np.testing.assert_allclose(a.cpu().numpy(), got.sum(axis=1), rtol=1e-6, atol=0)
        np.testing.assert_allclose(b.cpu().numpy(), got.sum(axis=2), rtol=1e-6, atol=0)
        oa, ob = oracle.checksums(orf)
        np.testing.assert_allclose(a.cpu().numpy(), oa, rtol=1e-6, atol=0)
        np.testing.assert_allclose(b.cpu().numpy(), ob, rtol=1e-6, atol=0)


def test_static_entry_refuses_grids_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1909_00709_gb300 import abi
    co = inputs.hotspot_coeffs(4096, 4096, 64)
    # pointers are never dereferenced: the size check comes first
    fake = 1 << 20
    st = abi.abft_sweep_checksums_static(fake, fake, fake + (1 << 12), fake, fake, (4096, 4096, 64), 4096, co, 0)
    assert st == 1
    st = abi.abft_sweep_checksums_static(fake, fake, fake + (1 << 12), fake, fake, (64, 64, 8), 62, co, 0)
    assert st == 1  # pitch not a multiple of 4
