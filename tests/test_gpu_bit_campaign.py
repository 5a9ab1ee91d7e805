"""The paper's per-bit campaign (Sec. 5.3, Fig. 7) on synthetic data: 64x64x8 HotSpot3D,
online ABFT at eps = 1e-5, one flip per sweep at a random point, per bit position.  The
paper states that flips in bits 0..12 are too small to be detected and that flips in
bits 13..31 are detected and corrected; the GPU must reproduce that split exactly, and
locate every detected flip at its true point."""
import numpy as np
import pytest

from paper_1909_00709_gb300 import inputs
from _util import gpu_context

pytestmark = pytest.mark.gpu

SHAPE = (64, 64, 8)
FLIPS_PER_BIT = 200


@pytest.fixture(scope="module")
def abi():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1909_00709_gb300 import abi, build
    build.build()
    abi.lib()
    return abi


@pytest.fixture(scope="module")
def campaign(abi):
    nx, ny, nz = SHAPE
    out = {}
    for bit in range(32):
        rng = np.random.default_rng(1000 + bit)
        fl = [(t, 0, int(rng.integers(nz)), int(rng.integers(ny)), int(rng.integers(nx)), bit)
              for t in range(1, FLIPS_PER_BIT + 1)]
        with gpu_context(abi, [SHAPE], [0]) as ctx:
            ctx.inject_list(inputs.flip_list(fl))
            ctx.step(FLIPS_PER_BIT + 1, 1)
            ev = ctx.events()
        got = {(int(e["step"]), int(e["z"]), int(e["y"]), int(e["x"])): int(e["kind"]) for e in ev}
        located = sum(1 for (t, _, z, y, x, _) in fl if got.get((t, z, y, x)) == 1)
        out[bit] = (located, len(got))
    return out


def test_undetectable_bits_match_the_paper(campaign, golden):
    for bit in golden["paper_claims"]["undetectable_bits_64x64x8"]["value"]:
        assert campaign[bit] == (0, 0), (bit, campaign[bit])


def test_detectable_bits_are_located_and_corrected(campaign, golden):
    for bit in golden["paper_claims"]["detectable_bits_64x64x8"]["value"]:
        assert campaign[bit] == (FLIPS_PER_BIT, FLIPS_PER_BIT), (bit, campaign[bit])
