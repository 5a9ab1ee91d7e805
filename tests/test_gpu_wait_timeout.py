"""Failure detection without a fault: the library's bounded device waits give up.

A grid barrier that one CTA never reaches (a block that died) and an mbarrier whose
transaction bytes never arrive (a copy that was lost) each run out after a short
limit; the kernel records the timeout in its status word and returns, the call
reports ABFT_E_TIMEOUT, and the CUDA context is still usable afterwards (a protected
run in the same process matches the oracle)."""
import pytest

from _util import gpu_context, oracle_run, rel_err

pytestmark = pytest.mark.gpu

E_TIMEOUT = 5
LIMIT_US = 200_000


@pytest.fixture(scope="module")
def abi():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1909_00709_gb300 import abi, build
    build.build()
    abi.lib()
    return abi


@pytest.mark.parametrize("which", [0, 1])
def test_wait_runs_out_and_returns(abi, orc, which):
    import torch
    st, ms = abi.abft_selftest_wait(which, LIMIT_US, torch.cuda.current_stream().cuda_stream)
    assert st == E_TIMEOUT
    assert LIMIT_US / 1e3 * 0.9 <= ms <= LIMIT_US / 1e3 + 2000.0, ms
    # the context survived: a protected run right after matches the oracle
    shape = (64, 64, 8)
    with gpu_context(abi, [shape], [5]) as ctx:
        ctx.step(20, 1)
        got = ctx.read(0)
        assert len(ctx.events()) == 0
    assert rel_err(got, oracle_run(orc, shape, 5, 20, orc.MODE_ONLINE)["u"]) < 1e-5


def test_selftest_rejects_bad_arguments(abi):
    assert abi.abft_selftest_wait(2, LIMIT_US)[0] == 1
    assert abi.abft_selftest_wait(0, 10)[0] == 1
