"""Failure detection on the GPU without faulting it: the bounded wait the
step kernels use for their tile copies gives up on a barrier that nothing
completes, and the block returns, so a copy that never lands becomes an
error status (LBM_ETIMEOUT from lbm_observe) instead of a hang."""
import time

import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbm():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2408_00146_gb300 import lbm as L
    L.load()
    return L


@pytest.mark.parametrize("limit_ms", [20, 200])
def test_bounded_wait_gives_up_on_time(lbm, limit_ms):
    t0 = time.perf_counter()
    assert lbm.lbm_probe_bounded_wait(limit_ms * 1_000_000)
    dt = time.perf_counter() - t0
    assert dt >= limit_ms * 1e-3 * 0.9
    assert dt < limit_ms * 1e-3 + 2.0          # the wait ended by itself


def test_probe_rejects_bad_limits(lbm):
    for bad in (0, -1, 20_000_000_000):
        with pytest.raises(lbm.LbmError) as e:
            lbm.lbm_probe_bounded_wait(bad)
        assert e.value.status == lbm.LBM_EINVAL
