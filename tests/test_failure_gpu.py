"""Device failure path without a GPU fault: a bounded wait that runs out.

Every spin-wait in the library's kernels (mbarrier waits of the TMA row
copies and of the tcgen05 pipelines) is bounded by %globaltimer; on expiry the
kernel records DEV_ERR_WAIT_TIMEOUT in the context's status word and returns.
se_check_wait_timeout queues one such wait that nothing completes; the test
checks that se_sync reports it, clears it, and that the context keeps working.
"""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2204_14194_gb300 import binding as B
from paper_2204_14194_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    c = B.Context(0)
    yield c
    c.close()


def test_bounded_wait_runs_out_and_is_reported(ctx):
    t0 = time.perf_counter()
    ctx.check_wait_timeout(100_000)          # 0.1 s
    with pytest.raises(B.SeError) as e:
        ctx.sync()
    dt = time.perf_counter() - t0
    assert e.value.status == -3          # SE_ERR_CUDA
    assert "bounded device wait" in str(e.value)
    assert 0.09 <= dt < 5.0, dt
    ctx.sync()                               # the word was cleared


def test_context_stays_usable_after_a_timeout(ctx):
    ctx.check_wait_timeout(50_000)
    with pytest.raises(B.SeError):
        ctx.sync()
    wl = W.config2(32)
    plan = ctx.plan(32, 32, "dct_wht", 2048, wl.rho_hat, wl.gamma, 40, prec="bf16x6")
    s = torch.from_numpy(wl.samples).cuda()
    out = torch.empty_like(s)
    plan.extrapolate_strided(s, out)
    ctx.sync()
    o = out.cpu().numpy()
    np.testing.assert_array_equal(o[:, wl.support > 0], wl.samples[:, wl.support > 0])
    assert np.isfinite(o).all()
    plan.close()


def test_wait_limit_is_validated(ctx):
    with pytest.raises(B.SeError):
        ctx.check_wait_timeout(10)
    with pytest.raises(B.SeError):
        ctx.check_wait_timeout(10_000_000)
