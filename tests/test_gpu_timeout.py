"""Failure detection of the tensor-core product without a GPU fault: every
mbarrier wait of the kernel is bounded, and on expiry the kernel raises an
error flag, stops issuing, waits (with the normal limit) for the copies and
MMAs it already issued, frees its tensor memory and returns; the host reports
BTA_ERR_TIMEOUT.

The test shortens the epilogue's wait for the accumulators to 100 cycles
(BTA_OZ_EPI_WAIT), far less than the first TMA copy takes, so that wait runs
out on every CTA.  The error must come back from bta_sync as
BTA_ERR_TIMEOUT, and the same context must then factor correctly with the
normal limit."""

import numpy as np
import pytest

from gpu_util import build_lib, need_gpu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", [1, 2])
def test_short_epilogue_wait_reports_timeout_and_context_recovers(precision, monkeypatch):
    need_gpu()
    build_lib()
    import torch
    from paper_2507_06938_gb300 import bta
    b = 512
    rng = np.random.default_rng(21)
    M = rng.standard_normal((b, b))
    S = M @ M.T / b + np.eye(b)
    ctx = bta.BtaContext(1, b, 0, precision)
    ctx.block(bta.BTA_QP, bta.BTA_STORE_Q, bta.BTA_BLK_D, 0).copy_(torch.as_tensor(S, device="cuda"))
    torch.cuda.synchronize()
    monkeypatch.setenv("BTA_OZ_EPI_WAIT", "100")
    ctx.factor(bta.BTA_QP)
    with pytest.raises(bta.BtaError) as e:
        ctx.sync()
    assert e.value.code == bta.BTA_ERR_TIMEOUT
    monkeypatch.delenv("BTA_OZ_EPI_WAIT")
    ctx.factor(bta.BTA_QP)
    ctx.sync()
    L = np.tril(ctx.block(bta.BTA_QP, bta.BTA_STORE_L, bta.BTA_BLK_D, 0).cpu().numpy())
    Lref = np.linalg.cholesky(S)
    assert np.max(np.abs(L - Lref)) <= 1e-8 * np.max(np.abs(Lref))
    ctx.close()
