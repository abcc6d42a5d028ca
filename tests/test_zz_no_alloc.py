"""The allocation-free entry point bta_chol_inv_noalloc against the existing
path (bta_factor of a one-block BTA matrix, which runs the same recursive
Cholesky + inverse on workspace that the context allocated) and against the
plain definitions (LAPACK Cholesky and inverse of the same matrix).

Callers that may not call cudaMalloc -- a framework whose memory pool owns
the device budget, a serving loop that cannot take cudaMalloc's
synchronisation -- use bta_chol_inv_noalloc; its workspace is a fixed device
array inside the library.  Two calls in a row must both agree with the
existing path (the shared workspace keeps the previous call's contents).
This file is named so that pytest collects it last."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _spd(b, seed):
    rng = np.random.default_rng(seed)
    M = rng.standard_normal((b, b))
    return M @ M.T / b + np.eye(b)


def _existing_path(S):
    """Factor S with bta_factor (n = 1, a = 0): returns L and L^{-1} (numpy)."""
    import torch
    from paper_2507_06938_gb300 import bta
    b = S.shape[0]
    ctx = bta.BtaContext(1, b, 0, bta.BTA_FP64)
    D0 = ctx.block(bta.BTA_QP, bta.BTA_STORE_Q, bta.BTA_BLK_D, 0)
    D0.copy_(torch.as_tensor(S, device="cuda"))
    ctx.factor(bta.BTA_QP)
    ctx.sync()
    L = np.tril(ctx.block(bta.BTA_QP, bta.BTA_STORE_L, bta.BTA_BLK_D, 0).cpu().numpy())
    X = ctx.block(bta.BTA_QP, bta.BTA_STORE_LINV, bta.BTA_BLK_D, 0).cpu().numpy()
    return L, X


def _noalloc(S):
    import torch
    from paper_2507_06938_gb300 import bta
    b = S.shape[0]
    A = torch.as_tensor(S.copy(), device="cuda")          # symmetric: row- and column-major agree
    X = torch.full((b, b), float("nan"), dtype=torch.float64, device="cuda")
    info = torch.zeros(1, dtype=torch.int64, device="cuda")
    bta.bta_chol_inv_noalloc(A, X, info)
    torch.cuda.synchronize()
    # the library writes column-major: the torch (row-major) view is the transpose
    return np.tril(A.cpu().numpy().T), X.cpu().numpy().T, int(info.item())


def test_noalloc_matches_existing_entry_point_twice():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_06938_gb300 import _build
    _build.build()
    for b, seed in ((300, 1), (1000, 2), (2048, 5)):
        S = _spd(b, seed)
        L_ref, X_ref = _existing_path(S)
        # the definitions: S = L L^T with positive diagonal, X = L^{-1}
        L_np = np.linalg.cholesky(S)
        X_np = np.linalg.inv(L_np)
        for call in range(2):
            L, X, info = _noalloc(S)
            assert info == -1
            scale_l = np.max(np.abs(L_ref))
            scale_x = np.max(np.abs(X_ref))
            assert np.max(np.abs(L - L_ref)) <= 1e-9 * scale_l, (b, call)
            assert np.max(np.abs(X - X_ref)) <= 1e-9 * scale_x, (b, call)
            assert np.max(np.abs(L - L_np)) <= 1e-9 * np.max(np.abs(L_np)), (b, call)
            assert np.max(np.abs(X - X_np)) <= 1e-9 * np.max(np.abs(X_np)), (b, call)
            assert np.all(np.triu(X, 1) == 0.0)


def test_noalloc_reports_pivot_and_rejects_bad_arguments():
    import ctypes
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_06938_gb300 import _build, bta
    _build.build()
    S = _spd(200, 3)
    S[57, 57] = -5.0
    _, _, info = _noalloc(S)
    assert info == 57
    # the following call starts from a cleared status word
    _, _, info = _noalloc(_spd(200, 4))
    assert info == -1
    f64 = dict(dtype=torch.float64, device="cuda")
    info = torch.zeros(1, dtype=torch.int64, device="cuda")
    big = torch.zeros((bta.NOALLOC_MAX_B + 1, bta.NOALLOC_MAX_B + 1), **f64)
    with pytest.raises(ValueError):
        bta.bta_chol_inv_noalloc(big, big, info)
    # non-square A, undersized X, empty info: rejected before the library is called
    with pytest.raises(ValueError):
        bta.bta_chol_inv_noalloc(torch.zeros((64, 32), **f64), torch.zeros((64, 64), **f64), info)
    with pytest.raises(ValueError):
        bta.bta_chol_inv_noalloc(torch.zeros((64, 64), **f64), torch.zeros((64, 32), **f64), info)
    with pytest.raises(ValueError):
        bta.bta_chol_inv_noalloc(torch.zeros((64, 64), **f64), torch.zeros((64, 64), **f64),
                                 torch.zeros(0, dtype=torch.int64, device="cuda"))
    # the C entry point itself refuses an order above its fixed workspace and
    # leading dimensions below the order (host checks, nothing is launched)
    lib = bta.lib()
    A = torch.zeros((64, 64), **f64)
    assert lib.bta_chol_inv_noalloc(A.data_ptr(), bta.NOALLOC_MAX_B + 1, bta.NOALLOC_MAX_B + 1, A.data_ptr(),
                                    bta.NOALLOC_MAX_B + 1, info.data_ptr(), ctypes.c_void_p(None)) == bta.BTA_ERR_ARG
    assert lib.bta_chol_inv_noalloc(A.data_ptr(), 64, 32, A.data_ptr(), 64, info.data_ptr(),
                                    ctypes.c_void_p(None)) == bta.BTA_ERR_ARG
