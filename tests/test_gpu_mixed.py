"""Mixed-precision path (BTA_MIXED): the large Schur-update, triangular and
selected-inversion products run as digit-split FP64 products on the tcgen05
tensor cores (5 bf16 slices of 7 bits per operand, ~36 significant bits
below each row/column maximum); the arrow, tip, log-det and refinement
residuals stay FP64.

Bounds (against the FP64 oracle): log-determinant relative error <= 1e-8
and, after two refinement steps with an FP64 residual, solve residual
<= 1e-10 (the mixed-path targets).  Selected-inverse blocks carry the
36-bit product error amplified by the conditioning of the recurrence; the
largest relative error measured (fixed-effect arrow/tip blocks of Q_c at
b = 1024) is 7.4e-6, so the bound here is 5e-5 relative to the block
maximum; the FP64 path keeps the 1e-9 bound."""

import numpy as np
import pytest

from oracle import bta as obta
from oracle import fobj as ofobj
from oracle import model as omodel

from gpu_util import GpuCase, blocks_of, build_lib, dev, need_gpu, problem, rel_max

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _setup():
    need_gpu()
    build_lib()


@pytest.mark.parametrize("name,min_dim", [("t_uni_mid", 64), ("t_coreg3_mid", 64), ("t_coreg3_mid", 128),
                                          ("c2s", 256)])
def test_mixed_factor_logdet_selinv(name, min_dim, monkeypatch):
    import torch
    from paper_2507_06938_gb300 import bta
    monkeypatch.setenv("BTA_OZ_MIN", str(min_dim))
    p = problem(name)
    prm = omodel.theta_to_params(p.theta0, p.nv)
    built = omodel.build(p, prm)
    run = GpuCase(p, precision=bta.BTA_MIXED)
    for which, Q in ((bta.BTA_QP, built.Qp), (bta.BTA_QC, built.Qc)):
        blk = obta.blocks_from_sparse(Q, p.nt, p.b, p.a)
        Lo = obta.factor(blk)
        run.assemble(prm, which)
        run.ctx.factor(which)
        ld = torch.zeros(1, dtype=torch.float64, device="cuda")
        run.ctx.logdet(which, ld)
        rng = np.random.default_rng(5)
        r = rng.standard_normal(p.N)
        x = torch.zeros(p.N, dtype=torch.float64, device="cuda")
        resid = torch.zeros(1, dtype=torch.float64, device="cuda")
        run.ctx.solve(which, dev(r), x, 2, resid)
        run.ctx.selinv(which)
        run.ctx.sync()
        ref = obta.logdet(Lo)
        err_ld = abs(ld.item() - ref) / abs(ref)
        assert err_ld <= 1e-8, err_ld
        assert resid.item() <= 1e-10, resid.item()
        S = blocks_of(run.ctx, which, bta.BTA_STORE_SIGMA, p.nt, p.b, p.a)
        So = obta.selinv(Lo)
        errs = {k: rel_max(S[k], So[k]) for k in ("D", "B", "R", "T")}
        print(name, which, "logdet", err_ld, "resid", resid.item(), "selinv", errs)
        for k, e in errs.items():
            assert e <= 5e-5, (k, e)


@pytest.mark.parametrize("name", ["t_coreg3", "t_uni_mid"])
def test_mixed_fobj(name, monkeypatch):
    import torch
    from paper_2507_06938_gb300 import bta
    monkeypatch.setenv("BTA_OZ_MIN", "64")
    p = problem(name)
    run = GpuCase(p, precision=bta.BTA_MIXED)
    th = p.theta0[None, :]
    f = torch.zeros(1, dtype=torch.float64, device="cuda")
    mu = torch.zeros(p.N, dtype=torch.float64, device="cuda")
    run.ctx.fobj_eval(run.model, dev(th), f, mu)
    run.ctx.sync()
    terms = ofobj.f_obj_terms(p, p.theta0)
    # f combines log-dets of size ~1e3-1e4 with 1e-8 relative error each
    tol = 1e-8 * (abs(terms["logdet_p"]) + abs(terms["logdet_c"]))
    assert abs(f.item() - terms["f"]) <= tol
    assert rel_max(mu.cpu().numpy(), terms["mu"]) < 1e-9


@pytest.mark.parametrize("b", [37, 100, 128])
def test_double_float_leaf(b):
    """Mixed precision factors diagonal blocks of order <= 128 in double-float
    (two FP32 words, about 48 bits): L and L^{-1} must match the FP64
    Cholesky to 1e-11 relative; a non-positive pivot is reported."""
    import torch
    from paper_2507_06938_gb300 import bta
    rng = np.random.default_rng(b)
    M = rng.standard_normal((b, b))
    S = M @ M.T / b + 0.5 * np.eye(b)
    ctx = bta.BtaContext(1, b, 0, bta.BTA_MIXED)
    ctx.block(bta.BTA_QP, bta.BTA_STORE_Q, bta.BTA_BLK_D, 0).copy_(torch.as_tensor(S, device="cuda"))
    ctx.factor(bta.BTA_QP)
    ctx.sync()
    L = np.tril(ctx.block(bta.BTA_QP, bta.BTA_STORE_L, bta.BTA_BLK_D, 0).cpu().numpy())
    X = ctx.block(bta.BTA_QP, bta.BTA_STORE_LINV, bta.BTA_BLK_D, 0).cpu().numpy()
    Lref = np.linalg.cholesky(S)
    assert rel_max(L, Lref) < 1e-11
    assert rel_max(X, np.linalg.inv(Lref)) < 1e-11
    S[b // 2, b // 2] = -1.0
    ctx.block(bta.BTA_QP, bta.BTA_STORE_Q, bta.BTA_BLK_D, 0).copy_(torch.as_tensor(S, device="cuda"))
    ctx.factor(bta.BTA_QP)
    with pytest.raises(bta.BtaError) as e:
        ctx.sync()
    assert e.value.code == bta.BTA_ERR_NOT_PD
    assert e.value.info <= b // 2


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_autotune_keeps_results_exact(precision):
    """The autotuner only changes launch shapes: after it runs, f_obj and the
    conditional mean still match the oracle at the bounds of the precision."""
    import torch
    from gpu_util import GpuCase, dev, problem, rel_max
    from oracle import fobj as ofobj
    p = problem("t_uni_mid")
    run = GpuCase(p, precision=precision, batch=2)
    leaf, df_leaf, tmin, tile, waves, ctas, band_tri, band_gen, band_low = run.ctx.autotune(reps=1)
    if precision == 0:
        assert leaf in (16, 32, 64) and ctas in (1, 2, 4)
    else:
        assert df_leaf in (32, 64, 128) and tmin in (128, 256, 384, 512)
        assert tile in ((0, 1) if precision == 1 else (0,)) and waves in (1, 2)
        assert band_tri in (1, 4, 8, 16) and band_gen in (1, 4, 8, 16) and band_low in (1, 4, 8, 16)
    th = np.stack([p.theta0, p.theta0 + 1e-3])
    f = torch.zeros(2, dtype=torch.float64, device="cuda")
    mu = torch.zeros((2, p.N), dtype=torch.float64, device="cuda")
    run.ctx.fobj_eval(run.model, dev(th), f, mu)
    run.ctx.sync()
    for j in range(2):
        terms = ofobj.f_obj_terms(p, th[j])
        tol = 1e-9 * abs(terms["f"]) if precision != 1 else 1e-8 * (abs(terms["logdet_p"]) + abs(terms["logdet_c"]))
        assert abs(f[j].item() - terms["f"]) <= tol
        assert rel_max(mu[j].cpu().numpy(), terms["mu"]) < 1e-8


@pytest.mark.parametrize("name", ["t_coreg3_mid", "c2s"])
def test_mixed_tile_128x64_three_stages(name, monkeypatch):
    """The second 35-bit tile configuration of the split product (128 x 64
    tiles, 3 TMA stages), which the autotuner may choose, at the same bounds
    as the default one."""
    import torch
    from paper_2507_06938_gb300 import bta
    monkeypatch.setenv("BTA_OZ_MIN", "128")
    monkeypatch.setenv("BTA_OZ_TILE", "1")
    p = problem(name)
    prm = omodel.theta_to_params(p.theta0, p.nv)
    built = omodel.build(p, prm)
    run = GpuCase(p, precision=bta.BTA_MIXED)
    Q = built.Qc
    Lo = obta.factor(obta.blocks_from_sparse(Q, p.nt, p.b, p.a))
    run.assemble(prm, bta.BTA_QC)
    run.ctx.factor(bta.BTA_QC)
    ld = torch.zeros(1, dtype=torch.float64, device="cuda")
    run.ctx.logdet(bta.BTA_QC, ld)
    run.ctx.selinv(bta.BTA_QC)
    run.ctx.sync()
    ref = obta.logdet(Lo)
    assert abs(ld.item() - ref) / abs(ref) <= 1e-8
    S = blocks_of(run.ctx, bta.BTA_QC, bta.BTA_STORE_SIGMA, p.nt, p.b, p.a)
    So = obta.selinv(Lo)
    for k in ("D", "B", "R", "T"):
        assert rel_max(S[k], So[k]) <= 5e-5, k
