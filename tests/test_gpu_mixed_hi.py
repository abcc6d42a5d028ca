"""Mixed precision with 49-bit digits (BTA_MIXED_HI): the same tensor-core
split products as BTA_MIXED with 7 bf16 slices per FP64 value instead of 5,
accumulated exactly per 512-long K chunk and summed across chunks in 64-bit
fixed point.  It exists for ill-conditioned models, such as the SPDE
precision on an irregular Delaunay mesh of uniform random points, whose
condition number reaches 1e10 and defeats the 35-bit digits.

The products then carry about 2^-49 of the operand scale, below the
double-float (about 2^-48) leaves of the diagonal recursion, so the results
sit close to the FP64 path.  Bounds against the FP64 oracle (tier B, itself
pinned to the dense tier): log-determinant 1e-10 relative, solve residual
1e-10 after two FP64-residual refinement steps, selected-inverse blocks 1e-8
of the block maximum, f 1e-9 of |log|Q_p|| + |log|Q_c||, mu 1e-9.  The tensor
threshold is lowered to 64 so that the small cases go through the tensor
kernel with several row and column tiles and ragged tails."""

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


@pytest.mark.parametrize("name,min_dim", [("t_uni_mid", 64), ("t_coreg3_mid", 64), ("t_coreg3_del", 64),
                                          ("c2s", 128)])
def test_mixed_hi_factor_logdet_selinv(name, min_dim, monkeypatch):
    import torch
    from paper_2507_06938_gb300 import bta
    monkeypatch.setenv("BTA_OZ_MIN", str(min_dim))
    p = problem(name)
    prm = omodel.theta_to_params(p.theta0, p.nv)
    built = omodel.build(p, prm)
    run = GpuCase(p, precision=bta.BTA_MIXED_HI)
    for which, Q in ((bta.BTA_QP, built.Qp), (bta.BTA_QC, built.Qc)):
        Lo = obta.factor(obta.blocks_from_sparse(Q, p.nt, p.b, p.a))
        run.assemble(prm, which)
        run.ctx.factor(which)
        ld = torch.zeros(1, dtype=torch.float64, device="cuda")
        run.ctx.logdet(which, ld)
        r = np.random.default_rng(5).standard_normal(p.N)
        x = torch.zeros(p.N, dtype=torch.float64, device="cuda")
        resid = torch.zeros(1, dtype=torch.float64, device="cuda")
        run.ctx.solve(which, dev(r), x, 2, resid)
        run.ctx.selinv(which)
        run.ctx.sync()
        ref = obta.logdet(Lo)
        err_ld = abs(ld.item() - ref) / abs(ref)
        S = blocks_of(run.ctx, which, bta.BTA_STORE_SIGMA, p.nt, p.b, p.a)
        So = obta.selinv(Lo)
        errs = {k: rel_max(S[k], So[k]) for k in ("D", "B", "R", "T")}
        print(name, which, "logdet", err_ld, "resid", resid.item(), "selinv", errs)
        assert err_ld <= 1e-10, err_ld
        assert resid.item() <= 1e-10, resid.item()
        for k, e in errs.items():
            assert e <= 1e-8, (k, e)


@pytest.mark.parametrize("name", ["t_coreg3", "t_coreg3_del"])
def test_mixed_hi_fobj_and_gradient(name, monkeypatch):
    import torch
    from paper_2507_06938_gb300 import bta
    monkeypatch.setenv("BTA_OZ_MIN", "64")
    p = problem(name)
    run = GpuCase(p, precision=bta.BTA_MIXED_HI)
    th = dev(p.theta0[None, :])
    f = torch.zeros(1, dtype=torch.float64, device="cuda")
    mu = torch.zeros(p.N, dtype=torch.float64, device="cuda")
    run.ctx.fobj_eval(run.model, th, f, mu)
    g = torch.zeros((1, p.theta0.shape[0]), dtype=torch.float64, device="cuda")
    run.ctx.fobj_grad(run.model, th, f, g)
    run.ctx.sync()
    terms = ofobj.f_obj_terms(p, p.theta0)
    tol = 1e-9 * (abs(terms["logdet_p"]) + abs(terms["logdet_c"]))
    assert abs(f.item() - terms["f"]) <= tol
    assert rel_max(mu.cpu().numpy(), terms["mu"]) < 1e-9
    gref = ofobj.grad_adjoint(p, p.theta0)
    scale = np.maximum(np.abs(gref), 1e-3 * np.max(np.abs(gref)))
    assert np.max(np.abs(g[0].cpu().numpy() - gref) / scale) < 1e-7


@pytest.mark.parametrize("band", [1, 4, 16])
def test_tile_order_bands(band, monkeypatch):
    """The tile order of the split product (row tiles per band, which the
    autotuner chooses) changes only which CTA computes which tile: the factor,
    log-determinant and selected inverse agree with the oracle at the 49-bit
    bounds for every band, on a case with several row bands and a ragged last
    band (b = 432: 4 row tiles of 128, 7 column tiles of 64)."""
    import torch
    from paper_2507_06938_gb300 import bta
    monkeypatch.setenv("BTA_OZ_MIN", "64")
    monkeypatch.setenv("BTA_OZ_BAND", str(band))
    p = problem("t_coreg3_mid")
    prm = omodel.theta_to_params(p.theta0, p.nv)
    built = omodel.build(p, prm)
    run = GpuCase(p, precision=bta.BTA_MIXED_HI)
    Lo = obta.factor(obta.blocks_from_sparse(built.Qc, p.nt, p.b, p.a))
    run.assemble(prm, bta.BTA_QC)
    run.ctx.factor(bta.BTA_QC)
    ld = torch.zeros(1, dtype=torch.float64, device="cuda")
    run.ctx.logdet(bta.BTA_QC, ld)
    run.ctx.selinv(bta.BTA_QC)
    run.ctx.sync()
    ref = obta.logdet(Lo)
    assert abs(ld.item() - ref) <= 1e-10 * abs(ref)
    S = blocks_of(run.ctx, bta.BTA_QC, bta.BTA_STORE_SIGMA, p.nt, p.b, p.a)
    So = obta.selinv(Lo)
    for k in ("D", "B", "R"):
        e = max(rel_max(S[k][i], So[k][i]) for i in range(So[k].shape[0]))
        assert e <= 1e-8, (band, k, e)
