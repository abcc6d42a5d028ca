"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Tolerances (FP64 path): assembled blocks 1e-12 relative to the block's
largest entry (same sums in another order); Cholesky blocks and their
inverses 1e-9; log-determinant 1e-10 relative; selected-inverse blocks 1e-9
relative to the block's largest entry; solve residual 1e-10; f_obj 1e-9
relative.  The log-det and selected-inverse bounds are the FP64 targets of
the hot path; the others follow from FP64 rounding (u = 1.1e-16) times
the condition numbers of these matrices (below 1e6)."""

import math

import numpy as np
import pytest

import synth
from oracle import bta as obta
from oracle import dense as odense
from oracle import fobj as ofobj
from oracle import model as omodel

from gpu_util import GpuCase, blocks_of, build_lib, dev, need_gpu, problem, rel_max

pytestmark = pytest.mark.gpu

SMALL = ["t_uni", "t_uni_ragged", "t_coreg2", "t_coreg3", "t_coreg3_del", "t_uni_nt1", "c1"]


@pytest.fixture(scope="module", autouse=True)
def _setup():
    need_gpu()
    build_lib()


def _params(p, theta=None, rho_override=None):
    prm = omodel.theta_to_params(p.theta0 if theta is None else theta, p.nv)
    if rho_override is not None:
        prm.rho[:] = rho_override
    return prm


def _oracle_blocks(p, prm):
    built = omodel.build(p, prm)
    return built, {w: obta.blocks_from_sparse(Q, p.nt, p.b, p.a)
                   for w, Q in ((0, built.Qp), (1, built.Qc))}


@pytest.mark.parametrize("name", SMALL)
def test_assembly_matches_oracle(name):
    from paper_2507_06938_gb300 import bta
    p = problem(name)
    prm = _params(p, rho_override=0.7 if name == "c1" else None)
    built, ref = _oracle_blocks(p, prm)
    run = GpuCase(p)
    for which in (bta.BTA_QP, bta.BTA_QC):
        run.assemble(prm, which)
        run.ctx.sync()
        got = blocks_of(run.ctx, which, bta.BTA_STORE_Q, p.nt, p.b, p.a)
        for k in ("D", "B", "R", "T"):
            assert rel_max(got[k], ref[which][k]) < 1e-12, (which, k)


@pytest.mark.parametrize("leaf", [32, 64])
@pytest.mark.parametrize("name", SMALL)
def test_factor_logdet_solve_selinv_match_dense(name, leaf, monkeypatch):
    from paper_2507_06938_gb300 import bta
    monkeypatch.setenv("BTA_LEAF", str(leaf))
    import torch
    p = problem(name)
    prm = _params(p)
    built, ref = _oracle_blocks(p, prm)
    run = GpuCase(p)
    rng = np.random.default_rng(7)
    for which, Q in ((bta.BTA_QP, built.Qp), (bta.BTA_QC, built.Qc)):
        Qd = Q.toarray()
        run.assemble(prm, which)
        run.ctx.factor(which)
        ld = torch.zeros(1, dtype=torch.float64, device="cuda")
        run.ctx.logdet(which, ld)
        r = rng.standard_normal(p.N)
        x = torch.zeros(p.N, dtype=torch.float64, device="cuda")
        resid = torch.zeros(1, dtype=torch.float64, device="cuda")
        run.ctx.solve(which, dev(r), x, 0, resid)
        run.ctx.selinv(which)
        run.ctx.sync()
        # factor == dense Cholesky on the pattern
        Lref = odense.bta_blocks(np.linalg.cholesky(Qd), p.nt, p.b, p.a)
        L = blocks_of(run.ctx, which, bta.BTA_STORE_L, p.nt, p.b, p.a)
        for k in ("D", "B", "R", "T"):
            got = np.tril(L[k]) if k in ("D", "T") else L[k]
            assert rel_max(got, Lref[k]) < 1e-9, k
        # inverses of the diagonal factor blocks
        for i in range(p.nt):
            Xi = run.ctx.block(which, bta.BTA_STORE_LINV, bta.BTA_BLK_D, i).cpu().numpy()
            assert rel_max(Xi, np.linalg.inv(Lref["D"][i])) < 1e-9
        # log-determinant
        sign, ref_ld = np.linalg.slogdet(Qd)
        assert abs(ld.item() - ref_ld) <= 1e-10 * max(1.0, abs(ref_ld))
        # solve
        assert resid.item() < 1e-10
        assert rel_max(x.cpu().numpy(), np.linalg.solve(Qd, r)) < 1e-9
        # selected inverse
        Sref = odense.bta_blocks(np.linalg.inv(Qd), p.nt, p.b, p.a)
        S = blocks_of(run.ctx, which, bta.BTA_STORE_SIGMA, p.nt, p.b, p.a)
        for k in ("D", "B", "R", "T"):
            assert rel_max(S[k], Sref[k]) < 1e-9, k


@pytest.mark.parametrize("name", ["t_uni", "t_uni_ragged", "t_coreg3", "c1"])
def test_fobj_matches_oracle(name):
    import torch
    p = problem(name)
    run = GpuCase(p)
    rng = np.random.default_rng(11)
    thetas = np.stack([p.theta0, p.theta0 + 0.1 * rng.standard_normal(p.theta0.shape)])
    f = torch.zeros(2, dtype=torch.float64, device="cuda")
    mu = torch.zeros((2, p.N), dtype=torch.float64, device="cuda")
    run.ctx.fobj_eval(run.model, dev(thetas), f, mu)
    run.ctx.sync()
    for j in range(2):
        terms = ofobj.f_obj_terms(p, thetas[j], tier="dense")
        assert abs(f[j].item() - terms["f"]) <= 1e-9 * abs(terms["f"]), j
        assert rel_max(mu[j].cpu().numpy(), terms["mu"]) < 1e-9


@pytest.mark.parametrize("name", ["t_uni_mid", "t_coreg3_mid"])
def test_mid_size_against_tier_b(name):
    """Several tiles per block (b = 289 ragged, b = 432) against the block
    recurrences of the oracle."""
    import torch
    from paper_2507_06938_gb300 import bta
    p = problem(name)
    prm = _params(p)
    built, ref = _oracle_blocks(p, prm)
    run = GpuCase(p)
    which = bta.BTA_QC
    Lo = obta.factor(ref[which])
    So = obta.selinv(Lo)
    run.assemble(prm, which)
    run.ctx.factor(which)
    ld = torch.zeros(1, dtype=torch.float64, device="cuda")
    run.ctx.logdet(which, ld)
    run.ctx.selinv(which)
    run.ctx.sync()
    ref_ld = obta.logdet(Lo)
    assert abs(ld.item() - ref_ld) <= 1e-10 * abs(ref_ld)
    S = blocks_of(run.ctx, which, bta.BTA_STORE_SIGMA, p.nt, p.b, p.a)
    for k in ("D", "B", "R", "T"):
        assert rel_max(S[k], So[k]) < 1e-9, k


def test_not_positive_definite_is_reported():
    import torch
    from paper_2507_06938_gb300 import bta
    p = problem("t_uni")
    prm = _params(p)
    run = GpuCase(p)
    run.assemble(prm, bta.BTA_QP)
    run.ctx.sync()
    D1 = run.ctx.block(bta.BTA_QP, bta.BTA_STORE_Q, bta.BTA_BLK_D, 1)
    D1[5, 5] = -1e6
    torch.cuda.synchronize()
    run.ctx.factor(bta.BTA_QP)
    with pytest.raises(bta.BtaError) as e:
        run.ctx.sync()
    assert e.value.code == bta.BTA_ERR_NOT_PD
    assert e.value.info == p.b + 5
    # the context stays usable: reassemble and factor again
    run.assemble(prm, bta.BTA_QP)
    run.ctx.factor(bta.BTA_QP)
    run.ctx.sync()


def test_argument_errors_are_returned():
    import torch
    from paper_2507_06938_gb300 import bta
    p = problem("t_uni")
    run = GpuCase(p)
    with pytest.raises(bta.BtaError) as e:
        run.ctx.solve(bta.BTA_QC, torch.zeros(p.N, dtype=torch.float64, device="cuda"),
                      torch.zeros(p.N, dtype=torch.float64, device="cuda"))
    assert e.value.code == bta.BTA_ERR_STATE
    with pytest.raises(bta.BtaError):
        run.ctx.factor(5)
