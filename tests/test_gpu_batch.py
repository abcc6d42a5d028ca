"""Batched evaluation: several theta points (the central-difference stencil of
Eq. 10) and both matrices of each go through the same kernel launches.
Each slot must agree with the oracle evaluated on its own theta, including a
partial last group, and errors must name the failing matrix."""

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


def _stencil(theta0, h=1e-3):
    pts = [theta0]
    for i in range(theta0.shape[0]):
        e = np.zeros_like(theta0)
        e[i] = h
        pts += [theta0 + e, theta0 - e]
    return np.stack(pts)


@pytest.mark.parametrize("name,precision,batch", [("t_uni", 0, 3), ("t_coreg2", 0, 4), ("t_uni_mid", 1, 4)])
def test_batched_fobj_and_selinv(name, precision, batch, monkeypatch):
    import torch
    from paper_2507_06938_gb300 import bta
    monkeypatch.setenv("BTA_OZ_MIN", "64")
    p = problem(name)
    thetas = _stencil(p.theta0)[:5]          # 5 points: one full group and a partial one when batch < 5
    run = GpuCase(p, precision=precision, batch=batch)
    f = torch.zeros(thetas.shape[0], dtype=torch.float64, device="cuda")
    mu = torch.zeros((thetas.shape[0], p.N), dtype=torch.float64, device="cuda")
    run.ctx.fobj_eval(run.model, dev(thetas), f, mu)
    run.ctx.sync()
    ftol = 1e-9 if precision == 0 else 1e-7
    for j in range(thetas.shape[0]):
        terms = ofobj.f_obj_terms(p, thetas[j])
        assert abs(f[j].item() - terms["f"]) <= ftol * abs(terms["f"]), j
        assert rel_max(mu[j].cpu().numpy(), terms["mu"]) < 1e-8, j
    # a full group evaluated last, then the selected inverse of every Q_c slot
    run.ctx.fobj_eval(run.model, dev(thetas[:batch]), f[:batch].contiguous(), None)
    run.ctx.selinv_batch(bta.BTA_QC)
    run.ctx.sync()
    stol = 1e-9 if precision == 0 else 5e-5
    for j in range(batch):
        built = omodel.build(p, omodel.theta_to_params(thetas[j], p.nv))
        So = obta.selinv(obta.factor(obta.blocks_from_sparse(built.Qc, p.nt, p.b, p.a)))
        S = blocks_of(run.ctx, 2 * j + bta.BTA_QC, bta.BTA_STORE_SIGMA, p.nt, p.b, p.a)
        for k in ("D", "B", "R", "T"):
            assert rel_max(S[k], So[k]) < stol, (j, k)


def test_batched_error_names_the_matrix():
    import torch
    from paper_2507_06938_gb300 import bta
    p = problem("t_uni")
    run = GpuCase(p, batch=3)
    prm = omodel.theta_to_params(p.theta0, p.nv)
    params = dev(omodel.params_vector(prm))
    for j in range(3):
        run.ctx.assemble(run.model, params, 2 * j + bta.BTA_QC)
    run.ctx.sync()
    D = run.ctx.block(2 * 2 + bta.BTA_QC, bta.BTA_STORE_Q, bta.BTA_BLK_D, 2)
    D[3, 3] = -1e6
    torch.cuda.synchronize()
    run.ctx.factor_batch(bta.BTA_QC)
    with pytest.raises(bta.BtaError) as e:
        run.ctx.sync()
    assert e.value.code == bta.BTA_ERR_NOT_PD
    assert e.value.info == 2 * p.b + 3
    assert e.value.matrix == 2 * 2 + bta.BTA_QC


@pytest.mark.parametrize("precision", [0, 1])
def test_graph_replay_matches_direct(precision, monkeypatch):
    """From the second full group on, fobj_eval replays a captured CUDA graph;
    its values must equal those of the direct launches, for new thetas too."""
    import torch
    monkeypatch.setenv("BTA_OZ_MIN", "64")
    p = problem("t_uni_mid")
    run = GpuCase(p, precision=precision, batch=3)
    rng = np.random.default_rng(21)
    tol = 1e-9 if precision == 0 else 1e-7
    for call in range(4):
        thetas = p.theta0 + 0.05 * rng.standard_normal((3, p.theta0.shape[0]))
        f = torch.zeros(3, dtype=torch.float64, device="cuda")
        mu = torch.zeros((3, p.N), dtype=torch.float64, device="cuda")
        run.ctx.fobj_eval(run.model, dev(thetas), f, mu)
        run.ctx.sync()
        for j in range(3):
            terms = ofobj.f_obj_terms(p, thetas[j])
            assert abs(f[j].item() - terms["f"]) <= tol * abs(terms["f"]), (call, j)
            assert rel_max(mu[j].cpu().numpy(), terms["mu"]) < 1e-8, (call, j)
