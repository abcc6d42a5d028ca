"""Low-memory layout (bta_set_low_memory): the inverse diagonal factor blocks
replace L_ii in the factor's diagonal slots, the log-determinant is summed
while the blocks are factored, and the selected inverse overwrites the
factor.  The arithmetic is that of the default layout, so every output is
checked against the oracle (block tier, pinned to the dense tier) at the
bounds of the precision: log-det 1e-10, solve and L_ii^{-1} 1e-9, every
selected-inverse block 1e-9 (FP64) or 1e-8 (49-bit), f and the adjoint
gradient as in the batched tests.  Also: a selected inversion consumes the
factor (a later solve is refused until the next factorisation), switching
layouts keeps the assembled matrices, and time partitions are refused."""

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


@pytest.mark.parametrize("name,precision", [("t_coreg3", 0), ("t_uni_mid", 0), ("t_coreg3_mid", 2)])
def test_factor_logdet_solve_selinv(name, precision, monkeypatch):
    import torch
    from paper_2507_06938_gb300 import bta
    monkeypatch.setenv("BTA_OZ_MIN", "64")
    p = problem(name)
    prm = omodel.theta_to_params(p.theta0, p.nv)
    built = omodel.build(p, prm)
    run = GpuCase(p, precision=precision)
    run.ctx.set_low_memory(True)
    stol = 1e-9 if precision == 0 else 1e-8
    rng = np.random.default_rng(5)
    for which, Q in ((bta.BTA_QP, built.Qp), (bta.BTA_QC, built.Qc)):
        Lo = obta.factor(obta.blocks_from_sparse(Q, p.nt, p.b, p.a))
        run.assemble(prm, which)
        run.ctx.factor(which)
        ld = torch.zeros(1, dtype=torch.float64, device="cuda")
        run.ctx.logdet(which, ld)
        r = rng.standard_normal(p.N)
        x = torch.zeros(p.N, dtype=torch.float64, device="cuda")
        run.ctx.solve(which, dev(r), x, 0, None)
        run.ctx.sync()
        ref = obta.logdet(Lo)
        assert abs(ld.item() - ref) <= 1e-10 * abs(ref), (which, ld.item(), ref)
        assert rel_max(x.cpu().numpy(), obta.solve(Lo, r)) <= 1e-9
        # the factor's diagonal slots hold L_ii^{-1}
        for i in (0, p.nt - 1):
            Xi = run.ctx.block(which, bta.BTA_STORE_LINV, bta.BTA_BLK_D, i).cpu().numpy()
            Xo = np.linalg.inv(Lo["D"][i])
            assert rel_max(np.tril(Xi), Xo) <= 1e-9, i
        run.ctx.selinv(which)
        run.ctx.sync()
        S = blocks_of(run.ctx, which, bta.BTA_STORE_SIGMA, p.nt, p.b, p.a)
        So = obta.selinv(Lo)
        for k in ("D", "B", "R", "T"):
            if So[k].size:
                e = max(rel_max(S[k][i], So[k][i]) for i in range(So[k].shape[0])) if k != "T" \
                    else rel_max(S[k], So[k])
                assert e <= stol, (which, k, e)
        # the selected inverse has replaced the factor
        with pytest.raises(bta.BtaError) as err:
            run.ctx.solve(which, dev(r), x, 0, None)
        assert err.value.code == bta.BTA_ERR_STATE
        run.ctx.factor(which)
        run.ctx.solve(which, dev(r), x, 0, None)
        run.ctx.sync()
        assert rel_max(x.cpu().numpy(), obta.solve(Lo, r)) <= 1e-9


@pytest.mark.parametrize("name,precision", [("t_coreg3_mid", 0), ("t_coreg3_mid", 2)])
def test_fobj_gradient_batch(name, precision, monkeypatch):
    import torch
    monkeypatch.setenv("BTA_OZ_MIN", "64")
    from paper_2507_06938_gb300 import bta
    p = problem(name)
    run = GpuCase(p, precision=precision, batch=2)
    if precision == 0:
        run.ctx.set_low_memory(True)
    else:
        # created in the low-memory layout
        run.ctx.close()
        run.ctx = bta.BtaContext(p.nt, p.b, p.a, precision, None, 2, low_memory=True)
    thetas = np.stack([p.theta0, p.theta0 + 0.03])
    f = torch.zeros(2, dtype=torch.float64, device="cuda")
    g = torch.zeros((2, p.theta0.shape[0]), dtype=torch.float64, device="cuda")
    for _ in range(3):                  # direct, graph capture, graph replay
        run.ctx.fobj_grad(run.model, dev(thetas), f, g)
    run.ctx.sync()
    for j in range(2):
        terms = ofobj.f_obj_terms(p, thetas[j])
        tol = 1e-9 * (abs(terms["logdet_p"]) + abs(terms["logdet_c"]))
        assert abs(f[j].item() - terms["f"]) <= tol
        gref = ofobj.grad_adjoint(p, thetas[j], tier="bta")
        scale = np.maximum(np.abs(gref), 1e-3 * np.max(np.abs(gref)))
        assert np.max(np.abs(g[j].cpu().numpy() - gref) / scale) <= 1e-7


def test_switching_keeps_assembled_matrices():
    import torch
    from paper_2507_06938_gb300 import bta
    p = problem("t_uni_mid")
    prm = omodel.theta_to_params(p.theta0, p.nv)
    built = omodel.build(p, prm)
    ref = obta.logdet(obta.factor(obta.blocks_from_sparse(built.Qc, p.nt, p.b, p.a)))
    run = GpuCase(p, precision=0)
    run.assemble(prm, bta.BTA_QC)
    ld = torch.zeros(1, dtype=torch.float64, device="cuda")
    for low in (True, False, True):
        run.ctx.set_low_memory(low)
        run.ctx.factor(bta.BTA_QC)
        run.ctx.logdet(bta.BTA_QC, ld)
        run.ctx.sync()
        assert abs(ld.item() - ref) <= 1e-10 * abs(ref), low
    with pytest.raises(bta.BtaError) as err:
        run.ctx.set_time_partitions(2)
    assert err.value.code == bta.BTA_ERR_STATE
    run.ctx.set_low_memory(False)
    run.ctx.set_time_partitions(2)
    with pytest.raises(bta.BtaError) as err:
        run.ctx.set_low_memory(True)
    assert err.value.code == bta.BTA_ERR_STATE


def test_laplace_in_the_low_memory_layout():
    """The Newton iterations of the non-Gaussian path factor, take log-dets and
    solve many times without a selected inversion: the low-memory layout gives
    the same f and mode as the default one."""
    import torch
    from paper_2507_06938_gb300 import bta
    p = problem("t_pois")
    thetas = dev(np.stack([p.theta0, p.theta0 + 0.05]))
    out = []
    for low in (False, True):
        model = bta.BtaModel(p)
        ctx = bta.BtaContext(p.nt, p.b, p.a, 0, None, 2, low_memory=low)
        f = torch.zeros(2, dtype=torch.float64, device="cuda")
        x = torch.zeros((2, p.N), dtype=torch.float64, device="cuda")
        step = torch.zeros(2, dtype=torch.float64, device="cuda")
        ctx.fobj_laplace(model, thetas, bta.BTA_LIK_POISSON, 12, f, x, step)
        ctx.sync()
        out.append((f.cpu().numpy(), x.cpu().numpy()))
        ctx.close()
        model.close()
    assert np.max(np.abs(out[0][0] - out[1][0])) <= 1e-11 * np.max(np.abs(out[0][0]))
    assert rel_max(out[1][1], out[0][1]) <= 1e-11


def test_partial_group_and_host_buffers():
    """Three theta points through a two-slot context (a full group, then a
    partial one) and the host-buffer entry, in the low-memory layout: the
    same f, gradient and marginal variances as the default layout."""
    import torch
    from paper_2507_06938_gb300 import bta
    p = problem("t_coreg3")
    dim = p.theta0.shape[0]
    th = np.stack([p.theta0, p.theta0 + 0.02, p.theta0 - 0.02])
    res = []
    for low in (False, True):
        model = bta.BtaModel(p)
        ctx = bta.BtaContext(p.nt, p.b, p.a, 0, None, 2, low_memory=low)
        f = torch.zeros(3, dtype=torch.float64, device="cuda")
        g = torch.zeros((3, dim), dtype=torch.float64, device="cuda")
        ctx.fobj_grad(model, dev(th), f, g)
        ctx.sync()
        fh = torch.zeros(2, dtype=torch.float64).pin_memory()
        gh = torch.zeros((2, dim), dtype=torch.float64).pin_memory()
        vh = torch.zeros((2, p.N), dtype=torch.float64).pin_memory()
        ctx.fobj_grad_host(model, torch.tensor(th[:2]).pin_memory(), fh, gh, vh)
        res.append((f.cpu().numpy(), g.cpu().numpy(), fh.numpy().copy(), gh.numpy().copy(), vh.numpy().copy()))
        ctx.close()
        model.close()
    for a, b in zip(res[0], res[1]):
        assert rel_max(b, a) <= 1e-11
