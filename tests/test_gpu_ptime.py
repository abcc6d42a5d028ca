"""Parallel-in-time BTA factorisation, solve and selected inversion on one
GPU (bta_set_time_partitions; the time-domain partitioning of Sections IV-C
and IV-D.3 run as one batch): P - 1 separator blocks cut the time blocks into
P partitions whose interiors are eliminated together, then the separators
form a reduced BTA system.  The results are the same quantities as the
sequential recurrences compute, so they are checked against the oracle
(block tier, pinned to the dense tier) at the FP64 bounds: log-det 1e-10,
every selected-inverse block 1e-9 of its maximum, the solve against a
dense solve 1e-9; and f and the adjoint gradient through bta_fobj_grad.
Partition counts cover a full last partition, a last partition padded with
identity blocks, interiors of one block and the largest P allowed; the
49-bit mixed path with the tensor-core products at the mixed bounds.  The
relayout keeps assembled matrices, and a failed pivot names its matrix."""

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


# (n, P): h = ceil((n + 1) / P) blocks per partition (its separator included),
# the last partition n - (P - 1) h >= 1 interior blocks
CASES = [("t_uni_ragged", 2), ("t_uni_ragged", 3), ("t_uni_ragged", 4), ("t_coreg3", 2), ("t_coreg3", 3),
         ("t_uni_mid", 2), ("t_uni_mid", 3), ("t_coreg3_mid", 3), ("t_coreg3_mid", 4)]


@pytest.mark.parametrize("name,P", CASES)
def test_partitioned_factor_solve_selinv(name, P):
    import torch
    from paper_2507_06938_gb300 import bta
    p = problem(name)
    prm = omodel.theta_to_params(p.theta0, p.nv)
    built = omodel.build(p, prm)
    run = GpuCase(p, precision=bta.BTA_FP64)
    run.ctx.set_time_partitions(P)
    rng = np.random.default_rng(P)
    for which, Q in ((bta.BTA_QP, built.Qp), (bta.BTA_QC, built.Qc)):
        Lo = obta.factor(obta.blocks_from_sparse(Q, p.nt, p.b, p.a))
        run.assemble(prm, which)
        run.ctx.factor(which)
        ld = torch.zeros(1, dtype=torch.float64, device="cuda")
        run.ctx.logdet(which, ld)
        r = rng.standard_normal(p.N)
        x = torch.zeros(p.N, dtype=torch.float64, device="cuda")
        run.ctx.solve(which, dev(r), x, 0, None)
        run.ctx.selinv(which)
        run.ctx.sync()
        ref = obta.logdet(Lo)
        assert abs(ld.item() - ref) <= 1e-10 * abs(ref), (which, ld.item(), ref)
        xr = obta.solve(Lo, r)
        assert rel_max(x.cpu().numpy(), xr) <= 1e-9
        S = blocks_of(run.ctx, which, bta.BTA_STORE_SIGMA, p.nt, p.b, p.a)
        So = obta.selinv(Lo)
        for k in ("D", "B", "R", "T"):
            if So[k].size:
                e = max(rel_max(S[k][i], So[k][i]) for i in range(So[k].shape[0])) if k != "T" \
                    else rel_max(S[k], So[k])
                assert e <= 1e-9, (which, k, e)


@pytest.mark.parametrize("name,P,precision", [("t_coreg3", 2, 0), ("t_uni_mid", 3, 0), ("t_coreg3_mid", 3, 2),
                                              ("t_coreg3_mid", 4, 1)])
def test_partitioned_fobj_and_gradient(name, P, precision, monkeypatch):
    import torch
    from paper_2507_06938_gb300 import bta
    monkeypatch.setenv("BTA_OZ_MIN", "64")
    p = problem(name)
    run = GpuCase(p, precision=precision, batch=2)
    run.ctx.set_time_partitions(P)
    thetas = np.stack([p.theta0, p.theta0 + 0.03])
    f = torch.zeros(2, dtype=torch.float64, device="cuda")
    g = torch.zeros((2, p.theta0.shape[0]), dtype=torch.float64, device="cuda")
    run.ctx.fobj_grad(run.model, dev(thetas), f, g)
    run.ctx.sync()
    for j in range(2):
        terms = ofobj.f_obj_terms(p, thetas[j])
        tol = 1e-9 * (abs(terms["logdet_p"]) + abs(terms["logdet_c"]))
        assert abs(f[j].item() - terms["f"]) <= tol
        gref = ofobj.grad_adjoint(p, thetas[j], tier="bta")
        scale = np.maximum(np.abs(gref), 1e-3 * np.max(np.abs(gref)))
        assert np.max(np.abs(g[j].cpu().numpy() - gref) / scale) <= 1e-7


def test_partition_count_limits():
    from paper_2507_06938_gb300 import bta
    p = problem("t_uni")          # n = 5: P = 2 (h = 3) and P = 3 (h = 2); P = 4 leaves no last interior
    run = GpuCase(p, precision=0)
    for P in (0, 4, 6):
        with pytest.raises(bta.BtaError) as e:
            run.ctx.set_time_partitions(P)
        assert e.value.code == bta.BTA_ERR_ARG
    run.ctx.set_time_partitions(3)
    run.ctx.set_time_partitions(1)
    # the inverse tip factor sits in one block slot: a > b is refused
    ctx = bta.BtaContext(6, 2, 3, 0, None, 1)
    with pytest.raises(bta.BtaError) as e:
        ctx.set_time_partitions(2)
    assert e.value.code == bta.BTA_ERR_ARG
    ctx.close()


def test_relayout_keeps_assembled_matrices():
    import torch
    from paper_2507_06938_gb300 import bta
    p = problem("t_coreg3_mid")
    prm = omodel.theta_to_params(p.theta0, p.nv)
    built = omodel.build(p, prm)
    run = GpuCase(p, precision=0)
    run.assemble(prm, bta.BTA_QC)
    ref = obta.logdet(obta.factor(obta.blocks_from_sparse(built.Qc, p.nt, p.b, p.a)))
    ld = torch.zeros(1, dtype=torch.float64, device="cuda")
    for P in (3, 4, 1, 2):
        run.ctx.set_time_partitions(P)
        run.ctx.factor(bta.BTA_QC)
        run.ctx.logdet(bta.BTA_QC, ld)
        run.ctx.sync()
        assert abs(ld.item() - ref) <= 1e-10 * abs(ref), P
        Q = blocks_of(run.ctx, bta.BTA_QC, bta.BTA_STORE_Q, p.nt, p.b, p.a)
        Qo = obta.blocks_from_sparse(built.Qc, p.nt, p.b, p.a)
        for k in ("D", "B", "R", "T"):
            assert rel_max(Q[k], Qo[k]) <= 1e-14, (P, k)


def test_partitioned_error_names_the_matrix():
    import torch
    from paper_2507_06938_gb300 import bta
    p = problem("t_uni_mid")      # n = 12, P = 3: h = 5, partition 1 holds blocks 5..8
    run = GpuCase(p, batch=3)
    run.ctx.set_time_partitions(3)
    prm = omodel.theta_to_params(p.theta0, p.nv)
    params = dev(omodel.params_vector(prm))
    for j in range(3):
        run.ctx.assemble(run.model, params, 2 * j + bta.BTA_QC)
    run.ctx.sync()
    D = run.ctx.block(2 * 1 + bta.BTA_QC, bta.BTA_STORE_Q, bta.BTA_BLK_D, 6)
    D[3, 3] = -1e6
    torch.cuda.synchronize()
    run.ctx.factor_batch(bta.BTA_QC)
    with pytest.raises(bta.BtaError) as e:
        run.ctx.sync()
    assert e.value.code == bta.BTA_ERR_NOT_PD
    assert e.value.info == 1 * p.b + 3        # block 6 is the second interior block of its partition
    assert e.value.matrix == 2 * 1 + bta.BTA_QC
