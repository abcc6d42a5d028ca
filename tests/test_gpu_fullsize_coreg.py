"""Parity at the size of the trivariate coregional workload: nv = 3 fields
on the 32 x 32 grid mesh, nt = 48, b = 3072, a = 6, N = 147,462, with
300 shared sites per time step (Eqs. 5, 11).

The oracle's block tier needs minutes of CPU time at this size, so the
checks use what holds exactly at any size:
  * log|Q_p| against its closed form: Q_p = Lambda^-T blockdiag(Q^u)
    Lambda^-1 with unit-triangular M, so log|Q_p| = sum_u [ns log|Q_t^u| +
    nt log|Q_s^u| + nr log p_beta - (ns nt + nr) log sigma_u^2];
  * sampled blocks of Sigma_p against the closed-form covariance
    Sigma_{(t,v),(t',v')} = sum_u Lambda_vu Lambda_v'u rho_u^|t-t'| Q_{s,u}^-1
    (Eq. 6 with the AR(1) correlation);
  * the conditional mean through its residual with the oracle's sparse Q_c;
  * the selected inverse of Q_c through the diagonal blocks of Sigma_c Q_c = I,
    which involve only entries of Sigma_c on the BTA pattern:
    (Sigma Q)_ii = Sigma_{i,i-1} Q_{i-1,i} + Sigma_ii Q_ii + Sigma_{i,i+1} Q_{i+1,i}
    + Sigma_{i,t} Q_{t,i}, and the tip block likewise.
  * f against the oracle's block tier (the block recurrences on the CPU,
    pinned to the dense tier at small sizes), computed once per module.
Tolerances as for the working-size univariate test: FP64 log-det 1e-10,
Sigma 1e-9, residual 1e-10, f 1e-10 of |log|Q_p|| + |log|Q_c||; mixed
precision log-det 1e-8, residual 1e-10, Sigma 5e-5 of the block maximum,
f 1e-8 of the log-determinant scale.
"""

import time

import numpy as np
import pytest

from oracle import model as omodel

from gpu_util import dev, need_gpu, problem

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def setup():
    need_gpu()
    from paper_2507_06938_gb300 import _build
    _build.build()
    p = problem("c3")
    fd = omodel.fem_data(p)
    from oracle import fobj as ofobj
    terms = ofobj.f_obj_terms(p, p.theta0, tier="bta", fd=fd)
    return dict(p=p, fd=fd, theta=p.theta0.copy(), f=terms["f"],
                ld_scale=abs(terms["logdet_p"]) + abs(terms["logdet_c"]))


def _closed_form(p, theta, fd):
    prm = omodel.theta_to_params(theta, p.nv)
    ld = 0.0
    Cs = []
    for u in range(p.nv):
        Qs = omodel.spde_precision(fd.C, fd.G, prm.kappa[u], prm.tau[u]).toarray()
        sgn, ld_s = np.linalg.slogdet(Qs)
        assert sgn > 0
        ld_t = -(p.nt - 1) * np.log(1.0 - prm.rho[u] ** 2)
        ld += (p.ns * ld_t + p.nt * ld_s + p.nr * np.log(p.beta_prior_prec)
               - (p.ns * p.nt + p.nr) * np.log(prm.sigma[u] ** 2))
        Cs.append(np.linalg.inv(Qs))
    Lam = omodel.mixing_matrix(prm)
    return ld, Cs, Lam, prm.rho


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


@pytest.mark.parametrize("precision", [0, 1])
def test_coregional_full_size(setup, precision):
    import torch
    from paper_2507_06938_gb300 import bta
    p, fd, theta = setup["p"], setup["fd"], setup["theta"]
    n, b, a, ns, nv = p.nt, p.b, p.a, p.ns, p.nv
    model = bta.BtaModel(p)
    ctx = bta.BtaContext(n, b, a, precision, None, 1)
    th = dev(theta[None, :])
    f = torch.zeros(1, dtype=torch.float64, device="cuda")
    mu = torch.zeros((1, p.N), dtype=torch.float64, device="cuda")
    ctx.fobj_eval(model, th, f, mu)
    ctx.sync()
    g = torch.zeros((1, theta.shape[0]), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ctx.fobj_grad(model, th, f, g)
    ctx.sync()
    dt = time.perf_counter() - t0
    print(f"\nc3 fobj+gradient+selinv of Q_p and Q_c, precision {precision}: {dt:.2f} s")
    ld = torch.zeros(1, dtype=torch.float64, device="cuda")
    ctx.logdet(bta.BTA_QP, ld)
    ctx.sync()
    ld_ref, Cs, Lam, rho = _closed_form(p, theta, fd)
    ld_tol = 1e-10 if precision == 0 else 1e-8
    s_tol = 1e-9 if precision == 0 else 5e-5
    assert abs(ld.item() - ld_ref) <= ld_tol * abs(ld_ref), (ld.item(), ld_ref)
    assert abs(f.item() - setup["f"]) <= ld_tol * setup["ld_scale"], (f.item(), setup["f"])
    # Sigma_p: diagonal and sub-diagonal blocks at a few time steps
    S = bta.BTA_STORE_SIGMA

    def sig_block(dt_):
        out = np.zeros((b, b))
        for v in range(nv):
            for w in range(nv):
                out[v * ns:(v + 1) * ns, w * ns:(w + 1) * ns] = sum(
                    Lam[v, u] * Lam[w, u] * rho[u] ** dt_ * Cs[u] for u in range(nv))
        return out

    D_ref, B_ref = sig_block(0), sig_block(1)
    for i in (0, n // 2, n - 1):
        assert _rel(ctx.block(bta.BTA_QP, S, bta.BTA_BLK_D, i).cpu().numpy(), D_ref) < s_tol, i
    for i in (0, n - 2):
        assert _rel(ctx.block(bta.BTA_QP, S, bta.BTA_BLK_B, i).cpu().numpy(), B_ref) < s_tol, i
    # conditional mean residual with the oracle's sparse Q_c
    built = omodel.build(p, omodel.theta_to_params(theta, p.nv), fd)
    r = built.Qc @ mu[0].cpu().numpy() - built.rhs
    assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(built.rhs)
    # diagonal blocks of Sigma_c Q_c = I (Q_c from the oracle's build, in BTA order)
    Qc = built.Qc.tocsr()
    qc = bta.BTA_QC

    def Qblk(r0, r1, c0, c1):
        return Qc[r0:r1, c0:c1].toarray()

    tip = slice(n * b, n * b + a)
    for i in (0, n // 2, n - 1):
        rows = slice(i * b, (i + 1) * b)
        acc = ctx.block(qc, S, bta.BTA_BLK_D, i).cpu().numpy() @ Qblk(rows.start, rows.stop, rows.start, rows.stop)
        if i > 0:
            Sig_i_im1 = ctx.block(qc, S, bta.BTA_BLK_B, i - 1).cpu().numpy()          # Sigma_{i,i-1}
            acc += Sig_i_im1 @ Qblk((i - 1) * b, i * b, rows.start, rows.stop)
        if i < n - 1:
            Sig_ip1_i = ctx.block(qc, S, bta.BTA_BLK_B, i).cpu().numpy()              # Sigma_{i+1,i}
            acc += Sig_ip1_i.T @ Qblk((i + 1) * b, (i + 2) * b, rows.start, rows.stop)
        Sig_t_i = ctx.block(qc, S, bta.BTA_BLK_R, i).cpu().numpy()                    # Sigma_{t,i}
        acc += Sig_t_i.T @ Qblk(tip.start, tip.stop, rows.start, rows.stop)
        # relative to the size of the summands: |Sigma| |Q| b
        scale = np.max(np.abs(ctx.block(qc, S, bta.BTA_BLK_D, i).cpu().numpy())) * abs(Qc).max() * 40
        err = np.max(np.abs(acc - np.eye(b)))
        assert err <= (1e-9 if precision == 0 else 5e-5) * max(scale, 1.0), (i, err, scale)
    accT = ctx.block(qc, S, bta.BTA_BLK_T).cpu().numpy() @ Qblk(tip.start, tip.stop, tip.start, tip.stop)
    for i in range(n):
        accT += ctx.block(qc, S, bta.BTA_BLK_R, i).cpu().numpy() @ Qblk(i * b, (i + 1) * b, tip.start, tip.stop)
    assert np.max(np.abs(accT - np.eye(a))) <= (1e-9 if precision == 0 else 5e-5) * 1e3
    ctx.close()
    model.close()
    torch.cuda.empty_cache()
