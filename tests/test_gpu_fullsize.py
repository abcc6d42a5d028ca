"""Parity at the working size of the throughput measurement: the univariate
AR(1) x SPDE model on the 32 x 32 grid mesh with nt = 64 time steps
(b = 1024, a = 4, N = 65,540, m = 65,536), in the launch configuration the
benchmark times: the 9 theta points of a central-difference stencil (Eq. 10),
all 18 BTA matrices through the same launches, FP64 and mixed precision.

The dense oracle tier cannot run at this size, so the checks use what holds
at any size, plus the oracle's block tier where it finishes in seconds:
  * log|Q_p| against its closed form: Q_p = sigma^-2 blockdiag(Q_t (x) Q_s,
    p_beta I), so log|Q_p| = -N log sigma^2 + ns log|Q_t| + nt log|Q_s| +
    a log p_beta with log|Q_t| = -(nt - 1) log(1 - rho^2);
  * sampled blocks of Sigma_p = Q_p^{-1} against the closed-form covariance
    sigma^2 rho^|t-t'| Q_s^{-1} (AR(1) correlation times the spatial
    covariance), zero arrow and sigma^2 / p_beta on the tip;
  * the conditional mean through its residual ||Q_c mu - A^T D y|| / ||A^T D y||
    with the oracle's sparse FP64 Q_c;
  * f_obj at the stencil centre against the oracle's block tier;
  * sampled columns of Sigma_c = Q_c^{-1} (oracle block-tier solves with unit
    vectors) against the selected-inverse blocks on the BTA pattern;
  * the adjoint gradient against central differences of the FP64 f values of
    the same stencil, and the mixed gradient against the FP64 one.
Tolerances: FP64 as in the small-size parity tests (log-det 1e-10, Sigma
1e-9, residual 1e-10, f 1e-9); mixed precision at its targets (log-det 1e-8,
residual 1e-10, Sigma 5e-5 of the block maximum, gradient 1e-5 of the FP64
gradient).  The central difference with h = 1e-3 carries a truncation error
of order h^2 f''' / 6, so it is held to 1e-4.
"""

import numpy as np
import pytest

from oracle import bta as obta
from oracle import fobj as ofobj
from oracle import model as omodel

from gpu_util import build_lib, dev, need_gpu, problem

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

H = 1e-3


@pytest.fixture(scope="module")
def setup():
    need_gpu()
    build_lib()
    p = problem("c2")
    theta = p.theta0.copy()
    pts = [theta]
    for i in range(theta.shape[0]):
        e = np.zeros_like(theta)
        e[i] = H
        pts += [theta + e, theta - e]
    thetas = np.stack(pts)
    fd = omodel.fem_data(p)
    terms = ofobj.f_obj_terms(p, theta, tier="bta", fd=fd)
    built = terms["built"]
    Lc = obta.factor(obta.blocks_from_sparse(built.Qc, p.nt, p.b, p.a))
    rng = np.random.default_rng(7)
    cols = sorted({0, p.b - 1, 31 * p.b + int(rng.integers(p.b)), 63 * p.b + int(rng.integers(p.b)),
                   p.nt * p.b + 1})
    sigma_cols = {}
    for j in cols:
        e = np.zeros(p.N)
        e[j] = 1.0
        sigma_cols[j] = obta.solve(Lc, e)
    return dict(p=p, thetas=thetas, fd=fd, terms=terms, sigma_cols=sigma_cols, results={})


def _run(setup, precision):
    import torch
    from paper_2507_06938_gb300 import bta
    if precision in setup["results"]:
        return setup["results"][precision]
    p, thetas = setup["p"], setup["thetas"]
    B = thetas.shape[0]
    model = bta.BtaModel(p)
    ctx = bta.BtaContext(p.nt, p.b, p.a, precision, None, B)
    th = dev(thetas)
    f = torch.zeros(B, dtype=torch.float64, device="cuda")
    mu = torch.zeros((B, p.N), dtype=torch.float64, device="cuda")
    ctx.fobj_eval(model, th, f, mu)
    ctx.sync()
    out = dict(f_eval=f.cpu().numpy(), mu=mu.cpu().numpy())
    del mu
    f2 = torch.zeros(B, dtype=torch.float64, device="cuda")
    g = torch.zeros((B, thetas.shape[1]), dtype=torch.float64, device="cuda")
    ctx.fobj_grad(model, th, f2, g)
    ld = torch.zeros(B, dtype=torch.float64, device="cuda")
    for j in range(B):
        ctx.logdet(2 * j + bta.BTA_QP, ld[j:j + 1])
    ctx.sync()
    out.update(f=f2.cpu().numpy(), g=g.cpu().numpy(), ld_p=ld.cpu().numpy())
    # sampled blocks of Sigma_p (slots 0 and 8) and the pattern entries of the
    # sampled columns of Sigma_c (slot 0)
    S = bta.BTA_STORE_SIGMA
    sp_blocks = {}
    for j in (0, B - 1):
        which = 2 * j + bta.BTA_QP
        for i in (0, 1, 31, p.nt - 1):
            sp_blocks[(j, "D", i)] = ctx.block(which, S, bta.BTA_BLK_D, i).cpu().numpy()
        for i in (0, 31, p.nt - 2):
            sp_blocks[(j, "B", i)] = ctx.block(which, S, bta.BTA_BLK_B, i).cpu().numpy()
        sp_blocks[(j, "R")] = np.stack([ctx.block(which, S, bta.BTA_BLK_R, i).cpu().numpy() for i in range(p.nt)])
        sp_blocks[(j, "T")] = ctx.block(which, S, bta.BTA_BLK_T).cpu().numpy()
    out["sp"] = sp_blocks
    qc = bta.BTA_QC
    b, n = p.b, p.nt
    sc = {}
    for col in setup["sigma_cols"]:
        ent = {}
        if col < n * b:
            t, l = divmod(col, b)
            ent["D"] = ctx.block(qc, S, bta.BTA_BLK_D, t).cpu().numpy()[:, l]
            if t < n - 1:
                ent["B+"] = ctx.block(qc, S, bta.BTA_BLK_B, t).cpu().numpy()[:, l]
            if t > 0:
                ent["B-"] = ctx.block(qc, S, bta.BTA_BLK_B, t - 1).cpu().numpy()[l, :]
            ent["R"] = ctx.block(qc, S, bta.BTA_BLK_R, t).cpu().numpy()[:, l]
        else:
            r = col - n * b
            ent["R"] = np.concatenate([ctx.block(qc, S, bta.BTA_BLK_R, i).cpu().numpy()[r, :] for i in range(n)])
            ent["T"] = ctx.block(qc, S, bta.BTA_BLK_T).cpu().numpy()[:, r]
        sc[col] = ent
    out["sc"] = sc
    ctx.close()
    model.close()
    torch.cuda.empty_cache()
    setup["results"][precision] = out
    return out


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _closed_form(p, theta, fd):
    prm = omodel.theta_to_params(theta, p.nv)
    kappa, tau, rho, sigma = prm.kappa[0], prm.tau[0], prm.rho[0], prm.sigma[0]
    Qs = omodel.spde_precision(fd.C, fd.G, kappa, tau).toarray()
    sgn, ld_s = np.linalg.slogdet(Qs)
    assert sgn > 0
    ld_t = -(p.nt - 1) * np.log(1.0 - rho ** 2)
    ld_p = -p.N * np.log(sigma ** 2) + p.ns * ld_t + p.nt * ld_s + p.a * np.log(p.beta_prior_prec)
    Cs = np.linalg.inv(Qs)
    return ld_p, Cs, rho, sigma


@pytest.mark.parametrize("precision", [0, 1])
def test_prior_logdet_and_covariance_closed_form(setup, precision):
    p, thetas, fd = setup["p"], setup["thetas"], setup["fd"]
    out = _run(setup, precision)
    ld_tol = 1e-10 if precision == 0 else 1e-8
    s_tol = 1e-9 if precision == 0 else 5e-5
    for j in range(thetas.shape[0]):
        ld_ref = _closed_form(p, thetas[j], fd)[0]
        assert abs(out["ld_p"][j] - ld_ref) <= ld_tol * abs(ld_ref), (j, out["ld_p"][j], ld_ref)
    for j in (0, thetas.shape[0] - 1):
        _, Cs, rho, sigma = _closed_form(p, thetas[j], fd)
        for (jj, kind, *idx), blk in out["sp"].items():
            if jj != j:
                continue
            if kind == "D":
                assert _rel(blk, sigma ** 2 * Cs) < s_tol, (j, kind, idx)
            elif kind == "B":
                assert _rel(blk, sigma ** 2 * rho * Cs) < s_tol, (j, kind, idx)
            elif kind == "R":
                assert np.max(np.abs(blk)) <= s_tol * sigma ** 2 * np.max(np.abs(Cs)), (j, kind)
            else:
                assert _rel(blk, sigma ** 2 / p.beta_prior_prec * np.eye(p.a)) < s_tol, (j, kind)


@pytest.mark.parametrize("precision", [0, 1])
def test_conditional_mean_residual_and_fobj(setup, precision):
    p, thetas, fd, terms = setup["p"], setup["thetas"], setup["fd"], setup["terms"]
    out = _run(setup, precision)
    for j in (0, 3, thetas.shape[0] - 1):
        built = omodel.build(p, omodel.theta_to_params(thetas[j], p.nv), fd)
        r = built.Qc @ out["mu"][j] - built.rhs
        assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(built.rhs), j
    ref = terms["f"]
    if precision == 0:
        tol = 1e-9 * abs(ref)
    else:
        tol = 1e-8 * (abs(terms["logdet_p"]) + abs(terms["logdet_c"]))
    assert abs(out["f_eval"][0] - ref) <= tol, (out["f_eval"][0], ref)
    assert abs(out["f"][0] - ref) <= tol, (out["f"][0], ref)
    # the gradient call evaluates f at the same points
    assert np.max(np.abs(out["f"] - out["f_eval"])) <= tol


@pytest.mark.parametrize("precision", [0, 1])
def test_conditional_selected_inverse_columns(setup, precision):
    p = setup["p"]
    out = _run(setup, precision)
    tol = 1e-9 if precision == 0 else 5e-5
    b, n = p.b, p.nt
    for col, x in setup["sigma_cols"].items():
        got = out["sc"][col]
        if col < n * b:
            t = col // b
            assert _rel(got["D"], x[t * b:(t + 1) * b]) < tol, (col, "D")
            if "B+" in got:
                assert _rel(got["B+"], x[(t + 1) * b:(t + 2) * b]) < tol, (col, "B+")
            if "B-" in got:
                assert _rel(got["B-"], x[(t - 1) * b:t * b]) < tol, (col, "B-")
            assert _rel(got["R"], x[n * b:]) < tol, (col, "R")
        else:
            assert _rel(got["R"], x[:n * b]) < tol, (col, "R")
            assert _rel(got["T"], x[n * b:]) < tol, (col, "T")


def test_adjoint_gradient_at_full_size(setup):
    out64 = _run(setup, 0)
    outmx = _run(setup, 1)
    f, g = out64["f"], out64["g"]
    dim = g.shape[1]
    gfd = np.array([(f[2 * k + 1] - f[2 * k + 2]) / (2 * H) for k in range(dim)])
    scale = np.maximum(np.abs(g[0]), 1e-3 * np.max(np.abs(g[0])))
    assert np.max(np.abs(g[0] - gfd) / scale) < 1e-4, (g[0], gfd)
    assert np.max(np.abs(outmx["g"] - g) / scale) < 1e-5, (outmx["g"][0], g[0])
