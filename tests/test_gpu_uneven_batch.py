"""Parity of the uneven batch: nine univariate problems of different shapes
(ns in {256, 512, 1024} on 16x16, 16x32 and 32x32 grids, nt in {16, 32, 64})
evaluated together through bta_fobj_eval_multi, each on its own context and
stream (the independent function evaluations of Section IV-D.1, Eq. 10).

Checks per problem, against what the paper and the mathematics fix:
  * log|Q_p| against its Kronecker closed form (Eq. 2): ns log|Q_t| +
    nt log|Q_s| + a log p_beta - N log sigma^2;
  * the conditional mean through its residual with the oracle's sparse Q_c;
  * f_obj (Eq. 8) against the oracle's block tier for the nt = 16 problems;
  * in FP64, the adjoint gradient against central differences (Eq. 10) of
    the same call's f values.
Tolerances as in the full-size tests: FP64 log-det 1e-10, f 1e-9; mixed
log-det 1e-8, f 1e-8 (|log|Q_p|| + |log|Q_c||); residual 1e-10.
"""

import numpy as np
import pytest

from oracle import fobj as ofobj
from oracle import model as omodel

from gpu_util import build_lib, dev, need_gpu, problem

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

NAMES = [f"c4b_{ns}_{nt}" for ns in (256, 512, 1024) for nt in (16, 32, 64)]
H = 1e-3


def _closed_form_logdet_p(p, theta, fd):
    prm = omodel.theta_to_params(theta, p.nv)
    kappa, tau, rho, sigma = prm.kappa[0], prm.tau[0], prm.rho[0], prm.sigma[0]
    Qs = omodel.spde_precision(fd.C, fd.G, kappa, tau).toarray()
    sgn, ld_s = np.linalg.slogdet(Qs)
    assert sgn > 0
    ld_t = -(p.nt - 1) * np.log(1.0 - rho ** 2)
    return -p.N * np.log(sigma ** 2) + p.ns * ld_t + p.nt * ld_s + p.a * np.log(p.beta_prior_prec)


@pytest.fixture(scope="module")
def setup():
    need_gpu()
    build_lib()
    probs = {}
    for name in NAMES:
        p = problem(name)
        theta = p.theta0.copy()
        e = np.zeros_like(theta)
        e[1] = H                      # range_t: every shape's AR(1) coefficient moves
        thetas = np.stack([theta, theta + e, theta - e])
        probs[name] = dict(p=p, thetas=thetas, fd=omodel.fem_data(p))
    return probs


def _run_multi(setup, names, precision, with_grad):
    """One bta_fobj_eval_multi call over `names`; returns per-problem results."""
    import torch
    from paper_2507_06938_gb300 import bta
    ctxs, models, ths, fs, mus, gs, streams = [], [], [], [], [], [], []
    for name in names:
        d = setup[name]
        p = d["p"]
        st = torch.cuda.Stream()
        streams.append(st)
        models.append(bta.BtaModel(p))
        ctxs.append(bta.BtaContext(p.nt, p.b, p.a, precision, st, 1))
        ths.append(dev(d["thetas"]))
        fs.append(torch.zeros(3, dtype=torch.float64, device="cuda"))
        if with_grad:
            gs.append(torch.zeros((3, d["thetas"].shape[1]), dtype=torch.float64, device="cuda"))
        else:
            mus.append(torch.zeros((3, p.N), dtype=torch.float64, device="cuda"))
    # no synchronisation here: the thetas and zeroed outputs were queued on the
    # current stream, which every problem's stream waits for inside the call
    bta.bta_fobj_eval_multi(ctxs, models, ths, fs, mu_outs=None if with_grad else mus,
                            grad_outs=gs if with_grad else None)
    torch.cuda.current_stream().synchronize()
    out = {}
    for k, name in enumerate(names):
        ctx = ctxs[k]
        ctx.sync()
        ld = torch.zeros(1, dtype=torch.float64, device="cuda")
        ctx.logdet(bta.BTA_QP, ld)    # slot 0 holds the last theta of the call
        ctx.sync()
        out[name] = dict(f=fs[k].cpu().numpy(), ld_p_last=float(ld.item()),
                         mu=None if with_grad else mus[k].cpu().numpy(),
                         g=gs[k].cpu().numpy() if with_grad else None)
        ctx.close()
        models[k].close()
    torch.cuda.empty_cache()
    return out


def test_mixed_uneven_batch(setup):
    out = _run_multi(setup, NAMES, 1, with_grad=False)
    for name in NAMES:
        d, o = setup[name], out[name]
        p, thetas, fd = d["p"], d["thetas"], d["fd"]
        ld_ref = _closed_form_logdet_p(p, thetas[2], fd)
        assert abs(o["ld_p_last"] - ld_ref) <= 1e-8 * abs(ld_ref), (name, o["ld_p_last"], ld_ref)
        for j in (0, 2):
            built = omodel.build(p, omodel.theta_to_params(thetas[j], p.nv), fd)
            r = built.Qc @ o["mu"][j] - built.rhs
            assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(built.rhs), (name, j)
        if p.nt == 16:
            terms = ofobj.f_obj_terms(p, thetas[0], tier="bta", fd=fd)
            tol = 1e-8 * (abs(terms["logdet_p"]) + abs(terms["logdet_c"]))
            assert abs(o["f"][0] - terms["f"]) <= tol, (name, o["f"][0], terms["f"])


def test_fp64_uneven_batch_with_gradients(setup):
    names = [n for n in NAMES if n.endswith("_16")]
    out = _run_multi(setup, names, 0, with_grad=True)
    for name in names:
        d, o = setup[name], out[name]
        p, thetas, fd = d["p"], d["thetas"], d["fd"]
        ld_ref = _closed_form_logdet_p(p, thetas[2], fd)
        assert abs(o["ld_p_last"] - ld_ref) <= 1e-10 * abs(ld_ref), (name, o["ld_p_last"], ld_ref)
        terms = ofobj.f_obj_terms(p, thetas[0], tier="bta", fd=fd)
        assert abs(o["f"][0] - terms["f"]) <= 1e-9 * abs(terms["f"]), (name, o["f"][0], terms["f"])
        g = o["g"][0]
        gfd = (o["f"][1] - o["f"][2]) / (2 * H)
        scale = max(abs(g[1]), 1e-3 * np.max(np.abs(g)))
        assert abs(g[1] - gfd) <= 1e-4 * scale, (name, g[1], gfd)
        assert np.all(np.isfinite(o["g"]))   # every point of the call carries a gradient


def test_multi_rejects_mismatched_shapes(setup):
    import torch
    from paper_2507_06938_gb300 import bta
    a, b = setup["c4b_256_16"]["p"], setup["c4b_512_16"]["p"]
    ma = bta.BtaModel(a)
    cb = bta.BtaContext(b.nt, b.b, b.a, 0, None, 1)
    th = dev(setup["c4b_256_16"]["thetas"])
    f = torch.zeros(3, dtype=torch.float64, device="cuda")
    with pytest.raises(bta.BtaError) as e:
        bta.bta_fobj_eval_multi([cb], [ma], [th], [f])
    assert e.value.code == bta.BTA_ERR_ARG
    cb.close()
    ma.close()
