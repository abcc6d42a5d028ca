"""The 31-point central-difference stencil of the trivariate coregional model
(Eq. 10 with dim(theta) = 15) at the c3 size (b = 3072, nt = 48,
N = 147,462), i.e. 62 BTA matrices, evaluated by fobj_eval in groups of the
context's batch (4 points, 8 matrices per group; the last group is
partial), in mixed precision.

Checks:
  * grouping is exact: f at points of the first, a middle and the last
    (partial) group equals a separate single-point evaluation to 1e-10
    relative (launch shapes that depend on the batch may change summation
    orders; a wrong point-to-slot mapping changes f by far more);
  * log|Q_p| of every point of the last group against its closed form
    (Eqs. 2, 5, 11): sum_u [ns log|Q_t^u| + nt log|Q_s^u| + nr log p_beta
    - (ns nt + nr) log sigma_u^2], to the mixed-precision bound 1e-8;
  * all 31 values finite.
The single-point path at this size is pinned further by the full-size
coregional test (closed-form Sigma_p, residual, Sigma_c Q_c = I).
"""

import numpy as np
import pytest

from oracle import model as omodel

from gpu_util import build_lib, dev, need_gpu, problem

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

H = 1e-3
GROUP = 4


def _closed_form_logdet_p(p, theta, fd):
    prm = omodel.theta_to_params(theta, p.nv)
    ld = 0.0
    for u in range(p.nv):
        Qs = omodel.spde_precision(fd.C, fd.G, prm.kappa[u], prm.tau[u]).toarray()
        sgn, ld_s = np.linalg.slogdet(Qs)
        assert sgn > 0
        ld_t = -(p.nt - 1) * np.log(1.0 - prm.rho[u] ** 2)
        ld += (p.ns * ld_t + p.nt * ld_s + p.nr * np.log(p.beta_prior_prec)
               - (p.ns * p.nt + p.nr) * np.log(prm.sigma[u] ** 2))
    return ld


def test_coregional_stencil_in_groups():
    need_gpu()
    build_lib()
    import torch
    from paper_2507_06938_gb300 import bta
    p = problem("c3")
    fd = omodel.fem_data(p)
    theta = p.theta0.copy()
    dim = theta.shape[0]
    assert dim == 15
    pts = [theta]
    for k in range(dim):
        e = np.zeros_like(theta)
        e[k] = H
        pts += [theta + e, theta - e]
    thetas = np.stack(pts)
    n_pts = thetas.shape[0]
    model = bta.BtaModel(p)
    ctx = bta.BtaContext(p.nt, p.b, p.a, bta.BTA_MIXED, None, GROUP)
    f = torch.zeros(n_pts, dtype=torch.float64, device="cuda")
    ctx.fobj_eval(model, dev(thetas), f)
    ld = torch.zeros(GROUP, dtype=torch.float64, device="cuda")
    last0 = (n_pts - 1) // GROUP * GROUP          # first point of the last group
    last_cnt = n_pts - last0
    for j in range(last_cnt):
        ctx.logdet(2 * j + bta.BTA_QP, ld[j:j + 1])
    ctx.sync()
    f_all = f.cpu().numpy()
    ld_last = ld.cpu().numpy()[:last_cnt]
    ctx.close()
    torch.cuda.empty_cache()
    assert np.all(np.isfinite(f_all))
    for j in range(last_cnt):
        ref = _closed_form_logdet_p(p, thetas[last0 + j], fd)
        assert abs(ld_last[j] - ref) <= 1e-8 * abs(ref), (last0 + j, ld_last[j], ref)
    single = bta.BtaContext(p.nt, p.b, p.a, bta.BTA_MIXED, None, 1)
    f1 = torch.zeros(1, dtype=torch.float64, device="cuda")
    for k in (0, 13, n_pts - 1):
        single.fobj_eval(model, dev(thetas[k:k + 1]), f1)
        single.sync()
        v = float(f1.item())
        assert abs(v - f_all[k]) <= 1e-10 * abs(v), (k, v, f_all[k])
    single.close()
    model.close()
    torch.cuda.empty_cache()
