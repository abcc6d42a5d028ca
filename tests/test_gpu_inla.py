"""The INLA optimiser on the GPU path (c1: 10x10 grid, nt = 8, N = 802,
dim(theta) = 4): the mode of f_obj by BFGS (Eq. 9), the Gaussian
hyperparameter marginals and the latent marginals at the mode.

Pins:
  * the mode against scipy.optimize.minimize(method="BFGS") on the oracle's
    f_obj and adjoint gradient (dense tier);
  * the latent means against the oracle's conditional mean and the
    variances against the diagonal of the oracle's dense Q_c^{-1}, both at
    the GPU's mode;
  * the Hessian diagonal against second differences of the oracle's f_obj;
  * mixed precision with the central-difference gradient of Eq. 10 (the
    paper's scheme, 2 dim + 1 points per batched call) reaches the same mode
    to the accuracy its gradient noise allows.
"""

import numpy as np
import pytest
import scipy.optimize

from oracle import dense as odense
from oracle import fobj as ofobj
from oracle import model as omodel

from gpu_util import build_lib, need_gpu, problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    need_gpu()
    build_lib()
    p = problem("c1")
    fd = omodel.fem_data(p)
    fun = lambda t: -ofobj.f_obj(p, t, tier="dense", fd=fd)
    jac = lambda t: -ofobj.grad_adjoint(p, t, fd=fd)
    ref = scipy.optimize.minimize(fun, p.theta0, jac=jac, method="BFGS", options=dict(gtol=1e-7, maxiter=500))
    return dict(p=p, fd=fd, ref=ref)


def test_mode_and_marginals_fp64(setup):
    from paper_2507_06938_gb300 import bta, inla
    p, fd, ref = setup["p"], setup["fd"], setup["ref"]
    obj = inla.Objective(p, precision=bta.BTA_FP64, gradient="adjoint")
    res = inla.inla(obj, gtol=1e-6, max_iter=200)
    obj.close()
    assert np.max(np.abs(res.mode.grad)) <= 1e-4, res.mode.grad   # stationary to the evaluations' noise
    assert np.max(np.abs(res.mode.theta - ref.x)) < 1e-4, (res.mode.theta, ref.x)
    th = res.mode.theta
    terms = ofobj.f_obj_terms(p, th, tier="dense", fd=fd)
    assert abs(res.mode.f - terms["f"]) <= 1e-9 * abs(terms["f"])
    mu_ref = terms["mu"]
    assert np.max(np.abs(res.mu - mu_ref)) <= 1e-9 * np.max(np.abs(mu_ref))
    var_ref = np.diag(odense.inverse(terms["built"].Qc))
    assert np.max(np.abs(res.var - var_ref) / var_ref) <= 1e-9
    assert res.cov_theta is not None and np.all(res.sd_theta > 0)
    h = 1e-3
    for i in range(th.shape[0]):
        e = np.zeros_like(th)
        e[i] = h
        d2 = (ofobj.f_obj(p, th + e, tier="dense", fd=fd) - 2 * terms["f"]
              + ofobj.f_obj(p, th - e, tier="dense", fd=fd)) / h ** 2
        assert abs(res.hessian[i, i] - d2) <= 1e-3 * max(abs(d2), 1.0), (i, res.hessian[i, i], d2)


def test_mode_mixed_with_fd_gradient(setup):
    from paper_2507_06938_gb300 import bta, inla
    p, ref = setup["p"], setup["ref"]
    obj = inla.Objective(p, precision=bta.BTA_MIXED, gradient="fd")
    mode = inla.bfgs(obj.value_grad, p.theta0, gtol=2e-2, max_iter=200)
    obj.close()
    assert np.max(np.abs(mode.theta - ref.x)) < 2e-2, (mode.theta, ref.x)
