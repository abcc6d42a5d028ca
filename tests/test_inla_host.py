"""Host logic of the INLA optimiser (mode by BFGS, Hessian, marginals), run on
the CPU with objectives that need no GPU:
  * Rosenbrock's function, whose maximiser of -f is (1, ..., 1);
  * a quadratic, whose central-difference Hessian of the gradient is exact;
  * the oracle's f_obj and adjoint gradient on a small univariate problem,
    against scipy.optimize.minimize(method="BFGS") on the same functions,
    and the Gaussian hyperparameter marginals there (-H positive definite at
    the mode, H the oracle's second differences of f).
"""

import numpy as np
import pytest
import scipy.optimize

from oracle import dense as odense
from oracle import fobj as ofobj
from oracle import model as omodel
from paper_2507_06938_gb300 import inla

import synth


def _rosen(x):
    return float(np.sum(100.0 * (x[1:] - x[:-1] ** 2) ** 2 + (1.0 - x[:-1]) ** 2))


def _rosen_grad(x):
    g = np.zeros_like(x)
    g[:-1] = -400.0 * x[:-1] * (x[1:] - x[:-1] ** 2) - 2.0 * (1.0 - x[:-1])
    g[1:] += 200.0 * (x[1:] - x[:-1] ** 2)
    return g


def test_bfgs_finds_the_rosenbrock_minimum():
    # the optimiser maximises f, so f = -rosen
    res = inla.bfgs(lambda x: (-_rosen(x), -_rosen_grad(x)), np.array([-1.2, 1.0, -0.5, 0.8]),
                    gtol=1e-8, max_iter=500)
    assert res.converged
    assert np.max(np.abs(res.theta - 1.0)) < 1e-6, res.theta


def test_hessian_of_a_quadratic_is_exact():
    rng = np.random.default_rng(3)
    A = rng.standard_normal((5, 5))
    H = -(A @ A.T + np.eye(5))
    b = rng.standard_normal(5)

    def grads(pts):
        pts = np.atleast_2d(pts)
        return None, np.stack([H @ p + b for p in pts])

    got = inla.hessian_from_gradients(grads, rng.standard_normal(5), 1e-2)
    assert np.max(np.abs(got - H)) < 1e-10 * np.max(np.abs(H))


def test_stencil_differences_match_eq10():
    f = lambda t: np.sin(t[0]) + t[1] ** 3 - t[0] * t[1]
    th = np.array([0.3, -0.7])
    h = 1e-4
    g = inla.fd_from_stencil([f(p) for p in inla.stencil(th, h)], h)
    exact = np.array([np.cos(th[0]) - th[1], 3 * th[1] ** 2 - th[0]])
    assert np.max(np.abs(g - exact)) < 1e-7


class _OracleObjective:
    """The oracle's f_obj (dense tier) and adjoint gradient: test stand-in for
    the GPU objective of the optimiser."""

    def __init__(self, problem):
        self.problem = problem
        self.fd = omodel.fem_data(problem)

    def value_grad(self, theta):
        f = ofobj.f_obj(self.problem, theta, tier="dense", fd=self.fd)
        return f, ofobj.grad_adjoint(self.problem, theta, fd=self.fd)

    def grads(self, pts):
        out = [self.value_grad(p) for p in np.atleast_2d(pts)]
        return np.array([o[0] for o in out]), np.stack([o[1] for o in out])

    def latent_marginals(self, theta):
        terms = ofobj.f_obj_terms(self.problem, theta, tier="dense", fd=self.fd)
        Sc = odense.inverse(terms["built"].Qc)
        return terms["mu"], np.diag(Sc).copy()


@pytest.fixture(scope="module")
def small():
    p = synth.problem_from_config("t_uni")
    obj = _OracleObjective(p)
    res = inla.inla(obj, gtol=1e-6, max_iter=200)
    return p, obj, res


def test_mode_agrees_with_scipy_bfgs(small):
    p, obj, res = small
    ref = scipy.optimize.minimize(lambda t: -obj.value_grad(t)[0], p.theta0,
                                  jac=lambda t: -obj.value_grad(t)[1], method="BFGS",
                                  options=dict(gtol=1e-7, maxiter=500))
    assert res.mode.converged
    assert np.max(np.abs(res.mode.grad)) <= 1e-6
    assert np.max(np.abs(res.mode.theta - ref.x)) < 1e-4, (res.mode.theta, ref.x)
    assert res.mode.f >= -ref.fun - 1e-8 * abs(ref.fun)


def test_gaussian_marginals_at_the_mode(small):
    p, obj, res = small
    # -H positive definite at a maximum; H against second differences of f
    assert res.cov_theta is not None and np.all(res.sd_theta > 0)
    th, h = res.mode.theta, 1e-3
    f0 = obj.value_grad(th)[0]
    for i in range(th.shape[0]):
        e = np.zeros_like(th)
        e[i] = h
        d2 = (obj.value_grad(th + e)[0] - 2 * f0 + obj.value_grad(th - e)[0]) / h ** 2
        assert abs(res.hessian[i, i] - d2) <= 1e-3 * max(abs(d2), 1.0), (i, res.hessian[i, i], d2)
    assert np.allclose(res.cov_theta @ (-res.hessian), np.eye(th.shape[0]), atol=1e-8)
    # latent marginals are the conditional mean and diag(Q_c^-1) at the mode
    terms = ofobj.f_obj_terms(p, th, tier="dense", fd=obj.fd)
    assert np.allclose(res.mu, terms["mu"], rtol=0, atol=1e-12 * np.max(np.abs(terms["mu"])))
    assert np.all(res.var > 0)


def test_line_search_returns_a_strong_wolfe_step():
    # phi along a descent direction of Rosenbrock's function from a far point
    x = np.array([-1.2, 1.0])
    g = _rosen_grad(x)
    p = -g / np.linalg.norm(g)
    c1, c2 = 1e-4, 0.9

    def phi(alpha):
        z = x + alpha * p
        return _rosen(z), float(_rosen_grad(z) @ p), None

    phi0, dphi0 = _rosen(x), float(g @ p)
    for alpha1 in (1.0, 1e-3, 10.0):
        alpha, v, _ = inla._line_search(phi, phi0, dphi0, c1=c1, c2=c2, alpha1=alpha1)
        d = phi(alpha)[1]
        assert v <= phi0 + c1 * alpha * dphi0          # sufficient decrease
        assert abs(d) <= c2 * abs(dphi0)               # curvature (strong form)
