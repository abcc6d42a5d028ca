"""f_obj (Eq. 8) for a non-Gaussian likelihood through the Laplace
approximation at the mode of the latent field (oracle; test infrastructure
only).

Section II-A.3 builds p_G from the GMRF prior and a second-order Taylor
expansion of the log-likelihood around x: Q_c = Q_p + A^T D A (Eq. 4), with
D the negative Hessian of the log-likelihood with respect to the linear
predictor eta = A x.  For a Gaussian likelihood p_G is exact and centred at
mu for any x.  Otherwise x is the mode x* of p(x | theta, y) (the point
where p_G is evaluated, Eq. 7/8 with x = x*, Q_c = Q_c(theta, x*)), found by
Newton's method on log p(x | theta) + log l(y | x): with g = d ell / d eta
and D = -d^2 ell / d eta^2 at eta = A x_k, the Taylor expansion gives the
Gaussian whose mean is the next iterate,
    Q_c(x_k) x_{k+1} = A^T (g + D A x_k).
At the mode the quadratic form of p_G vanishes (x* is its mean), and the
-N/2 log 2 pi terms of Eqs. 1 and 3 cancel:
    f = log p(theta) + ell(y | x*) + 1/2 log|Q_p| - 1/2 x*^T Q_p x*
        - 1/2 log|Q_c(x*)|.

Likelihoods (per observation, independent):
  "poisson"  (log link, y counts): ell = y eta - exp(eta) - log y!,
             g = y - exp(eta), D = exp(eta);
  "gaussian" (noise precision d of the observation's variable):
             ell = 1/2 log d - 1/2 log 2 pi - 1/2 d (y - eta)^2,
             g = d (y - eta), D = d.
"""

from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp
from scipy.special import gammaln

from . import fobj as fobj_mod
from . import model

LOG_2PI = math.log(2.0 * math.pi)


def loglik(likelihood: str, y: np.ndarray, eta: np.ndarray, d: np.ndarray | None = None):
    """(ell summed over the observations, g = d ell/d eta, D = -d^2 ell/d eta^2)."""
    if likelihood == "poisson":
        e = np.exp(eta)
        return float(np.sum(y * eta - e - gammaln(y + 1.0))), y - e, e
    if likelihood == "gaussian":
        r = y - eta
        return float(np.sum(0.5 * np.log(d) - 0.5 * LOG_2PI - 0.5 * d * r * r)), d * r, d.astype(np.float64)
    raise ValueError(likelihood)


def laplace_terms(problem, theta, likelihood: str, *, iters: int = 30, tol: float = 1e-12, tier=None, fd=None,
                  x0=None) -> dict:
    """Newton iterations for x* and every term of f_obj at x*.

    Stops after `iters` Newton steps or once max |x_{k+1} - x_k| <= tol max(1, max |x_{k+1}|);
    returns f, x*, the step sizes, the log-determinants and ell(y | x*)."""
    tier = tier or fobj_mod.default_tier(problem)
    fd = model.fem_data(problem) if fd is None else fd
    params = model.theta_to_params(theta, problem.nv)
    built = model.build(problem, params, fd)
    n, b, a = problem.nt, problem.b, problem.a
    A, Qp, y = built.A, built.Qp, problem.y
    d_noise = built.d if likelihood == "gaussian" else None
    fp = fobj_mod.Factorized(Qp, tier, n, b, a)
    x = np.zeros(problem.N) if x0 is None else np.asarray(x0, dtype=np.float64).copy()
    steps = []
    for _ in range(iters):
        eta = A @ x
        _, g, D = loglik(likelihood, y, eta, d_noise)
        Qc = (Qp + A.T @ sp.diags(D) @ A).tocsr()
        x_new = fobj_mod.Factorized(Qc, tier, n, b, a).solve(A.T @ (g + D * eta))
        step = float(np.max(np.abs(x_new - x)))
        steps.append(step)
        x = x_new
        if step <= tol * max(1.0, float(np.max(np.abs(x)))):
            break
    eta = A @ x
    ell, _, D = loglik(likelihood, y, eta, d_noise)
    Qc = (Qp + A.T @ sp.diags(D) @ A).tocsr()
    logdet_p = fp.logdet()
    logdet_c = fobj_mod.Factorized(Qc, tier, n, b, a).logdet()
    quad = float(x @ (Qp @ x))
    lpt = fobj_mod.log_prior_theta(theta, problem.theta0)
    f = lpt + ell + 0.5 * logdet_p - 0.5 * quad - 0.5 * logdet_c
    return dict(f=f, x=x, steps=steps, logdet_p=logdet_p, logdet_c=logdet_c, ell=ell, quad=quad,
                log_prior_theta=lpt, Qc=Qc, Qp=Qp, A=A)
