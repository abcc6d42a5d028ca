"""Pins of the oracle's Laplace approximation for non-Gaussian likelihoods
(oracle/laplace.py): the Gaussian special case reproduces the exact f_obj
in one Newton step; for Poisson counts the mode satisfies the first-order
condition, agrees with an independent trust-region optimiser, and every
term of f equals a library density (scipy.stats) at the mode.  CPU only."""

import numpy as np
import pytest
import scipy.optimize as so
import scipy.stats as st

import synth
from oracle import fobj, laplace, model


def test_gaussian_likelihood_is_exact_in_one_newton_step():
    """For a Gaussian likelihood the Taylor expansion is exact: the first
    Newton step from x = 0 lands on mu, the second does not move, and f
    equals the Gaussian f_obj of Eq. 8."""
    p = synth.problem_from_config("t_coreg3")
    theta = p.theta0 + 0.05 * np.random.default_rng(1).standard_normal(p.theta0.shape)
    r = laplace.laplace_terms(p, theta, "gaussian", iters=3, tier="dense")
    ref = fobj.f_obj_terms(p, theta, tier="dense")
    assert r["steps"][1] <= 1e-9 * np.max(np.abs(ref["mu"]))
    assert np.max(np.abs(r["x"] - ref["mu"])) <= 1e-10 * np.max(np.abs(ref["mu"]))
    assert abs(r["f"] - ref["f"]) <= 1e-10 * abs(ref["f"])


@pytest.mark.parametrize("name", ["t_pois", "t_pois_coreg3"])
def test_poisson_mode_first_order_condition_and_quadratic_convergence(name):
    p = synth.problem_from_config(name)
    r = laplace.laplace_terms(p, p.theta0, "poisson", tier="dense")
    x = r["x"]
    grad = -(r["Qp"] @ x) + r["A"].T @ (p.y - np.exp(r["A"] @ x))
    scale = np.max(np.abs(r["Qp"] @ x)) + np.max(np.abs(r["A"].T @ p.y))
    assert np.max(np.abs(grad)) <= 1e-10 * scale
    s = r["steps"]
    assert len(s) < 15 and s[-1] <= 1e-12 * max(1.0, np.max(np.abs(x)))
    # Newton: once close, each step squares the error
    k = next(i for i in range(len(s)) if s[i] < 1e-3)
    if k + 1 < len(s) and s[k + 1] > 1e-13:
        assert s[k + 1] <= 10 * s[k] ** 2


def test_poisson_mode_matches_an_independent_optimiser():
    """scipy's trust-region Newton on -(log p(x|theta) + ell(y|x)) with the
    exact Hessian reaches the same mode."""
    p = synth.problem_from_config("t_pois")
    r = laplace.laplace_terms(p, p.theta0, "poisson", tier="dense")
    Qp, A, y = r["Qp"].toarray(), r["A"].toarray(), p.y

    def fun(x):
        eta = A @ x
        return 0.5 * x @ Qp @ x - np.sum(y * eta - np.exp(eta))

    def jac(x):
        return Qp @ x - A.T @ (y - np.exp(A @ x))

    def hess(x):
        return Qp + A.T @ (np.exp(A @ x)[:, None] * A)

    res = so.minimize(fun, np.zeros(p.N), jac=jac, hess=hess, method="trust-exact",
                      options={"gtol": 1e-11, "maxiter": 500})
    assert np.max(np.abs(res.x - r["x"])) <= 1e-7 * np.max(np.abs(r["x"]))


@pytest.mark.parametrize("name", ["t_pois", "t_pois_coreg3"])
def test_poisson_f_terms_are_library_densities(name):
    """f = log p(theta) + sum log Poisson(y | exp(eta*)) + log N(x*; 0, Q_p^-1)
    - log N(x*; x*, Q_c(x*)^-1), each density from scipy.stats."""
    p = synth.problem_from_config(name)
    theta = p.theta0 + 0.05 * np.random.default_rng(2).standard_normal(p.theta0.shape)
    r = laplace.laplace_terms(p, theta, "poisson", tier="dense")
    x = r["x"]
    eta = r["A"] @ x
    ell = float(np.sum(st.poisson.logpmf(p.y.astype(int), np.exp(eta))))
    cov_p = np.linalg.inv(r["Qp"].toarray())
    cov_c = np.linalg.inv(r["Qc"].toarray())
    lpx = st.multivariate_normal.logpdf(x, mean=np.zeros(p.N), cov=(cov_p + cov_p.T) / 2, allow_singular=False)
    lpg = st.multivariate_normal.logpdf(x, mean=x, cov=(cov_c + cov_c.T) / 2, allow_singular=False)
    f = fobj.log_prior_theta(theta, p.theta0) + ell + lpx - lpg
    assert abs(r["ell"] - ell) <= 1e-10 * abs(ell)
    assert abs(r["f"] - f) <= 1e-8 * (abs(r["logdet_p"]) + abs(r["logdet_c"]))


def test_block_tier_matches_dense_tier():
    p = synth.problem_from_config("t_pois_coreg3")
    rd = laplace.laplace_terms(p, p.theta0, "poisson", tier="dense")
    rb = laplace.laplace_terms(p, p.theta0, "poisson", tier="bta")
    assert abs(rd["f"] - rb["f"]) <= 1e-10 * abs(rd["f"])
    assert np.max(np.abs(rd["x"] - rb["x"])) <= 1e-10 * np.max(np.abs(rd["x"]))
