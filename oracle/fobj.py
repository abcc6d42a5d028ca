"""The INLA objective f_obj(theta) of Eq. 8 and its gradient (oracle; test
infrastructure only).

f_obj(theta) = log p(theta) + log l(y | theta, x) + log p(x | theta)
               - log p_G(x | theta, y)                                  (Eq. 8)
with
  log p(x | theta)     = -N/2 log 2 pi + 1/2 log|Q_p| - 1/2 x^T Q_p x        (Eq. 1)
  log l(y | theta, x)  = sum_k [1/2 log d_k - 1/2 log 2 pi - 1/2 d_k (y_k - (A x)_k)^2]
  log p_G(x | theta,y) = -N/2 log 2 pi + 1/2 log|Q_c| - 1/2 (x-mu)^T Q_c (x-mu)  (Eq. 3)
  mu = Q_c^{-1} A^T D y   (zero prior mean, Gaussian likelihood).
For a Gaussian likelihood p_G is exact (Section II-A.3), so f_obj does not
depend on x; x = mu is used unless another point is given.

Reading of log p(theta) (the paper leaves the hyperprior unspecified): an
independent N(theta0_i, 1) density on every component of theta.

Central finite differences (Eq. 10): d f / d theta_i ~ (f(theta + h e_i) -
f(theta - h e_i)) / (2h), h = 1e-3 unless given.

Analytic gradient (the adjoint form of Eq. 8 for a Gaussian likelihood): with
b = A^T D y, mu = Q_c^{-1} b and Sigma = Q^{-1},
  d f / d theta_k = d log p(theta) + 1/2 tr(Sigma_p dQ_p) - 1/2 tr(Sigma_c dQ_c)
                    - 1/2 y^T dD y + db^T mu - 1/2 mu^T dQ_c mu + 1/2 tr(D^{-1} dD),
obtained by differentiating 1/2 log|Q_p| - 1/2 log|Q_c| - 1/2 (y^T D y - b^T mu)
+ 1/2 log|D| (d log|Q| = tr(Q^{-1} dQ), d mu = Q_c^{-1}(db - dQ_c mu)).  The
derivatives dQ, dD, db of the model build are taken by complex-step
differentiation, Im F(theta + i h e_k) / h (Squire and Trapp, 1998), which is
exact to rounding for a function analytic in theta.
"""

from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp

from . import bta as bta_mod
from . import dense
from . import model

LOG_2PI = math.log(2.0 * math.pi)


def log_prior_theta(theta: np.ndarray, theta0: np.ndarray) -> float:
    d = np.asarray(theta) - np.asarray(theta0)
    return float(-0.5 * np.sum(d * d) - 0.5 * d.shape[0] * LOG_2PI)


class Factorized:
    """log|Q| and solves with Q through either tier (dense or BTA blocks)."""

    def __init__(self, Q: sp.spmatrix, tier: str, n: int, b: int, a: int):
        self.tier = tier
        if tier == "dense":
            self.L = dense.cholesky(Q)
        elif tier == "bta":
            self.L = bta_mod.factor(bta_mod.blocks_from_sparse(Q, n, b, a))
        else:
            raise ValueError(tier)

    def logdet(self) -> float:
        if self.tier == "dense":
            return float(2.0 * np.sum(np.log(np.diag(self.L))))
        return bta_mod.logdet(self.L)

    def solve(self, r: np.ndarray) -> np.ndarray:
        if self.tier == "dense":
            import scipy.linalg as sla
            z = sla.solve_triangular(self.L, r, lower=True)
            return sla.solve_triangular(self.L, z, lower=True, trans="T")
        return bta_mod.solve(self.L, r)


def default_tier(problem) -> str:
    return "dense" if problem.N <= 6000 else "bta"


def f_obj_terms(problem, theta, *, x=None, tier=None, fd=None, params=None) -> dict:
    """Every term of Eq. 8 at theta (x defaults to the conditional mean mu).

    ``params`` overrides the theta map (model parameters given directly)."""
    tier = tier or default_tier(problem)
    fd = model.fem_data(problem) if fd is None else fd
    p = params if params is not None else model.theta_to_params(theta, problem.nv)
    built = model.build(problem, p, fd)
    n, b, a = problem.nt, problem.b, problem.a
    N = problem.N
    fp = Factorized(built.Qp, tier, n, b, a)
    fc = Factorized(built.Qc, tier, n, b, a)
    logdet_p = fp.logdet()
    logdet_c = fc.logdet()
    mu = fc.solve(built.rhs)
    xx = mu if x is None else np.asarray(x, dtype=np.float64)
    resid = problem.y - built.A @ xx
    d = built.d
    log_lik = float(np.sum(0.5 * np.log(d) - 0.5 * LOG_2PI - 0.5 * d * resid * resid))
    log_px = float(-0.5 * N * LOG_2PI + 0.5 * logdet_p - 0.5 * xx @ (built.Qp @ xx))
    dx = xx - mu
    log_pg = float(-0.5 * N * LOG_2PI + 0.5 * logdet_c - 0.5 * dx @ (built.Qc @ dx))
    log_pt = log_prior_theta(theta, problem.theta0) if theta is not None else 0.0
    f = log_pt + log_lik + log_px - log_pg
    return dict(f=f, log_prior_theta=log_pt, log_lik=log_lik, log_px=log_px,
                log_pg=log_pg, logdet_p=logdet_p, logdet_c=logdet_c, mu=mu,
                built=built)


def f_obj(problem, theta, **kw) -> float:
    return f_obj_terms(problem, theta, **kw)["f"]


def fd_gradient(problem, theta, h: float = 1e-3, **kw) -> np.ndarray:
    """Central finite-difference gradient of f_obj (Eq. 10); uses the
    2 dim(theta) points theta +- h e_i."""
    theta = np.asarray(theta, dtype=np.float64)
    g = np.empty_like(theta)
    for i in range(theta.shape[0]):
        e = np.zeros_like(theta)
        e[i] = h
        g[i] = (f_obj(problem, theta + e, **kw) - f_obj(problem, theta - e, **kw)) / (2 * h)
    return g


def model_derivatives(problem, theta, k, fd=None, h=1e-30):
    """dQ_p, dQ_c (sparse), d(A^T D y), dD (diagonal) with respect to theta_k,
    by complex-step differentiation of the model build."""
    fd = model.fem_data(problem) if fd is None else fd
    th = np.asarray(theta, dtype=np.complex128).copy()
    th[k] += 1j * h
    built = model.build(problem, model.theta_to_params(th, problem.nv), fd)
    return (built.Qp.imag / h).tocsr(), (built.Qc.imag / h).tocsr(), built.rhs.imag / h, built.d.imag / h


def trace_on_pattern(S: dict, dQ: sp.spmatrix, n: int, b: int, a: int) -> float:
    """tr(Sigma dQ) = sum_ij Sigma_ij dQ_ij for symmetric Sigma and a symmetric
    dQ whose non-zeros lie on the BTA block pattern, from the lower BTA
    blocks of Sigma: the diagonal blocks and the tip once, the sub-diagonal
    and arrow blocks twice (their transposes above the diagonal)."""
    d = bta_mod.blocks_from_sparse(dQ, n, b, a)
    t = float(np.sum(S["D"] * d["D"])) + float(np.sum(S["T"] * d["T"]))
    t += 2.0 * float(np.sum(S["B"] * d["B"])) + 2.0 * float(np.sum(S["R"] * d["R"]))
    return t


def grad_adjoint(problem, theta, *, fd=None, tier: str = "dense") -> np.ndarray:
    """Analytic gradient of f_obj (formula in the module docstring).

    tier "dense": Sigma_p, Sigma_c from the dense inverse (small problems).
    tier "bta": Sigma_p, Sigma_c on the BTA pattern from the block selected
    inversion (Section III-A); the traces need no entry outside that pattern,
    because every dQ has the pattern of Q."""
    fd = model.fem_data(problem) if fd is None else fd
    theta = np.asarray(theta, dtype=np.float64)
    terms = f_obj_terms(problem, theta, tier=tier, fd=fd)
    built = terms["built"]
    mu = terms["mu"]
    n, b, a = problem.nt, problem.b, problem.a
    if tier == "dense":
        Sp = dense.inverse(built.Qp)
        Sc = dense.inverse(built.Qc)

        def trace(S, dQ):
            return float(np.sum(S * dQ.toarray()))
    elif tier == "bta":
        Sp = bta_mod.selinv(bta_mod.factor(bta_mod.blocks_from_sparse(built.Qp, n, b, a)))
        Sc = bta_mod.selinv(bta_mod.factor(bta_mod.blocks_from_sparse(built.Qc, n, b, a)))

        def trace(S, dQ):
            return trace_on_pattern(S, dQ, n, b, a)
    else:
        raise ValueError(tier)
    y = problem.y
    g = np.empty_like(theta)
    for k in range(theta.shape[0]):
        dQp, dQc, drhs, dd = model_derivatives(problem, theta, k, fd)
        tr_p = trace(Sp, dQp)
        tr_c = trace(Sc, dQc)
        g[k] = (-(theta[k] - problem.theta0[k]) + 0.5 * tr_p - 0.5 * tr_c - 0.5 * float(y @ (dd * y))
                + float(drhs @ mu) - 0.5 * float(mu @ (dQc @ mu)) + 0.5 * float(np.sum(dd / built.d)))
    return g
