"""Model assembly in plain FP64 scipy.sparse (oracle; test infrastructure only).

Builds, for one hyperparameter vector theta, the prior precision Q_p and the
conditional precision Q_c = Q_p + A^T D A (Eq. 4) of the spatio-temporal
(multivariate) latent Gaussian model, in the permuted BTA order of
Section IV-B.1.

Readings of the paper used here (the paper gives no formulas for them):
  * SPDE precision (Section II-A.1): Matern alpha = 2 in d = 2,
    Q_s = tau^2 (kappa^4 C + 2 kappa^2 G + G C^{-1} G), kappa = sqrt(8)/range_s,
    tau^2 = 1 / (4 pi kappa^2) (unit marginal variance; the scale sigma of
    each field lives in the mixing matrix Lambda of Eq. 5).
  * Temporal AR(1) with rho = exp(-1/range_t), stationary unit-variance
    precision Q_t = tridiag(-rho; 1, 1+rho^2, ..., 1+rho^2, 1) / (1 - rho^2).
  * Each univariate precision Q^u = blockdiag(Q_t^u (x) Q_s^u, p_beta I_nr)
    (time-major field, then its nr fixed effects; Eq. 2 with x = [x_st, x_f]),
    p_beta = 1e-3.
  * Coregional mixing (Eqs. 5, 6, 11): Lambda = M diag(sigma) with M unit lower
    triangular; M^{-1} has entries -lambda below the diagonal, ordered by
    sub-diagonal (nv = 3: M^{-1}[1,0] = -lambda_1, M^{-1}[2,1] = -lambda_2,
    M^{-1}[2,0] = -lambda_3, which reproduces Eq. 5).  The joint precision is
    Q^{nv} = Lambda^{-T} blockdiag(Q^u) Lambda^{-1}, whose (v, v') block is
    sum_u M^{-1}[u,v] M^{-1}[u,v'] Q^u / sigma_u^2 (Eq. 11).  For nv = 1 this
    is Q^1 / sigma^2, fixed effects included.
  * Conditional precision: the observations see the mixed field z = Lambda x
    (Eq. 5 with shared locations is y = (I (x) A_0) z + eps); the noise of
    variable v has precision tau_eps,v, so Q_c = Q^{nv} + A^T D A in z
    coordinates, D = diag(tau_eps of each observation).
  * Permutation (Section IV-B.1): variable (t, v, s) of the field goes to
    t*b + v*ns + s and fixed effect (v, r) to n*b + v*nr + r, b = nv*ns,
    n = nt, a = nv*nr, N = n*b + a.
"""

from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp

from . import fem

BETA_PRIOR_PREC = 1e-3


@dataclass
class Params:
    kappa: np.ndarray       # (nv,)
    tau: np.ndarray         # (nv,)  SPDE scale with unit variance
    rho: np.ndarray         # (nv,)  AR(1) coefficient
    sigma: np.ndarray       # (nv,)  field standard deviation (diag of Lambda)
    noise_prec: np.ndarray  # (nv,)  Gaussian observation precision tau_eps
    lam: np.ndarray         # (nv(nv-1)/2,) coregionalisation coefficients


def theta_to_params(theta: np.ndarray, nv: int) -> Params:
    """Hyperparameters (log range_s, log range_t, log sigma, log tau_eps per
    variable, then lambda) to model parameters."""
    theta = np.asarray(theta)
    if not np.iscomplexobj(theta):          # complex theta: complex-step derivatives
        theta = theta.astype(np.float64)
    per = theta[: 4 * nv].reshape(nv, 4)
    range_s = np.exp(per[:, 0])
    range_t = np.exp(per[:, 1])
    kappa = math.sqrt(8.0) / range_s
    tau = np.sqrt(1.0 / (4.0 * math.pi * kappa ** 2))
    rho = np.exp(-1.0 / range_t)
    return Params(kappa=kappa, tau=tau, rho=rho, sigma=np.exp(per[:, 2]),
                  noise_prec=np.exp(per[:, 3]), lam=theta[4 * nv:].copy())


def params_vector(p: Params) -> np.ndarray:
    """Flat layout [kappa, tau, rho, sigma, tau_eps] per variable, then lambda."""
    nv = p.kappa.shape[0]
    per = np.stack([p.kappa, p.tau, p.rho, p.sigma, p.noise_prec], axis=1)
    return np.concatenate([per.ravel(), p.lam]).astype(np.float64)


def params_from_vector(vec: np.ndarray, nv: int) -> Params:
    per = np.asarray(vec[: 5 * nv]).reshape(nv, 5)
    return Params(kappa=per[:, 0].copy(), tau=per[:, 1].copy(), rho=per[:, 2].copy(),
                  sigma=per[:, 3].copy(), noise_prec=per[:, 4].copy(),
                  lam=np.asarray(vec[5 * nv:], dtype=np.float64).copy())


def mixing_inverse(lam: np.ndarray, nv: int) -> np.ndarray:
    """M^{-1}: unit lower triangular, -lambda below the diagonal, sub-diagonal
    by sub-diagonal (offset 1 first, top to bottom)."""
    Minv = np.eye(nv, dtype=np.result_type(lam, np.float64))
    k = 0
    for off in range(1, nv):
        for v in range(off, nv):
            Minv[v, v - off] = -lam[k]
            k += 1
    return Minv


def mixing_matrix(p: Params) -> np.ndarray:
    """Lambda of Eq. 5: M diag(sigma), M = (M^{-1})^{-1}."""
    nv = p.kappa.shape[0]
    M = np.linalg.inv(mixing_inverse(p.lam, nv))
    return M @ np.diag(p.sigma)


def spde_precision(C: np.ndarray, G: sp.csr_matrix, kappa: float, tau: float) -> sp.csr_matrix:
    """Q_s = tau^2 (kappa^4 C + 2 kappa^2 G + G C^{-1} G) (Matern, alpha = 2)."""
    Cm = sp.diags(C)
    Ci = sp.diags(1.0 / C)
    Q = (kappa ** 4) * Cm + 2.0 * kappa ** 2 * G + G @ Ci @ G
    return (tau ** 2 * Q).tocsr()


def ar1_precision(nt: int, rho: float) -> sp.csr_matrix:
    """Stationary unit-variance AR(1) precision (nt x nt)."""
    if nt == 1:
        return sp.csr_matrix(np.ones((1, 1)))
    main = np.full(nt, 1.0 + rho ** 2)
    main[0] = main[-1] = 1.0
    off = np.full(nt - 1, -rho)
    return (sp.diags([off, main, off], [-1, 0, 1]) / (1.0 - rho ** 2)).tocsr()


def univariate_precision(Qt: sp.spmatrix, Qs: sp.spmatrix, nr: int,
                         beta_prec: float = BETA_PRIOR_PREC) -> sp.csr_matrix:
    """Q^u = blockdiag(Q_t (x) Q_s, beta_prec I_nr), time-major field first."""
    Qst = sp.kron(Qt, Qs, format="csr")
    return sp.block_diag([Qst, beta_prec * sp.identity(nr)], format="csr")


@dataclass
class FemData:
    C: np.ndarray
    G: sp.csr_matrix
    obs_idx: np.ndarray
    obs_w: np.ndarray


def fem_data(problem) -> FemData:
    C = fem.lumped_mass(problem.nodes, problem.tri)
    G = fem.stiffness(problem.nodes, problem.tri)
    idx, w = fem.barycentric(problem.nodes, problem.tri, problem.obs_xy, problem.obs_tri)
    return FemData(C=C, G=G, obs_idx=idx, obs_w=w)


def joint_prior_variable_major(problem, p: Params, fd: FemData) -> sp.csr_matrix:
    """Q^{nv} of Eq. 11 in variable-major order (variable, then time, then
    space; each variable's fixed effects after its field)."""
    nv, nt, nr = problem.nv, problem.nt, problem.nr
    Qu = []
    for u in range(nv):
        Qs = spde_precision(fd.C, fd.G, p.kappa[u], p.tau[u])
        Qt = ar1_precision(nt, p.rho[u])
        Qu.append(univariate_precision(Qt, Qs, nr, problem.beta_prior_prec))
    Minv = mixing_inverse(p.lam, nv)
    blocks = [[None] * nv for _ in range(nv)]
    for v in range(nv):
        for w in range(nv):
            acc = None
            for u in range(nv):
                c = Minv[u, v] * Minv[u, w] / p.sigma[u] ** 2
                if c != 0.0:
                    term = c * Qu[u]
                    acc = term if acc is None else acc + term
            blocks[v][w] = acc
    return sp.bmat(blocks, format="csr")


def bta_permutation(nv: int, ns: int, nt: int, nr: int) -> np.ndarray:
    """perm[i] = BTA position of variable-major index i (Section IV-B.1)."""
    b = nv * ns
    n = nt
    per_var = nt * ns + nr
    perm = np.empty(nv * per_var, dtype=np.int64)
    for v in range(nv):
        base = v * per_var
        t = np.repeat(np.arange(nt), ns)
        s = np.tile(np.arange(ns), nt)
        perm[base: base + nt * ns] = t * b + v * ns + s
        perm[base + nt * ns: base + per_var] = n * b + v * nr + np.arange(nr)
    return perm


def permute(Q: sp.spmatrix, perm: np.ndarray) -> sp.csr_matrix:
    """Return P Q P^T with row/column i moved to perm[i]."""
    Qc = Q.tocoo()
    N = Q.shape[0]
    return sp.csr_matrix((Qc.data, (perm[Qc.row], perm[Qc.col])), shape=(N, N))


def observation_matrix(problem, fd: FemData) -> sp.csr_matrix:
    """A (m x N) in BTA order: observation k of variable v at time t sees the
    mixed field of variable v at its three triangle nodes (barycentric
    weights) and the fixed effects (v, r) through its covariates."""
    nv, ns, nt, nr = problem.nv, problem.ns, problem.nt, problem.nr
    b = nv * ns
    N = nt * b + nv * nr
    m = problem.m
    rows, cols, vals = [], [], []
    for j in range(3):
        rows.append(np.arange(m))
        cols.append(problem.obs_time * b + problem.obs_var * ns + fd.obs_idx[:, j])
        vals.append(fd.obs_w[:, j])
    for r in range(nr):
        rows.append(np.arange(m))
        cols.append(nt * b + problem.obs_var * nr + r)
        vals.append(problem.X[:, r])
    A = sp.coo_matrix((np.concatenate(vals),
                       (np.concatenate(rows), np.concatenate(cols))), shape=(m, N))
    return A.tocsr()


@dataclass
class Built:
    Qp: sp.csr_matrix     # prior precision, BTA order
    Qc: sp.csr_matrix     # conditional precision, BTA order
    A: sp.csr_matrix      # observation matrix, BTA order
    d: np.ndarray         # noise precision of each observation (diag of D)
    rhs: np.ndarray       # A^T D y
    params: Params


def build(problem, params: Params, fd: FemData | None = None) -> Built:
    """Q_p, Q_c = Q_p + A^T D A (Eq. 4), A, D and A^T D y for one parameter set."""
    fd = fem_data(problem) if fd is None else fd
    Qvm = joint_prior_variable_major(problem, params, fd)
    perm = bta_permutation(problem.nv, problem.ns, problem.nt, problem.nr)
    Qp = permute(Qvm, perm)
    A = observation_matrix(problem, fd)
    d = params.noise_prec[problem.obs_var]
    Qc = (Qp + A.T @ sp.diags(d) @ A).tocsr()
    rhs = A.T @ (d * problem.y)
    return Built(Qp=Qp, Qc=Qc, A=A, d=d, rhs=np.asarray(rhs).ravel(), params=params)
