"""Pins of the oracle's linear algebra and objective: tier B (block
recurrences) against tier D (LAPACK on the dense matrix), the determinant
lemma, the kriging form of the conditional mean and the Gaussian marginal
likelihood form of f_obj.  CPU only."""

import math

import numpy as np
import pytest
import scipy.linalg as sla

import synth
from oracle import bta, dense, fobj, model

CASES = ["t_uni", "t_uni_ragged", "t_coreg2", "t_coreg3", "t_coreg3_del", "t_uni_nt1", "c1"]


def _built(name, theta=None):
    p = synth.problem_from_config(name)
    th = p.theta0 if theta is None else theta
    return p, model.build(p, model.theta_to_params(th, p.nv))


@pytest.mark.parametrize("name", CASES)
def test_tier_b_factor_logdet_solve_selinv_match_dense(name):
    p, b = _built(name)
    n, bs, a = p.nt, p.b, p.a
    for Q in (b.Qp, b.Qc):
        Qd = Q.toarray()
        blk = bta.blocks_from_sparse(Q, n, bs, a)
        L = bta.factor(blk)
        # factor == dense Cholesky on the pattern
        Ld = np.linalg.cholesky(Qd)
        ref = dense.bta_blocks(Ld, n, bs, a)
        for k in ("D", "B", "R", "T"):
            assert np.max(np.abs(L[k] - ref[k]), initial=0) < 1e-10 * np.max(np.abs(Ld)), k
        # log-determinant
        sign, ld = np.linalg.slogdet(Qd)
        assert sign > 0
        assert abs(bta.logdet(L) - ld) < 1e-11 * max(1.0, abs(ld))
        # solve
        rng = np.random.default_rng(3)
        r = rng.standard_normal(p.N)
        x = bta.solve(L, r)
        assert np.linalg.norm(Qd @ x - r) <= 1e-12 * np.linalg.norm(r) * np.linalg.cond(Qd) ** 0.5
        assert np.max(np.abs(x - np.linalg.solve(Qd, r))) < 1e-9 * np.max(np.abs(x))
        # selected inverse == dense inverse on the pattern
        S = bta.selinv(L)
        Sref = dense.bta_blocks(np.linalg.inv(Qd), n, bs, a)
        for k in ("D", "B", "R", "T"):
            scale = max(np.max(np.abs(Sref[k]), initial=0), 1e-300)
            assert np.max(np.abs(S[k] - Sref[k]), initial=0) < 1e-9 * scale, k
        # block matvec
        bound = 1e-13 * (np.abs(Qd) @ np.abs(x))
        assert np.all(np.abs(bta.matvec(blk, x) - Qd @ x) <= bound)


@pytest.mark.parametrize("name", ["t_uni", "t_coreg3", "c1"])
def test_determinant_lemma(name):
    """log|Q_c| = log|Q_p| + log|I + D^{1/2} A Q_p^{-1} A^T D^{1/2}|."""
    p, b = _built(name)
    Ad = b.A.toarray()
    Sp = np.linalg.inv(b.Qp.toarray())
    sd = np.sqrt(b.d)
    M = np.eye(p.m) + (sd[:, None] * Ad) @ Sp @ (Ad.T * sd[None, :])
    lhs = dense.logdet(b.Qc)
    rhs = dense.logdet(b.Qp) + np.linalg.slogdet(M)[1]
    assert abs(lhs - rhs) < 1e-9 * abs(lhs)


@pytest.mark.parametrize("name", ["t_uni", "t_coreg3"])
def test_conditional_mean_kriging_form(name):
    """mu = Q_c^{-1} A^T D y equals Sigma_p A^T (A Sigma_p A^T + D^{-1})^{-1} y."""
    p, b = _built(name)
    Ad = b.A.toarray()
    Sp = np.linalg.inv(b.Qp.toarray())
    K = Ad @ Sp @ Ad.T + np.diag(1.0 / b.d)
    mu_krig = Sp @ Ad.T @ np.linalg.solve(K, p.y)
    mu = fobj.f_obj_terms(p, p.theta0, tier="dense")["mu"]
    assert np.max(np.abs(mu - mu_krig)) < 1e-8 * np.max(np.abs(mu))


@pytest.mark.parametrize("name", ["t_uni", "t_uni_ragged", "t_coreg2", "t_coreg3"])
def test_fobj_is_gaussian_marginal_likelihood(name):
    """For a Gaussian likelihood, Eq. 7/8 give log p(theta) + log N(y; 0,
    A Q_p^{-1} A^T + D^{-1}) exactly (Bayes' rule with p_G exact)."""
    p = synth.problem_from_config(name)
    theta = p.theta0 + 0.05 * np.random.default_rng(5).standard_normal(p.theta0.shape)
    b = model.build(p, model.theta_to_params(theta, p.nv))
    Ad = b.A.toarray()
    K = Ad @ np.linalg.inv(b.Qp.toarray()) @ Ad.T + np.diag(1.0 / b.d)
    Lk = np.linalg.cholesky(K)
    z = sla.solve_triangular(Lk, p.y, lower=True)
    log_ml = -0.5 * z @ z - np.sum(np.log(np.diag(Lk))) - 0.5 * p.m * math.log(2 * math.pi)
    expect = fobj.log_prior_theta(theta, p.theta0) + log_ml
    for tier in ("dense", "bta"):
        got = fobj.f_obj(p, theta, tier=tier)
        assert abs(got - expect) < 1e-9 * abs(expect)


@pytest.mark.parametrize("name", ["t_uni", "t_coreg3"])
def test_fobj_independent_of_evaluation_point(name):
    p = synth.problem_from_config(name)
    f_mu = fobj.f_obj(p, p.theta0, tier="dense")
    rng = np.random.default_rng(9)
    for x in (np.zeros(p.N), rng.standard_normal(p.N)):
        assert abs(fobj.f_obj(p, p.theta0, x=x, tier="dense") - f_mu) < 1e-9 * abs(f_mu)


def test_fd_gradient_matches_second_order_accuracy():
    """Central differences (Eq. 10): halving h changes the estimate by O(h^2)."""
    p = synth.problem_from_config("t_uni")
    g1 = fobj.fd_gradient(p, p.theta0, h=2e-3, tier="dense")
    g2 = fobj.fd_gradient(p, p.theta0, h=1e-3, tier="dense")
    assert np.max(np.abs(g1 - g2)) < 1e-3 * max(1.0, np.max(np.abs(g2)))


@pytest.mark.parametrize("name", ["t_uni", "t_coreg2", "t_coreg3"])
def test_adjoint_gradient_matches_finite_differences(name):
    """The analytic (adjoint) gradient against central differences of f_obj
    (Eq. 10, h = 1e-4: truncation error ~h^2)."""
    p = synth.problem_from_config(name)
    theta = p.theta0 + 0.1 * np.random.default_rng(3).standard_normal(p.theta0.shape)
    g = fobj.grad_adjoint(p, theta)
    gfd = fobj.fd_gradient(p, theta, h=1e-4, tier="dense")
    scale = np.maximum(np.abs(g), 1e-3 * np.max(np.abs(g)))
    assert np.max(np.abs(g - gfd) / scale) < 1e-5


def test_logdet_derivative_closed_forms():
    """1/2 tr(Q_p^{-1} dQ_p) is 1/2 d log|Q_p|: for the univariate prior,
    d/d log sigma = -(ns nt + nr) and d/d log range_t = ns (nt-1) rho^2 r / (1-rho^2)
    with r = 1/range_t (log|Q_t| = -(nt-1) log(1-rho^2), rho = exp(-r))."""
    p = synth.problem_from_config("t_uni")
    theta = p.theta0.copy()
    theta[1] = math.log(2.5)
    fd = model.fem_data(p)
    prm = model.theta_to_params(theta, 1)
    Sp = dense.inverse(model.build(p, prm, fd).Qp)
    dQs, _, _, _ = fobj.model_derivatives(p, theta, 2, fd)
    assert abs(0.5 * np.sum(Sp * dQs.toarray()) + (p.ns * p.nt + p.nr)) < 1e-8 * p.N
    dQt, _, _, _ = fobj.model_derivatives(p, theta, 1, fd)
    rho, r = prm.rho[0], 1.0 / 2.5
    expect = p.ns * (p.nt - 1) * rho * rho * r / (1 - rho * rho)
    assert abs(0.5 * np.sum(Sp * dQt.toarray()) - expect) < 1e-8 * abs(expect)


@pytest.mark.parametrize("name", ["t_uni_ragged", "t_coreg3", "t_coreg3_del"])
def test_adjoint_gradient_block_tier_matches_dense_tier(name):
    """The block-tier gradient (traces over the BTA pattern of the selected
    inverse) equals the dense-tier one (traces with the full inverse): dQ has
    no entry outside the pattern.  Also against central differences."""
    p = synth.problem_from_config(name)
    theta = p.theta0 + 0.05 * np.random.default_rng(4).standard_normal(p.theta0.shape)
    g_b = fobj.grad_adjoint(p, theta, tier="bta")
    g_d = fobj.grad_adjoint(p, theta, tier="dense")
    scale = np.maximum(np.abs(g_d), 1e-3 * np.max(np.abs(g_d)))
    assert np.max(np.abs(g_b - g_d) / scale) < 1e-9
    gfd = fobj.fd_gradient(p, theta, h=1e-4, tier="bta")
    assert np.max(np.abs(g_b - gfd) / scale) < 1e-5


def test_trace_on_pattern_counts_each_entry_once():
    """trace_on_pattern against the full elementwise sum for random symmetric
    Sigma and a symmetric dQ with the BTA pattern (a dropped factor 2 or a
    transposed block would fail)."""
    import scipy.sparse as sp
    n, b, a = 4, 5, 2
    N = n * b + a
    rng = np.random.default_rng(8)
    M = rng.standard_normal((N, N))
    Sig = M + M.T
    P = rng.standard_normal((N, N))
    P = P + P.T
    blk = np.minimum(np.arange(N) // b, n)
    inside = (np.abs(blk[:, None] - blk[None, :]) <= 1) | (blk[:, None] == n) | (blk[None, :] == n)
    P[~inside] = 0.0
    S = dense.bta_blocks(Sig, n, b, a)
    t = fobj.trace_on_pattern(S, sp.csr_matrix(P), n, b, a)
    assert abs(t - float(np.sum(Sig * P))) < 1e-12 * np.sum(np.abs(Sig * P))
