"""Pins of the oracle's model assembly against things other than itself:
closed forms, invariants, textbook special cases and the paper's printed
numbers.  CPU only."""

import math
import os

import numpy as np
import pytest
import scipy.sparse as sp
from scipy.special import kv

import synth
from oracle import dense, fem, model

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- FEM (II-A.1)

@pytest.mark.parametrize("mesh", [("grid", 7), ("grid", 9, 13), ("delaunay", 60)])
def test_fem_mass_and_stiffness_invariants(mesh):
    if mesh[0] == "grid":
        nodes, tri = synth.grid_mesh(*mesh[1:])
    else:
        nodes, tri, _ = synth.delaunay_mesh(mesh[1], 7)
    C = fem.lumped_mass(nodes, tri)
    G = fem.stiffness(nodes, tri)
    # lumped mass sums to the domain area (unit square)
    assert abs(C.sum() - 1.0) < 1e-13
    assert np.all(C > 0)
    # constants are in the kernel of the stiffness matrix; symmetric, PSD
    assert np.max(np.abs(G @ np.ones(nodes.shape[0]))) < 1e-12
    assert abs(G - G.T).max() < 1e-13
    ev = np.linalg.eigvalsh(G.toarray())
    assert ev.min() > -1e-10
    # linear functions: (G u)_k = 0 at interior nodes (u_h = u exactly)
    u = 0.3 * nodes[:, 0] - 1.7 * nodes[:, 1] + 0.2
    interior = ((nodes[:, 0] > 1e-12) & (nodes[:, 0] < 1 - 1e-12)
                & (nodes[:, 1] > 1e-12) & (nodes[:, 1] < 1 - 1e-12))
    assert np.max(np.abs((G @ u)[interior])) < 1e-12


def test_fem_regular_grid_closed_forms():
    g = 8
    h = 1.0 / (g - 1)
    nodes, tri = synth.grid_mesh(g)
    C = fem.lumped_mass(nodes, tri)
    G = fem.stiffness(nodes, tri).toarray()
    for j in range(1, g - 1):
        for i in range(1, g - 1):
            k = j * g + i
            # interior lumped mass = h^2; stiffness = 5-point Laplacian stencil
            assert abs(C[k] - h * h) < 1e-15
            row = G[k].copy()
            assert abs(row[k] - 4.0) < 1e-13
            for nb in (k - 1, k + 1, k - g, k + g):
                assert abs(row[nb] + 1.0) < 1e-13
                row[nb] = 0.0
            row[k] = 0.0
            assert np.max(np.abs(row)) < 1e-13
    # quadratic u = x^2: second difference is exact, (G u)_k = -2 h^2
    u = nodes[:, 0] ** 2
    Gu = G @ u
    for j in range(1, g - 1):
        for i in range(1, g - 1):
            assert abs(Gu[j * g + i] + 2 * h * h) < 1e-13


@pytest.mark.parametrize("name", ["t_uni", "t_coreg3_del"])
def test_barycentric_interpolation(name):
    p = synth.problem_from_config(name)
    idx, w = fem.barycentric(p.nodes, p.tri, p.obs_xy, p.obs_tri)
    assert np.max(np.abs(w.sum(axis=1) - 1.0)) < 1e-13
    assert w.min() > -1e-12
    # P1 interpolation reproduces linear functions: the coordinates themselves
    xy = np.einsum("kj,kjd->kd", w, p.nodes[idx])
    assert np.max(np.abs(xy - p.obs_xy)) < 1e-13


# ------------------------------------------------------------ SPDE (II-A.1)

def test_spde_matern_variance_and_correlation():
    """Unit variance and the Matern(nu = 1) correlation kappa r K_1(kappa r)
    in the middle of a fine grid (textbook limit of the SPDE discretisation)."""
    g = 48
    nodes, tri = synth.grid_mesh(g)
    C = fem.lumped_mass(nodes, tri)
    G = fem.stiffness(nodes, tri)
    kappa = math.sqrt(8.0) / 0.3
    tau = math.sqrt(1.0 / (4 * math.pi * kappa ** 2))
    S = np.linalg.inv(model.spde_precision(C, G, kappa, tau).toarray())
    c = (g // 2) * g + g // 2
    assert abs(S[c, c] - 1.0) < 0.05
    h = 1.0 / (g - 1)
    for k in (2, 4, 6, 8):
        corr = S[c, c + k] / math.sqrt(S[c, c] * S[c + k, c + k])
        r = k * h
        assert abs(corr - kappa * r * kv(1, kappa * r)) < 0.03


def test_spde_plane_wave_symbol():
    """On the regular grid, two rings away from the boundary, C = h^2 I and G
    acts on u = cos(w x) as multiplication by h^2 lam, lam = (4/h^2)
    sin^2(w h / 2) (5-point symbol), so Q_s u = tau^2 h^2 (kappa^2 + lam)^2 u
    exactly: pins every term of tau^2 (kappa^4 C + 2 kappa^2 G + G C^{-1} G)."""
    g = 12
    h = 1.0 / (g - 1)
    nodes, tri = synth.grid_mesh(g)
    C = fem.lumped_mass(nodes, tri)
    G = fem.stiffness(nodes, tri)
    kappa, tau = 3.7, 0.41
    Q = model.spde_precision(C, G, kappa, tau)
    w = 2.3
    u = np.cos(w * nodes[:, 0])
    lam = 4.0 / h ** 2 * math.sin(w * h / 2) ** 2
    Qu = Q @ u
    for j in range(2, g - 2):
        for i in range(2, g - 2):
            k = j * g + i
            expect = tau ** 2 * h ** 2 * (kappa ** 2 + lam) ** 2 * u[k]
            assert abs(Qu[k] - expect) < 1e-10 * max(1.0, abs(expect))


# ------------------------------------------------------------------- AR(1)

@pytest.mark.parametrize("nt,rho", [(1, 0.5), (2, 0.3), (9, 0.7), (16, -0.4)])
def test_ar1_precision_closed_forms(nt, rho):
    Qt = model.ar1_precision(nt, rho).toarray()
    cov = rho ** np.abs(np.subtract.outer(np.arange(nt), np.arange(nt)))
    assert np.max(np.abs(np.linalg.inv(Qt) - cov)) < 1e-12
    sign, ld = np.linalg.slogdet(Qt)
    assert sign > 0
    assert abs(ld + (nt - 1) * math.log(1 - rho ** 2)) < 1e-12


# --------------------------------------------------- Kronecker prior (IV-B)

def _closed_form_logdet_qp(problem, p, fd):
    """sum_u [ns log|Q_t^u| + nt log|Q_s^u| + nr log p_beta]
       - 2 sum_u (ns nt + nr) log sigma_u     (|M| = 1)."""
    ns, nt, nr = problem.ns, problem.nt, problem.nr
    total = 0.0
    for u in range(problem.nv):
        Qs = model.spde_precision(fd.C, fd.G, p.kappa[u], p.tau[u]).toarray()
        ld_s = np.linalg.slogdet(Qs)[1]
        ld_t = -(nt - 1) * math.log(1 - p.rho[u] ** 2)
        total += ns * ld_t + nt * ld_s + nr * math.log(problem.beta_prior_prec)
        total -= 2 * (ns * nt + nr) * math.log(p.sigma[u])
    return total


@pytest.mark.parametrize("name", ["t_uni", "t_uni_ragged", "t_coreg2", "t_coreg3"])
def test_prior_logdet_closed_form(name):
    p = synth.problem_from_config(name)
    theta = p.theta0.copy()
    theta[2::4][: p.nv] = np.linspace(-0.3, 0.4, p.nv)  # sigma != 1
    prm = model.theta_to_params(theta, p.nv)
    fd = model.fem_data(p)
    b = model.build(p, prm, fd)
    assert abs(dense.logdet(b.Qp) - _closed_form_logdet_qp(p, prm, fd)) < 1e-9 * p.N


def test_univariate_prior_covariance_closed_form():
    """Sigma_p[(t,s),(t',s')] = sigma^2 rho^|t-t'| Q_s^{-1}[s,s'] and the tip is
    sigma^2 / p_beta I: pins the Kronecker order and the permutation."""
    p = synth.problem_from_config("t_uni")
    theta = p.theta0.copy()
    theta[2] = 0.25
    prm = model.theta_to_params(theta, 1)
    fd = model.fem_data(p)
    S = dense.inverse(model.build(p, prm, fd).Qp)
    Ss = np.linalg.inv(model.spde_precision(fd.C, fd.G, prm.kappa[0], prm.tau[0]).toarray())
    ns, nt = p.ns, p.nt
    sig2 = prm.sigma[0] ** 2
    for t in range(nt):
        for t2 in range(nt):
            blk = S[t * ns:(t + 1) * ns, t2 * ns:(t2 + 1) * ns]
            assert np.max(np.abs(blk - sig2 * prm.rho[0] ** abs(t - t2) * Ss)) < 1e-9
    tip = S[nt * ns:, nt * ns:]
    assert np.max(np.abs(tip - sig2 / p.beta_prior_prec * np.eye(p.nr))) < 1e-6


# -------------------------------------------------- coregional model (II-B, IV-B)

def _paper_lambda_nv3(sig, lam):
    """Lambda exactly as printed in Eq. 5."""
    s1, s2, s3 = sig
    l1, l2, l3 = lam
    return np.array([[s1, 0, 0],
                     [l1 * s1, s2, 0],
                     [(l3 + l1 * l2) * s1, l2 * s2, s3]])


def _paper_qmvn_coefficients(sig, lam):
    """Coefficient of Q^u in block (v, v') of Eq. 11 (nv = 3), as printed."""
    s1, s2, s3 = sig
    l1, l2, l3 = lam
    c = np.zeros((3, 3, 3))  # [v, v', u]
    c[0, 0] = [1 / s1 ** 2, l1 ** 2 / s2 ** 2, l3 ** 2 / s3 ** 2]
    c[0, 1] = c[1, 0] = [0, -l1 / s2 ** 2, l2 * l3 / s3 ** 2]
    c[0, 2] = c[2, 0] = [0, 0, -l3 / s3 ** 2]
    c[1, 1] = [0, 1 / s2 ** 2, l2 ** 2 / s3 ** 2]
    c[1, 2] = c[2, 1] = [0, 0, -l2 / s3 ** 2]
    c[2, 2] = [0, 0, 1 / s3 ** 2]
    return c


def _coreg_case():
    p = synth.problem_from_config("t_coreg3")
    theta = p.theta0.copy()
    theta[0:12:4] = np.log([0.25, 0.4, 0.3])
    theta[1:12:4] = np.log([2.0, 3.0, 5.0])
    theta[2:12:4] = [0.3, -0.2, 0.1]
    theta[12:] = [0.35, -0.45, 0.2]
    return p, theta


def test_coreg_eq11_coefficients():
    p, theta = _coreg_case()
    prm = model.theta_to_params(theta, 3)
    fd = model.fem_data(p)
    Qvm = model.joint_prior_variable_major(p, prm, fd).toarray()
    per = p.nt * p.ns + p.nr
    Qu = []
    for u in range(3):
        Qs = model.spde_precision(fd.C, fd.G, prm.kappa[u], prm.tau[u])
        Qt = model.ar1_precision(p.nt, prm.rho[u])
        Qu.append(model.univariate_precision(Qt, Qs, p.nr).toarray())
    coef = _paper_qmvn_coefficients(prm.sigma, prm.lam)
    for v in range(3):
        for w in range(3):
            blk = Qvm[v * per:(v + 1) * per, w * per:(w + 1) * per]
            expect = sum(coef[v, w, u] * Qu[u] for u in range(3))
            assert np.max(np.abs(blk - expect)) < 1e-10 * np.max(np.abs(expect))


def test_coreg_covariance_eq6():
    """inv(Q^{nv}) = Lambda blockdiag(Sigma_u) Lambda^T with Lambda of Eq. 5."""
    p, theta = _coreg_case()
    prm = model.theta_to_params(theta, 3)
    fd = model.fem_data(p)
    Qvm = model.joint_prior_variable_major(p, prm, fd).toarray()
    Sig = []
    for u in range(3):
        Qs = model.spde_precision(fd.C, fd.G, prm.kappa[u], prm.tau[u])
        Qt = model.ar1_precision(p.nt, prm.rho[u])
        Sig.append(np.linalg.inv(model.univariate_precision(Qt, Qs, p.nr).toarray()))
    per = Sig[0].shape[0]
    Lam = np.kron(_paper_lambda_nv3(prm.sigma, prm.lam), np.eye(per))
    import scipy.linalg as sla
    expect = Lam @ sla.block_diag(*Sig) @ Lam.T
    got = np.linalg.inv(Qvm)
    assert np.max(np.abs(got - expect)) < 1e-8 * np.max(np.abs(expect))
    # the oracle's Lambda equals the printed one
    assert np.allclose(model.mixing_matrix(prm), _paper_lambda_nv3(prm.sigma, prm.lam),
                       rtol=0, atol=1e-15)


# ------------------------------------------------ BTA layout (IV-B.1, table)

def test_dimension_formula_matches_paper_table():
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "paper_datasets_table.txt"))
            if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 9
    for name, nv, ns, nr, nt, N in rows:
        nv, ns, nr, nt, N = map(int, (nv, ns, nr, nt, N))
        # N = nv (ns nt + nr) = n b + a with n = nt, b = nv ns, a = nv nr
        assert nt * (nv * ns) + nv * nr == N, name


@pytest.mark.parametrize("name", ["t_uni", "t_coreg2", "t_coreg3", "t_coreg3_del", "c1"])
def test_bta_pattern_and_symmetry(name):
    p = synth.problem_from_config(name)
    b = model.build(p, model.theta_to_params(p.theta0, p.nv))
    for Q in (b.Qp, b.Qc):
        assert abs(Q - Q.T).max() < 1e-12 * abs(Q).max()
        assert dense.outside_bta_pattern_max(Q, p.nt, p.b, p.a) == 0.0
    # the prior has no arrow: fixed effects are a priori independent of the field
    blk = dense.bta_blocks(b.Qp.toarray(), p.nt, p.b, p.a)
    assert np.max(np.abs(blk["R"])) == 0.0
    assert np.min(np.linalg.eigvalsh(b.Qc.toarray())) > 0


def test_permutation_is_a_bijection():
    for nv, ns, nt, nr in [(1, 5, 3, 2), (3, 4, 5, 2), (2, 7, 1, 3)]:
        perm = model.bta_permutation(nv, ns, nt, nr)
        assert np.array_equal(np.sort(perm), np.arange(nv * (ns * nt + nr)))
