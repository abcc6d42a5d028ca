"""Tier B: block recurrences on a BTA matrix (oracle; test infrastructure only).

A BTA matrix (Section IV, table of structured-matrix parameters) has n
diagonal blocks of size b, the sub-diagonal blocks, an arrow of height a and
an a x a tip; N = n b + a.  Its lower blocks are stored as
    D[i] = Q[i, i]        (n, b, b)
    B[i] = Q[i+1, i]      (n-1, b, b)
    R[i] = Q[tip, i]      (n, a, b)
    T    = Q[tip, tip]    (a, a)
Section III-A lists the three operations on it (Cholesky factorisation,
triangular solve, selected inversion) and Section IV-D.2 their O(n (b^3 +
a^3)) cost.  The recurrences below are the block-Cholesky steps in the order
the block elimination fixes them, written with scipy.linalg; they are checked
against the dense definitions (oracle.dense) on small cases.
"""

from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp


def blocks_from_sparse(Q: sp.spmatrix, n: int, b: int, a: int) -> dict:
    Q = Q.tocsr()
    tip = slice(n * b, n * b + a)
    D = np.empty((n, b, b))
    B = np.empty((max(n - 1, 0), b, b))
    R = np.empty((n, a, b))
    for i in range(n):
        cols = slice(i * b, (i + 1) * b)
        D[i] = Q[cols, cols].toarray()
        if i < n - 1:
            B[i] = Q[(i + 1) * b:(i + 2) * b, cols].toarray()
        R[i] = Q[tip, cols].toarray()
    T = Q[tip, tip].toarray()
    return dict(D=D, B=B, R=R, T=T)


def factor(blk: dict) -> dict:
    """Block Cholesky Q = L L^T of a BTA matrix.

    For i = 0..n-1: L_ii = chol(D_i); L_{i+1,i} = B_i L_ii^{-T};
    D_{i+1} -= L_{i+1,i} L_{i+1,i}^T; L_{t,i} = R_i L_ii^{-T};
    R_{i+1} -= L_{t,i} L_{i+1,i}^T; T -= L_{t,i} L_{t,i}^T.  Then L_tt = chol(T).
    """
    D = blk["D"].copy()
    B = blk["B"].copy()
    R = blk["R"].copy()
    T = blk["T"].copy()
    n = D.shape[0]
    Ld = np.empty_like(D)
    Lb = np.empty_like(B)
    Lr = np.empty_like(R)
    for i in range(n):
        Ld[i] = sla.cholesky(D[i], lower=True)
        if i < n - 1:
            Lb[i] = sla.solve_triangular(Ld[i], B[i].T, lower=True).T
            D[i + 1] -= Lb[i] @ Lb[i].T
        Lr[i] = sla.solve_triangular(Ld[i], R[i].T, lower=True).T
        if i < n - 1:
            R[i + 1] -= Lr[i] @ Lb[i].T
        T -= Lr[i] @ Lr[i].T
    Lt = sla.cholesky(T, lower=True) if T.shape[0] else T
    return dict(D=Ld, B=Lb, R=Lr, T=Lt)


def logdet(L: dict) -> float:
    """log|Q| = 2 sum log of the diagonal of the Cholesky factor (Eq. 1)."""
    s = 0.0
    for i in range(L["D"].shape[0]):
        s += np.sum(np.log(np.diag(L["D"][i])))
    if L["T"].shape[0]:
        s += np.sum(np.log(np.diag(L["T"])))
    return float(2.0 * s)


def solve(L: dict, r: np.ndarray) -> np.ndarray:
    """Solve L L^T x = r by forward then backward block substitution."""
    Ld, Lb, Lr, Lt = L["D"], L["B"], L["R"], L["T"]
    n, b, _ = Ld.shape
    a = Lt.shape[0]
    r = np.asarray(r, dtype=np.float64)
    z = np.empty(n * b + a)
    for i in range(n):
        ri = r[i * b:(i + 1) * b].copy()
        if i > 0:
            ri -= Lb[i - 1] @ z[(i - 1) * b:i * b]
        z[i * b:(i + 1) * b] = sla.solve_triangular(Ld[i], ri, lower=True)
    if a:
        rt = r[n * b:].copy()
        for i in range(n):
            rt -= Lr[i] @ z[i * b:(i + 1) * b]
        z[n * b:] = sla.solve_triangular(Lt, rt, lower=True)
    x = np.empty_like(z)
    if a:
        x[n * b:] = sla.solve_triangular(Lt, z[n * b:], lower=True, trans="T")
    for i in range(n - 1, -1, -1):
        zi = z[i * b:(i + 1) * b].copy()
        if i < n - 1:
            zi -= Lb[i].T @ x[(i + 1) * b:(i + 2) * b]
        if a:
            zi -= Lr[i].T @ x[n * b:]
        x[i * b:(i + 1) * b] = sla.solve_triangular(Ld[i], zi, lower=True, trans="T")
    return x


def selinv(L: dict) -> dict:
    """Selected inverse Sigma = Q^{-1} on the BTA pattern from the factor.

    Sigma_tt = L_tt^{-T} L_tt^{-1}.  For i = n-1..0 with G_i = L_{i+1,i} L_ii^{-1}
    and F_i = L_{t,i} L_ii^{-1}:
      Sigma_{i+1,i} = -Sigma_{i+1,i+1} G_i - Sigma_{t,i+1}^T F_i
      Sigma_{t,i}   = -Sigma_{t,i+1} G_i - Sigma_tt F_i
      Sigma_ii      = L_ii^{-T} L_ii^{-1} - Sigma_{i+1,i}^T G_i - Sigma_{t,i}^T F_i
    (terms with index i+1 are absent for i = n-1).  These follow from
    Sigma L = L^{-T} restricted to block rows j >= i of block column i.
    """
    Ld, Lb, Lr, Lt = L["D"], L["B"], L["R"], L["T"]
    n, b, _ = Ld.shape
    a = Lt.shape[0]
    Sd = np.empty_like(Ld)
    Sb = np.empty_like(Lb)
    Sr = np.empty_like(Lr)
    if a:
        Lti = sla.solve_triangular(Lt, np.eye(a), lower=True)
        St = Lti.T @ Lti
    else:
        St = np.zeros((0, 0))
    for i in range(n - 1, -1, -1):
        Lii_inv = sla.solve_triangular(Ld[i], np.eye(b), lower=True)
        F = Lr[i] @ Lii_inv
        if i < n - 1:
            Gi = Lb[i] @ Lii_inv
            Sb[i] = -Sd[i + 1] @ Gi - Sr[i + 1].T @ F
            Sr[i] = -Sr[i + 1] @ Gi - St @ F
            Sd[i] = Lii_inv.T @ Lii_inv - Sb[i].T @ Gi - Sr[i].T @ F
        else:
            Sr[i] = -St @ F
            Sd[i] = Lii_inv.T @ Lii_inv - Sr[i].T @ F
    return dict(D=Sd, B=Sb, R=Sr, T=St)


def matvec(blk: dict, x: np.ndarray) -> np.ndarray:
    """y = Q x using the lower BTA blocks of the symmetric matrix Q."""
    D, B, R, T = blk["D"], blk["B"], blk["R"], blk["T"]
    n, b, _ = D.shape
    a = T.shape[0]
    y = np.zeros(n * b + a)
    xt = x[n * b:]
    for i in range(n):
        xi = x[i * b:(i + 1) * b]
        y[i * b:(i + 1) * b] += D[i] @ xi + R[i].T @ xt
        if i < n - 1:
            y[(i + 1) * b:(i + 2) * b] += B[i] @ xi
            y[i * b:(i + 1) * b] += B[i].T @ x[(i + 1) * b:(i + 2) * b]
        y[n * b:] += R[i] @ xi
    y[n * b:] += T @ xt
    return y
