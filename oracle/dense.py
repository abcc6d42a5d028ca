"""Tier D: the plain definitions on the dense N x N matrix (oracle; test
infrastructure only).

The BTA factorisation, log-determinant, solve and selected inversion of
Section III-A compute, up to rounding order, the Cholesky factor of Q, the
log-determinant 2 sum log L_kk (Eq. 1 needs |Q|), the solution of Q x = r and
the entries of Q^{-1} on the BTA pattern.  This module writes those
definitions out with LAPACK (numpy.linalg) on the full dense matrix.
"""

from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def to_dense(Q) -> np.ndarray:
    return Q.toarray() if sp.issparse(Q) else np.asarray(Q, dtype=np.float64)


def cholesky(Q) -> np.ndarray:
    return np.linalg.cholesky(to_dense(Q))


def logdet(Q) -> float:
    L = cholesky(Q)
    return float(2.0 * np.sum(np.log(np.diag(L))))


def solve(Q, r: np.ndarray) -> np.ndarray:
    return np.linalg.solve(to_dense(Q), r)


def inverse(Q) -> np.ndarray:
    return np.linalg.inv(to_dense(Q))


def bta_blocks(M: np.ndarray, n: int, b: int, a: int) -> dict:
    """Cut a dense N x N matrix into the lower BTA blocks:
    D[i] = M[i,i], B[i] = M[i+1,i], R[i] = M[tip,i], T = M[tip,tip]."""
    M = to_dense(M)
    tip = slice(n * b, n * b + a)
    D = np.stack([M[i * b:(i + 1) * b, i * b:(i + 1) * b] for i in range(n)])
    B = (np.stack([M[(i + 1) * b:(i + 2) * b, i * b:(i + 1) * b] for i in range(n - 1)])
         if n > 1 else np.zeros((0, b, b)))
    R = np.stack([M[tip, i * b:(i + 1) * b] for i in range(n)])
    T = M[tip, tip].copy()
    return dict(D=D, B=B, R=R, T=T)


def outside_bta_pattern_max(M, n: int, b: int, a: int) -> float:
    """max |M_ij| over (i, j) outside the BTA block pattern (0 for a BTA matrix)."""
    M = to_dense(M)
    N = n * b + a
    blk = np.minimum(np.arange(N) // b, n)      # block index, tip = n
    bi = blk[:, None]
    bj = blk[None, :]
    inside = (np.abs(bi - bj) <= 1) | (bi == n) | (bj == n)
    return float(np.max(np.abs(M[~inside]), initial=0.0))
