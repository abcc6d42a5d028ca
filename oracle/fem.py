"""P1 finite elements on a triangle mesh (oracle; test infrastructure only).

Section II-A.1: the spatial field is discretised with finite elements on a
triangular mesh (SPDE approach).  The paper gives no formulas; the standard
P1 element matrices are used:
  lumped mass   C_kk = sum over triangles T containing node k of |T| / 3
  stiffness     G_kl = sum over triangles T of |T| grad(phi_k) . grad(phi_l)
and an observation at a point p inside triangle T is interpolated with the
barycentric coordinates of p in T (the values of the three hat functions).
"""

from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def triangle_areas(nodes: np.ndarray, tri: np.ndarray) -> np.ndarray:
    p0, p1, p2 = nodes[tri[:, 0]], nodes[tri[:, 1]], nodes[tri[:, 2]]
    d1 = p1 - p0
    d2 = p2 - p0
    return 0.5 * np.abs(d1[:, 0] * d2[:, 1] - d1[:, 1] * d2[:, 0])


def lumped_mass(nodes: np.ndarray, tri: np.ndarray) -> np.ndarray:
    """Diagonal of the lumped mass matrix C (length ns)."""
    ns = nodes.shape[0]
    area = triangle_areas(nodes, tri)
    c = np.zeros(ns)
    for corner in range(3):
        np.add.at(c, tri[:, corner], area / 3.0)
    return c


def stiffness(nodes: np.ndarray, tri: np.ndarray) -> sp.csr_matrix:
    """Stiffness matrix G as scipy CSR (ns x ns)."""
    ns = nodes.shape[0]
    area = triangle_areas(nodes, tri)
    rows, cols, vals = [], [], []
    for t in range(tri.shape[0]):
        v = tri[t]
        P = nodes[v]
        # gradient of each hat function: solve [1 x y] coefficients
        M = np.column_stack([np.ones(3), P])
        coef = np.linalg.inv(M)          # column i = coefficients of phi_i
        grads = coef[1:, :].T            # (3, 2): grad phi_i
        K = area[t] * grads @ grads.T
        for i in range(3):
            for j in range(3):
                rows.append(v[i])
                cols.append(v[j])
                vals.append(K[i, j])
    G = sp.coo_matrix((vals, (rows, cols)), shape=(ns, ns)).tocsr()
    G.sum_duplicates()
    return G


def barycentric(nodes: np.ndarray, tri: np.ndarray, obs_xy: np.ndarray,
                obs_tri: np.ndarray):
    """Barycentric coordinates of every observation in its triangle.

    Returns (idx, w): idx (m, 3) node indices and w (m, 3) weights so that the
    interpolated value of a nodal field u at observation k is
    sum_j w[k, j] * u[idx[k, j]].
    """
    idx = tri[obs_tri].astype(np.int64)
    w = np.zeros(idx.shape)
    for k in range(obs_xy.shape[0]):
        P = nodes[idx[k]]
        M = np.vstack([np.ones(3), P.T])   # [1;x;y] per vertex, 3x3
        w[k] = np.linalg.solve(M, np.array([1.0, obs_xy[k, 0], obs_xy[k, 1]]))
    return idx, w
