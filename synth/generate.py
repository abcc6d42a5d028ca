"""Seeded generator of spatio-temporal multivariate observation problems.

Everything here is geometry and random numbers; the model (SPDE precision,
AR(1) precision, coregional mixing, observation operator) is built elsewhere,
independently by the oracle and by the CUDA library.

Hyperparameter layout (shared convention, not arithmetic): for each response
variable u = 0..nv-1 four entries ``[log range_s, log range_t, log sigma,
log noise_precision]``, followed by the nv(nv-1)/2 coregionalisation
coefficients lambda (for nv = 3 in the order lambda_1, lambda_2, lambda_3 of
the paper's Eq. 5).  dim(theta) = 4 nv + nv(nv-1)/2, i.e. 4 for a univariate
model and 15 for the trivariate one (Section IV-D.1).
"""

from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class Problem:
    """One synthetic spatio-temporal problem (inputs only)."""

    name: str
    nv: int            # number of response variables
    ns: int            # mesh nodes
    nt: int            # time steps
    nr: int            # fixed effects per variable
    nodes: np.ndarray  # (ns, 2) float64 node coordinates in the unit square
    tri: np.ndarray    # (ntri, 3) int32 node indices, counter-clockwise
    obs_var: np.ndarray   # (m,) int32 response variable of each observation
    obs_time: np.ndarray  # (m,) int32 time step of each observation
    obs_xy: np.ndarray    # (m, 2) float64 observation location
    obs_tri: np.ndarray   # (m,) int32 triangle containing the location
    X: np.ndarray         # (m, nr) float64 covariates (column 0 = intercept)
    y: np.ndarray         # (m,) float64 observed values
    theta0: np.ndarray    # generating hyperparameters (layout above)
    beta_prior_prec: float = 1e-3

    @property
    def m(self) -> int:
        return int(self.y.shape[0])

    @property
    def b(self) -> int:
        return self.nv * self.ns

    @property
    def a(self) -> int:
        return self.nv * self.nr

    @property
    def N(self) -> int:
        return self.nt * self.b + self.a


def theta_layout(nv: int) -> int:
    """Length of the hyperparameter vector for nv response variables."""
    return 4 * nv + nv * (nv - 1) // 2


# ----------------------------------------------------------------------------
# meshes
# ----------------------------------------------------------------------------

def grid_mesh(gx: int, gy: int | None = None):
    """Regular triangulated gx x gy grid over the unit square.

    Node (i, j) (i along x, j along y) sits at (i/(gx-1), j/(gy-1)) and has
    index j*gx + i.  Every grid square is split along its (i,j)-(i+1,j+1)
    diagonal into two counter-clockwise triangles.
    """
    gy = gx if gy is None else gy
    xs = np.arange(gx) / (gx - 1)
    ys = np.arange(gy) / (gy - 1)
    X, Y = np.meshgrid(xs, ys)  # rows j, cols i
    nodes = np.stack([X.ravel(), Y.ravel()], axis=1).astype(np.float64)
    tris = []
    for j in range(gy - 1):
        for i in range(gx - 1):
            p00 = j * gx + i
            p10 = p00 + 1
            p01 = p00 + gx
            p11 = p01 + 1
            tris.append((p00, p10, p11))
            tris.append((p00, p11, p01))
    return nodes, np.asarray(tris, dtype=np.int32)


def _grid_locate(xy: np.ndarray, gx: int, gy: int) -> np.ndarray:
    """Triangle index (in grid_mesh order) containing each point."""
    hx = 1.0 / (gx - 1)
    hy = 1.0 / (gy - 1)
    i = np.minimum((xy[:, 0] / hx).astype(np.int64), gx - 2)
    j = np.minimum((xy[:, 1] / hy).astype(np.int64), gy - 2)
    fx = xy[:, 0] / hx - i
    fy = xy[:, 1] / hy - j
    upper = (fy > fx).astype(np.int64)  # above the diagonal -> second triangle
    return ((j * (gx - 1) + i) * 2 + upper).astype(np.int32)


def delaunay_mesh(npts: int, seed: int):
    """Delaunay triangulation of the 4 unit-square corners plus npts-4 seeded
    uniform points (host-side geometry only)."""
    from scipy.spatial import Delaunay

    rng = np.random.default_rng(seed)
    corners = np.array([[0.0, 0.0], [1.0, 0.0], [1.0, 1.0], [0.0, 1.0]])
    pts = np.concatenate([corners, rng.uniform(0.0, 1.0, size=(npts - 4, 2))])
    d = Delaunay(pts)
    tri = d.simplices.astype(np.int32)
    # orient counter-clockwise
    p = pts[tri]
    cross = (p[:, 1, 0] - p[:, 0, 0]) * (p[:, 2, 1] - p[:, 0, 1]) - (
        p[:, 1, 1] - p[:, 0, 1]) * (p[:, 2, 0] - p[:, 0, 0])
    flip = cross < 0
    tri[flip] = tri[flip][:, [0, 2, 1]]
    return pts.astype(np.float64), tri, d


# ----------------------------------------------------------------------------
# problems
# ----------------------------------------------------------------------------

def _true_field(v: int, xy: np.ndarray, t: np.ndarray, nt: int) -> np.ndarray:
    """Smooth synthetic signal of response variable v (data only)."""
    return (np.sin(2 * np.pi * xy[:, 0] + 0.7 * v) * np.cos(2 * np.pi * xy[:, 1])
            * np.cos(2 * np.pi * t / max(nt, 1)))


def make_problem(name: str, *, nv: int, mesh, nt: int, nr: int, seed: int,
                 m_total: int | None = None, per_step: int | None = None,
                 shared_sites: bool = False, theta0=None,
                 lam_range: float = 0.5, likelihood: str = "gaussian") -> Problem:
    """Build a seeded problem.

    mesh: ("grid", gx[, gy]) or ("delaunay", npts).
    Univariate style (shared_sites=False): ``m_total`` observations; when
    ``per_step`` is given each time step gets ``per_step`` sites, otherwise the
    time of each observation is uniform over the nt steps.
    Coregional style (shared_sites=True): each time step has ``per_step``
    uniform sites, observed once per response variable with shared covariates.
    likelihood "gaussian": y = signal + noise of precision exp(theta0 noise
    entry); "poisson": counts y ~ Poisson(exp(eta)) with the log-rate
    eta = 0.5 signal + 0.2 sum of the covariates (data only).
    """
    rng = np.random.default_rng(seed)
    kind = mesh[0]
    if kind == "grid":
        gx = mesh[1]
        gy = mesh[2] if len(mesh) > 2 else gx
        nodes, tri = grid_mesh(gx, gy)
        locate = lambda xy: _grid_locate(xy, gx, gy)  # noqa: E731
    elif kind == "delaunay":
        nodes, tri, d = delaunay_mesh(mesh[1], seed + 1000)
        def locate(xy):  # noqa: E306
            s = d.find_simplex(xy)
            if np.any(s < 0):
                raise RuntimeError("observation outside the mesh")
            return s.astype(np.int32)
    else:
        raise ValueError(kind)
    ns = nodes.shape[0]

    if shared_sites:
        assert per_step is not None
        sites_t = np.repeat(np.arange(nt), per_step)
        sites_xy = rng.uniform(0.0, 1.0, size=(nt * per_step, 2))
        sites_X = np.ones((nt * per_step, nr))
        if nr > 1:
            sites_X[:, 1:] = rng.standard_normal((nt * per_step, nr - 1))
        obs_var = np.repeat(np.arange(nv), nt * per_step)
        obs_time = np.tile(sites_t, nv)
        obs_xy = np.tile(sites_xy, (nv, 1))
        X = np.tile(sites_X, (nv, 1))
    else:
        if per_step is not None:
            obs_time = np.repeat(np.arange(nt), per_step)
        else:
            obs_time = rng.integers(0, nt, size=m_total)
        m = obs_time.shape[0]
        obs_xy = rng.uniform(0.0, 1.0, size=(m, 2))
        if m % nv:
            raise ValueError("observation count must be a multiple of nv")
        obs_var = np.repeat(np.arange(nv), m // nv)
        X = np.ones((m, nr))
        if nr > 1:
            X[:, 1:] = rng.standard_normal((m, nr - 1))
    obs_tri = locate(obs_xy)

    if theta0 is None:
        per_var = [math.log(0.3), math.log(3.0), 0.0, math.log(4.0)]
        lam = rng.uniform(-lam_range, lam_range, size=nv * (nv - 1) // 2)
        theta0 = np.array(per_var * nv + list(lam), dtype=np.float64)
    theta0 = np.asarray(theta0, dtype=np.float64)
    assert theta0.shape[0] == theta_layout(nv)

    noise_prec = np.exp(theta0[3:4 * nv:4])
    y = np.zeros(obs_var.shape[0])
    for v in range(nv):
        sel = obs_var == v
        signal = _true_field(v, obs_xy[sel], obs_time[sel], nt)
        if likelihood == "gaussian":
            y[sel] = (signal + X[sel].sum(axis=1)
                      + rng.standard_normal(int(sel.sum())) / math.sqrt(noise_prec[v]))
        elif likelihood == "poisson":
            y[sel] = rng.poisson(np.exp(0.5 * signal + 0.2 * X[sel].sum(axis=1)))
        else:
            raise ValueError(likelihood)

    return Problem(name=name, nv=nv, ns=ns, nt=nt, nr=nr,
                   nodes=np.ascontiguousarray(nodes, dtype=np.float64),
                   tri=np.ascontiguousarray(tri, dtype=np.int32),
                   obs_var=obs_var.astype(np.int32), obs_time=obs_time.astype(np.int32),
                   obs_xy=np.ascontiguousarray(obs_xy, dtype=np.float64),
                   obs_tri=obs_tri.astype(np.int32),
                   X=np.ascontiguousarray(X, dtype=np.float64),
                   y=y.astype(np.float64), theta0=theta0)


# Workload recipes.  c1..c5 mirror the sizes of the benchmark configurations
# (univariate 10x10 grid / 32x32 grid, trivariate coregional 32x32 grid,
# trivariate Delaunay 2000-node mesh); the t_* entries are small test cases
# that still span several kernel tiles and a ragged tail.
CONFIGS = {
    # univariate, ns=100, nt=8, nr=2, N=802; m=400 uniform in space and time
    "c1": dict(nv=1, mesh=("grid", 10), nt=8, nr=2, seed=1, m_total=400),
    # univariate, ns=1024, nt=64, nr=4, N=65,540; 1024 observations per step
    "c2": dict(nv=1, mesh=("grid", 32), nt=64, nr=4, seed=2, per_step=1024),
    # c2 with 8 time steps (same block size b=1024; for kernel profiling)
    "c2s": dict(nv=1, mesh=("grid", 32), nt=8, nr=4, seed=2, per_step=1024),
    # c2 with 2 time steps: one Schur update of b=1024 blocks per factorisation,
    # small enough on the device for multi-pass kernel captures
    "c2p": dict(nv=1, mesh=("grid", 32), nt=2, nr=4, seed=2, per_step=1024),
    # trivariate coregional, b=3072, nt=48, a=6, N=147,462; 300 sites per step
    "c3": dict(nv=3, mesh=("grid", 32), nt=48, nr=2, seed=3, per_step=300,
               shared_sites=True),
    # c3 with 2 time steps: one Schur update of b=3072 blocks per factorisation,
    # small enough on the device for multi-pass kernel captures
    "c3p": dict(nv=3, mesh=("grid", 32), nt=2, nr=2, seed=3, per_step=300, shared_sites=True),
    # trivariate coregional on a 2000-node Delaunay mesh, b=6000, N=288,006
    "c5": dict(nv=3, mesh=("delaunay", 2000), nt=48, nr=2, seed=5, per_step=1000,
               shared_sites=True),
    # c5 with 2 time steps: the b=6000 Schur-update products of c5 at about 11 GB on the device
    "c5p": dict(nv=3, mesh=("delaunay", 2000), nt=2, nr=2, seed=5, per_step=1000, shared_sites=True),
    # reduced copy of c5 with 200 mesh nodes (b=600, N=28,806)
    "c5r": dict(nv=3, mesh=("delaunay", 200), nt=48, nr=2, seed=5, per_step=100,
                shared_sites=True),
    # small test cases
    "t_uni": dict(nv=1, mesh=("grid", 6), nt=5, nr=2, seed=11, m_total=90),
    "t_uni_ragged": dict(nv=1, mesh=("grid", 9, 11), nt=7, nr=3, seed=12, m_total=300),
    "t_coreg2": dict(nv=2, mesh=("grid", 5), nt=4, nr=2, seed=13, per_step=12,
                     shared_sites=True),
    "t_coreg3": dict(nv=3, mesh=("grid", 6), nt=5, nr=2, seed=14, per_step=15,
                     shared_sites=True),
    "t_coreg3_del": dict(nv=3, mesh=("delaunay", 40), nt=4, nr=2, seed=15, per_step=20,
                         shared_sites=True),
    "t_uni_nt1": dict(nv=1, mesh=("grid", 7), nt=1, nr=1, seed=16, m_total=30),
    "t_uni_mid": dict(nv=1, mesh=("grid", 17), nt=12, nr=2, seed=17, per_step=200),
    # count data (Poisson likelihood, log link) for the Laplace approximation
    "t_pois": dict(nv=1, mesh=("grid", 6), nt=5, nr=2, seed=21, m_total=90, likelihood="poisson"),
    "t_pois_coreg3": dict(nv=3, mesh=("grid", 5), nt=4, nr=2, seed=22, per_step=12, shared_sites=True,
                          likelihood="poisson"),
    "t_pois_mid": dict(nv=1, mesh=("grid", 17), nt=12, nr=2, seed=23, per_step=200, likelihood="poisson"),
    "t_pois_coreg3_mid": dict(nv=3, mesh=("grid", 12), nt=10, nr=2, seed=24, per_step=60, shared_sites=True,
                              likelihood="poisson"),
    # univariate count model at the working size (b = 1024, nt = 64)
    "c2pois": dict(nv=1, mesh=("grid", 32), nt=64, nr=4, seed=25, per_step=1024, likelihood="poisson"),
    "t_coreg3_mid": dict(nv=3, mesh=("grid", 12), nt=10, nr=2, seed=18, per_step=60,
                         shared_sites=True),
}


# The uneven batch of univariate instances (ns in {256, 512, 1024} on 16x16,
# 16x32 and 32x32 grids, nt in {16, 32, 64}; one site per mesh node and
# time step on average), evaluated together through one call.
for _gx, _gy in ((16, 16), (16, 32), (32, 32)):
    for _nt in (16, 32, 64):
        CONFIGS[f"c4b_{_gx * _gy}_{_nt}"] = dict(nv=1, mesh=("grid", _gx, _gy), nt=_nt, nr=4,
                                                 seed=40 + _nt + _gx * _gy, per_step=_gx * _gy)


def problem_from_config(name: str, **overrides) -> Problem:
    spec = dict(CONFIGS[name])
    spec.update(overrides)
    return make_problem(name, **spec)
