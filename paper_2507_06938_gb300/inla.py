"""The INLA steps above the BTA path (Section II-B): the hyperparameter mode,
the Gaussian approximation of the hyperparameter marginals, and the latent
marginals at the mode.

  * Mode: theta* = argmin_theta -f_obj(theta) (Eq. 9) by BFGS (Nocedal and
    Wright, Numerical Optimization, Algorithm 6.1) with a line search that
    enforces the strong Wolfe conditions (their Algorithms 3.5 and 3.6).  The
    gradient comes from the adjoint form of Eq. 8 (bta_fobj_grad), or, as in
    the paper, from the central differences of Eq. 10, whose 2 dim(theta) + 1
    points go through one batched fobj_eval call.
  * Hyperparameter marginals: Gaussian, with covariance (-H)^{-1} where H is
    the Hessian of f_obj at theta*, here the central differences of the
    gradient (2 dim(theta) points in one batched call), symmetrised.
  * Latent marginals at theta*: means mu and variances diag(Q_c^{-1}) from
    the selected inversion.

Host logic only: every evaluation of f_obj, its gradient, mu and the
selected inverse runs through the C ABI of libbta.
"""

from __future__ import annotations

import dataclasses

import numpy as np

from . import bta


class Objective:
    """f_obj of one model on one GPU context, with batched evaluation.

    gradient: "adjoint" (bta_fobj_grad) or "fd" (Eq. 10 in one batch).
    batch: theta points per group of the context (default 2 dim + 1, which
    holds one stencil or one Hessian column set in a single group).  Single
    points go to a second context of batch 1: a group smaller than its
    context's batch factors Q_p and Q_c as two chains (their storage ranges
    are not adjacent), a full group as one."""

    def __init__(self, problem, precision: int = bta.BTA_MIXED, gradient: str = "adjoint", h: float = 1e-3,
                 batch: int | None = None, stream=None):
        import torch
        if gradient not in ("adjoint", "fd"):
            raise ValueError("gradient must be 'adjoint' or 'fd'")
        self.problem = problem
        self.dim = int(np.asarray(problem.theta0).shape[0])
        self.gradient = gradient
        self.h = float(h)
        self.batch = int(batch) if batch else 2 * self.dim + 1
        self.model = bta.BtaModel(problem)
        self.ctx = bta.BtaContext(problem.nt, problem.b, problem.a, precision, stream, self.batch)
        self._ctx1 = None
        self._precision, self._stream = precision, stream
        self._torch = torch
        self.n_eval = 0

    def _context(self, count: int):
        if count != 1 or self.batch == 1:
            return self.ctx
        if self._ctx1 is None:
            p = self.problem
            self._ctx1 = bta.BtaContext(p.nt, p.b, p.a, self._precision, self._stream, 1)
        return self._ctx1

    def _dev(self, x):
        return self._torch.as_tensor(np.ascontiguousarray(x, dtype=np.float64), device="cuda")

    def values(self, thetas) -> np.ndarray:
        """f_obj at each row of thetas (one batched call)."""
        th = np.atleast_2d(np.asarray(thetas, dtype=np.float64))
        f = self._torch.zeros(th.shape[0], dtype=self._torch.float64, device="cuda")
        ctx = self._context(th.shape[0])
        ctx.fobj_eval(self.model, self._dev(th), f)
        ctx.sync()
        self.n_eval += th.shape[0]
        return f.cpu().numpy()

    def grads(self, thetas):
        """(f, gradient) at each row of thetas by the adjoint form."""
        th = np.atleast_2d(np.asarray(thetas, dtype=np.float64))
        t = self._torch
        f = t.zeros(th.shape[0], dtype=t.float64, device="cuda")
        g = t.zeros(th.shape, dtype=t.float64, device="cuda")
        ctx = self._context(th.shape[0])
        ctx.fobj_grad(self.model, self._dev(th), f, g)
        ctx.sync()
        self.n_eval += th.shape[0]
        return f.cpu().numpy(), g.cpu().numpy()

    def value_grad(self, theta):
        theta = np.asarray(theta, dtype=np.float64)
        if self.gradient == "adjoint":
            f, g = self.grads(theta[None, :])
            return float(f[0]), g[0]
        pts = stencil(theta, self.h)
        f = self.values(pts)
        return float(f[0]), fd_from_stencil(f, self.h)

    def latent_marginals(self, theta):
        """Conditional means mu and marginal variances diag(Q_c^{-1}) at theta."""
        t = self._torch
        N = self.problem.N
        f = t.zeros(1, dtype=t.float64, device="cuda")
        mu = t.zeros((1, N), dtype=t.float64, device="cuda")
        ctx = self._context(1)
        ctx.fobj_eval(self.model, self._dev(np.asarray(theta)[None, :]), f, mu)
        which = 2 * 0 + bta.BTA_QC          # slot 0 holds the last (only) point
        ctx.selinv(which)
        var = t.zeros(N, dtype=t.float64, device="cuda")
        ctx.selinv_diag(which, var)
        ctx.sync()
        self.n_eval += 1
        return mu[0].cpu().numpy(), var.cpu().numpy()

    def close(self):
        if self._ctx1 is not None:
            self._ctx1.close()
        self.ctx.close()
        self.model.close()


class DistributedObjective:
    """An objective whose batched evaluations are split over the ranks of a
    torch.distributed process group: the independent function evaluations
    of Section IV-D.1 (the 2 dim + 1 stencil points of Eq. 10, the Hessian
    columns), each rank on its own GPU.  Rank r evaluates rows r, r + W,
    r + 2 W, ... of every batch through its local objective; the values (and
    gradients) are then combined on the host by one all-reduce of a
    zero-filled array in which every row is written by exactly one rank (the
    sum is the gather of the paper's reduction, exact).  Every rank returns
    the full result, so BFGS runs identically everywhere.  With gloo the
    exchange is a host collective; the data path needs none."""

    def __init__(self, local, group=None):
        import torch.distributed as dist
        self.local = local
        self.dist = dist
        self.group = group
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)
        self.problem = local.problem
        self.dim = local.dim
        self.gradient = local.gradient
        self.h = local.h
        self.n_eval = 0

    def _mine(self, count: int) -> np.ndarray:
        return np.arange(self.rank, count, self.world)

    def _combine(self, full: np.ndarray) -> np.ndarray:
        import torch
        t = torch.as_tensor(full, dtype=torch.float64)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.SUM, group=self.group)
        return t.numpy()

    def values(self, thetas) -> np.ndarray:
        th = np.atleast_2d(np.asarray(thetas, dtype=np.float64))
        idx = self._mine(th.shape[0])
        full = np.zeros(th.shape[0])
        if idx.size:
            full[idx] = self.local.values(th[idx])
            self.n_eval += idx.size
        return self._combine(full)

    def grads(self, thetas):
        th = np.atleast_2d(np.asarray(thetas, dtype=np.float64))
        idx = self._mine(th.shape[0])
        full = np.zeros((th.shape[0], 1 + th.shape[1]))
        if idx.size:
            f, g = self.local.grads(th[idx])
            full[idx, 0] = f
            full[idx, 1:] = g
            self.n_eval += idx.size
        out = self._combine(full)
        return out[:, 0], out[:, 1:]

    def value_grad(self, theta):
        theta = np.asarray(theta, dtype=np.float64)
        if self.gradient == "adjoint":
            f, g = self.grads(theta[None, :])
            return float(f[0]), g[0]
        pts = stencil(theta, self.h)
        f = self.values(pts)
        return float(f[0]), fd_from_stencil(f, self.h)

    def latent_marginals(self, theta):
        return self.local.latent_marginals(theta)


def stencil(theta, h: float) -> np.ndarray:
    """The 2 dim + 1 points of Eq. 10: theta, then theta + h e_i, theta - h e_i."""
    theta = np.asarray(theta, dtype=np.float64)
    pts = [theta]
    for i in range(theta.shape[0]):
        e = np.zeros_like(theta)
        e[i] = h
        pts += [theta + e, theta - e]
    return np.stack(pts)


def fd_from_stencil(f, h: float) -> np.ndarray:
    """Central differences of Eq. 10 from f at the points of `stencil`."""
    f = np.asarray(f)
    d = (f.shape[0] - 1) // 2
    return np.array([(f[1 + 2 * i] - f[2 + 2 * i]) / (2.0 * h) for i in range(d)])


# ----------------------------------------------------------------------------- BFGS on -f_obj


def _line_search(phi, phi0, dphi0, c1=1e-4, c2=0.9, alpha1=1.0, alpha_max=50.0, max_iter=25):
    """Step length satisfying the strong Wolfe conditions for phi(alpha) =
    -f_obj(theta + alpha p): bracketing (Algorithm 3.5) then zoom (Algorithm
    3.6) with safeguarded quadratic interpolation.  phi(alpha) returns
    (value, derivative, payload).  Returns (alpha, value, payload) or None."""
    best = None
    prev = (0.0, phi0, dphi0, None)
    a = alpha1

    def zoom(lo, hi):
        nonlocal best
        for _ in range(max_iter):
            (al, vl, dl, _), (ah, vh, _, _) = lo, hi
            w = ah - al
            denom = 2.0 * (vh - vl - dl * w)
            a_q = al - dl * w * w / denom if denom > 0 else al + 0.5 * w
            lo_b, hi_b = sorted((al + 0.1 * w, ah - 0.1 * w))
            aj = min(max(a_q, lo_b), hi_b)
            vj, dj, pj = phi(aj)
            if vj <= phi0 + c1 * aj * dphi0 and (best is None or vj < best[1]):
                best = (aj, vj, pj)
            if vj > phi0 + c1 * aj * dphi0 or vj >= vl:
                hi = (aj, vj, dj, pj)
            else:
                if abs(dj) <= -c2 * dphi0:
                    return aj, vj, pj
                if dj * (ah - al) >= 0:
                    hi = lo
                lo = (aj, vj, dj, pj)
        return best

    for i in range(max_iter):
        v, d, pay = phi(a)
        if v <= phi0 + c1 * a * dphi0 and (best is None or v < best[1]):
            best = (a, v, pay)
        if v > phi0 + c1 * a * dphi0 or (i > 0 and v >= prev[1]):
            return zoom(prev, (a, v, d, pay))
        if abs(d) <= -c2 * dphi0:
            return a, v, pay
        if d >= 0:
            return zoom((a, v, d, pay), prev)
        prev = (a, v, d, pay)
        a = min(2.0 * a, alpha_max)
    return best


@dataclasses.dataclass
class BfgsResult:
    theta: np.ndarray
    f: float
    grad: np.ndarray
    n_iter: int
    converged: bool
    history: list


def bfgs(value_grad, theta0, gtol: float = 1e-3, ftol: float = 1e-13, max_iter: int = 100) -> BfgsResult:
    """Maximise f_obj: BFGS on phi = -f_obj with an inverse-Hessian update
    H <- (I - rho s y^T) H (I - rho y s^T) + rho s s^T, rho = 1 / (y^T s),
    skipped when y^T s is not positive; H0 = I, rescaled by y^T s / y^T y
    before the first update.  value_grad(theta) -> (f_obj, gradient).
    Stops when max |gradient| <= gtol, or when an iteration changes phi by
    less than ftol |phi| (the noise floor of the evaluations)."""
    x = np.asarray(theta0, dtype=np.float64).copy()
    f, g = value_grad(x)
    phi, gphi = -f, -np.asarray(g, dtype=np.float64)
    n = x.shape[0]
    Hinv = np.eye(n)
    history = [(x.copy(), f)]
    for it in range(max_iter):
        if np.max(np.abs(gphi)) <= gtol:
            return BfgsResult(x, f, -gphi, it, True, history)
        p = -Hinv @ gphi
        if gphi @ p >= 0:                      # not a descent direction: restart
            Hinv = np.eye(n)
            p = -gphi

        def line(alpha, x=x, p=p):
            fv, gv = value_grad(x + alpha * p)
            gv = np.asarray(gv, dtype=np.float64)
            return -fv, float(-gv @ p), (fv, gv)

        alpha1 = 1.0 if it > 0 else min(1.0, 1.0 / max(np.max(np.abs(gphi)), 1e-300))
        res = _line_search(line, phi, float(gphi @ p), alpha1=alpha1)
        if res is None:
            return BfgsResult(x, f, -gphi, it, False, history)
        alpha, phi_new, (f_new, g_new) = res
        s = alpha * p
        y = -g_new - gphi
        ys = float(y @ s)
        if ys > 1e-12 * np.linalg.norm(y) * np.linalg.norm(s):
            if it == 0:
                Hinv = (ys / float(y @ y)) * np.eye(n)
            rho = 1.0 / ys
            V = np.eye(n) - rho * np.outer(s, y)
            Hinv = V @ Hinv @ V.T + rho * np.outer(s, s)
        done = abs(phi_new - phi) <= ftol * abs(phi)
        x, f, phi, gphi = x + s, f_new, phi_new, -g_new
        history.append((x.copy(), f))
        if done:
            return BfgsResult(x, f, -gphi, it + 1, np.max(np.abs(gphi)) <= gtol, history)
    return BfgsResult(x, f, -gphi, max_iter, np.max(np.abs(gphi)) <= gtol, history)


def hessian_from_gradients(grads, theta, h: float = 1e-3) -> np.ndarray:
    """Hessian of f_obj at theta by central differences of the gradient,
    H[:, j] = (g(theta + h e_j) - g(theta - h e_j)) / 2h, symmetrised.
    grads(points) -> (f, gradients) for the 2 dim points in one call."""
    theta = np.asarray(theta, dtype=np.float64)
    d = theta.shape[0]
    pts = stencil(theta, h)[1:]
    _, G = grads(pts)
    G = np.asarray(G)
    H = np.stack([(G[2 * j] - G[2 * j + 1]) / (2.0 * h) for j in range(d)], axis=1)
    return 0.5 * (H + H.T)


@dataclasses.dataclass
class InlaResult:
    mode: BfgsResult
    hessian: np.ndarray
    cov_theta: np.ndarray | None      # (-H)^{-1}; None when -H is not positive definite
    sd_theta: np.ndarray | None
    mu: np.ndarray                    # latent means at the mode
    var: np.ndarray                   # latent marginal variances at the mode


def inla(objective, theta0=None, gtol: float = 1e-3, max_iter: int = 100, h_hess: float = 1e-3) -> InlaResult:
    """Mode of the hyperparameters, their Gaussian marginals, and the latent
    marginals at the mode for an `Objective`."""
    theta0 = objective.problem.theta0 if theta0 is None else theta0
    mode = bfgs(objective.value_grad, theta0, gtol=gtol, max_iter=max_iter)
    H = hessian_from_gradients(objective.grads, mode.theta, h_hess)
    cov = sd = None
    try:
        Lc = np.linalg.cholesky(-H)
        Linv = np.linalg.inv(Lc)
        cov = Linv.T @ Linv
        sd = np.sqrt(np.diag(cov))
    except np.linalg.LinAlgError:
        pass
    mu, var = objective.latent_marginals(mode.theta)
    return InlaResult(mode, H, cov, sd, mu, var)
