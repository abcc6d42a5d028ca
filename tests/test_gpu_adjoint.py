"""Adjoint gradient of f_obj on the GPU (selected inverses + trace kernels)
against the oracle's analytic gradient (dense inverses, complex-step model
derivatives) and against central finite differences of the oracle f_obj
(Eq. 10).  Bounds: 1e-7 relative to max(|g_k|, 1e-3 |g|_inf) in FP64 (sums of
traces of size ~N with FP64 rounding); 1e-5 in mixed precision (the
selected-inverse error of the mixed path) and against finite differences."""

import numpy as np
import pytest

from oracle import fobj as ofobj

from gpu_util import GpuCase, build_lib, dev, need_gpu, problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _setup():
    need_gpu()
    build_lib()


def _rel(g, ref):
    scale = np.maximum(np.abs(ref), 1e-3 * np.max(np.abs(ref)))
    return float(np.max(np.abs(g - ref) / scale))


@pytest.mark.parametrize("name,precision,batch", [("t_uni", 0, 1), ("t_uni_ragged", 0, 2), ("t_coreg2", 0, 3),
                                                  ("t_coreg3", 0, 2), ("t_coreg3", 1, 2), ("t_uni_mid", 1, 1)])
def test_adjoint_gradient(name, precision, batch, monkeypatch):
    import torch
    monkeypatch.setenv("BTA_OZ_MIN", "64")
    p = problem(name)
    rng = np.random.default_rng(4)
    thetas = p.theta0 + 0.1 * rng.standard_normal((3, p.theta0.shape[0]))
    run = GpuCase(p, precision=precision, batch=batch)
    f = torch.zeros(3, dtype=torch.float64, device="cuda")
    g = torch.zeros((3, p.theta0.shape[0]), dtype=torch.float64, device="cuda")
    run.ctx.fobj_grad(run.model, dev(thetas), f, g)
    run.ctx.sync()
    tol = 1e-7 if precision == 0 else 1e-5
    for j in range(3):
        ref = ofobj.grad_adjoint(p, thetas[j])
        assert _rel(g[j].cpu().numpy(), ref) < tol, (j, g[j].cpu().numpy(), ref)
        assert abs(f[j].item() - ofobj.f_obj(p, thetas[j])) < 1e-7 * abs(f[j].item())
    gfd = ofobj.fd_gradient(p, thetas[0], h=1e-4, tier="dense")
    assert _rel(g[0].cpu().numpy(), gfd) < 1e-5


def test_autograd_function():
    import torch
    from paper_2507_06938_gb300.autograd import fobj
    p = problem("t_coreg2")
    run = GpuCase(p, batch=2)
    th = torch.tensor(p.theta0 + 0.05, dtype=torch.float64, device="cuda", requires_grad=True)
    val = fobj(th, run.ctx, run.model)
    val.backward()
    ref = ofobj.grad_adjoint(p, p.theta0 + 0.05)
    assert _rel(th.grad.cpu().numpy(), ref) < 1e-7
