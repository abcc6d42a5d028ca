"""The host-buffer entry point bta_fobj_grad_host (thetas in host memory,
f, gradient and marginal variances back in host memory) gives the results
of the device-pointer path: bta_fobj_grad and bta_selinv_diag on the same
context shape, for a number of thetas that leaves a partial last group."""

import numpy as np
import pytest

from gpu_util import build_lib, dev, need_gpu, problem

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", [0, 2])
def test_host_buffers_match_device_path(precision):
    need_gpu()
    build_lib()
    import torch
    from paper_2507_06938_gb300 import bta
    p = problem("t_coreg3")
    rng = np.random.default_rng(31)
    thetas = np.ascontiguousarray(p.theta0 + 0.05 * rng.standard_normal((3, p.theta0.shape[0])))
    model = bta.BtaModel(p)
    ctx = bta.BtaContext(p.nt, p.b, p.a, precision, None, 2)
    f_h = torch.zeros(3, dtype=torch.float64).pin_memory()
    g_h = torch.zeros((3, thetas.shape[1]), dtype=torch.float64).pin_memory()
    v_h = np.zeros((3, p.N))
    ctx.fobj_grad_host(model, torch.as_tensor(thetas).pin_memory(), f_h, g_h, v_h)
    for j in range(3):
        ref = bta.BtaContext(p.nt, p.b, p.a, precision, None, 1)
        f = torch.zeros(1, dtype=torch.float64, device="cuda")
        g = torch.zeros((1, thetas.shape[1]), dtype=torch.float64, device="cuda")
        v = torch.zeros(p.N, dtype=torch.float64, device="cuda")
        ref.fobj_grad(model, dev(thetas[j:j + 1]), f, g)
        ref.selinv_diag(bta.BTA_QC, v)
        ref.sync()
        assert abs(f_h[j].item() - f.item()) <= 1e-12 * abs(f.item())
        assert np.max(np.abs(g_h[j].numpy() - g[0].cpu().numpy())) <= 1e-10 * np.max(np.abs(g.cpu().numpy()))
        assert np.max(np.abs(v_h[j] - v.cpu().numpy())) <= 1e-12 * np.max(np.abs(v.cpu().numpy()))
        ref.close()
    with pytest.raises(TypeError):
        ctx.fobj_grad_host(model, dev(thetas), f_h, g_h)
    ctx.close()
    model.close()
