"""Non-Gaussian likelihood (bta_fobj_laplace): Newton iterations for the mode
x* of the latent field, each an assembly of Q_c(x_k) = Q_p + A^T D(x_k) A
with per-observation weights, a BTA factorisation and a solve, then f_obj at
x* through the Laplace approximation (Section II-A.3, Eqs. 4, 7, 8).

Against the oracle (oracle/laplace.py, pinned by tests/test_oracle_laplace.py)
on Poisson count data: f, the mode and the convergence of the last Newton
step; FP64 at the FP64 bounds (f 1e-10 of the log-determinant scale, x* 1e-9),
the 35-bit mixed path at its log-det target (1e-8) and the 49-bit one at 1e-9.
The Gaussian likelihood through the same entry point reproduces fobj_eval
(the Taylor expansion is exact, one step reaches mu).  12 Newton steps: the
oracle needs 7 to 9 from x = 0 on these cases (quadratic convergence)."""

import numpy as np
import pytest

from oracle import fobj as ofobj
from oracle import laplace as olap

from gpu_util import build_lib, dev, need_gpu, problem, rel_max

pytestmark = pytest.mark.gpu

ITERS = 12


@pytest.fixture(scope="module", autouse=True)
def _setup():
    need_gpu()
    build_lib()


def _run(p, precision, thetas, lik, iters=ITERS, batch=1):
    import torch
    from paper_2507_06938_gb300 import bta
    model = bta.BtaModel(p)
    ctx = bta.BtaContext(p.nt, p.b, p.a, precision, None, batch)
    k = thetas.shape[0]
    f = torch.zeros(k, dtype=torch.float64, device="cuda")
    x = torch.zeros((k, p.N), dtype=torch.float64, device="cuda")
    step = torch.zeros(k, dtype=torch.float64, device="cuda")
    ctx.fobj_laplace(model, dev(thetas), lik, iters, f, x, step)
    ctx.sync()
    out = f.cpu().numpy(), x.cpu().numpy(), step.cpu().numpy()
    ctx.close()
    model.close()
    return out


@pytest.mark.parametrize("name,precision,tol", [("t_pois", 0, 1e-10), ("t_pois_coreg3", 0, 1e-10),
                                                ("t_pois_mid", 1, 1e-8), ("t_pois_coreg3_mid", 1, 1e-8),
                                                ("t_pois_mid", 2, 1e-9), ("t_pois_coreg3_mid", 2, 1e-9),
                                                ("t_pois_coreg3_mid", 0, 1e-10)])
def test_poisson_laplace_matches_oracle(name, precision, tol, monkeypatch):
    from paper_2507_06938_gb300 import bta
    monkeypatch.setenv("BTA_OZ_MIN", "64")   # small cases through the tensor-core products
    p = problem(name)
    rng = np.random.default_rng(41)
    thetas = np.stack([p.theta0, p.theta0 + 0.05 * rng.standard_normal(p.theta0.shape)])
    f, x, step = _run(p, precision, thetas, bta.BTA_LIK_POISSON, batch=2)
    for j in range(2):
        ref = olap.laplace_terms(p, thetas[j], "poisson")
        scale = abs(ref["logdet_p"]) + abs(ref["logdet_c"])
        print(name, precision, j, "f", f[j], ref["f"], "rel", abs(f[j] - ref["f"]) / scale, "step", step[j])
        assert abs(f[j] - ref["f"]) <= tol * scale
        assert rel_max(x[j], ref["x"]) <= (1e-9 if precision == 0 else 1e-7)
        assert step[j] <= 1e-9 * max(1.0, np.max(np.abs(ref["x"])))


def test_gaussian_likelihood_reproduces_fobj_eval():
    import torch
    from paper_2507_06938_gb300 import bta
    p = problem("t_coreg3")
    thetas = np.stack([p.theta0, p.theta0 + 0.02])
    f, x, step = _run(p, 0, thetas, bta.BTA_LIK_GAUSSIAN, iters=2, batch=2)
    for j in range(2):
        ref = ofobj.f_obj_terms(p, thetas[j], tier="dense")
        assert abs(f[j] - ref["f"]) <= 1e-10 * abs(ref["f"])
        assert rel_max(x[j], ref["mu"]) <= 1e-10
        assert step[j] <= 1e-9 * np.max(np.abs(ref["mu"]))


def test_partial_group_and_bad_arguments():
    import torch
    from paper_2507_06938_gb300 import bta
    p = problem("t_pois")
    rng = np.random.default_rng(42)
    thetas = p.theta0 + 0.05 * rng.standard_normal((3, p.theta0.shape[0]))
    f3, x3, _ = _run(p, 0, thetas, bta.BTA_LIK_POISSON, batch=2)
    f1, x1, _ = _run(p, 0, thetas[2:3], bta.BTA_LIK_POISSON, batch=1)
    assert abs(f3[2] - f1[0]) <= 1e-11 * abs(f1[0])
    assert rel_max(x3[2], x1[0]) <= 1e-11
    model = bta.BtaModel(p)
    ctx = bta.BtaContext(p.nt, p.b, p.a, 0, None, 1)
    f = torch.zeros(1, dtype=torch.float64, device="cuda")
    th = dev(p.theta0[None, :])
    for lik, iters in ((7, 5), (bta.BTA_LIK_POISSON, 0)):
        with pytest.raises(bta.BtaError) as e:
            ctx.fobj_laplace(model, th, lik, iters, f)
        assert e.value.code == bta.BTA_ERR_ARG
    ctx.close()
    model.close()
