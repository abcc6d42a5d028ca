"""Measurement aids of the C ABI: bta_profile / bta_profile_read (events
around the Schur-update products of the factorisation) and
bta_profile_phases (events at the phase boundaries of a gradient group).
Checks that the phases cover the step: each positive, their sum within a few
percent of the whole call timed on the same stream, for the graph capture
and its replays; the product events count two launches
per factorisation step and matrix group with b^3 nominal flops per matrix;
and the state errors.  Profiling leaves the results unchanged."""

import numpy as np
import pytest

from gpu_util import build_lib, dev, need_gpu, problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _setup():
    need_gpu()
    build_lib()


@pytest.mark.parametrize("precision", [0, 2])
def test_phases_cover_the_gradient_step(precision, monkeypatch):
    import torch
    from paper_2507_06938_gb300 import bta
    monkeypatch.setenv("BTA_OZ_MIN", "64")
    p = problem("t_coreg3_mid")
    B = 3
    stream = torch.cuda.Stream()
    model = bta.BtaModel(p)
    ctx = bta.BtaContext(p.nt, p.b, p.a, precision, stream, B)
    dim = p.theta0.shape[0]
    thetas = dev(np.stack([p.theta0 + 0.01 * j for j in range(B)]))
    f = torch.zeros(B, dtype=torch.float64, device="cuda")
    g = torch.zeros((B, dim), dtype=torch.float64, device="cuda")
    with torch.cuda.stream(stream):
        ctx.fobj_grad(model, thetas, f, g)
        ctx.sync()
        f0, g0 = f.clone(), g.clone()
        with pytest.raises(bta.BtaError) as e:
            ctx.profile_phases()
        assert e.value.code == bta.BTA_ERR_STATE
        ctx.profile(True)
        with pytest.raises(bta.BtaError) as e:
            ctx.profile_phases()
        assert e.value.code == bta.BTA_ERR_STATE
        for _ in range(3):                 # direct, graph capture, graph replay
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ctx.fobj_grad(model, thetas, f, g)
            e1.record(stream)
            e1.synchronize()
            ph = ctx.profile_phases()
            total = e0.elapsed_time(e1)
            assert set(ph) == set(bta.PHASE_NAMES)
            assert all(v > 0 for v in ph.values()), ph
            assert sum(ph.values()) <= total * 1.02 + 0.05
            assert sum(ph.values()) >= total * 0.85 - 0.2, (ph, total)
        ms, launches, flops = ctx.profile_read()
        assert launches == 2 * (p.nt - 1) and ms > 0
        assert abs(flops - launches * 2 * B * float(p.b) ** 3) <= 1e-9 * flops
        ctx.profile(False)
        ctx.sync()
    # the same values as unprofiled (the graph replay may sum in another order)
    assert torch.allclose(f, f0, rtol=1e-12, atol=0) and torch.allclose(g, g0, rtol=1e-9, atol=1e-12)
    ctx.close()
    model.close()
