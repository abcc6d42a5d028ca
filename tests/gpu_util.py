"""Helpers shared by the GPU parity tests: run the CUDA path through the
C ABI on a synth problem and fetch results as numpy arrays."""

from __future__ import annotations

import numpy as np

import synth
from oracle import model as omodel


def need_gpu():
    import pytest
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def build_lib():
    from paper_2507_06938_gb300 import _build
    _build.build()


def dev(x):
    import torch
    return torch.as_tensor(np.ascontiguousarray(x, dtype=np.float64), device="cuda")


def blocks_of(ctx, which, store, n, b, a):
    """Copy all BTA blocks of one storage to host numpy (row-major arrays of
    the matrices themselves)."""
    from paper_2507_06938_gb300 import bta
    D = np.stack([ctx.block(which, store, bta.BTA_BLK_D, i).cpu().numpy() for i in range(n)])
    B = (np.stack([ctx.block(which, store, bta.BTA_BLK_B, i).cpu().numpy() for i in range(n - 1)])
         if n > 1 else np.zeros((0, b, b)))
    R = np.stack([ctx.block(which, store, bta.BTA_BLK_R, i).cpu().numpy() for i in range(n)]) if a else np.zeros((n, 0, b))
    T = ctx.block(which, store, bta.BTA_BLK_T).cpu().numpy() if a else np.zeros((0, 0))
    return dict(D=D, B=B, R=R, T=T)


class GpuCase:
    """A model + context for one problem; params given directly or by theta."""

    def __init__(self, problem, precision=0, stream=None, batch=1):
        from paper_2507_06938_gb300 import bta
        self.p = problem
        self.model = bta.BtaModel(problem)
        self.ctx = bta.BtaContext(problem.nt, problem.b, problem.a, precision, stream, batch)

    def assemble(self, params: omodel.Params, which):
        self.params_dev = dev(omodel.params_vector(params))
        self.ctx.assemble(self.model, self.params_dev, which)


def problem(name, **kw):
    return synth.problem_from_config(name, **kw)


def rel_max(a, b):
    """max |a - b| / max |b| (0 if both empty)."""
    a = np.asarray(a)
    b = np.asarray(b)
    if b.size == 0:
        return 0.0
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))
