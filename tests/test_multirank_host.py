"""Host logic of the multi-rank benchmark on CPU ranks (gloo, world size 2):
every rank draws its own stencils (weak scaling over independent theta points,
no exchange on the data path), the job time is the slowest rank's, and the
job throughput counts the points of all ranks."""

import os
import socket

import numpy as np
import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    import bench
    import synth
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        p = synth.problem_from_config("t_uni")
        stencils = bench.thetas_for(p, 3, rank)
        # per-rank timings: rank 1 is slower on the first entry, rank 0 on the second
        mine = [10.0 + rank, 5.0 - rank]
        worst = bench.max_over_ranks(mine, dist, "cpu")
        q.put((rank, np.stack(stencils), worst))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_ranks_shard_points_and_take_the_slowest_time():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    out = {}
    for _ in range(2):
        rank, st, worst = q.get(timeout=120)
        out[rank] = (st, worst)
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    s0, w0 = out[0]
    s1, w1 = out[1]
    # same shape (steps x (2 dim + 1) x dim), different points on different ranks
    assert s0.shape == s1.shape and s0.shape[1] == 2 * s0.shape[2] + 1
    assert np.min(np.abs(s0 - s1)) > 0.0
    # every stencil is a central-difference stencil around its first point
    h = s0[0, 1, 0] - s0[0, 0, 0]
    assert np.allclose(s0[:, 1::2] - s0[:, :1], h * np.eye(s0.shape[2]))
    assert np.allclose(s0[:, 2::2] - s0[:, :1], -h * np.eye(s0.shape[2]))
    # the job time is the slowest rank's, on every rank
    assert w0 == w1 == [11.0, 5.0]


def test_job_throughput_counts_all_ranks():
    import bench
    assert bench.job_throughput(steps=5, world=4, batch=9, ms=1000.0) == pytest.approx(180.0)
    assert bench.job_throughput(steps=1, world=1, batch=9, ms=500.0) == pytest.approx(18.0)


class _OracleObjective:
    """An objective with the interface of inla.Objective evaluated by the CPU
    oracle (f_obj and its block-tier adjoint gradient): stands in for a GPU
    context on a CPU rank."""

    def __init__(self, problem, gradient):
        self.problem = problem
        self.dim = problem.theta0.shape[0]
        self.gradient = gradient
        self.h = 1e-3
        self.rows = 0

    def values(self, thetas):
        from oracle import fobj
        self.rows += len(thetas)
        return np.array([fobj.f_obj(self.problem, t, tier="dense") for t in thetas])

    def grads(self, thetas):
        from oracle import fobj
        self.rows += len(thetas)
        f = np.array([fobj.f_obj(self.problem, t, tier="dense") for t in thetas])
        g = np.stack([fobj.grad_adjoint(self.problem, t) for t in thetas])
        return f, g


def _inla_worker(rank, world, port, q):
    import torch.distributed as dist
    import synth
    from paper_2507_06938_gb300 import inla
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        p = synth.problem_from_config("t_uni")
        local = _OracleObjective(p, "fd")
        obj = inla.DistributedObjective(local)
        pts = inla.stencil(p.theta0, 1e-3)
        f = obj.values(pts)
        fv, g = obj.value_grad(p.theta0)
        fa, ga = inla.DistributedObjective(_OracleObjective(p, "adjoint")).grads(pts[:3])
        res = inla.bfgs(obj.value_grad, p.theta0, gtol=1e-4, max_iter=30)
        q.put((rank, f, g, local.rows, fa, ga, res.theta))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_inla_stencil_points_split_over_two_ranks():
    """DistributedObjective: the 2 dim + 1 points of Eq. 10 are split
    round-robin over the ranks, every rank gets the full vector of f values
    (and gradients), identical to a single-process evaluation, and BFGS
    reaches the same mode on every rank."""
    import torch.multiprocessing as mp
    import synth
    from paper_2507_06938_gb300 import inla
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_inla_worker, args=(r, 2, port, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    out = {}
    for _ in range(2):
        r = q.get(timeout=300)
        out[r[0]] = r[1:]
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    p = synth.problem_from_config("t_uni")
    single = _OracleObjective(p, "fd")
    pts = inla.stencil(p.theta0, 1e-3)
    f_ref = single.values(pts)
    f_a, g_a = _OracleObjective(p, "adjoint").grads(pts[:3])
    for rank in (0, 1):
        f, g, rows, fa, ga, mode = out[rank]
        assert np.array_equal(f, f_ref)
        assert np.allclose(g, inla.fd_from_stencil(f_ref, 1e-3), rtol=0, atol=1e-12)
        assert np.array_equal(fa, f_a) and np.array_equal(ga, g_a)
    # the work was split: 9 stencil points -> 5 rows on rank 0, 4 on rank 1 (first call)
    assert out[0][2] > out[1][2]
    assert np.array_equal(out[0][5], out[1][5])
