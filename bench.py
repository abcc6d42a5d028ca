#!/usr/bin/env python
"""Throughput of the BTA hot path of one f_obj(theta) evaluation on GB300.

One step = one batch of 2 dim(theta) + 1 = 9 theta points (the stencil of
Eq. 10) of the univariate AR(1) x SPDE model at working size (32 x 32 grid
mesh: ns = 1024, nt = 64, nb = 4 fixed effects, m = 65,536 observations,
N = 65,540), each with the whole hot path: assembly, factorisation and
log-determinant of Q_p and Q_c, the conditional-mean solve, f_obj, the
selected inversion of Q_p and Q_c and the adjoint gradient of f_obj.  All 18
BTA matrices of a step go through the same kernel launches.  Each step uses a
different stencil centre.

value  = f_obj evaluations / s with inputs resident in HBM (device-timed)
e2e    = the same through the C ABI with the thetas copied host->device and
         f, mu and the marginal variances copied device->host inside the
         timed region (pinned host buffers)
--impl reference times the CPU FP64 oracle (oracle/) on the host cores.
"""

from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "f_obj evals/s and BTA Cholesky+selinv TFLOP/s: mixed vs FP64 on one GB300"
UNIT = "f_obj evals/s"
L2_BYTES = 129e6


def workload(p, B) -> str:
    """The measured workload, described from the problem itself."""
    kind = "univariate AR(1) x SPDE Matern" if p.nv == 1 else f"{p.nv}-variate coregional AR(1) x SPDE Matern"
    return (f"{kind}, mesh ns={p.ns}, nt={p.nt}, nb={p.a} fixed effects, m={int(p.y.shape[0])} observations, "
            f"N={p.N}; per step: {B} theta points (2 dim(theta)+1 stencil), each assemble+factor+log-det of "
            "Q_p and Q_c, conditional-mean solve, f_obj, selected inversion of Q_p and Q_c, adjoint gradient")


def l2_note(p, B) -> str:
    per = (2 * p.nt - 1) * p.b * p.b * 8.0
    rel = "larger" if 2 * B * per > L2_BYTES else "smaller"
    return f"inputs {rel} than L2 (BTA blocks ~{per / 1e9:.3g} GB per matrix, {2 * B} matrices)"


CONFIG_NAME = "c2"
# FP64 peak of the GB300: the nominal FP64 rate (no FP64 figure is measured by
# the driver); a DFMA throughput probe on this machine read 1.20 TFLOP/s at 1995 MHz.
FP64_PEAK_TFLOPS = 1.25


def _measured_bf16():
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["bf16_tflops"])
    except (OSError, ValueError, KeyError):
        return 1900.0   # fallback figure of the profiling recipe


BF16_PEAK_TFLOPS = _measured_bf16()


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["fp64", "mixed"])
    ap.add_argument("--config", default=CONFIG_NAME)
    ap.add_argument("--batch", type=int, default=0, help="theta points per step (default 2 dim(theta) + 1)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default launch shapes")
    ap.add_argument("--no-compare", action="store_true",
                    help="skip the FP64 comparison run of the mixed-precision bench")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.gpu)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def kernel_source_sha1(source: str, region=None):
    """sha1 of a kernel's source text: the file, or the part of it between two
    marker lines (the device code of the captured kernels)."""
    try:
        text = open(os.path.join(ROOT, source), "rb").read()
    except OSError:
        return None
    if region:
        start, end = (m.encode() for m in region)
        i = text.find(start)
        j = text.find(end, i + 1) if i >= 0 else -1
        if i < 0 or j < 0:
            return None
        text = text[i:j]
    return hashlib.sha1(text).hexdigest()


def traffic_record(kernel_key: str):
    """DRAM bytes per launch of the dominant kernel from a committed ncu summary,
    null if the kernel's source changed since the capture."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        rec = json.load(open(path)).get(kernel_key)
    except (OSError, ValueError):
        return None
    if not rec:
        return None
    h = kernel_source_sha1(rec["source"], rec.get("region"))
    return rec["bytes_per_launch"] if h is not None and h == rec["source_sha1"] else None


def cpu_threads():
    try:
        from threadpoolctl import threadpool_info
        n = [d.get("num_threads") for d in threadpool_info() if d.get("user_api") == "blas"]
        if n and n[0]:
            return int(n[0])
    except Exception:
        pass
    return os.cpu_count()


def oracle_step(problem, theta, fd):
    """One theta point of the workload on the CPU oracle (tier B): f_obj and the
    selected inversion of Q_p and Q_c (the inputs of the adjoint gradient)."""
    from oracle import bta as obta
    from oracle import fobj as ofobj
    terms = ofobj.f_obj_terms(problem, theta, tier="bta", fd=fd)
    built = terms["built"]
    for Q in (built.Qp, built.Qc):
        obta.selinv(obta.factor(obta.blocks_from_sparse(Q, problem.nt, problem.b, problem.a)))
    return terms["f"]


def stencil(center, h=1e-3):
    """The 2 dim + 1 points of the central-difference gradient (Eq. 10)."""
    import numpy as np
    pts = [center]
    for i in range(center.shape[0]):
        e = np.zeros_like(center)
        e[i] = h
        pts += [center + e, center - e]
    return np.stack(pts)


def thetas_for(problem, count, rank):
    """One stencil per step around a different seeded center."""
    import numpy as np
    rng = np.random.default_rng(1000 + rank)
    return [stencil(problem.theta0 + 0.02 * rng.standard_normal(problem.theta0.shape)) for _ in range(count)]


def max_over_ranks(values, dist, device):
    """Element-wise maximum of per-rank timings (the job's time is the slowest
    rank's); identity without a process group."""
    import torch
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.tolist()]


def job_throughput(steps, world, batch, ms):
    """Evaluations per second of the whole job: every rank evaluates its own
    `batch` theta points per step (weak scaling), over the slowest rank's time."""
    return steps * world * batch / (ms / 1e3)


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import synth
    from oracle import model as omodel
    p = synth.problem_from_config(args.config)
    fd = omodel.fem_data(p)
    # bounded sample: one theta point of each step's stencil (the oracle takes
    # tens of seconds per point at this size); value in f_obj evaluations / s
    thetas = thetas_for(p, args.warmup + args.steps, 0)
    for j in range(min(args.warmup, 1)):     # the CPU path has nothing further to warm up
        oracle_step(p, thetas[j][0], fd)
    t0 = time.perf_counter()
    for j in range(args.steps):
        oracle_step(p, thetas[args.warmup + j][0], fd)
    dt = time.perf_counter() - t0
    value = args.steps / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": workload(p, len(thetas[0])), "name": args.config},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cpu_threads(), "kind": "oracle",
                         "sample": "one theta point (f_obj + selinv of Q_p and Q_c) of each step's 9 points, "
                                   "numpy/scipy FP64 block recurrences"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def _roofline(precision, prof_ms, prof_n, prof_flops):
    """Roofline record of the dominant kernel from the profiling events of the
    last timed step (the graph replays the same launches every step)."""
    achieved = (prof_flops / (prof_ms / 1e3) / 1e12) if prof_ms > 0 else None
    if precision == "fp64":
        return {
            "bound": "alu", "kernel": "gemm64_kernel (FP64 DFMA Schur-update GEMMs L_{i+1,i}=B_i L_ii^-T and "
                                      "D_{i+1}-=L L^T, batched over the step's matrices)",
            "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": (achieved / FP64_PEAK_TFLOPS) if achieved else None,
            "traffic": traffic_record("gemm64_bxbxb"),
            "launches_timed": prof_n, "flops_per_launch": (prof_flops / prof_n) if prof_n else None,
            "peak_source": "nominal GB300 FP64 rate (no FP64 entry in the measured peaks)",
        }
    # executed bf16 tensor flops: 15 digit-pair products per FP64-equivalent flop
    tensor = 15.0 * achieved if achieved else None
    peak = BF16_PEAK_TFLOPS
    return {
        "bound": "tensor", "kernel": "ozaki_gemm (digit split + tcgen05 bf16 15-pair products) for the "
                                    "Schur-update GEMMs, batched over the step's matrices",
        "achieved": tensor, "peak": peak, "unit": "TFLOP/s", "frac": (tensor / peak) if tensor else None,
        "achieved_fp64_equivalent": achieved,
        "traffic": traffic_record("ozaki_bxbxb"),
        "launches_timed": prof_n, "flops_per_launch": (prof_flops / prof_n) if prof_n else None,
        "peak_source": "measured bf16 dense (burst) of this pool, of measured",
    }


def measure(args, precision_name, warmup, steps, with_e2e, dist, rank, world, local):
    """Time `steps` batched f_obj+gradient+selinv steps of one precision after
    `warmup` untimed ones; returns the measurements of this rank."""
    import numpy as np
    import torch
    from paper_2507_06938_gb300 import bta
    import synth

    p = synth.problem_from_config(args.config)
    precision = bta.BTA_FP64 if precision_name == "fp64" else bta.BTA_MIXED
    B = args.batch or (2 * p.theta0.shape[0] + 1)
    stream = torch.cuda.Stream()
    model = bta.BtaModel(p)
    ctx = bta.BtaContext(p.nt, p.b, p.a, precision, stream, B)
    tuned = None if args.no_autotune else ctx.autotune(reps=2)
    nsteps = warmup + steps
    thetas_h = np.stack([t[:B] if t.shape[0] >= B else np.resize(t, (B, t.shape[1]))
                         for t in thetas_for(p, nsteps, rank)])          # steps x B x dim
    thetas_d = torch.tensor(thetas_h, dtype=torch.float64, device="cuda")
    f_d = torch.zeros((nsteps, B), dtype=torch.float64, device="cuda")
    g_d = torch.zeros((nsteps, B, p.theta0.shape[0]), dtype=torch.float64, device="cuda")
    var_d = torch.zeros((B, p.N), dtype=torch.float64, device="cuda")

    def step(j, theta_dev, f_out):
        ctx.fobj_grad(model, theta_dev, f_out, g_d[j])

    def barrier_sync():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    out = {"problem": p, "B": B, "thetas_h": thetas_h, "tuned": tuned}
    with torch.cuda.stream(stream):
        # the dominant GEMM launches carry timing events; the f_obj graph that
        # the timed steps replay is captured with them during the warm-up
        ctx.profile(True)
        for j in range(warmup):
            step(j, thetas_d[j], f_d[j])
        ctx.sync()
        barrier_sync()
        # ---- device-resident timed region
        launches0 = bta.bta_launch_count()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        with ClockSampler(local) as clk:
            e0.record(stream)
            for j in range(steps):
                step(warmup + j, thetas_d[warmup + j], f_d[warmup + j])
            e1.record(stream)
            e1.synchronize()
        ctx.sync()
        out["launches"] = bta.bta_launch_count() - launches0
        out["prof"] = ctx.profile_read()
        ctx.profile(False)
        out["ms"] = e0.elapsed_time(e1)
        out["clocks"] = clk.summary()
        barrier_sync()
        out["ms_e2e"] = None
        if with_e2e:
            # ---- end-to-end through the C ABI with host buffers
            th_pin = torch.tensor(thetas_h, dtype=torch.float64).pin_memory()
            f_pin = torch.zeros((steps, B), dtype=torch.float64).pin_memory()
            g_pin = torch.zeros((steps, B, p.theta0.shape[0]), dtype=torch.float64).pin_memory()
            var_pin = torch.zeros((B, p.N), dtype=torch.float64).pin_memory()
            theta_stage = torch.zeros((B, p.theta0.shape[0]), dtype=torch.float64, device="cuda")
            g0 = torch.cuda.Event(enable_timing=True)
            g1 = torch.cuda.Event(enable_timing=True)
            g0.record(stream)
            for j in range(steps):
                theta_stage.copy_(th_pin[warmup + j], non_blocking=True)
                ctx.fobj_grad(model, theta_stage, f_d[j], g_d[j])
                for k in range(B):
                    ctx.selinv_diag(2 * k + bta.BTA_QC, var_d[k])
                f_pin[j].copy_(f_d[j], non_blocking=True)
                g_pin[j].copy_(g_d[j], non_blocking=True)
                var_pin.copy_(var_d, non_blocking=True)
            g1.record(stream)
            g1.synchronize()
            ctx.sync()
            out["ms_e2e"] = g0.elapsed_time(g1)
    ctx.close()
    model.close()
    del thetas_d, f_d, g_d, var_d
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    out["ms"], out["ms_e2e"] = max_over_ranks([out["ms"], out["ms_e2e"] or 0.0], dist, "cuda")
    total_evals = steps * world * B
    out["value"] = job_throughput(steps, world, B, out["ms"])
    out["e2e_value"] = job_throughput(steps, world, B, out["ms_e2e"]) if with_e2e else None
    flops_eval = 2 * bta.bta_flops_factor(p.nt, p.b, p.a) + 2 * bta.bta_flops_selinv(p.nt, p.b, p.a)
    out["tflops"] = flops_eval * total_evals / (out["ms"] / 1e3) / 1e12
    out["roofline"] = _roofline(precision_name, *out["prof"])
    return out


def run_ours(args):
    import torch

    rank, world, local = dist_env()
    if not torch.cuda.is_available():
        raise RuntimeError("bench.py needs a CUDA device")
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_2507_06938_gb300 import _build
    if rank == 0 or world == 1:
        _build.build()
    if dist is not None:
        dist.barrier()

    r = measure(args, args.precision, args.warmup, args.steps, True, dist, rank, world, local)
    cmp = None
    if args.precision == "mixed" and not args.no_compare:
        # the FP64 path on the same workload, shorter (one FP64 step takes seconds)
        cmp = measure(args, "fp64", 1, 1, False, dist, rank, world, local)
    p, B = r["problem"], r["B"]

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    line = {
        "metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": r["ms"] / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if args.precision == "fp64" else "mixed (f64 with bf16-digit tensor-core products)",
        "data": "synthetic",
        "config": {"workload": workload(p, B), "name": args.config, "precision": args.precision, "theta_points": B,
                   "l2": l2_note(p, B),
                   "parallelism": f"replicas x{world} (independent theta points per GPU)"},
        "tflops": r["tflops"], "tflops_unit": "nominal (2 F_fact + 2 F_selinv) per f_obj evaluation / time",
        "roofline": r["roofline"],
        "e2e": {"value": r["e2e_value"], "unit": UNIT, "h2d_bytes_per_step": int(B * p.theta0.shape[0] * 8),
                "d2h_bytes_per_step": int(B * (8 + p.theta0.shape[0] * 8 + p.N * 8))},
        "batch": B,
        "autotuned": (None if r["tuned"] is None else
                      dict(zip(("fp64_leaf", "df32_leaf", "tensor_min_dim"), r["tuned"]))),
        "gpu_launches": int(r["launches"]),
        "clocks": r["clocks"],
    }
    if cmp is not None:
        line["fp64"] = {"value": cmp["value"], "unit": UNIT, "ms_per_step": cmp["ms"], "steps": 1, "warmup": 1,
                        "tflops": cmp["tflops"], "roofline": cmp["roofline"], "gpu_launches": int(cmp["launches"]),
                        "clocks": cmp["clocks"], "mixed_over_fp64": r["value"] / cmp["value"]}
    if world == 1 and not args.no_cpu_baseline:
        from oracle import model as omodel
        fd = omodel.fem_data(p)
        th = r["thetas_h"][args.warmup][0]
        t0 = time.perf_counter()
        oracle_step(p, th, fd)
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": 1.0 / dt, "unit": UNIT, "cores": cpu_threads(), "kind": "oracle",
                                "sample": "one theta point (f_obj + selinv of Q_p and Q_c) on the FP64 "
                                          "numpy/scipy block recurrences"}
    print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
