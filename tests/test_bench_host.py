"""Host logic of bench.py that decides what the JSON line claims: the DRAM
traffic record is only reported while the captured kernels' source region is
unchanged, and the workload text and L2 note describe the measured problem."""

import json

import bench
import synth


def test_traffic_record_follows_the_captured_source_and_shape(tmp_path, monkeypatch):
    root = tmp_path
    (root / "profiles").mkdir()
    src_rel = "kernel.cu"
    (root / src_rel).write_text("prologue\n// begin\nkernel body\n// end\nhost code\n")
    rec = {"kernel": "k", "M": 64, "N": 64, "K": 64, "batch": 2, "slices": 7, "source": src_rel,
           "region": ["// begin", "// end"], "bytes_per_launch": 123}
    monkeypatch.setattr(bench, "ROOT", str(root))
    rec["source_sha1"] = bench.kernel_source_sha1(src_rel, rec["region"])
    (root / "profiles" / "traffic.json").write_text(json.dumps({"records": [rec]}))
    shape = {"M": 64, "N": 64, "K": 64, "batch": 2, "slices": 7}
    assert bench.traffic_record("k", shape) == 123
    # another launch shape (batch, size or digit slices) has no capture
    assert bench.traffic_record("k", dict(shape, batch=18)) is None
    assert bench.traffic_record("k", dict(shape, M=6000)) is None
    assert bench.traffic_record("k", dict(shape, slices=5)) is None
    # host code outside the region may change
    (root / src_rel).write_text("prologue\n// begin\nkernel body\n// end\nother host code\n")
    assert bench.traffic_record("k", shape) == 123
    # the kernel may not
    (root / src_rel).write_text("prologue\n// begin\nkernel body v2\n// end\nhost code\n")
    assert bench.traffic_record("k", shape) is None
    # nor may its markers disappear
    (root / src_rel).write_text("prologue\nkernel body\n")
    assert bench.traffic_record("k", shape) is None
    assert bench.traffic_record("missing", shape) is None


def test_workload_text_and_l2_note_describe_the_problem():
    p = synth.problem_from_config("c2")
    text = bench.workload(p, 9)
    for part in ("ns=1024", "nt=64", "nb=4", "m=65536", "N=65540", "9 theta point"):
        assert part in text, part
    assert bench.l2_note(p, 9).startswith("inputs larger than L2")
    small = synth.problem_from_config("t_uni")
    assert bench.l2_note(small, 1).startswith("inputs smaller than L2")


def test_workload_of_the_default_configuration():
    p = synth.problem_from_config(bench.CONFIG_NAME)
    text = bench.workload(p, 1)
    for part in ("3-variate coregional", "Delaunay", "ns=2000", "b=6000", "nt=48", "N=288006", "1 theta point"):
        assert part in text, part
    # about 96 GB per matrix with factor, inverse blocks and selected inverse
    assert 90e9 < bench.matrix_bytes(p) < 100e9


def test_errors_against_reference():
    import numpy as np
    ref = dict(ld_p=-2e5, ld_c=3e5, f=10.0, resid=1e-13, g=np.array([1.0, -2.0, 1e-6]),
               sigma={(0, "D", 0): np.array([[2.0, 1.0], [1.0, 2.0]])})
    mix = dict(ld_p=-2e5 * (1 + 1e-9), ld_c=3e5, f=10.0 + 5e-4, resid=2e-12, g=np.array([1.0, -2.0 + 2e-6, 0.0]),
               sigma={(0, "D", 0): np.array([[2.0, 1.0 + 1e-8], [1.0, 2.0]])})
    e = bench.errors_against(mix, ref)
    assert abs(e["logdet_p_rel"] - 1e-9) < 1e-15
    assert e["logdet_c_rel"] == 0.0
    assert abs(e["f_rel_to_logdets"] - 5e-4 / 5e5) < 1e-15
    assert e["solve_residual"] == 2e-12
    assert abs(e["sigma_block_rel_max"] - 0.5e-8) < 1e-15
    assert list(e["sigma_block_rel"]) == ["Q_p D0"]
    # gradient error relative to max(|g_k|, 1e-3 |g|_inf): the third entry's scale is 2e-3
    assert abs(e["grad_rel_max"] - 1e-6 / 2e-3) < 1e-12


def test_roofline_records_of_both_precisions():
    """The roofline record from the profiling events: achieved rate, the
    measured peak it divides by, and the traffic lookup keyed on the launch
    shape and, for the split product, the tuned tile order."""
    import bench
    import synth
    from paper_2507_06938_gb300 import bta
    p = synth.problem_from_config("c5p")
    prof = (10.0, 2, 2 * 4.32e11)            # ms, launches, nominal flops
    peak = {"dfma": 1.25, "dmma": 1.1}
    r = bench._roofline("fp64", prof, p, 1, peak)
    assert r["bound"] == "alu" and abs(r["achieved"] - 86.4) < 1e-9 and r["peak"] == 1.25
    tuned = (32, 64, 256, 0, 1, 2, 1, 8, 1)
    assert len(tuned) == len(bta.BtaContext.AUTOTUNE_KEYS)
    r = bench._roofline("mixed_hi", prof, p, 1, peak, tuned)
    assert r["bound"] == "tensor" and abs(r["achieved_fp64_equivalent"] - 86.4) < 1e-9
    assert abs(r["achieved"] - 28 * 86.4) < 1e-6 and r["frac"] == r["achieved"] / bench.BF16_PEAK_TFLOPS
    r2 = bench._roofline("mixed_hi", prof, p, 1, peak, None)
    assert r2["achieved"] == r["achieved"]


def test_memory_layouts_of_the_batch_sizing():
    """The low-memory layout keeps Q, the factor (one spare slot each way) and
    one buffer per matrix; the default adds the selected inverse and the n
    inverse blocks: about 0.6 of the bytes at n = 48."""
    import bench
    import synth
    p = synth.problem_from_config("c5")
    full, low = bench.matrix_bytes(p), bench.matrix_bytes(p, True)
    bb = 8.0 * p.b * p.b
    assert abs(full / bb - (3 * (2 * p.nt - 1) + p.nt + 8.5)) < 1e-9
    assert abs(low / bb - ((2 * p.nt - 1) + 2 * (p.nt + 1) + 1 + 8.5)) < 1e-9
    assert 0.55 < low / full < 0.62


def test_layout_choice_follows_the_free_memory(monkeypatch):
    """--memory auto takes the low-memory layout exactly when it fits more
    theta points per step; an explicit batch or time partitions keep the
    default layout, and --memory low/full force it."""
    import types
    import bench
    import synth
    import torch
    p = synth.problem_from_config("c5")
    free = {"v": 290e9}
    monkeypatch.setattr(torch.cuda, "mem_get_info", lambda *a: (free["v"], 298e9))
    args = types.SimpleNamespace(memory="auto", batch=0, time_partitions=1)
    assert bench.choose_layout(args, p) == (2, True)
    free["v"] = 120e9                      # one point either way: keep the default layout
    assert bench.choose_layout(args, p) == (1, False)
    free["v"] = 290e9
    assert bench.choose_layout(args, p, batch=1) == (1, False)
    args.time_partitions = 4
    assert bench.choose_layout(args, p) == (1, False)
    args.memory = "low"
    assert bench.choose_layout(args, p) == (1, False)
    args.memory = "auto"
    args.time_partitions, args.memory = 1, "low"
    assert bench.choose_layout(args, p, batch=1) == (1, True)
    args.memory = "full"
    assert bench.choose_layout(args, p) == (1, False)
