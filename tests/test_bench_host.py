"""Host logic of bench.py that decides what the JSON line claims: the DRAM
traffic record is only reported while the captured kernels' source region is
unchanged, and the workload text and L2 note describe the measured problem."""

import json

import bench
import synth


def test_traffic_record_follows_the_captured_source(tmp_path, monkeypatch):
    root = tmp_path
    (root / "profiles").mkdir()
    src_rel = "kernel.cu"
    (root / src_rel).write_text("prologue\n// begin\nkernel body\n// end\nhost code\n")
    rec = {"source": src_rel, "region": ["// begin", "// end"], "bytes_per_launch": 123}
    monkeypatch.setattr(bench, "ROOT", str(root))
    rec["source_sha1"] = bench.kernel_source_sha1(src_rel, rec["region"])
    (root / "profiles" / "traffic.json").write_text(json.dumps({"k": rec}))
    assert bench.traffic_record("k") == 123
    # host code outside the region may change
    (root / src_rel).write_text("prologue\n// begin\nkernel body\n// end\nother host code\n")
    assert bench.traffic_record("k") == 123
    # the kernel may not
    (root / src_rel).write_text("prologue\n// begin\nkernel body v2\n// end\nhost code\n")
    assert bench.traffic_record("k") is None
    # nor may its markers disappear
    (root / src_rel).write_text("prologue\nkernel body\n")
    assert bench.traffic_record("k") is None
    assert bench.traffic_record("missing") is None


def test_workload_text_and_l2_note_describe_the_problem():
    p = synth.problem_from_config("c2")
    text = bench.workload(p, 9)
    for part in ("ns=1024", "nt=64", "nb=4", "m=65536", "N=65540", "9 theta points"):
        assert part in text, part
    assert bench.l2_note(p, 9).startswith("inputs larger than L2")
    small = synth.problem_from_config("t_uni")
    assert bench.l2_note(small, 1).startswith("inputs smaller than L2")
