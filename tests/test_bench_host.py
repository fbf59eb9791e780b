"""Host logic of bench.py that needs no GPU: the recorded DRAM traffic is
tied to the kernel file's code, not its comments."""
from __future__ import annotations

import os

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
BLEND = os.path.join(ROOT, "paper_2503_08217_gb300", "csrc", "k_blend.cu")


def test_code_hash_ignores_comments_and_blank_lines(tmp_path):
    src = open(BLEND).read()
    base = bench.code_hash(BLEND)
    a = tmp_path / "a.cu"
    a.write_text("// a new leading comment\n\n" + src.replace("\n\n", "\n\n/* note */\n\n", 1) + "\n\n")
    assert bench.code_hash(str(a)) == base


def test_code_hash_sees_code_and_string_changes(tmp_path):
    a = tmp_path / "a.cu"
    a.write_text('int f() { return 1; }  // x\nconst char* s = "// not a comment";\n')
    b = tmp_path / "b.cu"
    b.write_text('int f() { return 2; }  // x\nconst char* s = "// not a comment";\n')
    c = tmp_path / "c.cu"
    c.write_text('int f() { return 1; }  // y\nconst char* s = "// changed";\n')
    ha, hb, hc = (bench.code_hash(str(p)) for p in (a, b, c))
    assert ha != hb and ha != hc


def test_recorded_traffic_only_for_its_code_and_workload():
    t = bench.NCU_TRAFFIC["blend_bwd"]
    same = bench.code_hash(os.path.join(ROOT, t["source"])) == t["code_sha256_16"]
    assert bench.measured_traffic("blend_bwd", "rig") == (t["bytes"] if same else None)
    assert bench.measured_traffic("blend_bwd", "small-rig") is None
    assert bench.measured_traffic("blend_fwd", "rig") is None


def test_the_bench_line_names_its_launch_shapes(monkeypatch):
    import bench
    from paper_2503_08217_gb300 import autotune, build
    monkeypatch.delenv("S3R_LIBRARY", raising=False)
    assert bench.launch_shapes() == autotune.source_defaults()
    monkeypatch.setenv("S3R_LIBRARY", build.variant_path({"S3R_SORT_ITEMS": 11}))
    assert bench.launch_shapes() == {"variant": "sort_items11"}
