"""Host-side tests of the launch-shape autotuner and the variant builds (no GPU)."""
from __future__ import annotations

import concurrent.futures
import ctypes
import os
import shutil
import subprocess
import sys

import pytest

from paper_2503_08217_gb300 import autotune, binding
from paper_2503_08217_gb300 import build as libbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HAVE_NVCC = shutil.which("nvcc") is not None or os.path.exists("/usr/local/cuda/bin/nvcc")


def test_every_tuned_define_has_a_source_default_among_its_candidates():
    d = autotune.source_defaults()
    assert set(d) == {p.name for p in autotune.PARAMS}
    for p in autotune.PARAMS:
        assert d[p.name] in p.candidates, p.name
        assert len(set(p.candidates)) == len(p.candidates)


def test_every_overridable_launch_shape_is_in_the_tuner():
    """Each `#ifndef S3R_X / #define S3R_X <int>` default in the CUDA sources is
    a launch shape the tuner searches (S3R_ARCH, the build's target, and
    S3R_SCAN_CTAS and S3R_TIN_MAX_GRID, which only the variant parity test
    sets, aside)."""
    import re
    found = set()
    for path in sorted(os.listdir(libbuild.CSRC)):
        with open(os.path.join(libbuild.CSRC, path)) as f:
            found |= set(re.findall(r"^#ifndef (S3R_\w+)\n#define \1 \d+\b", f.read(), re.M))
    assert found - {"S3R_ARCH", "S3R_SCAN_CTAS", "S3R_TIN_MAX_GRID"} == {p.name for p in autotune.PARAMS}


def test_defines_reach_only_the_units_that_see_them():
    blend = libbuild.relevant_defines("k_blend.cu", {"S3R_BLEND_FWD_BATCH": 32})
    assert blend == {"S3R_BLEND_FWD_BATCH": 32}
    for src in libbuild.SOURCES:
        if src != "k_blend.cu":
            assert libbuild.relevant_defines(src, {"S3R_BLEND_FWD_BATCH": 32}) == {}, src
    # the radix tile is declared in the shared internal header: every unit sees it
    for src in libbuild.SOURCES:
        assert libbuild.relevant_defines(src, {"S3R_SORT_ITEMS": 11}) == {"S3R_SORT_ITEMS": 11}, src


def test_bad_define_names_and_values_are_rejected():
    with pytest.raises(ValueError):
        libbuild.build(defines={"NOT_OURS": 3})
    with pytest.raises(ValueError):
        libbuild.build(defines={"S3R_SORT_ITEMS": "15; rm"})


def _fake_cost(target):
    def measure(values):
        return 10.0 + sum((values[k] - t) ** 2 for k, t in target.items())
    return measure


def test_coordinate_descent_reaches_the_minimum_of_a_separable_cost():
    start = {"A": 1, "B": 5}
    params = [("A", (1, 2, 3)), ("B", (4, 5, 6))]
    best, ms, trials = autotune.coordinate_descent(start, params, _fake_cost({"A": 3, "B": 4}),
                                                   min_gain=0.0)
    assert best == {"A": 3, "B": 4} and ms == 10.0
    assert trials[0] == (start, 10.0 + 4 + 1)


def test_coordinate_descent_times_each_configuration_once():
    calls = []

    def measure(v):
        calls.append(dict(v))
        return {1: 5.0, 2: 6.0, 3: 7.0}[v["A"]] + v["B"]

    start = {"A": 2, "B": 0}
    best, ms, trials = autotune.coordinate_descent(start, [("A", (3, 2, 1)), ("B", (0, 1))],
                                                   measure, passes=3)
    assert best == {"A": 1, "B": 0} and ms == 5.0
    keys = [tuple(sorted(c.items())) for c in calls]
    assert len(keys) == len(set(keys)) == len(trials)


def test_coordinate_descent_keeps_the_incumbent_below_the_minimum_gain():
    start = {"A": 2}
    costs = {1: 100.0, 2: 100.5, 3: 101.0}
    best, ms, _ = autotune.coordinate_descent(start, [("A", (1, 2, 3))],
                                              lambda v: costs[v["A"]], min_gain=0.01)
    assert best == {"A": 2} and ms == 100.5


def test_coordinate_descent_skips_failing_variants_and_honours_the_deadline():
    def measure(v):
        if v["A"] == 1:
            raise RuntimeError("nvcc failed for k_blend.cu")
        return float(v["A"])
    best, ms, trials = autotune.coordinate_descent({"A": 3}, [("A", (1, 2))], measure)
    assert best == {"A": 2} and ms == 2.0
    assert isinstance(trials[1][1], str) and "nvcc failed" in trials[1][1]
    _, _, trials = autotune.coordinate_descent({"A": 3}, [("A", (1, 2))], measure, deadline=0.0)
    assert len(trials) == 1


def test_a_failing_start_is_an_error():
    with pytest.raises(RuntimeError):
        autotune.coordinate_descent({"A": 1}, [("A", (1, 2))], lambda v: 1 / 0)


def test_write_defaults_rewrites_only_the_chosen_define(tmp_path):
    csrc = tmp_path / "csrc"
    shutil.copytree(libbuild.CSRC, csrc)
    before = {p: (csrc / p).read_text() for p in os.listdir(csrc)}
    changed = autotune.write_defaults({"S3R_BLEND_BWD_BATCH": 128, "S3R_SORT_ITEMS": 15}, str(csrc))
    assert changed == ["S3R_BLEND_BWD_BATCH"]   # the sort default already was 15
    d = autotune.source_defaults(str(csrc))
    assert d["S3R_BLEND_BWD_BATCH"] == 128
    assert {k: v for k, v in d.items() if k != "S3R_BLEND_BWD_BATCH"} == \
        {k: v for k, v in autotune.source_defaults().items() if k != "S3R_BLEND_BWD_BATCH"}
    after = (csrc / "k_blend.cu").read_text()
    diff = [(a, b) for a, b in zip(before["k_blend.cu"].splitlines(), after.splitlines()) if a != b]
    assert diff == [("#define S3R_BLEND_BWD_BATCH 64    // splats staged per batch (backward)",
                     "#define S3R_BLEND_BWD_BATCH 128    // splats staged per batch (backward)")]
    for p, text in before.items():
        if p != "k_blend.cu":
            assert (csrc / p).read_text() == text


def test_report_lists_every_trial():
    start = {"A": 1, "B": 5}
    trials = [(start, 12.0), ({"A": 2, "B": 5}, 11.0), ({"A": 2, "B": 6}, "RuntimeError: x")]
    text = autotune.report(start, {"A": 2, "B": 5}, 11.0, trials, "rig", 10, 3)
    assert "| 1 | A=2 | 11.000 | 0.917 |" in text
    assert "failed: RuntimeError: x" in text
    assert "| A | 1 | 2 |" in text


@pytest.mark.skipif(not HAVE_NVCC, reason="nvcc is needed to compile")
def test_every_candidate_passes_the_sources_compile_time_checks():
    cc = libbuild.nvcc()
    flags = ["-arch=sm_103a", "-O3", "-std=c++17", "-I" + libbuild.INCLUDE, "-DS3R_ARCH=103",
             "-cubin", "-o", os.devnull]
    jobs = []
    for p in autotune.PARAMS:
        src = "k_sort.cu" if p.source.endswith(".cuh") else p.source
        for v in p.candidates:
            jobs.append((p.name, v, True, [cc, *flags, f"-D{p.name}={v}", os.path.join(libbuild.CSRC, src)]))
    # and one value past each checked limit is refused at compile time
    bad = [("S3R_SORT_ITEMS", 19, "k_sort.cu"), ("S3R_DUP_EXPAND_ITEMS", 16, "k_sort.cu"),
           ("S3R_DUP_EXPAND_ITEMS", 2, "k_sort.cu"), ("S3R_BLEND_FWD_BATCH", 48, "k_blend.cu"),
           ("S3R_BLEND_BWD_BLOCKS", 33, "k_blend.cu")]
    for name, v, src in bad:
        jobs.append((name, v, False, [cc, *flags, f"-D{name}={v}", os.path.join(libbuild.CSRC, src)]))

    def run(job):
        return job[0], job[1], job[2], subprocess.run(job[3], capture_output=True, text=True).returncode

    with concurrent.futures.ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        for name, v, legal, rc in ex.map(run, jobs):
            if legal:
                assert rc == 0, f"{name}={v} does not compile"
            else:
                assert rc != 0, f"{name}={v} should be refused"


@pytest.mark.skipif(not HAVE_NVCC, reason="nvcc is needed to build")
def test_a_variant_library_builds_loads_and_exports_the_abi():
    lib = libbuild.build(defines={"S3R_PROJECT_MASK_BLOCKS": 4})
    assert lib == libbuild.variant_path({"S3R_PROJECT_MASK_BLOCKS": 4})
    assert lib != libbuild.LIB and os.path.exists(lib)
    L = ctypes.CDLL(lib)
    for name in binding.EXPORTS:
        assert hasattr(L, name), name


def test_the_binding_loads_the_library_the_environment_names():
    env = dict(os.environ, S3R_LIBRARY="/nonexistent/libs3r.so")
    code = ("from paper_2503_08217_gb300 import binding\n"
            "print(binding.LIB_PATH)\n"
            "try:\n    binding.load()\nexcept RuntimeError as e:\n    print('missing' in str(e))\n")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True,
                       text=True, check=True)
    assert r.stdout.split() == ["/nonexistent/libs3r.so", "True"]


def test_recorded_traffic_is_not_claimed_for_a_variant_library(monkeypatch):
    import bench
    # a record taken on the current source of the kernel's file
    src = "paper_2503_08217_gb300/csrc/k_blend.cu"
    monkeypatch.setitem(bench.NCU_TRAFFIC, "blend_bwd",
                        {"bytes": 123, "source": src, "profile": "profiles/x.md",
                         "code_sha256_16": bench.code_hash(os.path.join(ROOT, src))})
    monkeypatch.delenv("S3R_LIBRARY", raising=False)
    assert bench.measured_traffic("blend_bwd", "rig") == 123
    assert bench.measured_traffic("blend_bwd", "mid") is None
    monkeypatch.setenv("S3R_LIBRARY", libbuild.variant_path({"S3R_BLEND_BWD_BATCH": 32}))
    assert bench.measured_traffic("blend_bwd", "rig") is None


def test_report_carries_each_trials_clocks_and_the_second_timing():
    start = {"A": 1}
    trials = [(start, 5.0), ({"A": 2}, 5.5)]
    notes = {(("A", 1),): autotune.clock_note({"clocks": {"sm_mhz": 2070.0, "sm_max_mhz": 2070,
                                                          "reasons": []}}),
             (("A", 2),): autotune.clock_note({"clocks": {"sm_mhz": 1800.0, "sm_max_mhz": 2070,
                                                          "reasons": ["sw_power_cap"]}})}
    text = autotune.report(start, start, 5.0, trials, "rig", 20, 5, notes, retimed=5.05)
    assert "| 0 | (start) | 5.000 | 1.000 | 2070 / 2070 MHz, no reason |" in text
    assert "| 1 | A=2 | 5.500 | 1.100 | 1800 / 2070 MHz, sw_power_cap |" in text
    assert "timed again in a fresh process: 5.050 ms / step (+1.00 %" in text
    assert autotune.clock_note({"clocks": {"sm_mhz": None, "reasons": ["no samples"]}}) == "not sampled"
