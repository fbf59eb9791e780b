"""The launch shapes the autotuner varies change no result.

A library built with every tuned define below its default, and one with every
define above it, each pass the end-to-end parity tests against the FP64
oracle (stages, images, gradients, the row-table overflow path, ragged
sizes). The tests run in a child pytest with S3R_LIBRARY naming the variant,
so this process's loaded library is not replaced. The larger batches stage
two Gaussians per thread (a loop the 64-Gaussian default takes once), the
smaller radix tiles and expansion chunks multiply the look-back tiles and
chunk-map entries. Two more libraries set shapes the tuner does not search:
one caps the chunked scans (compaction, splat and pair offsets) at two CTAs,
so that on these small inputs a chunk spans many tiles and each CTA takes
several chunks; one sends every view of the tile-count kernel down the path
for views too large for the packed splat record (the separate arrays).
"""
from __future__ import annotations

import os
import subprocess
import sys

import pytest

from paper_2503_08217_gb300 import autotune
from paper_2503_08217_gb300 import build as libbuild

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PARITY = ("tiny_forward_stages or tiny_gradients or multiview_rig_sh3_lod or "
          "row_table_overflow or single_gaussian_and_ragged_sizes")
N_PARITY = 5


def _shapes(pick):
    out = {}
    for p in autotune.PARAMS:
        d = autotune.source_defaults()[p.name]
        out[p.name] = pick([c for c in p.candidates if c != d] or [d])
    return out


LOW = _shapes(min)
HIGH = _shapes(max)


def _parity_with(defines):
    lib = libbuild.build(defines=defines)
    env = dict(os.environ, S3R_LIBRARY=lib)
    cmd = [sys.executable, "-m", "pytest", "tests/test_gpu_parity.py", "-m", "gpu", "-x", "-q",
           "-p", "no:cacheprovider", "-k", PARITY]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0, r.stdout[-4000:] + r.stderr[-2000:]
    assert f"{N_PARITY} passed" in r.stdout, r.stdout[-2000:]


@pytest.mark.parametrize("defines", [LOW, HIGH], ids=["below_defaults", "above_defaults"])
def test_off_default_launch_shapes_pass_parity(defines):
    d = autotune.source_defaults()
    assert all(defines[k] != d[k] for k in d)
    _parity_with(defines)


@pytest.mark.parametrize("defines", [{"S3R_SCAN_CTAS": 2}, {"S3R_TIN_MAX_GRID": 0}],
                         ids=["two_scan_ctas", "unpacked_tile_inputs"])
def test_untuned_shapes_pass_parity(defines):
    _parity_with(defines)
