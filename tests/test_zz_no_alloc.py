"""The allocation-free selection entry point (s3r_select_visible_static).

Some callers cannot allocate device memory at all: code inside a host
framework whose caching allocator owns the whole device, or a real-time loop
that may not call cudaMalloc after start-up. For them the library offers the
temporal selection with its scratch in a fixed array of the library's device
image. This test calls it through the C ABI twice in a row, on two different
visibility records and times over the same number of Gaussians (the scratch
keeps the previous call's contents, and its look-back words would hold the
first call's prefixes if the call did not clear them), and compares both
results with the oracle's selection and with the selection that s3r_project
computes in a workspace. It is self-contained, so it passes alone in a fresh
process and after the other tests (this file is collected last).
"""
import numpy as np
import pytest

import oracle
from paper_2503_08217_gb300 import scenegen

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_static_selection_matches_oracle_and_workspace():
    from paper_2503_08217_gb300 import binding, build
    from paper_2503_08217_gb300.render import DeviceScene, Renderer
    build.build()
    binding.load()
    # 102,001 Gaussians: 25 look-back tiles of 4,096 and a ragged tail
    scene = scenegen.generate("tiny", seed=3, n_static=100_001)
    n = scene.n
    rng = np.random.default_rng(8)
    records = []
    for lo, hi, never in ((-1.2, 1.2, 0.1), (-0.3, 0.9, 0.4)):
        vis = np.sort(rng.uniform(lo, hi, (n, 2)).astype(np.float32), axis=1)
        vis[rng.random(n) < never] = (0.9, -0.9)          # never-visible windows
        records.append(vis)
    steps = (4, 7)

    dev = DeviceScene.from_host(scene)
    out_idx = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    out_count = torch.zeros(1, dtype=torch.int32, device="cuda")
    for vis, step in zip(records, steps):
        t = float(scene.times[step])
        vis_t = torch.from_numpy(vis).cuda()
        expect = oracle.select(vis, t)
        assert 0 < expect.size < n
        # the existing path: s3r_project in a workspace
        cams = scene.cams[step]
        r = Renderer(n, scene.n_inst, cams)
        iq = torch.from_numpy(scene.inst_quat[step]).cuda()
        it = torch.from_numpy(scene.inst_trans[step]).cuda()
        r.ws.project(dev.c_scene(), binding.make_poses(iq, it), cams, t, vis_t, None, 0.0)
        c = r.counts()
        ref = r.ws.debug("selected", torch.int32, c["n_selected"]).cpu().numpy().view(np.uint32)
        np.testing.assert_array_equal(ref.astype(np.int64), expect)
        # the allocation-free entry point
        out_idx.fill_(-1)
        out_count.fill_(-7)
        binding.select_visible_static(vis_t, t, out_idx, out_count)
        torch.cuda.synchronize()
        m = int(out_count.item()) & 0xFFFFFFFF
        assert m != 0xFFFFFFFF                            # no look-back wait gave up
        assert m == expect.size
        np.testing.assert_array_equal(out_idx[:m].cpu().numpy().view(np.uint32).astype(np.int64), expect)


def test_static_selection_rejects_too_many_gaussians():
    from paper_2503_08217_gb300 import binding
    L = binding.load()
    out = torch.zeros(1, dtype=torch.int32, device="cuda")
    st = L.s3r_select_visible_static((1 << 26) + 1, 0.0, None, None, out.data_ptr(), None)
    assert st == 1 and b"2^26" in L.s3r_last_error()
