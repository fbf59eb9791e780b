"""The allocation-free selection entry point (s3r_select_visible_static).

Some callers cannot allocate device memory at all: code inside a host
framework whose caching allocator owns the whole device, or a real-time loop
that may not call cudaMalloc after start-up. For them the library offers the
temporal selection with its scratch in a fixed array of the library's device
image. This test calls it through the C ABI twice in a row (the scratch keeps
the previous call's contents, so the second call checks that it is cleared)
and compares both results with the selection that s3r_project computes in a
workspace. It is self-contained, so it passes alone in a fresh process and
after the other tests (this file is collected last).
"""
import numpy as np
import pytest

from paper_2503_08217_gb300 import scenegen

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_static_selection_matches_workspace_selection():
    from paper_2503_08217_gb300 import binding, build
    from paper_2503_08217_gb300.render import DeviceScene, Renderer
    build.build()
    binding.load()
    # 102,001 Gaussians: 25 look-back tiles of 4,096 and a ragged tail
    scene = scenegen.generate("tiny", seed=3, n_static=100_001)
    n = scene.n
    rng = np.random.default_rng(8)
    vis = np.sort(rng.uniform(-1.2, 1.2, (n, 2)).astype(np.float32), axis=1)
    vis[rng.random(n) < 0.1] = (0.9, -0.9)            # some never-visible windows
    step = 4
    t = float(scene.times[step])
    vis_t = torch.from_numpy(vis).cuda()

    # the existing path: s3r_project in a workspace
    dev = DeviceScene.from_host(scene)
    cams = scene.cams[step]
    r = Renderer(n, scene.n_inst, cams)
    iq = torch.from_numpy(scene.inst_quat[step]).cuda()
    it = torch.from_numpy(scene.inst_trans[step]).cuda()
    r.ws.project(dev.c_scene(), binding.make_poses(iq, it), cams, t, vis_t, None, 0.0)
    c = r.counts()
    ref = r.ws.debug("selected", torch.int32, c["n_selected"]).cpu().numpy().view(np.uint32)
    assert 0 < ref.size < n

    # the allocation-free entry point, twice in a row
    out_idx = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    out_count = torch.zeros(1, dtype=torch.int32, device="cuda")
    for _ in range(2):
        out_idx.fill_(-1)
        out_count.fill_(-7)
        binding.select_visible_static(vis_t, t, out_idx, out_count)
        torch.cuda.synchronize()
        m = int(out_count.item())
        assert m == ref.size
        np.testing.assert_array_equal(out_idx[:m].cpu().numpy().view(np.uint32), ref)


def test_static_selection_rejects_too_many_gaussians():
    from paper_2503_08217_gb300 import binding
    L = binding.load()
    out = torch.zeros(1, dtype=torch.int32, device="cuda")
    st = L.s3r_select_visible_static((1 << 26) + 1, 0.0, None, None, out.data_ptr(), None)
    assert st == 1 and b"2^26" in L.s3r_last_error()
