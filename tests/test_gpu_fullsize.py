"""Full-size parity on sampled outputs: the surround-rig workload the bench
times (9.0M Gaussians, 7 cameras, 12.8 Mpix, SH3, LOD 1 px) at the bench's
timestep and in its state and launch configuration (one batched call
sequence over all cameras, after a first-epoch sweep has recorded the point
lives, Eq. 5, and Eq. 6 has turned them into visibility windows), against
the FP64 oracle computed one sample at a time:

  * the visibility record: the oracle's own sweep of 20,000 sampled
    Gaussians over all 300 timesteps and 7 cameras, then Eq. 6, equals the
    GPU's record at those Gaussians exactly (away from near-threshold
    projection decisions);
  * the selection of the bench's timestep from the GPU's record equals the
    oracle's selection of the same record, every index;
  * 3000 sampled selected Gaussians: frustum/keep masks exactly, splat
    records within the FP32 tolerances, for every camera;
  * the sort of all pairs over the 50,400 tiles (two tile-digit passes)
    equals the oracle's stable sort of the GPU's FP32 splats with only
    unreachable pairs left out (a sample of them checked), and the tile
    ranges are those of the sorted list;
  * 24 sampled pixels per camera: Eq. 2 at those pixels (<= 1e-4);
  * the gradient of a loss supported on those pixels w.r.t. every parameter
    and pose (<= 1e-3 relative per tensor).
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_2503_08217_gb300 import scenegen

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _mt_ambiguous(rec, cam):
    """Gaussians whose M_t decision (in front of the near plane, a non-empty
    tile rectangle) lies within the oracle's margins of a threshold: a
    flagged near plane, or flagged rectangle edges (or 3-sigma radius) whose
    other possible floor (or ceiling) would change whether the clamped
    rectangle is empty. A flagged edge of a Gaussian far off screen, or of a
    wide rectangle, moves a border that does not decide M_t."""
    import itertools
    b = rec["near_bits"]
    amb = (b & 1) != 0
    front = (rec["p"][:, 2] > 0) & ((b & (2 | 4 | 8 | 16 | 32)) != 0)
    idx = np.nonzero(front & ~amb)[0]
    if idx.size == 0:
        return amb
    gx, gy = (cam.width + 15) // 16, (cam.height + 15) // 16
    u, v, rad, bb = rec["uv"][idx, 0], rec["uv"][idx, 1], rec["radius"][idx], b[idx]

    def alts(q, bit):
        f = np.floor(q)
        m = np.round(q)
        return [np.where((bb & bit) != 0, m - 1, f), np.where((bb & bit) != 0, m, f)]

    empties = []
    for dr in (-1.0, 0.0, 1.0):
        r = np.where((bb & 32) != 0, rad + dr, rad)
        for x0, x1, y0, y1 in itertools.product(alts((u - r) / 16, 2), alts((u + r + 15) / 16, 4),
                                                alts((v - r) / 16, 8), alts((v + r + 15) / 16, 16)):
            w = np.clip(x1, 0, gx) - np.clip(x0, 0, gx)
            h = np.clip(y1, 0, gy) - np.clip(y0, 0, gy)
            empties.append((w <= 0) | (h <= 0))
    e = np.stack(empties)
    amb = amb.copy()
    amb[idx] = e.any(0) != e.all(0)
    return amb


def _full_rig_pairs_isolated(res, cams, rng, n_unreached=200_000):
    """The stage-isolated sort check of the parity tests at full size: the
    GPU's pairs against the oracle's keys and stable sort of the GPU's FP32
    splats (every pair), unreachability of a sample of the left-out pairs."""
    from test_gpu_parity import _assert_unreached, _oracle_pairs
    ov, ot = _oracle_pairs(res, cams)
    gv = res["sorted_splats"].astype(np.int64)
    gt = res["sorted_tiles"].astype(np.int64)
    S = max(int(res["xy"].shape[0]), 1)
    keep = np.isin(ot * S + ov, gt * S + gv)
    assert int(keep.sum()) == gv.size
    np.testing.assert_array_equal(gv, ov[keep])
    np.testing.assert_array_equal(gt, ot[keep])
    out = np.nonzero(~keep)[0]
    pick = out if out.size <= n_unreached else rng.choice(out, n_unreached, replace=False)
    _assert_unreached(res, cams, ov[pick], ot[pick])
    ranges = np.zeros((res["ranges"].shape[0], 2), np.int64)
    first = np.r_[0, np.nonzero(np.diff(gt))[0] + 1]
    last = np.r_[first[1:], gt.size]
    ranges[gt[first], 0] = first
    ranges[gt[first], 1] = last
    np.testing.assert_array_equal(res["ranges"].astype(np.int64), ranges)
    return int(ov.size), int(out.size), int(pick.size)


def test_rig_full_size_sampled():
    import gpu_helpers
    from paper_2503_08217_gb300 import binding, build
    from paper_2503_08217_gb300.render import DeviceScene, Renderer
    build.build()
    binding.load()
    scene = scenegen.generate("rig", seed=0)
    k = scene.n_steps // 2
    cams = scene.cams[k]
    lod = 1.0
    n = scene.n
    rng = np.random.default_rng(5)

    # GPU, bench launch configuration and state: the first-epoch sweep with
    # every Gaussian selectable, Eq. 5 into the point lives, then Eq. 6
    max_splats = max(4096, int(n * min(len(cams), 3)))
    r = Renderer(n, scene.n_inst, cams, max_splats=max_splats, max_duplicates=min(2**31 - 1, 6 * max_splats))
    dev = DeviceScene.from_host(scene)
    cs = dev.c_scene()
    vis_t = torch.empty((n, 2), device="cuda")
    life_t = torch.empty((n, 2), device="cuda")
    binding.update_visibility(n, 0.0, None, life_t, vis_t, binding.VIS_RESET)
    all_vis = vis_t.clone()
    for kk in range(scene.n_steps):
        iq = torch.from_numpy(scene.inst_quat[kk]).cuda()
        it = torch.from_numpy(scene.inst_trans[kk]).cuda()
        r.ws.project(cs, binding.make_poses(iq, it), scene.cams[kk], float(scene.times[kk]), all_vis,
                     life_t, lod)
    binding.update_visibility(n, 0.0, None, life_t, vis_t, binding.VIS_FINALIZE)
    torch.cuda.synchronize()
    r.counts()      # a capacity flag of the sweep's projections is not part of this check
    vis = vis_t.cpu().numpy()
    life = life_t.cpu().numpy()
    del all_vis

    # the oracle's own sweep of sampled Gaussians (M_t is per Gaussian: with
    # every window open, a Gaussian's record depends on its own projections only)
    samp = np.sort(rng.choice(n, 20_000, replace=False))
    _, life_o = oracle.vis_reset(samp.size)
    near_any = np.zeros(samp.size, bool)
    for kk in range(scene.n_steps):
        mt = np.zeros(samp.size, bool)
        for cam in scene.cams[kk]:
            rec = oracle.project(scene, samp, kk, cam, lod)
            mt |= rec["infrustum"]
            near_any |= _mt_ambiguous(rec, cam)
        oracle.vis_record(life_o, mt, np.float32(scene.times[kk]))
    vis_o = oracle.vis_finalize(life_o)
    ok = ~near_any
    np.testing.assert_array_equal(life[samp][ok], life_o[ok])
    np.testing.assert_array_equal(vis[samp][ok], vis_o[ok])
    assert near_any.sum() <= 3e-3 * samp.size
    t = float(scene.times[k])
    sel = oracle.select(vis, t)
    # (seven cameras that look all around see every Gaussian of the straight
    # corridor at some timestep before or after the middle one, so here every
    # window contains t: the record selects all of them)
    assert sel.size > 0

    # oracle projection of every camera (FP64), and the pixel samples
    recs = [oracle.project(scene, sel, k, cam, lod) for cam in cams]
    samples, dL = [], []
    cand = excl = flagged = 0
    for v, cam in enumerate(cams):
        bad = gpu_helpers.bad_pixels(cam, recs[v], np.zeros((cam.height, cam.width), bool))
        py = rng.integers(0, cam.height, 400)
        px = rng.integers(0, cam.width, 400)
        keep = ~bad[py, px]
        cand += py.size
        excl += int((~keep).sum())
        pix = np.unique(np.stack([py[keep], px[keep]], 1), axis=0)
        pix = pix[rng.permutation(pix.shape[0])][:48]
        o = oracle.render_pixels(oracle.select_splats(recs[v]), pix[:, 1], pix[:, 0])
        flagged += int(o["flag"].sum())
        pix = pix[~o["flag"]][:24]          # no near-threshold blend decision
        assert pix.shape[0] == 24
        samples.append((pix[:, 1], pix[:, 0]))
        d = np.zeros((3, cam.height, cam.width))
        d[:, pix[:, 0], pix[:, 1]] = rng.standard_normal((3, pix.shape[0]))
        dL.append(d)

    res = gpu_helpers.gpu_step(scene, k, cams, vis, life=life, lod=lod, dL=dL, renderer=r, dev=dev)
    assert res["counts"]["n_splats"] > 1_000_000 and res["counts"]["n_duplicates"] > 10_000_000
    np.testing.assert_array_equal(res["selected"], sel)
    # Eq. 5 at the bench's timestep leaves the finalised lives as they were
    # (every Gaussian in a frustum now was in it when the record was taken)
    np.testing.assert_array_equal(res["life"], life)

    # sampled Gaussians: masks and splat records
    gids = gpu_helpers.splat_gids(res)
    picks = rng.choice(sel.shape[0], 3000, replace=False)
    checked = near_picks = 0
    for j in picks:
        near = any(recs[v]["near"][j] for v in range(len(cams)))
        if near:
            near_picks += 1
            continue
        fm = sum(int(recs[v]["infrustum"][j]) << v for v in range(len(cams)))
        km = sum(int(recs[v]["kept"][j]) << v for v in range(len(cams)))
        assert int(res["frustum_mask"][j]) == fm
        assert int(res["keep_mask"][j]) == km
        s = int(res["splat_start"][j])
        for v in range(len(cams)):
            if not (km >> v) & 1:
                continue
            rec = recs[v]
            assert gids[s] == sel[j] and res["view"][s] == v
            u, vv = rec["uv"][j]
            assert abs(res["xy"][s, 0] - u) <= 1e-5 * abs(u) + 2e-4
            assert abs(res["xy"][s, 1] - vv) <= 1e-5 * abs(vv) + 2e-4
            np.testing.assert_allclose(res["conic_o"][s, :3], rec["conic"][j], rtol=1e-3,
                                       atol=1e-5 * np.abs(rec["conic"][j]).max())
            np.testing.assert_allclose(res["rgb_d"][s, :3], rec["rgb"][j], atol=2e-5)
            np.testing.assert_array_equal(res["rect"][s], rec["rect"][j])
            s += 1
            checked += 1
    assert checked > 500 and near_picks <= 3e-3 * len(cams) * picks.size

    # every pair of the 50,400 tiles, sorted with two tile-digit passes
    assert res["ranges"].shape[0] == 50_400
    n_rect, n_out, n_checked = _full_rig_pairs_isolated(res, cams, rng)

    # sampled pixels and the gradient of a loss on them
    grads = oracle.zero_grads(scene)
    for v, cam in enumerate(cams):
        sp = oracle.select_splats(recs[v])
        px, py = samples[v]
        o = oracle.render_pixels(sp, px, py)
        assert not o["flag"].any()
        got = res["images"][v][:, py, px].T
        assert np.abs(got - o["rgb"]).max() <= 1e-4
        dpix = dL[v][:, py, px].T.copy()
        gs = oracle.render_backward_pixels(sp, px, py, dpix)
        touched = np.nonzero((np.abs(gs["uv"]).sum(1) + np.abs(gs["rgb"]).sum(1) + np.abs(gs["opacity"])) > 0)[0]
        kept_idx = np.nonzero(recs[v]["kept"])[0][touched]
        sub = {key: gs[key][touched] for key in ("uv", "conic", "opacity", "rgb")}
        oracle.project_backward(scene, sel[kept_idx], k, cam, lod, sub, grads)
    for name in ("means", "log_scales", "quats", "opacity_logits", "sh"):
        a = res["grads"][name].reshape(-1)
        b = grads[name].reshape(-1)
        nz = np.abs(b) > 0
        assert nz.sum() > 100, name
        rel = np.linalg.norm(a - b) / np.linalg.norm(b)
        assert rel <= 1e-3, (name, rel)
    for name in ("inst_quat", "inst_trans"):
        b = grads[name]
        if np.abs(b).max() > 0:
            rel = np.linalg.norm(res["grads"][name] - b) / np.linalg.norm(b)
            assert rel <= 1e-3, (name, rel)
    gpu_helpers.report("full rig", selected=f"{sel.size}/{n}",
                       record_sample_near_threshold=f"{int(near_any.sum())}/{samp.size}",
                       gaussian_sample_near_threshold=f"{near_picks}/{picks.size}",
                       pixel_candidates_excluded=f"{excl}/{cand}",
                       pixel_blend_flagged=f"{flagged}/{48 * len(cams)}",
                       sorted_pairs=int(res["sorted_tiles"].size), rectangle_pairs=n_rect,
                       left_out_checked_unreachable=f"{n_checked}/{n_out}")


def test_corridor_x4_sampled():
    """The largest scale of the scene-size sweep (Fig. 4 analogue): the large
    corridor stretched four times at constant density (36M Gaussians, 320
    instances, 6 km), one 1920x1280 camera at the middle timestep, every
    Gaussian selected, LOD 1 px: masks and splat records of 3000 sampled
    Gaussians, 24 sampled pixels, and the gradient of a loss on those pixels,
    against the FP64 oracle. Index widths: the splat and pair counts of the
    sweep's largest scene."""
    import gpu_helpers
    from paper_2503_08217_gb300 import binding, build
    from paper_2503_08217_gb300.render import DeviceScene, Renderer
    build.build()
    binding.load()
    scene = scenegen.generate("large", seed=0, length_scale=4.0)
    n = scene.n
    assert n > 35_000_000
    k = scene.n_steps // 2
    cams = scene.cams[k]
    cam = cams[0]
    lod = 1.0
    rng = np.random.default_rng(8)
    vis, _ = oracle.vis_reset(n)
    sel = np.arange(n)
    rec = oracle.project(scene, sel, k, cam, lod)
    bad = gpu_helpers.bad_pixels(cam, rec, np.zeros((cam.height, cam.width), bool))
    py = rng.integers(0, cam.height, 400)
    px = rng.integers(0, cam.width, 400)
    keep = ~bad[py, px]
    pix = np.unique(np.stack([py[keep], px[keep]], 1), axis=0)
    pix = pix[rng.permutation(pix.shape[0])][:48]
    sp = oracle.select_splats(rec)
    o = oracle.render_pixels(sp, pix[:, 1], pix[:, 0])
    flagged = int(o["flag"].sum())
    pix = pix[~o["flag"]][:24]
    assert pix.shape[0] == 24
    d = np.zeros((3, cam.height, cam.width))
    d[:, pix[:, 0], pix[:, 1]] = rng.standard_normal((3, pix.shape[0]))

    max_splats = n
    r = Renderer(n, scene.n_inst, cams, max_splats=max_splats, max_duplicates=min(2**31 - 1, 6 * max_splats))
    dev = DeviceScene.from_host(scene)
    res = gpu_helpers.gpu_step(scene, k, cams, vis, lod=lod, dL=[d], renderer=r, dev=dev)
    assert res["counts"]["n_selected"] == n and res["counts"]["n_splats"] > 500_000

    gids = gpu_helpers.splat_gids(res)
    # half of the samples from everywhere (most are outside the one camera's
    # frustum), half from the Gaussians the oracle keeps
    picks = np.unique(np.concatenate([rng.choice(n, 1500, replace=False),
                                      rng.choice(np.nonzero(rec["kept"])[0], 1500, replace=False)]))
    checked = near_picks = 0
    for j in picks:
        if rec["near"][j]:
            near_picks += 1
            continue
        assert int(res["frustum_mask"][j]) == int(rec["infrustum"][j])
        assert int(res["keep_mask"][j]) == int(rec["kept"][j])
        if rec["kept"][j]:
            s = int(res["splat_start"][j])
            assert gids[s] == j
            u, vv = rec["uv"][j]
            assert abs(res["xy"][s, 0] - u) <= 1e-5 * abs(u) + 2e-4
            assert abs(res["xy"][s, 1] - vv) <= 1e-5 * abs(vv) + 2e-4
            np.testing.assert_allclose(res["conic_o"][s, :3], rec["conic"][j], rtol=1e-3,
                                       atol=1e-5 * np.abs(rec["conic"][j]).max())
            np.testing.assert_allclose(res["rgb_d"][s, :3], rec["rgb"][j], atol=2e-5)
            np.testing.assert_array_equal(res["rect"][s], rec["rect"][j])
            checked += 1
    assert checked > 1000 and near_picks <= 3e-3 * picks.size

    got = res["images"][0][:, pix[:, 0], pix[:, 1]].T
    o = oracle.render_pixels(sp, pix[:, 1], pix[:, 0])
    assert np.abs(got - o["rgb"]).max() <= 1e-4
    grads = oracle.zero_grads(scene)
    gs = oracle.render_backward_pixels(sp, pix[:, 1], pix[:, 0], d[:, pix[:, 0], pix[:, 1]].T.copy())
    touched = np.nonzero((np.abs(gs["uv"]).sum(1) + np.abs(gs["rgb"]).sum(1) + np.abs(gs["opacity"])) > 0)[0]
    kept_idx = np.nonzero(rec["kept"])[0][touched]
    sub = {key: gs[key][touched] for key in ("uv", "conic", "opacity", "rgb")}
    oracle.project_backward(scene, sel[kept_idx], k, cam, lod, sub, grads)
    for name in ("means", "log_scales", "quats", "opacity_logits", "sh"):
        a = res["grads"][name].reshape(-1)
        b = grads[name].reshape(-1)
        assert (np.abs(b) > 0).sum() > 50, name
        rel = np.linalg.norm(a - b) / np.linalg.norm(b)
        assert rel <= 1e-3, (name, rel)
    gpu_helpers.report("corridor x4 (36M)", gaussians=n, splats=res["counts"]["n_splats"],
                       pairs=res["counts"]["n_duplicates"],
                       gaussian_sample_near_threshold=f"{near_picks}/{picks.size}",
                       pixel_blend_flagged=f"{flagged}/48")



def test_training_corridor_rig_sampled():
    """The training configuration's scene (16M static Gaussians over 2 km,
    120 instances, SH3) seen by the 7-camera rig in one batched call, every
    Gaussian selected, LOD 1 px: masks and splat records of sampled
    Gaussians in every view, 16 sampled pixels of each camera, and the
    gradient of a loss on them, against the FP64 oracle. The oracle keeps
    one view's full records at a time; the sampled Gaussians' records are
    projected again on their own (a record depends only on its Gaussian)."""
    import gpu_helpers
    from paper_2503_08217_gb300 import binding, build
    from paper_2503_08217_gb300.render import DeviceScene, Renderer
    build.build()
    binding.load()
    scene = scenegen.generate("train", seed=0)
    n = scene.n
    assert n > 16_000_000
    k = scene.n_steps // 2
    cams = scene.cams[k]
    V = len(cams)
    lod = 1.0
    rng = np.random.default_rng(21)
    vis, _ = oracle.vis_reset(n)
    sel = np.arange(n)
    kept = np.zeros((V, n), bool)
    splats, samples, dL, flagged = [], [], [], 0
    for v, cam in enumerate(cams):
        rec = oracle.project(scene, sel, k, cam, lod, view=v)
        kept[v] = rec["kept"]
        bad = gpu_helpers.bad_pixels(cam, rec, np.zeros((cam.height, cam.width), bool))
        sp = oracle.select_splats(rec)
        del rec
        py = rng.integers(0, cam.height, 300)
        px = rng.integers(0, cam.width, 300)
        keep = ~bad[py, px]
        pix = np.unique(np.stack([py[keep], px[keep]], 1), axis=0)
        pix = pix[rng.permutation(pix.shape[0])][:32]
        o = oracle.render_pixels(sp, pix[:, 1], pix[:, 0])
        flagged += int(o["flag"].sum())
        pix = pix[~o["flag"]][:16]
        assert pix.shape[0] == 16
        splats.append(sp)
        samples.append((pix[:, 1], pix[:, 0]))
        d = np.zeros((3, cam.height, cam.width))
        d[:, pix[:, 0], pix[:, 1]] = rng.standard_normal((3, pix.shape[0]))
        dL.append(d)

    max_splats = int(n * 3)
    r = Renderer(n, scene.n_inst, cams, max_splats=max_splats, max_duplicates=min(2**31 - 1, 6 * max_splats))
    dev = DeviceScene.from_host(scene)
    res = gpu_helpers.gpu_step(scene, k, cams, vis, lod=lod, dL=dL, renderer=r, dev=dev)
    assert res["counts"]["n_selected"] == n

    gids = gpu_helpers.splat_gids(res)
    picks = np.unique(np.concatenate([rng.choice(n, 1000, replace=False),
                                      rng.choice(np.nonzero(kept.any(0))[0], 2000, replace=False)]))
    precs = [oracle.project(scene, picks, k, cam, lod, view=v) for v, cam in enumerate(cams)]
    for v in range(V):
        assert (precs[v]["kept"] == kept[v, picks]).all()
    checked = near_picks = 0
    for i, j in enumerate(picks):
        if any(pr["near"][i] for pr in precs):
            near_picks += 1
            continue
        fm = sum(int(precs[v]["infrustum"][i]) << v for v in range(V))
        km = sum(int(precs[v]["kept"][i]) << v for v in range(V))
        assert int(res["frustum_mask"][j]) == fm and int(res["keep_mask"][j]) == km
        s = int(res["splat_start"][j])
        for v in range(V):
            if not (km >> v) & 1:
                continue
            pr = precs[v]
            assert gids[s] == j and res["view"][s] == v
            u, vv = pr["uv"][i]
            assert abs(res["xy"][s, 0] - u) <= 1e-5 * abs(u) + 2e-4
            assert abs(res["xy"][s, 1] - vv) <= 1e-5 * abs(vv) + 2e-4
            np.testing.assert_allclose(res["rgb_d"][s, :3], pr["rgb"][i], atol=2e-5)
            np.testing.assert_array_equal(res["rect"][s], pr["rect"][i])
            s += 1
            checked += 1
    assert checked > 1000 and near_picks <= 3e-3 * V * picks.size

    grads = oracle.zero_grads(scene)
    for v, cam in enumerate(cams):
        sp = splats[v]
        px, py = samples[v]
        o = oracle.render_pixels(sp, px, py)
        assert np.abs(res["images"][v][:, py, px].T - o["rgb"]).max() <= 1e-4
        gs = oracle.render_backward_pixels(sp, px, py, dL[v][:, py, px].T.copy())
        touched = np.nonzero((np.abs(gs["uv"]).sum(1) + np.abs(gs["rgb"]).sum(1) + np.abs(gs["opacity"])) > 0)[0]
        sub = {key: gs[key][touched] for key in ("uv", "conic", "opacity", "rgb")}
        oracle.project_backward(scene, sp["gid"][touched], k, cam, lod, sub, grads)
    for name in ("means", "log_scales", "quats", "opacity_logits", "sh"):
        a = res["grads"][name].reshape(-1)
        b = grads[name].reshape(-1)
        assert (np.abs(b) > 0).sum() > 50, name
        rel = np.linalg.norm(a - b) / np.linalg.norm(b)
        assert rel <= 1e-3, (name, rel)
    gpu_helpers.report("training corridor rig (16M+)", gaussians=n, splats=res["counts"]["n_splats"],
                       pairs=res["counts"]["n_duplicates"],
                       gaussian_sample_near_threshold=f"{near_picks}/{picks.size}",
                       pixel_blend_flagged=f"{flagged}/{32 * V}")
