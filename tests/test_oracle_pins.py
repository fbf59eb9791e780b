"""Pins for the FP64 oracle: closed forms, special cases, invariants, brute
force, finite differences and an independent float64 torch restatement.

These run on the CPU only. Each pin is chosen so that a plausible slip in the
oracle (a dropped term, a wrong sign, a transposed matrix, a wrong constant)
fails at least one of them.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2503_08217_gb300 import scenegen
import torch_ref


def _single_scene(gaussians, cam, *, sh_degree=0, n_inst=0, inst_q=None, inst_t=None, offsets=None):
    """A hand-built scene: gaussians = list of (mean, log_scale, quat, opac_logit, sh[K,3])."""
    n = len(gaussians)
    K = (sh_degree + 1) ** 2
    means = np.array([g[0] for g in gaussians], np.float32).reshape(n, 3)
    ls = np.array([g[1] for g in gaussians], np.float32).reshape(n, 3)
    qs = np.array([g[2] for g in gaussians], np.float32).reshape(n, 4)
    ol = np.array([g[3] for g in gaussians], np.float32).reshape(n)
    sh = np.array([g[4] for g in gaussians], np.float32).reshape(n, K, 3)
    if offsets is None:
        offsets = np.array([0, n], np.int64)
    iq = np.zeros((1, n_inst, 4), np.float32) if inst_q is None else inst_q[None].astype(np.float32)
    it = np.zeros((1, n_inst, 3), np.float32) if inst_t is None else inst_t[None].astype(np.float32)
    return scenegen.Scene(name="hand", means=means, log_scales=ls, quats=qs, opacity_logits=ol,
                          sh=sh, sh_degree=sh_degree, inst_offsets=np.asarray(offsets, np.int64),
                          inst_quat=iq, inst_trans=it, times=np.zeros(1, np.float32),
                          cams=[[cam]], lod_threshold=0.0)


def _render_scene(scene, lod_r=0.0, bg=(0.0, 0.0, 0.0), tiled=False):
    vis, life = oracle.vis_reset(scene.n)
    return oracle.step_forward(scene, 0, vis, life, lod_r, bg=bg, tiled=tiled)


# ---------------------------------------------------------------- SH basis
def test_sh_basis_orthonormal_on_sphere():
    """Real SH up to degree 3 integrate to the identity over the sphere
    (Gauss-Legendre in cos(theta) x uniform phi, exact for these degrees)."""
    xs, ws = np.polynomial.legendre.leggauss(16)
    nphi = 32
    G = np.zeros((16, 16))
    for ct, w in zip(xs, ws):
        st = math.sqrt(1 - ct * ct)
        for j in range(nphi):
            ph = 2 * math.pi * j / nphi
            d = np.array([st * math.cos(ph), st * math.sin(ph), ct])
            Y, _ = oracle.sh_basis(d)
            G += w * (2 * math.pi / nphi) * np.outer(Y, Y)
    np.testing.assert_allclose(G, np.eye(16), atol=1e-12)


def test_sh_basis_gradient_matches_difference_quotient():
    rng = np.random.default_rng(3)
    for _ in range(5):
        d = rng.standard_normal(3)
        _, dY = oracle.sh_basis(d)
        h = 1e-6
        for r in range(3):
            e = np.zeros(3)
            e[r] = h
            fd = (oracle.sh_basis(d + e)[0] - oracle.sh_basis(d - e)[0]) / (2 * h)
            np.testing.assert_allclose(dY[:, r], fd, rtol=1e-7, atol=1e-8)


def test_sh_degree1_is_linear_in_direction():
    """Degree-1 real SH are sqrt(3/(4 pi)) * (-y, z, -x) (textbook, CS phase)."""
    d = np.array([0.36, -0.48, 0.8])
    Y, _ = oracle.sh_basis(d)
    k = math.sqrt(3 / (4 * math.pi))
    np.testing.assert_allclose(Y[1:4], k * np.array([0.48, 0.8, -0.36]), rtol=1e-14)
    assert Y[0] == pytest.approx(1 / (2 * math.sqrt(math.pi)), rel=1e-15)


# ---------------------------------------------------------------- closed forms
IDENTITY_W2C = np.array([[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 1, 0]], np.float32)


def _cam(w=64, h=64, f=250.0):
    return scenegen.Camera(width=w, height=h, fx=f, fy=f, cx=0.5 * w, cy=0.5 * h, near=0.2,
                           world_to_cam=IDENTITY_W2C)


def _closed_form_alpha(o, s, z, f, W, H):
    """Isotropic Gaussian on the optical axis: Sigma2 = (f s / z)^2 I, dilated
    by 0.3, centred on the principal point (W/2, H/2)."""
    var = (f * s / z) ** 2 + 0.3
    py, px = np.mgrid[0:H, 0:W]
    r2 = (px + 0.5 - W / 2) ** 2 + (py + 0.5 - H / 2) ** 2
    a = np.minimum(0.99, o * np.exp(-0.5 * r2 / var))
    return np.where(a >= 1 / 255, a, 0.0), var


def _s32(s):
    """The scale the oracle sees: exp of the float32-rounded log-scale."""
    return math.exp(float(np.float32(math.log(s))))


def test_single_gaussian_closed_form_footprint():
    s, z, f, W, H = _s32(0.1), 10.0, 250.0, 64, 64
    logit = 0.25
    o = 1 / (1 + math.exp(-logit))
    dc = np.array([0.5, -1.0, 1.5])
    g = ((0, 0, z), [math.log(s)] * 3, (0.6, 0.0, 0.8, 0.0), logit, dc[None])
    sc = _single_scene([g], _cam(W, H, f))
    out = _render_scene(sc)
    view = out["views"][0]
    rec = view["rec"]
    # 2D scale = f s / z exactly; colour = 0.5 + dc / (2 sqrt(pi))
    assert rec["sigma_lod"][0] == pytest.approx(f * s / z, rel=1e-12)
    rgb = 0.5 + dc * (0.5 / math.sqrt(math.pi))
    np.testing.assert_allclose(rec["rgb"][0], rgb, rtol=1e-12)
    alpha, var = _closed_form_alpha(o, s, z, f, W, H)
    np.testing.assert_allclose(rec["conic"][0], [1 / var, 0.0, 1 / var], rtol=1e-12, atol=1e-15)
    x0, y0, x1, y1 = rec["rect"][0]
    inside = np.zeros((H, W), bool)
    inside[y0 * 16:y1 * 16, x0 * 16:x1 * 16] = True
    for ch in range(3):
        np.testing.assert_allclose(view["image"][ch][inside], rgb[ch] * alpha[inside], rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(view["T"][inside], 1 - alpha[inside], rtol=1e-12)


def test_two_gaussians_analytic_blend():
    """Two isotropic Gaussians on the axis: C = c1 a1 + c2 a2 (1 - a1)."""
    f, W, H = 250.0, 64, 64
    g1 = ((0, 0, 10.0), [math.log(0.1)] * 3, (1, 0, 0, 0), 0.5, np.array([[1.0, 0.0, -1.0]]))
    g2 = ((0, 0, 20.0), [math.log(0.3)] * 3, (1, 0, 0, 0), 1.5, np.array([[-1.0, 1.0, 0.25]]))
    sc = _single_scene([g2, g1], _cam(W, H, f))          # index order != depth order
    out = _render_scene(sc)
    img = out["views"][0]["image"]
    a1, _ = _closed_form_alpha(1 / (1 + math.exp(-0.5)), _s32(0.1), 10.0, f, W, H)
    a2, _ = _closed_form_alpha(1 / (1 + math.exp(-1.5)), _s32(0.3), 20.0, f, W, H)
    k = 0.5 / math.sqrt(math.pi)
    c1 = 0.5 + k * np.array([1.0, 0.0, -1.0])
    c2 = 0.5 + k * np.array([-1.0, 1.0, 0.25])
    # both rects cover the full 64 x 64 image for these footprints
    for ch in range(3):
        np.testing.assert_allclose(img[ch], c1[ch] * a1 + c2[ch] * a2 * (1 - a1), rtol=1e-12, atol=1e-15)


def test_near_plane_and_offscreen_are_not_visible():
    f, W, H = 250.0, 64, 64
    gs = [((0, 0, 0.1), [-2] * 3, (1, 0, 0, 0), 0.0, np.zeros((1, 3))),     # in front of near plane
          ((0, 0, -5.0), [-2] * 3, (1, 0, 0, 0), 0.0, np.zeros((1, 3))),    # behind the camera
          ((100.0, 0, 5.0), [-2] * 3, (1, 0, 0, 0), 0.0, np.zeros((1, 3))),  # far off to the side
          ((0, 0, 5.0), [-2] * 3, (1, 0, 0, 0), 0.0, np.zeros((1, 3)))]     # visible
    sc = _single_scene(gs, _cam(W, H, f))
    rec = _render_scene(sc)["views"][0]["rec"]
    assert list(rec["infrustum"]) == [False, False, False, True]


# ---------------------------------------------------------------- invariants
@pytest.fixture(scope="module")
def tiny():
    return scenegen.generate("tiny", seed=0)


def test_untiled_brute_force_equals_tiled(tiny):
    vis, _ = oracle.vis_reset(tiny.n)
    for step in (0, 4, 9):
        a = oracle.step_forward(tiny, step, vis, None, 0.0)
        for view in a["views"]:
            b = oracle.render(320, 192, view["splats"], tiled=True)
            np.testing.assert_array_equal(view["image"], b["image"])
            np.testing.assert_array_equal(view["n_contrib"], b["n_contrib"])


def test_tile_keys_match_numpy_stable_sort(tiny):
    vis, _ = oracle.vis_reset(tiny.n)
    sp = oracle.step_forward(tiny, 3, vis, None, 0.0)["views"][0]["splats"]
    keys, vals, ranges = oracle.tile_keys(320, 192, sp["depth32"], sp["rect"], tile_base=7)
    gx = 20
    ks, vs = [], []
    for i, (x0, y0, x1, y1) in enumerate(sp["rect"]):
        for ty in range(y0, y1):
            for tx in range(x0, x1):
                ks.append(((7 + ty * gx + tx) << 32) | int(sp["depth32"][i].view(np.uint32)))
                vs.append(i)
    ks = np.array(ks, np.uint64)
    order = np.argsort(ks, kind="stable")
    np.testing.assert_array_equal(keys, ks[order])
    np.testing.assert_array_equal(vals, np.array(vs)[order])
    tiles = (keys >> np.uint64(32)).astype(np.int64) - 7
    for t in range(ranges.shape[0]):
        idx = np.nonzero(tiles == t)[0]
        if idx.size:
            assert ranges[t, 0] == idx[0] and ranges[t, 1] == idx[-1] + 1
        else:
            assert ranges[t, 0] == ranges[t, 1]


def test_transmittance_and_image_bounds(tiny):
    vis, _ = oracle.vis_reset(tiny.n)
    black = oracle.step_forward(tiny, 2, vis, None, 0.0)["views"][0]
    white = oracle.step_forward(tiny, 2, vis, None, 0.0, bg=(1.0, 1.0, 1.0))["views"][0]
    # SH degree 0 colours lie in [0, 1]; the composite with a white background
    # stays in [0, 1] and differs from the black one by exactly T
    assert black["splats"]["rgb"].min() >= 0 and black["splats"]["rgb"].max() <= 1
    assert white["image"].min() >= 0 and white["image"].max() <= 1 + 1e-12
    np.testing.assert_allclose(white["image"] - black["image"], np.broadcast_to(black["T"], (3, 192, 320)),
                               atol=1e-12)
    assert black["T"].max() <= 1 and black["T"].min() >= 1e-4 * (1 - 0.99)
    # pixels with no contributor keep T = 1
    assert np.all(black["T"][black["n_contrib"] == 0] == 1.0)


def test_transmittance_monotone_along_each_list(tiny):
    """Cutting every list after its first k entries can only raise T."""
    vis, _ = oracle.vis_reset(tiny.n)
    sp = oracle.step_forward(tiny, 5, vis, None, 0.0)["views"][0]["splats"]
    order = np.lexsort((sp["gid"], sp["depth32"]))
    prev = np.zeros((192, 320))
    for frac in (0.0, 0.25, 0.5, 0.75, 1.0):
        keep = order[: int(frac * order.size)]
        sub = {k: v[keep] for k, v in sp.items()}
        T = oracle.render(320, 192, sub)["T"]
        # T of a prefix of the front-to-back list is >= T of a longer prefix
        if frac > 0:
            assert np.all(T <= prev + 1e-15)
        prev = T


def test_lod_zero_equals_no_culling_and_is_monotone(tiny):
    vis, _ = oracle.vis_reset(tiny.n)
    a = oracle.step_forward(tiny, 4, vis, None, 0.0)["views"][0]
    b = oracle.step_forward(tiny, 4, vis, None, -1.0)["views"][0]
    np.testing.assert_array_equal(a["rec"]["kept"], a["rec"]["infrustum"])
    np.testing.assert_array_equal(a["rec"]["kept"], b["rec"]["kept"])
    np.testing.assert_array_equal(a["image"], b["image"])
    prev = a["rec"]["kept"]
    for r in (0.25, 0.5, 1.0, 2.0, 4.0):
        k = oracle.step_forward(tiny, 4, vis, None, r)["views"][0]["rec"]["kept"]
        assert np.all(prev >= k) and k.sum() < prev.sum()
        prev = k
    empty = oracle.step_forward(tiny, 4, vis, None, 1e9, bg=(0.2, 0.3, 0.4))["views"][0]
    for ch, val in enumerate((0.2, 0.3, 0.4)):
        assert np.all(empty["image"][ch] == val)


def test_instance_matrix_equals_transform_then_project():
    """Sec. 3.3 instance-specific projection: M = V * P gives the same 2D
    Gaussians as transforming to the world frame first (Fig. 1(a))."""
    sc = scenegen.generate("fd", seed=5)
    vis, _ = oracle.vis_reset(sc.n)
    sel = oracle.select(vis, float(sc.times[1]))
    for cam in (sc.cams[1][0], scenegen.make_camera(96, 80, 70.0, (0.5, -0.2, -1.0), 0.2)):
        a = oracle.project(sc, sel, 1, cam, 0.0)
        b = oracle.project(sc, sel, 1, cam, 0.0, conventional=True)
        dyn = a["inst"] > 0
        assert dyn.sum() == 20 and a["infrustum"][dyn].sum() > 0
        np.testing.assert_array_equal(a["infrustum"], b["infrustum"])
        np.testing.assert_array_equal(a["rect"], b["rect"])
        for k in ("p", "uv", "conic", "opacity", "rgb", "sigma_lod", "radius"):
            np.testing.assert_allclose(a[k], b[k], rtol=1e-10, atol=1e-10, err_msg=k)


# ---------------------------------------------------------------- visibility record
def test_visibility_record_exact_values():
    """Eq. 5 and Eq. 6 on a scripted sequence, FP32 throughout."""
    vis, life = oracle.vis_reset(4)
    np.testing.assert_array_equal(vis, [[-1, 1]] * 4)        # initial v (Sec. 3.3)
    np.testing.assert_array_equal(life, [[1, -1]] * 4)       # initial l
    seen = {0.2: [True, False, True, False], -0.5: [False, False, True, False],
            0.25: [False, False, True, True]}
    for t, m in seen.items():
        oracle.vis_record(life, np.array(m), np.float32(t))
    v = oracle.vis_finalize(life)
    # seen only at t = 0.2: window [0.1, 0.3] (exact in FP32)
    assert v[0, 0] == np.float32(0.1) and v[0, 1] == np.float32(0.3)
    # never seen: l stays (1, -1), giving the empty window [0.9, -0.9]
    assert v[1, 0] == np.float32(0.9) and v[1, 1] == np.float32(-0.9)
    # seen at -0.5, 0.2, 0.25: window [-0.6, 0.35]
    assert v[2, 0] == np.float32(-0.6) and v[2, 1] == np.float32(0.35)
    assert v[3, 0] == np.float32(0.15) and v[3, 1] == np.float32(0.35)
    sel = oracle.select(v, np.float32(0.3))
    assert list(sel) == [0, 2, 3]
    assert list(oracle.select(v, np.float32(0.3000001))) == [2, 3]
    assert list(oracle.select(v, np.float32(-1.0))) == []


def test_selection_is_inclusive_fp32():
    vis = np.array([[-0.5, 0.5], [0.5, 0.5], [0.5000001, 1.0], [1.0, -1.0]], np.float32)
    assert list(oracle.select(vis, np.float32(0.5))) == [0, 1]


def test_record_uses_frustum_mask_before_lod(tiny):
    """M_t updates the point life for in-frustum Gaussians whether or not LOD
    culls them (Sec. 3.3 order: project -> M_t -> LOD)."""
    vis, life_a = oracle.vis_reset(tiny.n)
    _, life_b = oracle.vis_reset(tiny.n)
    fa = oracle.step_forward(tiny, 3, vis, life_a, 0.0)
    fb = oracle.step_forward(tiny, 3, vis, life_b, 3.0)
    assert fb["views"][0]["rec"]["kept"].sum() < fa["views"][0]["rec"]["kept"].sum()
    np.testing.assert_array_equal(life_a, life_b)
    t = np.float32(tiny.times[3])
    full = np.zeros(tiny.n, bool)
    full[fa["sel"][fa["mt"]]] = True
    assert np.all(life_a[full] == t) and np.all(life_a[~full] == [1, -1])


# ---------------------------------------------------------------- gradients
def _fd_setup(seed=11, step=1):
    sc = scenegen.generate("fd", seed=seed)
    cam = sc.cams[step][0]
    vis, _ = oracle.vis_reset(sc.n)
    f = oracle.step_forward(sc, step, vis, None, 0.0)
    rec = f["views"][0]["rec"]
    assert not rec["near"][rec["infrustum"]].any()
    return sc, cam, f


def _loss(sc, step, cam, w, **over):
    sc2 = dataclasses.replace(sc, **{k: v for k, v in over.items() if k not in ("inst_quat", "inst_trans")})
    vis, _ = oracle.vis_reset(sc2.n)
    sel = oracle.select(vis, float(sc2.times[step]))
    rec = oracle.project(sc2, sel, step, cam, 0.0, inst_quat=over.get("inst_quat"),
                         inst_trans=over.get("inst_trans"))
    img = oracle.render(cam.width, cam.height, oracle.select_splats(rec))["image"]
    return float((w * img).sum())


def test_gradient_matches_central_finite_differences():
    """FP64 central differences, h = 1e-6, on a 500-Gaussian 64 x 64 crop.
    Pixels whose blend has a decision near a threshold get weight 0."""
    step = 1
    oracle.set_margins(alpha_tol=1e-4, T_tol=1e-6, power_tol=1e-7)
    try:
        sc, cam, f = _fd_setup(step=step)
        rng = np.random.default_rng(0)
        w = rng.standard_normal((3, 64, 64))
        w *= ~f["views"][0]["flag"][None]
        g = oracle.step_backward(sc, step, f, [w], 0.0)
        w *= ~g["pixel_flags"][0][None]
        g = oracle.step_backward(sc, step, f, [w], 0.0)
        # sample parameters of kept Gaussians
        kept = f["sel"][f["views"][0]["rec"]["kept"]]
        picks = rng.choice(kept, size=25, replace=False)
        dyn = kept[kept >= sc.inst_offsets[1]]
        picks = np.concatenate([picks, dyn[:5]])
        h = 1e-6
        checked = 0
        for name, shape in (("means", 3), ("log_scales", 3), ("quats", 4), ("opacity_logits", 1), ("sh", 48)):
            base = getattr(sc, name).astype(np.float64)
            for gi in picks:
                comps = range(shape) if shape <= 4 else rng.choice(shape, 6, replace=False)
                for c in comps:
                    plus, minus = base.copy(), base.copy()
                    idx = (gi,) if shape == 1 else ((gi, c) if name != "sh" else (gi, c // 3, c % 3))
                    plus[idx] += h
                    minus[idx] -= h
                    fd = (_loss(sc, step, cam, w, **{name: plus}) - _loss(sc, step, cam, w, **{name: minus})) / (2 * h)
                    an = g[name][idx]
                    assert abs(fd - an) <= 2e-5 + 2e-4 * abs(an), (name, gi, c, fd, an)
                    checked += 1
        for name in ("inst_quat", "inst_trans"):
            base = getattr(sc, name)[step].astype(np.float64)
            for idx in np.ndindex(base.shape):
                plus, minus = base.copy(), base.copy()
                plus[idx] += h
                minus[idx] -= h
                fd = (_loss(sc, step, cam, w, **{name: plus}) - _loss(sc, step, cam, w, **{name: minus})) / (2 * h)
                an = g[name][idx]
                assert abs(fd - an) <= 2e-5 + 2e-4 * abs(an), (name, idx, fd, an)
                checked += 1
        assert checked > 400
    finally:
        oracle.set_margins()


def test_gradient_matches_torch_autograd_restatement():
    """Independent float64 torch forward + autograd vs the hand-derived
    oracle gradient, including the per-instance pose (q, t)."""
    step = 2
    sc = scenegen.generate("fd", seed=4)
    cam = scenegen.make_camera(48, 40, 45.0, (0.3, 0.1, 0.0), 0.05)
    vis, _ = oracle.vis_reset(sc.n)
    f = oracle.step_forward(sc, step, vis, None, 0.0, cams=[cam])
    rng = np.random.default_rng(1)
    w = rng.standard_normal((3, 40, 48))
    g = oracle.step_backward(sc, step, f, [w], 0.0, cams=[cam])

    params = torch_ref.params_from_scene(sc, step)
    img, T = torch_ref.render_view(params, sc.inst_offsets, cam, 0.0, f["sel"])
    np.testing.assert_allclose(img.detach().numpy(), f["views"][0]["image"], rtol=0, atol=1e-12)
    np.testing.assert_allclose(T.detach().numpy(), f["views"][0]["T"], rtol=0, atol=1e-12)
    (img * torch.as_tensor(w)).sum().backward()
    for name in ("means", "log_scales", "quats", "opacity_logits", "sh", "inst_quat", "inst_trans"):
        ref = params[name].grad.numpy()
        ours = g[name]
        scale = np.abs(ref).max()
        assert scale > 0, name
        np.testing.assert_allclose(ours, ref, rtol=1e-8, atol=1e-10 * scale, err_msg=name)


def test_torch_restatement_matches_oracle_forward_on_tiny_crop():
    sc = scenegen.subset(scenegen.generate("tiny", seed=2), 3000, 300)
    cam = scenegen.make_camera(80, 48, 60.0, (0.0, 0.0, 3.0), 0.0)
    vis, _ = oracle.vis_reset(sc.n)
    f = oracle.step_forward(sc, 3, vis, None, 0.0, cams=[cam], bg=(0.1, 0.2, 0.3))
    params = torch_ref.params_from_scene(sc, 3, requires_grad=False)
    img, _ = torch_ref.render_view(params, sc.inst_offsets, cam, 0.0, f["sel"], bg=(0.1, 0.2, 0.3))
    np.testing.assert_allclose(img.numpy(), f["views"][0]["image"], rtol=0, atol=1e-12)


def test_pixel_subset_render_equals_full_render(tiny):
    """The spot-check entry points (a chosen pixel set) agree with the
    full-image blend and its backward exactly."""
    vis, _ = oracle.vis_reset(tiny.n)
    f = oracle.step_forward(tiny, 4, vis, None, 0.0)
    sp = f["views"][0]["splats"]
    rng = np.random.default_rng(0)
    pix = np.unique(np.stack([rng.integers(0, 192, 80), rng.integers(0, 320, 80)], 1), axis=0)
    py, px = pix[:, 0], pix[:, 1]
    r = oracle.render_pixels(sp, px, py)
    np.testing.assert_array_equal(r["rgb"], f["views"][0]["image"][:, py, px].T)
    np.testing.assert_array_equal(r["n_contrib"], f["views"][0]["n_contrib"][py, px])
    dL = rng.standard_normal((3, 192, 320))
    mask = np.zeros((192, 320), bool)
    mask[py, px] = True
    full = oracle.render_backward(320, 192, sp, dL * mask)
    part = oracle.render_backward_pixels(sp, px, py, dL[:, py, px].T)
    for k in ("uv", "conic", "opacity", "rgb"):
        np.testing.assert_allclose(part[k], full[k], rtol=1e-12, atol=1e-12 * np.abs(full[k]).max())


def test_adam_first_step_closed_form():
    # from zero moments the bias corrections cancel: m_hat = g, v_hat = g^2,
    # so the step is lr * g / (|g| + eps) (Kingma and Ba, Algorithm 1)
    rng = np.random.default_rng(3)
    g = rng.standard_normal(257) * np.exp(rng.uniform(-6, 3, 257))
    g[:3] = [0.0, 1e-12, -1e-12]
    p0 = rng.standard_normal(257)
    lr, b1, b2, eps = 0.01, 0.9, 0.999, 1e-8
    p, m, v = oracle.adam_step(p0, g, np.zeros(257), np.zeros(257), lr, 1, b1, b2, eps)
    np.testing.assert_allclose(m, (1 - b1) * g, rtol=1e-15, atol=0)
    np.testing.assert_allclose(v, (1 - b2) * g * g, rtol=1e-15, atol=0)
    np.testing.assert_allclose(p, p0 - lr * g / (np.abs(g) + eps), rtol=0, atol=1e-15)
    assert p[0] == p0[0]


def test_adam_without_momentum_is_normalised_gradient_every_step():
    # beta1 = beta2 = 0: m = g and v = g^2 at every step, bias corrections are 1
    rng = np.random.default_rng(4)
    p = rng.standard_normal(64)
    m = rng.standard_normal(64)
    v = rng.uniform(0, 1, 64)
    for step in range(1, 4):
        g = rng.standard_normal(64)
        p_new, m, v = oracle.adam_step(p, g, m, v, 0.1, step, 0.0, 0.0, 1e-3)
        np.testing.assert_allclose(p_new, p - 0.1 * g / (np.abs(g) + 1e-3), rtol=0, atol=1e-15)
        np.testing.assert_array_equal(m, g)
        p = p_new


def test_adam_matches_torch_optim_adam_float64():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(5)
    p0 = rng.standard_normal(1000)
    tp = torch.nn.Parameter(torch.tensor(p0, dtype=torch.float64))
    opt = torch.optim.Adam([tp], lr=3e-3, betas=(0.8, 0.95), eps=1e-6)
    p, m, v = p0.copy(), np.zeros(1000), np.zeros(1000)
    for step in range(1, 8):
        g = rng.standard_normal(1000) * (0.1 if step % 2 else 10.0)
        tp.grad = torch.tensor(g, dtype=torch.float64)
        opt.step()
        p, m, v = oracle.adam_step(p, g, m, v, 3e-3, step, 0.8, 0.95, 1e-6)
    st = opt.state[tp]
    np.testing.assert_allclose(p, tp.detach().numpy(), rtol=0, atol=1e-13)
    np.testing.assert_allclose(m, st["exp_avg"].numpy(), rtol=1e-13, atol=0)
    np.testing.assert_allclose(v, st["exp_avg_sq"].numpy(), rtol=1e-13, atol=0)
