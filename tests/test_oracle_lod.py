"""Pins for the oracle's stochastic LOD (Eq. 7) and its counter-based
generator. CPU only.

Eq. 7 draws, for each in-frustum (Gaussian, view) whose 2D scale is below r,
a Bernoulli drop with p = p_max + (p_max - 0.01) min(0, (d - D)/D) and, for
the survivors, a noisy offset [dx, dy, dz] * min(1, d/D) * N(0, 1) per axis.
The draws come from Philox4x32-10 (Salmon et al., SC 2011) with counter
(Gaussian id, view, epoch, block) and key (seed low, seed high).
"""
from __future__ import annotations

import dataclasses
import os

import numpy as np
import pytest

import oracle
from paper_2503_08217_gb300 import scenegen


@pytest.fixture
def lod_off():
    yield
    oracle.set_lod(0)


def test_philox_known_answer_vectors():
    """The known-answer vectors published with the Random123 library for
    philox4x32_10 (zero, all-ones, and pi-digit counter/key), stored in
    tests/golden/philox4x32_10_kat.txt with their citation."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "philox4x32_10_kat.txt")
    cases = 0
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        ctr, key, want = (np.array([int(w, 16) for w in part.split()], np.uint32)
                          for part in line.split("|"))
        np.testing.assert_array_equal(oracle.philox(ctr, key), want)
        cases += 1
    assert cases == 3


def test_philox_outputs_are_uniform_and_balanced():
    """40,000 consecutive counters: the top byte of every output word passes a
    chi-square test over 256 bins, and every one of the 128 output bits is set
    about half the time."""
    n = 40_000
    out = np.array([oracle.philox([i, 7, 3, 0], [0x1234, 0x5678]) for i in range(n)], np.uint32)
    for w in range(4):
        hist = np.bincount(out[:, w] >> 24, minlength=256)
        chi2 = ((hist - n / 256) ** 2 / (n / 256)).sum()
        assert chi2 < 255 + 6 * np.sqrt(2 * 255), (w, chi2)
    bits = ((out[:, :, None] >> np.arange(32, dtype=np.uint32)) & 1).mean(axis=0)
    assert np.abs(bits - 0.5).max() < 5 * 0.5 / np.sqrt(n)


def _cone_scene(n, depths, rng, log_scale=-7.0, cam_w=256, f=200.0):
    """n tiny Gaussians spread over the image of an identity camera at the
    given depths (so the camera frame is the world frame)."""
    u = rng.uniform(16, cam_w - 16, n)
    v = rng.uniform(16, cam_w - 16, n)
    x = (u - cam_w / 2) * depths / f
    y = (v - cam_w / 2) * depths / f
    means = np.stack([x, y, depths], 1).astype(np.float32)
    cam = scenegen.Camera(width=cam_w, height=cam_w, fx=f, fy=f, cx=cam_w / 2, cy=cam_w / 2,
                          near=0.2, world_to_cam=np.hstack([np.eye(3), np.zeros((3, 1))]).astype(np.float32))
    sc = scenegen.Scene(name="cone", means=means,
                        log_scales=np.full((n, 3), log_scale, np.float32),
                        quats=np.tile(np.array([1, 0, 0, 0], np.float32), (n, 1)),
                        opacity_logits=np.zeros(n, np.float32), sh=np.zeros((n, 1, 3), np.float32),
                        sh_degree=0, inst_offsets=np.array([0, n], np.int64),
                        inst_quat=np.zeros((1, 0, 4), np.float32), inst_trans=np.zeros((1, 0, 3), np.float32),
                        times=np.zeros(1, np.float32), cams=[[cam]], lod_threshold=1.0)
    return sc, cam


def test_eq7_drop_rate_follows_depth(lod_off):
    """Dropped fraction per depth bin equals p(d): 0.01 at d -> 0, linear up to
    p_max at d = D, p_max beyond (within 5 binomial standard deviations)."""
    rng = np.random.default_rng(0)
    n = 60_000
    D, pmax = 40.0, 0.6
    d = rng.uniform(1.0, 80.0, n)
    sc, cam = _cone_scene(n, d, rng)
    sel = np.arange(n)
    oracle.set_lod(1, p_max=pmax, dist=D, offset=(0, 0, 0), seed=99, epoch=5)
    rec = oracle.project(sc, sel, 0, cam, 1.0)
    assert rec["infrustum"].all() and (rec["sigma_lod"] < 1.0).all()
    dropped = ~rec["kept"]
    edges = np.linspace(1, 80, 17)
    for lo, hi in zip(edges[:-1], edges[1:]):
        m = (d >= lo) & (d < hi)
        mid = np.clip(d[m], None, None)
        p = pmax + (pmax - 0.01) * np.minimum(0.0, (mid - D) / D)
        exp = p.mean()
        sd = np.sqrt((p * (1 - p)).sum()) / m.sum()
        assert abs(dropped[m].mean() - exp) < 5 * sd + 1e-3, (lo, hi, dropped[m].mean(), exp)
    # beyond D the probability is exactly p_max, below D strictly less
    far = d >= D
    assert abs(dropped[far].mean() - pmax) < 5 * np.sqrt(pmax * (1 - pmax) / far.sum())
    near = d < 5
    assert dropped[near].mean() < 0.2


def test_eq7_spares_gaussians_at_or_above_r(lod_off):
    """Gaussians whose 2D scale is at least r are neither dropped nor moved:
    their records are identical to the deterministic path's."""
    rng = np.random.default_rng(1)
    n = 4000
    d = rng.uniform(2.0, 30.0, n)
    sc, cam = _cone_scene(n, d, rng, log_scale=-1.0)
    sel = np.arange(n)
    oracle.set_lod(0)
    det = oracle.project(sc, sel, 0, cam, 1.0)
    oracle.set_lod(1, p_max=0.9, dist=10.0, offset=(0.5, 0.5, 0.5), seed=3, epoch=1)
    sto = oracle.project(sc, sel, 0, cam, 1.0)
    big = det["kept"]
    assert big.sum() > 100
    np.testing.assert_array_equal(sto["raw"][big], det["raw"][big])
    # and the small ones in the deterministic path are all culled
    assert not det["kept"][det["infrustum"] & ~big].any()


def test_eq7_offset_is_a_scaled_standard_normal(lod_off):
    """Survivors move by offset * min(1, d/D) * N(0, 1) per axis: the
    normalised displacements have mean 0, variance 1, no cross-correlation,
    and the scale saturates at d = D."""
    rng = np.random.default_rng(2)
    n = 30_000
    D = 20.0
    d = rng.uniform(2.0, 40.0, n)
    sc, cam = _cone_scene(n, d, rng)
    off = np.array([0.3, 0.2, 0.5])
    oracle.set_lod(1, p_max=0.01, dist=D, offset=off, seed=11, epoch=2)
    rec = oracle.project(sc, np.arange(n), 0, cam, 1.0)
    k = rec["kept"]
    assert k.mean() > 0.97
    disp = rec["p"][k] - sc.means[k].astype(np.float64)       # identity camera
    z = disp / (off * np.minimum(1.0, d[k] / D)[:, None])
    m = k.sum()
    assert np.abs(z.mean(0)).max() < 5 / np.sqrt(m)
    assert np.abs(z.var(0) - 1).max() < 5 * np.sqrt(2 / m)
    c = np.corrcoef(z.T)
    assert np.abs(c - np.eye(3)).max() < 5 / np.sqrt(m)
    # a fourth-moment check that rules out a uniform or clipped draw
    assert abs((z ** 4).mean() - 3) < 0.15


def test_eq7_draws_depend_on_seed_epoch_and_view_only(lod_off):
    rng = np.random.default_rng(3)
    n = 5000
    sc, cam = _cone_scene(n, rng.uniform(5, 60, n), rng)
    sel = np.arange(n)

    def run(seed, epoch, view):
        oracle.set_lod(1, p_max=0.5, dist=30.0, offset=(0.2, 0.2, 0.2), seed=seed, epoch=epoch)
        return oracle.project(sc, sel, 0, cam, 1.0, view=view)["raw"]

    a = run(5, 1, 0)
    np.testing.assert_array_equal(a, run(5, 1, 0))
    for other in (run(6, 1, 0), run(5 + (1 << 32), 1, 0), run(5, 2, 0), run(5, 1, 1)):
        assert (other[:, 1] != a[:, 1]).mean() > 0.2


def test_eq7_gradient_matches_central_finite_differences(lod_off):
    """With D below the near plane, p = p_max and the offset scale is 1 for
    every Gaussian, so the draws are constants and the render is a smooth
    function of the parameters: FP64 central differences of the stochastic
    render equal the oracle's gradient (noisy means included)."""
    step = 1
    oracle.set_margins(alpha_tol=1e-4, T_tol=1e-6, power_tol=1e-7)
    try:
        sc = scenegen.generate("fd", seed=11)
        cam = sc.cams[step][0]
        oracle.set_lod(0)
        vis, _ = oracle.vis_reset(sc.n)
        sel = oracle.select(vis, float(sc.times[step]))
        r = float(np.median(oracle.project(sc, sel, step, cam, 0.0)["sigma_lod"]))
        oracle.set_lod(1, p_max=0.3, dist=0.05, offset=(0.02, 0.02, 0.02), seed=21, epoch=4)
        f = oracle.step_forward(sc, step, vis, None, r)
        rec = f["views"][0]["rec"]
        assert not rec["near"][rec["infrustum"]].any()
        small = rec["infrustum"] & (rec["sigma_lod"] < r)
        assert small.sum() > 50 and (small & rec["kept"]).sum() > 30 and (small & ~rec["kept"]).sum() > 10
        rng = np.random.default_rng(0)
        w = rng.standard_normal((3, 64, 64))
        w *= ~f["views"][0]["flag"][None]
        g = oracle.step_backward(sc, step, f, [w], r)
        w *= ~g["pixel_flags"][0][None]
        g = oracle.step_backward(sc, step, f, [w], r)

        def loss(**over):
            sc2 = dataclasses.replace(sc, **{k: v for k, v in over.items() if k not in ("inst_quat", "inst_trans")})
            rec2 = oracle.project(sc2, sel, step, cam, r, inst_quat=over.get("inst_quat"),
                                  inst_trans=over.get("inst_trans"))
            return float((w * oracle.render(cam.width, cam.height, oracle.select_splats(rec2))["image"]).sum())

        moved = sel[small & rec["kept"]]
        picks = np.concatenate([rng.choice(moved, 12, replace=False),
                                rng.choice(sel[rec["kept"] & ~small], 6, replace=False)])
        h = 1e-6
        checked = 0
        for name, shape in (("means", 3), ("log_scales", 3), ("quats", 4), ("opacity_logits", 1), ("sh", 48)):
            base = getattr(sc, name).astype(np.float64)
            for gi in picks:
                comps = range(shape) if shape <= 4 else rng.choice(shape, 4, replace=False)
                for c in comps:
                    plus, minus = base.copy(), base.copy()
                    idx = (gi,) if shape == 1 else ((gi, c) if name != "sh" else (gi, c // 3, c % 3))
                    plus[idx] += h
                    minus[idx] -= h
                    fd = (loss(**{name: plus}) - loss(**{name: minus})) / (2 * h)
                    an = g[name][idx]
                    assert abs(fd - an) <= 2e-5 + 2e-4 * abs(an), (name, gi, c, fd, an)
                    checked += 1
        for name in ("inst_quat", "inst_trans"):
            base = getattr(sc, name)[step].astype(np.float64)
            for idx in np.ndindex(base.shape):
                plus, minus = base.copy(), base.copy()
                plus[idx] += h
                minus[idx] -= h
                fd = (loss(**{name: plus}) - loss(**{name: minus})) / (2 * h)
                an = g[name][idx]
                assert abs(fd - an) <= 2e-5 + 2e-4 * abs(an), (name, idx, fd, an)
                checked += 1
        assert checked > 150
    finally:
        oracle.set_margins()
        oracle.set_lod(0)
