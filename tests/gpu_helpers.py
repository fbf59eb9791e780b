"""Helpers for the GPU parity tests: run one timestep through the C ABI and
copy the workspace intermediates out; build the oracle's per-splat view of
the same inputs; and mark the pixels and Gaussians whose integer decisions
sit within rounding distance of a threshold (where FP32 and FP64 may
legitimately differ)."""
from __future__ import annotations

import numpy as np
import torch

import oracle
from paper_2503_08217_gb300 import binding
from paper_2503_08217_gb300.render import DeviceScene, Renderer, pixel_count, split_views


# Lines for the "parity exclusions" section of the pytest summary: what each
# comparison left out (near-threshold Gaussians, excluded pixels) and why.
REPORT: list = []


def report(test: str, **counts) -> None:
    REPORT.append(test + ": " + ", ".join(f"{k} {v}" for k, v in counts.items()))


def gpu_step(scene, step, cams, vis, life=None, lod=0.0, bg=(0.0, 0.0, 0.0), dL=None,
             renderer=None, max_splats=None, max_duplicates=None, dev=None):
    """Run project/sort/fwd (and bwd if dL is given) on cuda:0."""
    dev = DeviceScene.from_host(scene) if dev is None else dev
    r = renderer or Renderer(scene.n, scene.n_inst, cams, max_splats=max_splats,
                             max_duplicates=max_duplicates)
    vis_t = torch.from_numpy(np.ascontiguousarray(vis, np.float32)).cuda()
    life_t = None if life is None else torch.from_numpy(np.ascontiguousarray(life, np.float32)).cuda()
    iq = torch.from_numpy(np.ascontiguousarray(scene.inst_quat[step], np.float32)).cuda()
    it = torch.from_numpy(np.ascontiguousarray(scene.inst_trans[step], np.float32)).cuda()
    bg_t = torch.tensor(bg, dtype=torch.float32, device="cuda")
    t = float(scene.times[step])
    out = r.forward(dev, iq, it, cams, t, vis_t, life_t, lod, bg_t)
    res = {"renderer": r, "out": out, "images": [v.double().cpu().numpy() for v in split_views(out, cams)]}
    c = r.counts()
    res["counts"] = c
    _raise_status(c)
    n_sel, n_sp, n_dup = c["n_selected"], c["n_splats"], c["n_duplicates"]
    ws = r.ws
    res["selected"] = ws.debug("selected", torch.int32, n_sel).cpu().numpy().astype(np.int64)
    res["frustum_mask"] = ws.debug("frustum_mask", torch.int32, n_sel).cpu().numpy().view(np.uint32)
    res["keep_mask"] = ws.debug("keep_mask", torch.int32, n_sel).cpu().numpy().view(np.uint32)
    res["splat_start"] = ws.debug("splat_start", torch.int32, n_sel).cpu().numpy().view(np.uint32)
    sp = min(n_sp, r.ws.capacity.max_splats)
    rec = ws.debug("splat_record", torch.float32, 8 * sp).cpu().numpy().reshape(-1, 8)
    res["xy"] = rec[:, 0:2].copy()
    res["conic_o"] = rec[:, 2:6].copy()
    res["record_ext"] = rec[:, 6:8].copy().view(np.uint32)   # x0 | y0 << 16, w | h << 13 | view << 26 | moved << 31
    res["rgb_d"] = ws.debug("splat_rgb_depth", torch.float32, 4 * sp).cpu().numpy().reshape(-1, 4)
    rect = ws.debug("splat_rect", torch.int32, 2 * sp).cpu().numpy().view(np.uint32).reshape(-1, 2)
    res["rect"] = np.stack([rect[:, 0] & 0xFFFF, rect[:, 0] >> 16, rect[:, 1] & 0xFFFF, rect[:, 1] >> 16],
                           1).astype(np.int32)
    vb = ws.debug("splat_view", torch.uint8, sp).cpu().numpy().astype(np.int32)
    res["view"] = vb & 0x7F
    res["moved"] = (vb >> 7).astype(bool)          # Eq. 7: rendered at its noisy mean
    # the packed record repeats the rectangle, view and Eq. 7 flag (its last
    # word is all ones for views too large to pack: then the arrays serve)
    ext, r4 = res["record_ext"], res["rect"].astype(np.uint32)
    packed = ext[:, 1] != 0xFFFFFFFF
    same = ((ext[:, 0] == (r4[:, 0] | (r4[:, 1] << 16)))
            & ((ext[:, 1] & 0x1FFF) == r4[:, 2] - r4[:, 0])
            & (((ext[:, 1] >> 13) & 0x1FFF) == r4[:, 3] - r4[:, 1])
            & (((ext[:, 1] >> 26) & 0x1F) == res["view"])
            & (((ext[:, 1] >> 31) & 1).astype(bool) == res["moved"]))
    assert (same | ~packed).all(), "packed splat record disagrees with the rect/view arrays"
    nd = min(n_dup, r.ws.capacity.max_duplicates)
    res["sorted_splats"] = ws.debug("sorted_splats", torch.int32, nd).cpu().numpy().view(np.uint32)
    res["sorted_tiles"] = ws.debug("sorted_tiles", torch.int32, nd).cpu().numpy().view(np.uint32)
    n_tiles = sum(((cm.width + 15) // 16) * ((cm.height + 15) // 16) for cm in cams)
    res["ranges"] = ws.debug("tile_ranges", torch.int32, 2 * n_tiles).cpu().numpy().view(np.uint32).reshape(-1, 2)
    P = pixel_count(cams)
    res["final_T"] = ws.debug("final_T", torch.float32, P).cpu().numpy()
    res["n_contrib"] = ws.debug("n_contrib", torch.int32, P).cpu().numpy()
    if life_t is not None:
        res["life"] = life_t.cpu().numpy()
    if dL is not None:
        grads = {"means": torch.zeros_like(dev.means), "log_scales": torch.zeros_like(dev.log_scales),
                 "quats": torch.zeros_like(dev.quats), "opacity_logits": torch.zeros_like(dev.opacity_logits),
                 "sh": torch.zeros_like(dev.sh), "inst_quat": torch.zeros_like(iq),
                 "inst_trans": torch.zeros_like(it)}
        dL_t = torch.from_numpy(np.concatenate([np.asarray(d, np.float32).reshape(-1) for d in dL])).cuda()
        r.backward(dev, iq, it, bg_t, dL_t, grads)
        torch.cuda.synchronize()
        res["grads"] = {k: v.double().cpu().numpy() for k, v in grads.items()}
        res["splat_grads"] = ws.debug("splat_grads", torch.float32, 12 * sp).cpu().numpy().reshape(-1, 12)
    _raise_status(r.counts())
    return res


def _raise_status(c):
    if c["device_status"] & 2:
        raise binding.S3RError(4, "a bounded device-side wait gave up")
    if c["device_status"] & 1:
        raise binding.S3RError(2, f"capacity exceeded ({c})")


def popcount32(a):
    a = np.asarray(a, np.uint32)
    if hasattr(np, "bitwise_count"):
        return np.bitwise_count(a).astype(np.int64)
    return np.unpackbits(a.view(np.uint8).reshape(-1, 4), axis=1).sum(1).astype(np.int64)


def splat_gids(res):
    """Gaussian id of every GPU splat: a selected Gaussian's splats are
    contiguous from its splat_start, one per kept view."""
    counts = popcount32(res["keep_mask"])
    assert np.array_equal(np.cumsum(counts) - counts, res["splat_start"].astype(np.int64))
    return np.repeat(res["selected"], counts)


def sweep_visibility(scene, cams_fn=None, lod=0.0):
    """Oracle forward-only sweep over every timestep, then Eq. 6: the
    visibility record a first training epoch would produce."""
    vis, life = oracle.vis_reset(scene.n)
    for k in range(scene.n_steps):
        cams = scene.cams[k] if cams_fn is None else cams_fn(k)
        sel = oracle.select(vis, float(scene.times[k]))
        mt = np.zeros(sel.shape[0], bool)
        for cam in cams:
            mt |= oracle.project(scene, sel, k, cam, lod)["infrustum"]
        full = np.zeros(scene.n, bool)
        full[sel[mt]] = True
        oracle.vis_record(life, full, np.float32(scene.times[k]))
    return oracle.vis_finalize(life), life


def bad_pixels(cam, rec, flag, alpha_margin=1e-3):
    """Pixels to leave out of an image comparison: the oracle's blend flagged
    them (a decision within its margins of a threshold), or a near-threshold
    decision of one Gaussian's projection may flip between FP32 and FP64 and
    that Gaussian reaches the pixel. The decisions and the tiles they can
    change: a rectangle edge (the tile column or row on either side of it), the
    3-sigma radius (one tile on either side of every edge), the near plane,
    the LOD threshold or an Eq. 7 draw (the whole rectangle grown by one tile).
    Within those tiles only the pixels where the Gaussian's FP64 alpha = min(0.99,
    o exp(-q/2)) reaches 1/255 (less a relative margin far above the FP32
    rounding of alpha) are left out: at every other pixel the blend skips the
    Gaussian, so whether it is in the tile's list does not matter. A Gaussian
    whose record has no usable conic (behind the near plane in FP64) leaves
    out every pixel of those tiles."""
    bad = flag.copy()
    H, W = cam.height, cam.width
    gx, gy = (W + 15) // 16, (H + 15) // 16
    bits = rec.get("near_bits", rec["near"].astype(np.int32) * 1)
    cand = np.nonzero((bits != 0) & (rec["infrustum"] | (rec["p"][:, 2] > 0)))[0]
    thr = (1.0 / 255.0) * (1.0 - alpha_margin)

    for i in cand:
        b = int(bits[i])
        x0, y0, x1, y1 = (int(q) for q in rec["rect"][i])
        u, v = (float(q) for q in rec["uv"][i])
        A, B, C = (float(q) for q in rec["conic"][i])
        o = float(rec["opacity"][i])
        usable = (np.isfinite([u, v, A, B, C, o]).all() and A > 0 and C > 0 and A * C - B * B > 0
                  and bool(rec["infrustum"][i] or rec["p"][i, 2] > 0))
        boxes = []
        if (b & (1 | 64 | 128)) or x1 <= x0 or y1 <= y0:
            if x1 <= x0 or y1 <= y0:   # a rect that may be empty on one side: around the centre
                r = int(rec["radius"][i]) // 16 + 2
                x0, x1 = int(u // 16) - r, int(u // 16) + r + 1
                y0, y1 = int(v // 16) - r, int(v // 16) + r + 1
            boxes.append((x0 - 1, y0 - 1, x1 + 1, y1 + 1))
        else:
            if b & 32:
                b |= 2 | 4 | 8 | 16
            if b & 2:
                boxes.append((x0 - 1, y0 - 1, x0 + 1, y1 + 1))
            if b & 4:
                boxes.append((x1 - 1, y0 - 1, x1 + 1, y1 + 1))
            if b & 8:
                boxes.append((x0 - 1, y0 - 1, x1 + 1, y0 + 1))
            if b & 16:
                boxes.append((x0 - 1, y1 - 1, x1 + 1, y1 + 1))
        for xa, ya, xb, yb in boxes:
            xa, ya = max(0, xa), max(0, ya)
            xb, yb = min(gx, xb), min(gy, yb)
            if not (xb > xa and yb > ya):
                continue
            ys, ye = ya * 16, min(H, yb * 16)
            xs, xe = xa * 16, min(W, xb * 16)
            if not usable:
                bad[ys:ye, xs:xe] = True
                continue
            dy = (np.arange(ys, ye) + 0.5 - v)[:, None]
            dx = (np.arange(xs, xe) + 0.5 - u)[None, :]
            q = A * dx * dx + 2.0 * B * dx * dy + C * dy * dy
            alpha = np.minimum(0.99, o * np.exp(-0.5 * q))
            bad[ys:ye, xs:xe] |= alpha >= thr
    return bad
