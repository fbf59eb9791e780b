"""FP64 CPU oracle for the S3R-GS per-timestep render-and-backprop path.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
bench's CPU-baseline leg use it to check and to time against; the product
path (the CUDA library and its binding) never imports it, and it imports
nothing from the product package.

The arithmetic lives in ``s3r_oracle.cpp`` (plain C++17, double precision,
OpenMP over independent pixels and Gaussians); this module only marshals
numpy arrays and strings the stages together in the paper's order
(Sec. 3.3): temporal selection -> instance-specific projection (Eq. 1) ->
M_t and the point-life update (Eq. 5) -> adaptive-LOD cull -> SH colour ->
alpha blending (Eq. 2); Eq. 6 and the reset act on the record between
epochs. ``step_backward`` is the exact hand-derived gradient of the step.

Every function here is pinned by ``tests/test_oracle_pins.py`` against
closed forms, brute force, finite differences and an independent float64
torch restatement.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "s3r_oracle.cpp")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
REC = 24  # doubles per projected record

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with the host C++ compiler (no GPU involved)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        # no contraction of a*b+c into FMA: the arithmetic is the written one on
        # every host (the Eq. 7 draw threshold is compared in FP32)
        cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
               "-o", _LIB_PATH, _SRC]
        subprocess.run(cmd, check=True)
    return _LIB_PATH


def _P(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB_PATH)
        vp, i64, i32, f32, f64 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_float, ctypes.c_double
        L.orc_select.argtypes = [i64, vp, f32, vp]
        L.orc_select.restype = i64
        L.orc_vis_record.argtypes = [i64, vp, f32, vp]
        L.orc_vis_finalize.argtypes = [i64, vp, vp]
        L.orc_vis_reset.argtypes = [i64, vp, vp]
        proj = [i64, vp, vp, vp, vp, vp, vp, i32, vp, i32, vp, vp, vp, f64, vp]
        L.orc_project.argtypes = proj[:-1] + [i32, vp]
        L.orc_project_conventional.argtypes = proj
        L.orc_render.argtypes = [i32, i32, i32, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]
        L.orc_render_tiled.argtypes = [i32, i32, i32, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]
        L.orc_tile_keys.argtypes = [i32, i32, i32, vp, vp, i64, vp, vp, vp]
        L.orc_tile_keys.restype = i64
        L.orc_render_backward.argtypes = [i32, i32, i32, vp, vp, vp, vp, vp, vp, vp, vp, vp,
                                          vp, vp, vp, vp, vp, vp]
        L.orc_project_backward.argtypes = [i64, vp, vp, vp, vp, vp, vp, i32, vp, i32, vp, vp, vp,
                                           f64, i32, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]
        u32 = ctypes.c_uint32
        L.orc_set_lod.argtypes = [i32, f64, f64, f64, f64, f64, u32, u32, u32]
        L.orc_philox.argtypes = [vp, vp, vp]
        L.orc_sh_basis.argtypes = [vp, vp, vp]
        L.orc_render_pixels.argtypes = [i32, i32, i32, vp, vp, vp, vp, vp, vp, vp, vp, vp, i32,
                                        vp, vp, vp, vp, vp, vp]
        L.orc_render_backward_pixels.argtypes = [i32, vp, vp, vp, vp, vp, vp, vp, vp, vp, i32, vp,
                                                 vp, vp, vp, vp, vp, vp]
        L.orc_num_threads.restype = i32
        L.orc_adam_step.argtypes = [i64, vp, vp, vp, vp, f64, f64, f64, f64, i32]
        L.orc_set_margins.argtypes = [f64, f64, f64]
        _lib = L
    return _lib


def set_margins(alpha_tol=1e-6, T_tol=1e-8, power_tol=1e-9) -> None:
    """Margins for flagging blend decisions near their thresholds."""
    lib().orc_set_margins(alpha_tol, T_tol, power_tol)


def num_threads() -> int:
    return int(lib().orc_num_threads())


# ------------------------------------------------------------------ records
def vis_reset(n: int):
    """Initial record (Sec. 3.3): v = (-1, 1), l = (1, -1), float32 [n,2]."""
    life = np.empty((n, 2), np.float32)
    vis = np.empty((n, 2), np.float32)
    lib().orc_vis_reset(n, _P(life), _P(vis))
    return vis, life


def vis_record(life: np.ndarray, mask: np.ndarray, t: float) -> None:
    """Eq. 5 in place on `life` for the Gaussians with mask[i] set."""
    m = np.ascontiguousarray(mask.astype(np.uint8))
    lib().orc_vis_record(life.shape[0], _P(m), ctypes.c_float(t), _P(life))


def vis_finalize(life: np.ndarray) -> np.ndarray:
    """Eq. 6: the visibility window from the point life, in FP32."""
    vis = np.empty_like(life)
    lib().orc_vis_finalize(life.shape[0], _P(life), _P(vis))
    return vis


def select(vis: np.ndarray, t: float) -> np.ndarray:
    """Temporal selection: ascending int64 indices with v_s <= t <= v_e."""
    vis = np.ascontiguousarray(vis, np.float32)
    out = np.empty(vis.shape[0], np.int64)
    m = lib().orc_select(vis.shape[0], _P(vis), ctypes.c_float(t), _P(out))
    return out[:m].copy()


# ------------------------------------------------------------------ projection
def cam_array(cam) -> np.ndarray:
    w2c = np.asarray(cam.world_to_cam, np.float64).reshape(12)
    return np.concatenate([[cam.width, cam.height, cam.fx, cam.fy, cam.cx, cam.cy, cam.near],
                           w2c]).astype(np.float64)


def _scene_arrays(scene):
    """Parameters widened (exactly) to float64; the oracle computes in FP64.
    The widened copies are kept on the scene object (large scenes)."""
    cache = getattr(scene, "_oracle_f64", None)
    if cache is not None and cache[0] is scene.means:
        return cache[1]
    arrays = _widen(scene)
    try:
        object.__setattr__(scene, "_oracle_f64", (scene.means, arrays))
    except (AttributeError, TypeError):
        pass
    return arrays


def _widen(scene):
    return (np.ascontiguousarray(scene.means, np.float64),
            np.ascontiguousarray(scene.log_scales, np.float64),
            np.ascontiguousarray(scene.quats, np.float64),
            np.ascontiguousarray(scene.opacity_logits, np.float64),
            np.ascontiguousarray(scene.sh, np.float64),
            np.ascontiguousarray(scene.inst_offsets, np.int64))


def project(scene, sel: np.ndarray, step: int, cam, lod_r: float, *, conventional=False,
            inst_quat=None, inst_trans=None, view: int = 0) -> dict:
    """Project the selected Gaussians into one camera at timestep `step`;
    `view` is the camera's index in its call (a counter word of the
    stochastic LOD's draws)."""
    means, ls, qs, ol, sh, off = _scene_arrays(scene)
    iq = np.ascontiguousarray(scene.inst_quat[step] if inst_quat is None else inst_quat, np.float64)
    it = np.ascontiguousarray(scene.inst_trans[step] if inst_trans is None else inst_trans, np.float64)
    sel = np.ascontiguousarray(sel, np.int64)
    rec = np.zeros((sel.shape[0], REC), np.float64)
    args = [sel.shape[0], _P(sel), _P(means), _P(ls), _P(qs), _P(ol), _P(sh), scene.sh_degree,
            _P(off), scene.n_inst, _P(iq), _P(it), _P(cam_array(cam)), float(lod_r)]
    if conventional:
        lib().orc_project_conventional(*args, _P(rec))
    else:
        lib().orc_project(*args, int(view), _P(rec))
    return unpack_records(rec)


def unpack_records(rec: np.ndarray) -> dict:
    return {
        "infrustum": rec[:, 0] > 0.5, "kept": rec[:, 1] > 0.5, "near": rec[:, 2] > 0.5,
        "near_bits": rec[:, 2].astype(np.int32),
        "p": rec[:, 3:6], "uv": rec[:, 6:8], "conic": rec[:, 8:11], "opacity": rec[:, 11],
        "rgb": rec[:, 12:15], "radius": rec[:, 15], "rect": rec[:, 16:20].astype(np.int32),
        "sigma_lod": rec[:, 20], "depth32": rec[:, 21].astype(np.float32),
        "inst": rec[:, 22].astype(np.int32), "gid": rec[:, 23].astype(np.int64), "raw": rec,
    }


# ------------------------------------------------------------------ blending
def _splat_args(sp):
    u = np.ascontiguousarray(sp["uv"][:, 0], np.float64)
    v = np.ascontiguousarray(sp["uv"][:, 1], np.float64)
    conic = np.ascontiguousarray(sp["conic"], np.float64)
    opac = np.ascontiguousarray(sp["opacity"], np.float64)
    rgb = np.ascontiguousarray(sp["rgb"], np.float64)
    depth = np.ascontiguousarray(sp["depth32"], np.float32)
    order = np.ascontiguousarray(sp.get("order", np.arange(u.shape[0])), np.int64)
    rect = np.ascontiguousarray(sp["rect"], np.int32)
    return u, v, conic, opac, rgb, depth, order, rect


def select_splats(rec: dict, mask=None) -> dict:
    """The kept records of one view as the blend sees them (order = gid)."""
    keep = rec["kept"] if mask is None else mask
    sp = {k: rec[k][keep] for k in ("uv", "conic", "opacity", "rgb", "depth32", "rect", "gid")}
    sp["order"] = sp["gid"]
    return sp


def render(width: int, height: int, sp: dict, bg=(0.0, 0.0, 0.0), *, tiled=False) -> dict:
    """Alpha blending of one view (Eq. 2). Untiled brute force by default."""
    u, v, conic, opac, rgb, depth, order, rect = _splat_args(sp)
    n = u.shape[0]
    bgv = np.asarray(bg, np.float64)
    img = np.zeros((3, height, width), np.float64)
    T = np.zeros((height, width), np.float64)
    nc = np.zeros((height, width), np.int32)
    flag = np.zeros((height, width), np.int32)
    if tiled:
        lib().orc_render_tiled(width, height, n, _P(u), _P(v), _P(conic), _P(opac), _P(rgb),
                               _P(depth), _P(rect), _P(bgv), _P(img), _P(T), _P(nc))
    else:
        lib().orc_render(width, height, n, _P(u), _P(v), _P(conic), _P(opac), _P(rgb), _P(depth),
                         _P(order), _P(rect), _P(bgv), _P(img), _P(T), _P(nc), _P(flag))
    return {"image": img, "T": T, "n_contrib": nc, "flag": flag.astype(bool)}


def render_pixels(sp: dict, px, py, bg=(0.0, 0.0, 0.0)) -> dict:
    """Eq. 2 at chosen pixels only (rgb [n,3], T, n_contrib, flag)."""
    u, v, conic, opac, rgb, depth, order, rect = _splat_args(sp)
    px = np.ascontiguousarray(px, np.int32)
    py = np.ascontiguousarray(py, np.int32)
    m = px.shape[0]
    out = np.zeros((m, 3))
    T = np.zeros(m)
    nc = np.zeros(m, np.int32)
    flag = np.zeros(m, np.int32)
    bgv = np.asarray(bg, np.float64)
    lib().orc_render_pixels(0, 0, u.shape[0], _P(u), _P(v), _P(conic), _P(opac), _P(rgb), _P(depth),
                            _P(order), _P(rect), _P(bgv), m, _P(px), _P(py), _P(out), _P(T), _P(nc),
                            _P(flag))
    return {"rgb": out, "T": T, "n_contrib": nc, "flag": flag.astype(bool)}


def render_backward_pixels(sp: dict, px, py, dL, bg=(0.0, 0.0, 0.0)) -> dict:
    """Per-splat gradients of sum_q dL[q] . image(px[q], py[q])."""
    u, v, conic, opac, rgb, depth, order, rect = _splat_args(sp)
    n = u.shape[0]
    px = np.ascontiguousarray(px, np.int32)
    py = np.ascontiguousarray(py, np.int32)
    d = np.ascontiguousarray(dL, np.float64)
    g = {"uv": np.zeros((n, 2)), "conic": np.zeros((n, 3)), "opacity": np.zeros(n),
         "rgb": np.zeros((n, 3))}
    bgv = np.asarray(bg, np.float64)
    lib().orc_render_backward_pixels(n, _P(u), _P(v), _P(conic), _P(opac), _P(rgb), _P(depth),
                                     _P(order), _P(rect), _P(bgv), px.shape[0], _P(px), _P(py),
                                     _P(d), _P(g["uv"]), _P(g["conic"]), _P(g["opacity"]),
                                     _P(g["rgb"]))
    return g


def tile_keys(width: int, height: int, depth32, rect, tile_base: int = 0):
    """(keys u64, vals i32, ranges i64 [tiles,2]) of the duplicated pairs."""
    depth32 = np.ascontiguousarray(depth32, np.float32)
    rect = np.ascontiguousarray(rect, np.int32)
    n = depth32.shape[0]
    m = lib().orc_tile_keys(width, height, n, _P(depth32), _P(rect), tile_base, None, None, None)
    keys = np.zeros(m, np.uint64)
    vals = np.zeros(m, np.int32)
    gx, gy = (width + 15) // 16, (height + 15) // 16
    ranges = np.zeros((gx * gy, 2), np.int64)
    lib().orc_tile_keys(width, height, n, _P(depth32), _P(rect), tile_base, _P(keys), _P(vals),
                        _P(ranges))
    return keys, vals, ranges


def render_backward(width: int, height: int, sp: dict, dL_dimg: np.ndarray, bg=(0.0, 0.0, 0.0)):
    """Per-splat gradients of sum(dL_dimg * image) for one view."""
    u, v, conic, opac, rgb, depth, order, rect = _splat_args(sp)
    n = u.shape[0]
    g = {"uv": np.zeros((n, 2)), "conic": np.zeros((n, 3)), "opacity": np.zeros(n),
         "rgb": np.zeros((n, 3))}
    flag = np.zeros((height, width), np.int32)
    d = np.ascontiguousarray(dL_dimg, np.float64)
    bgv = np.asarray(bg, np.float64)
    lib().orc_render_backward(width, height, n, _P(u), _P(v), _P(conic), _P(opac), _P(rgb),
                              _P(depth), _P(order), _P(rect), _P(bgv), _P(d), _P(g["uv"]),
                              _P(g["conic"]), _P(g["opacity"]), _P(g["rgb"]), _P(flag))
    g["flag"] = flag.astype(bool)
    return g


def zero_grads(scene) -> dict:
    n = scene.n
    k = (scene.sh_degree + 1) ** 2
    return {"means": np.zeros((n, 3)), "log_scales": np.zeros((n, 3)), "quats": np.zeros((n, 4)),
            "opacity_logits": np.zeros(n), "sh": np.zeros((n, k, 3)),
            "inst_quat": np.zeros((scene.n_inst, 4)), "inst_trans": np.zeros((scene.n_inst, 3))}


def project_backward(scene, sel, step, cam, lod_r, sg: dict, grads: dict, *, inst_quat=None,
                     inst_trans=None, view: int = 0) -> np.ndarray:
    """Chain splat gradients (indexed like `sel`, zero where not kept) into
    `grads` (accumulated). Returns this view's composed-matrix gradient
    dL/dM [n_inst+1, 3, 4] (row 0 = static)."""
    means, ls, qs, ol, sh, off = _scene_arrays(scene)
    iq = np.ascontiguousarray(scene.inst_quat[step] if inst_quat is None else inst_quat, np.float64)
    it = np.ascontiguousarray(scene.inst_trans[step] if inst_trans is None else inst_trans, np.float64)
    sel = np.ascontiguousarray(sel, np.int64)
    gm = np.zeros((scene.n_inst + 1, 12), np.float64)
    args = [np.ascontiguousarray(sg[k], np.float64) for k in ("uv", "conic", "opacity", "rgb")]
    L = lib()
    L.orc_project_backward(sel.shape[0], _P(sel), _P(means), _P(ls), _P(qs), _P(ol), _P(sh),
                           scene.sh_degree, _P(off), scene.n_inst, _P(iq), _P(it),
                           _P(cam_array(cam)), float(lod_r), int(view), *[_P(a) for a in args],
                           _P(grads["means"]), _P(grads["log_scales"]), _P(grads["quats"]),
                           _P(grads["opacity_logits"]), _P(grads["sh"]), _P(gm),
                           _P(grads["inst_quat"]), _P(grads["inst_trans"]))
    return gm.reshape(scene.n_inst + 1, 3, 4)


def set_lod(mode: int = 0, p_max: float = 0.0, dist: float = 1.0, offset=(0.0, 0.0, 0.0),
            seed: int = 0, epoch: int = 0) -> None:
    """Select the LOD of the projection: mode 0 = deterministic threshold
    cull, 1 = Eq. 7 (depth-dependent Bernoulli drop and noisy offset of the
    Gaussians below r), drawn by Philox4x32-10 with counter (Gaussian id,
    view, epoch, block) and key (seed low, seed high 32 bits)."""
    lib().orc_set_lod(int(mode), float(p_max), float(dist), float(offset[0]), float(offset[1]),
                      float(offset[2]), int(seed) & 0xffffffff, (int(seed) >> 32) & 0xffffffff,
                      int(epoch) & 0xffffffff)


def philox(ctr, key) -> np.ndarray:
    """Philox4x32-10 of one 4-word counter under a 2-word key."""
    c = np.ascontiguousarray(ctr, np.uint32)
    k = np.ascontiguousarray(key, np.uint32)
    out = np.zeros(4, np.uint32)
    lib().orc_philox(_P(c), _P(k), _P(out))
    return out


def sh_basis(direction) -> tuple:
    d = np.ascontiguousarray(direction, np.float64)
    Y = np.zeros(16)
    dY = np.zeros((16, 3))
    lib().orc_sh_basis(_P(d), _P(Y), _P(dY))
    return Y, dY


# ------------------------------------------------------------------ whole step
def step_forward(scene, step: int, vis: np.ndarray, life: np.ndarray | None, lod_r: float,
                 cams=None, bg=(0.0, 0.0, 0.0), *, tiled=False) -> dict:
    """One timestep over all cameras: select, project, record (Eq. 5, on the
    union of the views' frustum masks, before LOD), cull, render."""
    cams = scene.cams[step] if cams is None else cams
    t = float(scene.times[step])
    sel = select(vis, t)
    views = []
    mt = np.zeros(sel.shape[0], bool)
    for vi, cam in enumerate(cams):
        rec = project(scene, sel, step, cam, lod_r, view=vi)
        mt |= rec["infrustum"]
        sp = select_splats(rec)
        out = render(cam.width, cam.height, sp, bg, tiled=tiled)
        views.append({"rec": rec, "splats": sp, **out})
    if life is not None:
        full = np.zeros(scene.n, bool)
        full[sel] = mt
        vis_record(life, full, np.float32(t))
    return {"sel": sel, "mt": mt, "views": views, "t": t}


def step_backward(scene, step: int, fwd: dict, dL_dimgs, lod_r: float, cams=None,
                  bg=(0.0, 0.0, 0.0)) -> dict:
    """Exact gradient of sum_v <dL_dimgs[v], image_v> w.r.t. all parameters
    and the instance poses at this timestep."""
    cams = scene.cams[step] if cams is None else cams
    grads = zero_grads(scene)
    gms = []
    flags = []
    for vi, cam in enumerate(cams):
        view = fwd["views"][vi]
        sp = view["splats"]
        g = render_backward(cam.width, cam.height, sp, dL_dimgs[vi], bg)
        flags.append(g["flag"])
        kept = view["rec"]["kept"]
        full = {"uv": np.zeros((kept.shape[0], 2)), "conic": np.zeros((kept.shape[0], 3)),
                "opacity": np.zeros(kept.shape[0]), "rgb": np.zeros((kept.shape[0], 3))}
        for k in full:
            full[k][kept] = g[k]
        gms.append(project_backward(scene, fwd["sel"], step, cam, lod_r, full, grads, view=vi))
    grads["M"] = gms
    grads["pixel_flags"] = flags
    return grads


def adam_step(param, grad, exp_avg, exp_avg_sq, lr, step, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step in float64 (Kingma and Ba, Algorithm 1; PyTorch's form
    without weight decay). Returns new (param, exp_avg, exp_avg_sq) arrays."""
    p = np.array(param, dtype=np.float64, copy=True).reshape(-1)
    g = np.ascontiguousarray(np.asarray(grad, dtype=np.float64).reshape(-1))
    m = np.array(exp_avg, dtype=np.float64, copy=True).reshape(-1)
    v = np.array(exp_avg_sq, dtype=np.float64, copy=True).reshape(-1)
    assert p.shape == g.shape == m.shape == v.shape
    lib().orc_adam_step(p.size, _P(p), _P(g), _P(m), _P(v), float(lr), float(beta1), float(beta2),
                        float(eps), int(step))
    shape = np.shape(param)
    return p.reshape(shape), m.reshape(shape), v.reshape(shape)
