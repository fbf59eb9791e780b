"""An independent float64 restatement of one rendered view in plain PyTorch.

Used only as a third opinion on the oracle: it re-derives the forward from
the definitions (Eq. 1 with composed instance matrices, SH colour, Eq. 2 with
the 3DGS thresholds) using dense tensor algebra, and gets gradients from
torch.autograd instead of a hand-derived chain rule. It shares no code with
the C++ oracle or with the CUDA library. Small inputs only: it materialises a
[pixels, splats] matrix.
"""
from __future__ import annotations

import math

import numpy as np
import torch


def _rot(q):
    q = q / torch.linalg.vector_norm(q, dim=-1, keepdim=True)
    w, x, y, z = q.unbind(-1)
    return torch.stack([
        torch.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], -1),
        torch.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], -1),
        torch.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], -1),
    ], -2)


def _sh_eval(sh, d, degree):
    """Real SH (orthonormal, Condon-Shortley sign) times coefficients."""
    x, y, z = d.unbind(-1)
    pi = math.pi
    basis = [torch.full_like(x, 0.5 / math.sqrt(pi))]
    if degree >= 1:
        k1 = math.sqrt(3 / (4 * pi))
        basis += [-k1 * y, k1 * z, -k1 * x]
    if degree >= 2:
        basis += [math.sqrt(15 / (4 * pi)) * x * y,
                  -math.sqrt(15 / (4 * pi)) * y * z,
                  math.sqrt(5 / (16 * pi)) * (3 * z * z - 1),
                  -math.sqrt(15 / (4 * pi)) * x * z,
                  math.sqrt(15 / (16 * pi)) * (x * x - y * y)]
    if degree >= 3:
        basis += [-math.sqrt(35 / (32 * pi)) * y * (3 * x * x - y * y),
                  math.sqrt(105 / (4 * pi)) * x * y * z,
                  -math.sqrt(21 / (32 * pi)) * y * (5 * z * z - 1),
                  math.sqrt(7 / (16 * pi)) * z * (5 * z * z - 3),
                  -math.sqrt(21 / (32 * pi)) * x * (5 * z * z - 1),
                  math.sqrt(105 / (16 * pi)) * z * (x * x - y * y),
                  -math.sqrt(35 / (32 * pi)) * x * (x * x - 3 * y * y)]
    Y = torch.stack(basis, -1)                     # [n, K]
    return torch.einsum("nk,nkc->nc", Y, sh)


def render_view(params: dict, inst_offsets: np.ndarray, cam, lod_r: float, sel: np.ndarray,
                bg=(0.0, 0.0, 0.0)):
    """Render one camera. params: float64 tensors means, log_scales, quats,
    opacity_logits, sh, inst_quat, inst_trans (leaf tensors may require grad).
    Returns (image [3,H,W], T_final [H,W])."""
    dev = params["means"].device
    sel_t = torch.as_tensor(sel, dtype=torch.long, device=dev)
    mu = params["means"][sel_t]
    ls = params["log_scales"][sel_t]
    q = params["quats"][sel_t]
    ol = params["opacity_logits"][sel_t]
    sh = params["sh"][sel_t]
    degree = int(round(math.sqrt(sh.shape[1]))) - 1

    inst = np.searchsorted(inst_offsets, sel, side="right") - 1       # segment per Gaussian
    n_inst = inst_offsets.shape[0] - 2
    V = torch.as_tensor(np.asarray(cam.world_to_cam, np.float64), device=dev)
    Vr, Vt = V[:, :3], V[:, 3]
    eye = torch.eye(3, dtype=torch.float64, device=dev)
    Pr = torch.cat([eye[None], _rot(params["inst_quat"])], 0) if n_inst else eye[None]
    Pt = torch.cat([torch.zeros(1, 3, dtype=torch.float64, device=dev), params["inst_trans"]], 0) \
        if n_inst else torch.zeros(1, 3, dtype=torch.float64, device=dev)
    Ak = Vr[None] @ Pr                                                  # [n_inst+1,3,3]
    bk = (Vr[None] @ Pt[..., None])[..., 0] + Vt[None]
    it = torch.as_tensor(inst, dtype=torch.long, device=dev)
    A, b = Ak[it], bk[it]

    p = (A @ mu[..., None])[..., 0] + b
    x, y, z = p.unbind(-1)
    near = cam.near
    R = _rot(q)
    s2 = torch.exp(2 * ls)
    S3 = R @ torch.diag_embed(s2) @ R.transpose(-1, -2)
    Sc = A @ S3 @ A.transpose(-1, -2)
    W, H = cam.width, cam.height
    limx = 1.3 * (0.5 * W / cam.fx)
    limy = 1.3 * (0.5 * H / cam.fy)
    zs = torch.where(z > near, z, torch.ones_like(z))                  # avoid 0-division off-frustum
    tx = torch.clamp(x / zs, -limx, limx) * zs
    ty = torch.clamp(y / zs, -limy, limy) * zs
    zero = torch.zeros_like(zs)
    J = torch.stack([torch.stack([cam.fx / zs, zero, -cam.fx * tx / zs ** 2], -1),
                     torch.stack([zero, cam.fy / zs, -cam.fy * ty / zs ** 2], -1)], -2)
    S2 = J @ Sc @ J.transpose(-1, -2)
    a, bb, c = S2[:, 0, 0], S2[:, 0, 1], S2[:, 1, 1]
    lam_max = 0.5 * (a + c) + torch.sqrt(torch.clamp(0.25 * (a - c) ** 2 + bb * bb, min=0.0))
    sigma_lod = torch.sqrt(lam_max).detach()
    X = S2 + 0.3 * torch.eye(2, dtype=torch.float64, device=dev)
    det = X[:, 0, 0] * X[:, 1, 1] - X[:, 0, 1] ** 2
    Q = torch.linalg.inv(X)
    mid = 0.5 * (X[:, 0, 0] + X[:, 1, 1])
    lam = mid + torch.sqrt(torch.clamp(mid * mid - det, min=0.1))
    radius = torch.ceil(3 * torch.sqrt(lam)).detach()
    u = cam.fx * x / zs + cam.cx
    v = cam.fy * y / zs + cam.cy
    gx, gy = (W + 15) // 16, (H + 15) // 16
    ud, vd = u.detach(), v.detach()
    x0 = torch.clamp(torch.floor((ud - radius) / 16), 0, gx)
    x1 = torch.clamp(torch.floor((ud + radius + 15) / 16), 0, gx)
    y0 = torch.clamp(torch.floor((vd - radius) / 16), 0, gy)
    y1 = torch.clamp(torch.floor((vd + radius + 15) / 16), 0, gy)
    infr = (z.detach() > near) & (det.detach() > 0) & ((x1 - x0) * (y1 - y0) > 0)
    kept = infr & (sigma_lod >= lod_r)

    # colour from the camera centre in the Gaussian's own frame
    cpos = -torch.linalg.solve(A, b[..., None])[..., 0]
    d = mu - cpos
    d = d / torch.linalg.vector_norm(d, dim=-1, keepdim=True)
    rgb = torch.clamp(_sh_eval(sh, d, degree) + 0.5, min=0.0)
    opac = torch.sigmoid(ol)

    k = torch.nonzero(kept).flatten()
    depth32 = z.detach()[k].cpu().numpy().astype(np.float32)
    gid = np.asarray(sel)[k.cpu().numpy()]
    order = np.lexsort((gid, depth32))                                 # depth, then index
    k = k[torch.as_tensor(order, device=dev)]
    uu, vv = u[k], v[k]
    QA, QB, QC = Q[k, 0, 0], Q[k, 0, 1], Q[k, 1, 1]
    oo, cc = opac[k], rgb[k]
    rx0, rx1, ry0, ry1 = x0[k], x1[k], y0[k], y1[k]

    py, px = torch.meshgrid(torch.arange(H, device=dev, dtype=torch.float64),
                            torch.arange(W, device=dev, dtype=torch.float64), indexing="ij")
    px, py = px.reshape(-1, 1), py.reshape(-1, 1)
    tix, tiy = torch.floor(px / 16), torch.floor(py / 16)
    cover = (tix >= rx0) & (tix < rx1) & (tiy >= ry0) & (tiy < ry1)    # [P, S]
    dx = uu[None] - (px + 0.5)
    dy = vv[None] - (py + 0.5)
    power = -0.5 * (QA[None] * dx * dx + QC[None] * dy * dy) - QB[None] * dx * dy
    alpha = torch.clamp(oo[None] * torch.exp(power), max=0.99)
    live = cover & (power <= 0) & (alpha >= 1.0 / 255.0)
    alpha = torch.where(live, alpha, torch.zeros_like(alpha))
    one_minus = 1 - alpha
    t_incl = torch.cumprod(one_minus, dim=1)
    valid = live & (t_incl.detach() >= 1e-4)
    alpha = torch.where(valid, alpha, torch.zeros_like(alpha))
    one_minus = 1 - alpha
    t_incl = torch.cumprod(one_minus, dim=1)
    t_excl = torch.cat([torch.ones_like(t_incl[:, :1]), t_incl[:, :-1]], 1)
    w = alpha * t_excl
    Cimg = w @ cc                                                       # [P, 3]
    Tfin = t_incl[:, -1] if t_incl.shape[1] else torch.ones(px.shape[0], dtype=torch.float64, device=dev)
    bgt = torch.as_tensor(bg, dtype=torch.float64, device=dev)
    out = Cimg + Tfin[:, None] * bgt[None]
    return out.T.reshape(3, H, W), Tfin.reshape(H, W)


def params_from_scene(scene, step: int, requires_grad=True) -> dict:
    def t(a):
        return torch.tensor(np.asarray(a, np.float64), dtype=torch.float64, requires_grad=requires_grad)
    return {"means": t(scene.means), "log_scales": t(scene.log_scales), "quats": t(scene.quats),
            "opacity_logits": t(scene.opacity_logits), "sh": t(scene.sh),
            "inst_quat": t(scene.inst_quat[step]), "inst_trans": t(scene.inst_trans[step])}
