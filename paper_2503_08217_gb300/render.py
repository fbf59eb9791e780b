"""Renderer and autograd function over the libs3r C ABI.

``Renderer`` owns one workspace and runs the per-timestep sequence
project -> sort -> render_fwd (-> render_bwd) for any number of cameras in
one call; ``Renderer.capture`` records the whole forward+backward sequence
into a CUDA graph for replay. ``S3RRender`` exposes it as a
``torch.autograd.Function`` whose backward is the library's hand-written
adjoint (parameters and per-instance poses). PyTorch provides device memory
and streams only; every arithmetic step runs in libs3r.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import torch

from . import binding


@dataclasses.dataclass
class DeviceScene:
    means: torch.Tensor
    log_scales: torch.Tensor
    quats: torch.Tensor
    opacity_logits: torch.Tensor
    sh: torch.Tensor
    inst_offsets: torch.Tensor
    sh_degree: int

    @classmethod
    def from_host(cls, scene, device="cuda") -> "DeviceScene":
        def f(a):
            return torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(device)
        return cls(means=f(scene.means), log_scales=f(scene.log_scales), quats=f(scene.quats),
                   opacity_logits=f(scene.opacity_logits), sh=f(scene.sh),
                   inst_offsets=torch.from_numpy(np.asarray(scene.inst_offsets, np.int64)).to(device),
                   sh_degree=int(scene.sh_degree))

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    @property
    def n_inst(self) -> int:
        return int(self.inst_offsets.shape[0]) - 2

    def params(self):
        return [self.means, self.log_scales, self.quats, self.opacity_logits, self.sh]

    def c_scene(self, means=None, log_scales=None, quats=None, opacity_logits=None, sh=None):
        return binding.make_scene(self.means if means is None else means,
                                  self.log_scales if log_scales is None else log_scales,
                                  self.quats if quats is None else quats,
                                  self.opacity_logits if opacity_logits is None else opacity_logits,
                                  self.sh if sh is None else sh, self.inst_offsets, self.sh_degree)


def pixel_count(cams) -> int:
    return int(sum(int(c.width) * int(c.height) for c in cams))


def tile_count(cams) -> int:
    return int(sum(((int(c.width) + 15) // 16) * ((int(c.height) + 15) // 16) for c in cams))


class Renderer:
    """One workspace sized for a scene and a camera rig."""

    def __init__(self, n: int, n_inst: int, cams, *, max_splats: int | None = None,
                 max_duplicates: int | None = None, max_rows: int = 0, device=None):
        self.n_views_max = len(cams)
        splats = max_splats if max_splats is not None else max(1024, n * min(len(cams), 2))
        dups = max_duplicates if max_duplicates is not None else max(4096, 8 * splats)
        self.ws = binding.Workspace(max_gaussians=max(n, 1), max_splats=splats,
                                    max_duplicates=dups, max_views=len(cams),
                                    max_instances=max(n_inst, 0), max_tiles=tile_count(cams),
                                    max_pixels=pixel_count(cams), max_rows=max_rows,
                                    device=device)
        self.graph = None
        self._grad_mode = binding.GRAD_ACCUMULATE

    # ---------------------------------------------------------------- stages
    def forward(self, scene: DeviceScene, inst_quat, inst_trans, cams, t: float, vis_window,
                point_life, lod: float, background, out=None, *, c_scene=None):
        """project + sort + render_fwd; returns the flat planar image buffer."""
        cs = scene.c_scene() if c_scene is None else c_scene
        poses = binding.make_poses(inst_quat, inst_trans)
        if out is None:
            out = torch.empty(3 * pixel_count(cams), dtype=torch.float32,
                              device=scene.means.device)
        self.ws.project(cs, poses, cams, t, vis_window, point_life, lod)
        self.ws.sort()
        self.ws.render_fwd(background, out)
        return out

    def backward(self, scene: DeviceScene, inst_quat, inst_trans, background, dL, grads: dict,
                 *, c_scene=None, overwrite: bool = False):
        """render_bwd into `grads`: added to them, or with `overwrite` every
        element written (the buffers need no zeroing)."""
        cs = scene.c_scene() if c_scene is None else c_scene
        poses = binding.make_poses(inst_quat, inst_trans)
        mode = binding.GRAD_OVERWRITE if overwrite else binding.GRAD_ACCUMULATE
        if mode != self._grad_mode:
            self.ws.set_grad_mode(mode)
            self._grad_mode = mode
        self.ws.render_bwd(cs, poses, background, dL.contiguous(), grads)

    def counts(self):
        return self.ws.counts()

    def sync_status(self):
        self.ws.sync_status()

    # ---------------------------------------------------------------- graphs
    def capture(self, fn, stream=None):
        """Record `fn()` (a sequence of calls on this renderer) into a CUDA
        graph after one eager warm-up run; returns the torch CUDA graph."""
        s = torch.cuda.Stream() if stream is None else stream
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            fn()
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            fn()
        torch.cuda.synchronize()
        self.graph = g
        return g


def split_views(flat: torch.Tensor, cams):
    """Per-view [3,H,W] views of the flat planar image buffer."""
    out, off = [], 0
    for c in cams:
        n = 3 * int(c.width) * int(c.height)
        out.append(flat[off:off + n].view(3, int(c.height), int(c.width)))
        off += n
    return out


class S3RRender(torch.autograd.Function):
    """images = render(params, poses) for one timestep and a camera rig.

    Non-differentiable inputs (renderer, cameras, t, LOD threshold,
    background, visibility record) get None gradients; the visibility record
    (point life) is updated in place by Eq. 5 during the forward."""

    @staticmethod
    def forward(ctx, renderer: Renderer, scene: DeviceScene, cams, t, lod, background, vis_window,
                point_life, means, log_scales, quats, opacity_logits, sh, inst_quat, inst_trans):
        cs = scene.c_scene(means, log_scales, quats, opacity_logits, sh)
        out = renderer.forward(scene, inst_quat, inst_trans, cams, t, vis_window, point_life, lod,
                               background, c_scene=cs)
        ctx.renderer = renderer
        ctx.scene = scene
        ctx.save_for_backward(background, means, log_scales, quats, opacity_logits, sh, inst_quat,
                              inst_trans)
        return out

    @staticmethod
    def backward(ctx, dout):
        background, means, log_scales, quats, opacity_logits, sh, inst_quat, inst_trans = \
            ctx.saved_tensors
        # every element is written by the library (overwrite mode)
        grads = {"means": torch.empty_like(means), "log_scales": torch.empty_like(log_scales),
                 "quats": torch.empty_like(quats), "opacity_logits": torch.empty_like(opacity_logits),
                 "sh": torch.empty_like(sh), "inst_quat": torch.empty_like(inst_quat),
                 "inst_trans": torch.empty_like(inst_trans)}
        cs = ctx.scene.c_scene(means, log_scales, quats, opacity_logits, sh)
        ctx.renderer.backward(ctx.scene, inst_quat, inst_trans, background, dout.contiguous(), grads,
                              c_scene=cs, overwrite=True)
        return (None, None, None, None, None, None, None, None, grads["means"], grads["log_scales"],
                grads["quats"], grads["opacity_logits"], grads["sh"], grads["inst_quat"],
                grads["inst_trans"])


def render(renderer: Renderer, scene: DeviceScene, cams, t: float, lod: float, background,
           vis_window, point_life, inst_quat, inst_trans, params=None):
    """Differentiable render of all cameras at time t (flat planar output)."""
    p = scene.params() if params is None else params
    return S3RRender.apply(renderer, scene, cams, t, lod, background, vis_window, point_life, *p,
                           inst_quat, inst_trans)


class FusedAdam:
    """Adam over up to 8 float32 CUDA tensors, one `s3r_adam_step` launch per
    step; the moments live beside the parameters. `step(grads)` takes one
    gradient tensor per parameter, in the same order."""

    def __init__(self, params, lr: float, betas=(0.9, 0.999), eps: float = 1e-8):
        self.params = list(params)
        if len(self.params) > 8:
            raise ValueError("FusedAdam takes at most 8 tensors per launch")
        self.lr, self.betas, self.eps = float(lr), tuple(float(b) for b in betas), float(eps)
        self.exp_avg = [torch.zeros_like(p) for p in self.params]
        self.exp_avg_sq = [torch.zeros_like(p) for p in self.params]
        self.t = 0

    def step(self, grads, stream=None):
        self.t += 1
        binding.adam_step(self.params, list(grads), self.exp_avg, self.exp_avg_sq, self.lr, self.t,
                          self.betas[0], self.betas[1], self.eps, stream)
