"""One optimisation step of the reconstruction, its state between steps, and
checkpoint / resume of that state.

The state (``TrainState``) is what the next step reads:
  * the Gaussian parameters (means, log-scales, quaternions, opacity logits,
    SH coefficients) and the instance layout;
  * the per-timestep instance poses (quaternion, translation), which the pose
    adjoints of the backward optimise (the instance matrices of Sec. 3.3);
  * the Adam moments of both, with their step counts (one count for the
    Gaussians, one per timestep for that timestep's poses);
  * the temporal-visibility record, windows v and point lives l (Eq. 5, 6);
  * the LOD configuration (threshold r; for Eq. 7 also p_max, D, the offset
    and the Philox seed) and the workspace's call counter, which numbers the
    Eq. 7 draws;
  * the number of steps taken.

``Trainer.step(k, target)`` renders timestep k's cameras, takes the L1 loss
against ``target``, runs the backward (Gaussian and pose adjoints), and takes
one Adam step on the Gaussians and one on timestep k's poses; the projection
records Eq. 5 into the point lives as it goes. Every arithmetic step runs in
libs3r.

``save(path, state)`` writes the state with torch.save (tensors on the CPU,
with a format number); ``load(path, device)`` reads it back. A trainer built
on a loaded state continues where the saved run stopped: the forward is
deterministic, so its images are bit-identical to the uninterrupted run's;
the backward sums with float atomics in an unspecified order, so gradients,
and the parameters after the step, agree to that rounding (as two runs of
one step do).
"""
from __future__ import annotations

import dataclasses

import torch

from . import binding
from .render import DeviceScene, Renderer, pixel_count

FORMAT = 1
PARAM_NAMES = ("means", "log_scales", "quats", "opacity_logits", "sh")


@dataclasses.dataclass
class TrainState:
    scene: DeviceScene
    inst_quat: torch.Tensor          # [T, n_inst, 4]
    inst_trans: torch.Tensor         # [T, n_inst, 3]
    vis_window: torch.Tensor         # [n, 2] v = (v_s, v_e)
    point_life: torch.Tensor         # [n, 2] l = (l_s, l_e)
    exp_avg: list                    # Adam first moments, one per PARAM_NAMES entry
    exp_avg_sq: list                 # Adam second moments
    pose_exp_avg: list               # [quat, trans] first moments, shaped like the poses
    pose_exp_avg_sq: list            # [quat, trans] second moments
    pose_steps: list                 # Adam steps taken by each timestep's poses
    adam_steps: int = 0              # Adam steps taken by the Gaussians
    step: int = 0
    epoch: int = 0                   # workspace call counter after the last projection
    # "mode": "threshold" or "stochastic"; "r" in px; for "stochastic" (Eq. 7)
    # also "p_max", "distance", "offset" (3 floats) and "seed"
    lod: dict = dataclasses.field(default_factory=lambda: {"mode": "threshold", "r": 0.0})

    @classmethod
    def initial(cls, scene: DeviceScene, inst_quat, inst_trans, vis_window, point_life,
                lod: dict | None = None) -> "TrainState":
        """A state before the first step: zero moments, no steps taken."""
        params = scene.params()
        return cls(scene=scene, inst_quat=inst_quat.contiguous(), inst_trans=inst_trans.contiguous(),
                   vis_window=vis_window, point_life=point_life,
                   exp_avg=[torch.zeros_like(p) for p in params],
                   exp_avg_sq=[torch.zeros_like(p) for p in params],
                   pose_exp_avg=[torch.zeros_like(inst_quat), torch.zeros_like(inst_trans)],
                   pose_exp_avg_sq=[torch.zeros_like(inst_quat), torch.zeros_like(inst_trans)],
                   pose_steps=[0] * int(inst_quat.shape[0]),
                   lod=dict(lod) if lod else {"mode": "threshold", "r": 0.0})

    def tensors(self) -> dict:
        """Every tensor of the state by name (the checkpoint's contents)."""
        out = {f"scene.{n}": p for n, p in zip(PARAM_NAMES, self.scene.params())}
        out["scene.inst_offsets"] = self.scene.inst_offsets
        out.update({"inst_quat": self.inst_quat, "inst_trans": self.inst_trans,
                    "vis_window": self.vis_window, "point_life": self.point_life})
        for n, m, v in zip(PARAM_NAMES, self.exp_avg, self.exp_avg_sq):
            out[f"exp_avg.{n}"], out[f"exp_avg_sq.{n}"] = m, v
        for n, m, v in zip(("quat", "trans"), self.pose_exp_avg, self.pose_exp_avg_sq):
            out[f"pose_exp_avg.{n}"], out[f"pose_exp_avg_sq.{n}"] = m, v
        return out


def save(path, state: TrainState) -> None:
    """Write the state to `path` (torch.save; tensors copied to the CPU)."""
    blob = {"format": FORMAT,
            "tensors": {k: t.detach().cpu() for k, t in state.tensors().items()},
            "sh_degree": int(state.scene.sh_degree), "pose_steps": [int(x) for x in state.pose_steps],
            "adam_steps": int(state.adam_steps), "step": int(state.step),
            "epoch": int(state.epoch), "lod": dict(state.lod)}
    torch.save(blob, path)


def load(path, device="cuda") -> TrainState:
    """Read a state written by save() onto `device`."""
    blob = torch.load(path, map_location="cpu", weights_only=True)
    if blob.get("format") != FORMAT:
        raise ValueError(f"{path}: checkpoint format {blob.get('format')!r}, expected {FORMAT}")
    t = {k: v.to(device) for k, v in blob["tensors"].items()}
    scene = DeviceScene(means=t["scene.means"], log_scales=t["scene.log_scales"],
                        quats=t["scene.quats"], opacity_logits=t["scene.opacity_logits"],
                        sh=t["scene.sh"], inst_offsets=t["scene.inst_offsets"],
                        sh_degree=int(blob["sh_degree"]))
    return TrainState(scene=scene, inst_quat=t["inst_quat"], inst_trans=t["inst_trans"],
                      vis_window=t["vis_window"], point_life=t["point_life"],
                      exp_avg=[t[f"exp_avg.{n}"] for n in PARAM_NAMES],
                      exp_avg_sq=[t[f"exp_avg_sq.{n}"] for n in PARAM_NAMES],
                      pose_exp_avg=[t["pose_exp_avg.quat"], t["pose_exp_avg.trans"]],
                      pose_exp_avg_sq=[t["pose_exp_avg_sq.quat"], t["pose_exp_avg_sq.trans"]],
                      pose_steps=list(blob["pose_steps"]), adam_steps=int(blob["adam_steps"]),
                      step=int(blob["step"]), epoch=int(blob["epoch"]), lod=dict(blob["lod"]))


class Trainer:
    """Steps a TrainState. `cams_of_step[k]` and `times[k]` are timestep k's
    cameras and time; the workspace is sized for the largest camera set."""

    def __init__(self, state: TrainState, cams_of_step, times, *, lr: float = 1e-3,
                 pose_lr: float = 1e-4, betas=(0.9, 0.999), eps: float = 1e-8, background=None,
                 max_splats: int | None = None, max_duplicates: int | None = None):
        self.state = state
        self.cams, self.times = cams_of_step, times
        self.lr, self.pose_lr, self.betas, self.eps = float(lr), float(pose_lr), betas, float(eps)
        sc = state.scene
        rig = max(cams_of_step, key=lambda c: (len(c), pixel_count(c)))
        self.renderer = Renderer(sc.n, sc.n_inst, rig, max_splats=max_splats,
                                 max_duplicates=max_duplicates)
        ws = self.renderer.ws
        lod = state.lod
        if lod.get("mode") == "stochastic":
            ws.set_lod(binding.LOD_STOCHASTIC, p_max=lod["p_max"], distance=lod["distance"],
                       offset=tuple(lod["offset"]), seed=lod["seed"])
        if state.epoch:
            ws.set_epoch(state.epoch)
        dev = sc.means.device
        self.background = (torch.zeros(3, device=dev) if background is None
                           else background.to(dev, torch.float32))
        self.grads = {n: torch.zeros_like(p) for n, p in zip(PARAM_NAMES, sc.params())}
        n_inst = int(state.inst_quat.shape[1])
        self.grads["inst_quat"] = torch.zeros((n_inst, 4), device=dev)
        self.grads["inst_trans"] = torch.zeros((n_inst, 3), device=dev)
        self.loss = torch.zeros(1, device=dev)

    def step(self, k: int, target: torch.Tensor, *, check: bool = True):
        """One optimisation step on timestep k; returns (loss [1], rendered
        image, flat planar per view) as device tensors.

        Both Adam updates are gated on the device by the workspace's latched
        status: if a call of this step (or an earlier unchecked one) dropped
        splats or pairs for lack of capacity, or a bounded wait gave up, the
        parameters and moments are left as they were. With `check` (the
        default) the status is read after the step (one host
        synchronisation): a failure raises binding.S3RError and the step is not
        counted. With check=False no synchronisation happens; call check()
        before relying on the step counters, which then count steps that the
        device may have skipped."""
        s = self.state
        cams, t = self.cams[k], float(self.times[k])
        out = torch.empty(3 * pixel_count(cams), device=s.scene.means.device)
        dL = torch.empty_like(out)
        iq, it = s.inst_quat[k], s.inst_trans[k]
        self.renderer.forward(s.scene, iq, it, cams, t, s.vis_window, s.point_life,
                              float(s.lod.get("r", 0.0)), self.background, out=out)
        binding.l1_loss(out, target, dL, self.loss)
        # every gradient element is written (overwrite mode): no zeroing
        self.renderer.backward(s.scene, iq, it, self.background, dL, self.grads, overwrite=True)
        b1, b2 = self.betas
        gate = self.renderer.ws.status_word()
        counters = (s.adam_steps, s.pose_steps[k], s.step)
        s.adam_steps += 1
        binding.adam_step(s.scene.params(), [self.grads[n] for n in PARAM_NAMES], s.exp_avg,
                          s.exp_avg_sq, self.lr, s.adam_steps, b1, b2, self.eps, gate=gate)
        if iq.numel():
            s.pose_steps[k] += 1
            binding.adam_step([iq, it], [self.grads["inst_quat"], self.grads["inst_trans"]],
                              [s.pose_exp_avg[0][k], s.pose_exp_avg[1][k]],
                              [s.pose_exp_avg_sq[0][k], s.pose_exp_avg_sq[1][k]],
                              self.pose_lr, s.pose_steps[k], b1, b2, self.eps, gate=gate)
        s.step += 1
        if check:
            try:
                self.check()
            except binding.S3RError:
                s.adam_steps, s.pose_steps[k], s.step = counters
                raise
        return self.loss, out

    def check(self) -> None:
        """Synchronise and raise binding.S3RError if a call of the workspace
        latched a failure since the last check (reading clears it)."""
        self.renderer.sync_status()

    def save(self, path) -> None:
        """Checkpoint the state after the steps so far. Synchronises; raises
        if the device latched an error; records the workspace call counter."""
        self.renderer.sync_status()
        self.state.epoch = int(self.renderer.counts()["epoch"])
        save(path, self.state)
