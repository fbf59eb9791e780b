"""Seeded synthetic street-corridor scenes.

This module only draws inputs: Gaussian parameters, per-timestep instance
poses, cameras and rendering times. It holds none of the rendering method's
arithmetic, so both the GPU path and the CPU oracle can consume its output.

The scenes stand in for the driving sequences the paper evaluates on
(Argoverse 2 with seven surround cameras, KITTI with up to 127 vehicles,
nuScenes with six cameras; Sec. 4.1 and Tab. 2), none of which is available
here. Each scene is a straight corridor along +z:

* static Gaussians: means uniform in x and z, y either uniform or a two-part
  mixture that is 3x denser within 5 m of y = 0; log-scales ~ N(-2, 0.5);
  rotations are normalised N(0, I4) quaternions (w, x, y, z); opacity logits
  ~ N(0, 1); SH degree 0 or 3 with the DC term drawn so that it alone spans
  colours in [0, 1] and higher bands ~ N(0, 0.05^2);
* dynamic instances: Gaussians in a local 2 x 2 x 4 m box (4 m along the
  heading), moving rigidly at a constant speed along a heading yawed about
  the vertical axis;
* cameras: OpenCV pinhole (x right, y down, z forward). The world frame equals
  the first front camera's frame, so the corridor runs along +z; a rig is
  several cameras at one position, yawed about the world y axis.

Layouts (all float32 / int64, C-contiguous):
  means [N,3], log_scales [N,3], quats [N,4], opacity_logits [N],
  sh [N,(deg+1)^2,3], inst_offsets [n_inst+2] (segment 0 = static,
  segment k = instance k), inst_quat [T,n_inst,4], inst_trans [T,n_inst,3],
  times [T] (normalised rendering times in [-1, 1], Sec. 3.3).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class Camera:
    width: int
    height: int
    fx: float
    fy: float
    cx: float
    cy: float
    near: float
    world_to_cam: np.ndarray  # float32 [3,4], row-major, OpenCV axes


@dataclasses.dataclass
class Scene:
    name: str
    means: np.ndarray
    log_scales: np.ndarray
    quats: np.ndarray
    opacity_logits: np.ndarray
    sh: np.ndarray
    sh_degree: int
    inst_offsets: np.ndarray
    inst_quat: np.ndarray
    inst_trans: np.ndarray
    times: np.ndarray
    cams: list  # cams[k] = list of Camera at timestep k
    lod_threshold: float

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    @property
    def n_inst(self) -> int:
        return int(self.inst_offsets.shape[0] - 2)

    @property
    def n_steps(self) -> int:
        return int(self.times.shape[0])


@dataclasses.dataclass
class CorridorSpec:
    name: str
    n_static: int
    x_range: tuple
    y_range: tuple
    z_range: tuple
    y_dense: bool            # 3x density within 5 m of y = 0
    inst_sizes: tuple        # (lo, hi) inclusive Gaussians per instance
    n_inst: int
    inst_speed: tuple        # m/s, uniform
    inst_yaw: float          # |yaw| bound, rad
    inst_fixed: tuple | None  # explicit (x, z0) per instance, or None
    sh_degree: int
    n_steps: int
    dt: float                # seconds per timestep
    cam_step: float          # metres the rig advances per timestep
    rig: tuple               # ((width, height, f, yaw), ...)
    lod_threshold: float
    inst_x: tuple = (-8.0, 8.0)  # lateral start position of instances, uniform


SPECS = {
    # Tiny plain pipeline: 20k static + 2 x 1,000 dynamic, 320 x 192 camera.
    "tiny": CorridorSpec(
        name="tiny", n_static=20_000, x_range=(-40.0, 40.0), y_range=(-2.0, 8.0),
        z_range=(0.0, 80.0), y_dense=False, inst_sizes=(1000, 1000), n_inst=2,
        inst_speed=(8.0, 8.0), inst_yaw=0.0, inst_fixed=((-3.0, 10.0), (3.0, 25.0)),
        sh_degree=0, n_steps=10, dt=0.1, cam_step=1.0,
        rig=((320, 192, 250.0, 0.0),), lod_threshold=0.0),
    # Mid corridor: 1M static over 300 m, 20 x 5,000 dynamic, 1080p, SH3.
    "mid": CorridorSpec(
        name="mid", n_static=1_000_000, x_range=(-20.0, 20.0), y_range=(-2.0, 15.0),
        z_range=(0.0, 300.0), y_dense=True, inst_sizes=(5000, 5000), n_inst=20,
        inst_speed=(0.0, 15.0), inst_yaw=0.1, inst_fixed=None,
        sh_degree=3, n_steps=100, dt=0.1, cam_step=3.0,
        rig=((1920, 1080, 960.0, 0.0),), lod_threshold=1.0),
    # Large corridor: 8M static over 1.5 km, 80 x U{5k..20k} dynamic, 1920 x 1280.
    "large": CorridorSpec(
        name="large", n_static=8_000_000, x_range=(-20.0, 20.0), y_range=(-2.0, 15.0),
        z_range=(0.0, 1500.0), y_dense=True, inst_sizes=(5000, 20000), n_inst=80,
        inst_speed=(0.0, 15.0), inst_yaw=0.1, inst_fixed=None,
        sh_degree=3, n_steps=300, dt=0.1, cam_step=5.0,
        rig=((1920, 1280, 960.0, 0.0),), lod_threshold=1.0),
    # Surround rig on the large corridor: 5 x 1080p (f 960) + 2 x 1280 x 960 (f 640).
    "rig": CorridorSpec(
        name="rig", n_static=8_000_000, x_range=(-20.0, 20.0), y_range=(-2.0, 15.0),
        z_range=(0.0, 1500.0), y_dense=True, inst_sizes=(5000, 20000), n_inst=80,
        inst_speed=(0.0, 15.0), inst_yaw=0.1, inst_fixed=None,
        sh_degree=3, n_steps=300, dt=0.1, cam_step=5.0,
        rig=tuple((1920, 1080, 960.0, 2.0 * math.pi * k / 7.0) for k in range(5))
        + tuple((1280, 960, 640.0, 2.0 * math.pi * k / 7.0) for k in range(5, 7)),
        lod_threshold=1.0),
    # Finite-difference crop: 480 static + 2 x 10 dynamic (yawed) Gaussians in
    # front of a 64 x 64 camera, SH degree 3.
    "fd": CorridorSpec(
        name="fd", n_static=480, x_range=(-4.0, 4.0), y_range=(-3.0, 3.0),
        z_range=(4.0, 16.0), y_dense=False, inst_sizes=(10, 10), n_inst=2,
        inst_speed=(2.0, 4.0), inst_yaw=0.3, inst_fixed=None,
        sh_degree=3, n_steps=4, dt=0.1, cam_step=0.5,
        rig=((64, 64, 50.0, 0.0),), lod_threshold=0.0, inst_x=(-2.0, 2.0)),
    # Training-step scene: 16M static over 2 km, 120 instances, the same rig.
    "train": CorridorSpec(
        name="train", n_static=16_000_000, x_range=(-20.0, 20.0), y_range=(-2.0, 15.0),
        z_range=(0.0, 2000.0), y_dense=True, inst_sizes=(5000, 20000), n_inst=120,
        inst_speed=(0.0, 15.0), inst_yaw=0.1, inst_fixed=None,
        sh_degree=3, n_steps=400, dt=0.1, cam_step=5.0,
        rig=tuple((1920, 1080, 960.0, 2.0 * math.pi * k / 7.0) for k in range(5))
        + tuple((1280, 960, 640.0, 2.0 * math.pi * k / 7.0) for k in range(5, 7)),
        lod_threshold=1.0),
}


def _yaw_quat(yaw: float) -> np.ndarray:
    """Unit quaternion (w, x, y, z) of a rotation by `yaw` about the y axis."""
    return np.array([math.cos(0.5 * yaw), 0.0, math.sin(0.5 * yaw), 0.0], np.float64)


def _yaw_matrix(yaw: float) -> np.ndarray:
    c, s = math.cos(yaw), math.sin(yaw)
    return np.array([[c, 0.0, s], [0.0, 1.0, 0.0], [-s, 0.0, c]], np.float64)


def make_camera(width: int, height: int, f: float, position, yaw: float,
                near: float = 0.2) -> Camera:
    """Pinhole camera at `position` looking along the yawed +z axis."""
    r_cw = _yaw_matrix(yaw)                # camera -> world rotation
    r_wc = r_cw.T
    t_wc = -r_wc @ np.asarray(position, np.float64)
    w2c = np.concatenate([r_wc, t_wc[:, None]], axis=1).astype(np.float32)
    return Camera(width=int(width), height=int(height), fx=float(f), fy=float(f),
                  cx=0.5 * width, cy=0.5 * height, near=float(near), world_to_cam=w2c)


def _sh_coeffs(rng, n: int, degree: int) -> np.ndarray:
    k = (degree + 1) ** 2
    sh = np.empty((n, k, 3), np.float32)
    # The DC band alone maps U[-sqrt(pi), sqrt(pi)] onto colours in [0, 1].
    root_pi = math.sqrt(math.pi)
    sh[:, 0, :] = rng.uniform(-root_pi, root_pi, size=(n, 3)).astype(np.float32)
    if k > 1:
        sh[:, 1:, :] = 0.05 * rng.standard_normal((n, k - 1, 3), dtype=np.float32)
    return sh


def _gaussian_attrs(rng, n: int):
    log_scales = (-2.0 + 0.5 * rng.standard_normal((n, 3), dtype=np.float32)).astype(np.float32)
    q = rng.standard_normal((n, 4), dtype=np.float32)
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    opac = rng.standard_normal(n, dtype=np.float32)
    return log_scales, q.astype(np.float32), opac


def _static_means(rng, spec: CorridorSpec, n: int) -> np.ndarray:
    m = np.empty((n, 3), np.float32)
    m[:, 0] = rng.uniform(*spec.x_range, size=n)
    m[:, 2] = rng.uniform(*spec.z_range, size=n)
    ylo, yhi = spec.y_range
    if spec.y_dense:
        # two segments: [ylo, 5] at density 3, [5, yhi] at density 1
        w_dense = 3.0 * (5.0 - ylo)
        w_sparse = 1.0 * (yhi - 5.0)
        dense = rng.random(n) < w_dense / (w_dense + w_sparse)
        y = np.where(dense, rng.uniform(ylo, 5.0, size=n), rng.uniform(5.0, yhi, size=n))
        m[:, 1] = y
    else:
        m[:, 1] = rng.uniform(ylo, yhi, size=n)
    return m


def generate(name: str, seed: int = 0, *, n_static: int | None = None,
             n_inst: int | None = None, n_steps: int | None = None,
             rig=None, sh_degree: int | None = None, length_scale: float | None = None) -> Scene:
    """Draw the named corridor scene from a PCG64 stream seeded with `seed`.

    The keyword overrides shrink a scene (fewer Gaussians, instances or
    timesteps, a smaller camera) while keeping its distributions; tests use
    them for crops the oracle finishes in seconds. `length_scale` stretches the
    corridor at constant density: its length, static Gaussians, instances and
    timesteps all scale by that factor (a scene-scale sweep).
    """
    spec = SPECS[name]
    if length_scale is not None:
        f = float(length_scale)
        z0, z1 = spec.z_range
        spec = dataclasses.replace(spec, z_range=(z0, z0 + (z1 - z0) * f),
                                   n_static=max(1, int(round(spec.n_static * f))),
                                   n_inst=max(1, int(round(spec.n_inst * f))),
                                   n_steps=max(2, int(round(spec.n_steps * f))),
                                   inst_fixed=None)
    if n_static is not None or n_inst is not None or n_steps is not None or rig is not None \
            or sh_degree is not None:
        spec = dataclasses.replace(
            spec,
            n_static=spec.n_static if n_static is None else int(n_static),
            n_inst=spec.n_inst if n_inst is None else int(n_inst),
            n_steps=spec.n_steps if n_steps is None else int(n_steps),
            rig=spec.rig if rig is None else tuple(rig),
            sh_degree=spec.sh_degree if sh_degree is None else int(sh_degree),
            inst_fixed=spec.inst_fixed if (n_inst is None or spec.inst_fixed is None
                                           or n_inst == len(spec.inst_fixed)) else None)
    rng = np.random.Generator(np.random.PCG64(seed))

    # --- static background
    ns = spec.n_static
    means_s = _static_means(rng, spec, ns)
    ls_s, q_s, o_s = _gaussian_attrs(rng, ns)

    # --- dynamic instances (local frames)
    if spec.inst_sizes[0] == spec.inst_sizes[1]:
        sizes = np.full(spec.n_inst, spec.inst_sizes[0], np.int64)
    else:
        sizes = rng.integers(spec.inst_sizes[0], spec.inst_sizes[1] + 1, size=spec.n_inst)
    nd = int(sizes.sum())
    means_d = np.empty((nd, 3), np.float32)
    means_d[:, 0] = rng.uniform(-1.0, 1.0, size=nd)
    means_d[:, 1] = rng.uniform(-1.0, 1.0, size=nd)
    means_d[:, 2] = rng.uniform(-2.0, 2.0, size=nd)
    ls_d, q_d, o_d = _gaussian_attrs(rng, nd)

    n = ns + nd
    sh = _sh_coeffs(rng, n, spec.sh_degree)
    offsets = np.zeros(spec.n_inst + 2, np.int64)
    offsets[1] = ns
    offsets[2:] = ns + np.cumsum(sizes)

    # --- instance trajectories: constant speed along a fixed yawed heading
    if spec.inst_fixed is not None:
        start = np.array([[x, 1.0, z0] for (x, z0) in spec.inst_fixed], np.float64)
        speed = np.full(spec.n_inst, spec.inst_speed[0])
        yaw = np.zeros(spec.n_inst)
    else:
        start = np.stack([rng.uniform(*spec.inst_x, size=spec.n_inst),
                          np.full(spec.n_inst, 1.0),
                          rng.uniform(*spec.z_range, size=spec.n_inst)], axis=1)
        speed = rng.uniform(*spec.inst_speed, size=spec.n_inst)
        yaw = rng.uniform(-spec.inst_yaw, spec.inst_yaw, size=spec.n_inst)
    T = spec.n_steps
    inst_quat = np.empty((T, spec.n_inst, 4), np.float32)
    inst_trans = np.empty((T, spec.n_inst, 3), np.float32)
    for i in range(spec.n_inst):
        heading = _yaw_matrix(yaw[i]) @ np.array([0.0, 0.0, 1.0])
        q = _yaw_quat(yaw[i])
        for k in range(T):
            inst_quat[k, i] = q
            inst_trans[k, i] = start[i] + speed[i] * (k * spec.dt) * heading

    # --- rendering times normalised to [-1, 1] and the rig's cameras
    if T > 1:
        times = (-1.0 + 2.0 * np.arange(T, dtype=np.float32) / np.float32(T - 1)).astype(np.float32)
    else:
        times = np.zeros(1, np.float32)
    cams = []
    for k in range(T):
        pos = (0.0, 0.0, k * spec.cam_step)
        cams.append([make_camera(w, h, f, pos, cy) for (w, h, f, cy) in spec.rig])

    return Scene(
        name=spec.name,
        means=np.ascontiguousarray(np.concatenate([means_s, means_d])),
        log_scales=np.ascontiguousarray(np.concatenate([ls_s, ls_d])),
        quats=np.ascontiguousarray(np.concatenate([q_s, q_d])),
        opacity_logits=np.ascontiguousarray(np.concatenate([o_s, o_d])),
        sh=sh, sh_degree=spec.sh_degree, inst_offsets=offsets,
        inst_quat=inst_quat, inst_trans=inst_trans, times=times, cams=cams,
        lod_threshold=spec.lod_threshold)


def subset(scene: Scene, n_static: int, per_inst: int, seed: int = 0) -> Scene:
    """A crop of `scene`: the first `n_static` static Gaussians and the first
    `per_inst` Gaussians of every instance (the instance layout is kept)."""
    off = scene.inst_offsets
    pick = [np.arange(min(n_static, off[1]))]
    new_off = [0, len(pick[0])]
    for k in range(1, len(off) - 1):
        idx = np.arange(off[k], min(off[k] + per_inst, off[k + 1]))
        pick.append(idx)
        new_off.append(new_off[-1] + len(idx))
    sel = np.concatenate(pick)
    return dataclasses.replace(
        scene, means=scene.means[sel].copy(), log_scales=scene.log_scales[sel].copy(),
        quats=scene.quats[sel].copy(), opacity_logits=scene.opacity_logits[sel].copy(),
        sh=scene.sh[sel].copy(), inst_offsets=np.asarray(new_off, np.int64))


def with_cameras(scene: Scene, cams_per_step) -> Scene:
    return dataclasses.replace(scene, cams=cams_per_step)


def ode_model(seed: int, n_inst: int, embed_dim: int = 8, scale: float = 0.6,
              z0_positions=None):
    """Seeded parameters of the NeuralODE pose model (flat FP32 vector in the
    library's layout, hidden width 64), instance embeddings [K, D] and initial
    states [K, 6] (the given positions, or uniform in a 20 m box, and zero
    rotation). Random draws only."""
    rng = np.random.Generator(np.random.PCG64(seed))
    H = 64
    n = H * (7 + embed_dim) + H + H * H + H + 6 * H + 6
    params = (rng.standard_normal(n) * (scale / np.sqrt(H))).astype(np.float32)
    embed = (rng.standard_normal((n_inst, embed_dim)) * 0.5).astype(np.float32)
    z0 = np.zeros((n_inst, 6), np.float32)
    if z0_positions is None:
        z0[:, :3] = rng.uniform(-10.0, 10.0, (n_inst, 3))
    else:
        z0[:, :3] = np.asarray(z0_positions, np.float32)
    return params, embed, z0
