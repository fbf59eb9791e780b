"""ctypes binding of libs3r (include/s3r.h), argument marshalling only.

Every computation runs in the CUDA library; this module turns torch tensors
into device pointers, cameras into ``s3r_camera`` structs, and non-OK status
codes into exceptions. It loads ``libs3r.so`` from the package directory (or
the variant build that the environment variable ``S3R_LIBRARY`` names, which
is how the autotuner times alternative launch shapes) and raises if it is
missing: there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_LIB_PATH = os.path.join(HERE, "libs3r.so")
LIB_PATH = os.environ.get("S3R_LIBRARY") or DEFAULT_LIB_PATH

S3R_MAX_VIEWS = 32
VIS_RECORD, VIS_FINALIZE, VIS_RESET = 0, 1, 2
STATUS_NAMES = {0: "S3R_OK", 1: "S3R_ERR_INVALID", 2: "S3R_ERR_CAPACITY", 3: "S3R_ERR_CUDA",
                4: "S3R_ERR_TIMEOUT", 5: "S3R_ERR_STATE"}

# every entry point declared in include/s3r.h
EXPORTS = ("s3r_workspace_create", "s3r_workspace_destroy", "s3r_workspace_bytes", "s3r_project",
           "s3r_sort", "s3r_render_fwd", "s3r_render_bwd", "s3r_update_visibility",
           "s3r_query_counts", "s3r_sync_status", "s3r_debug_buffer", "s3r_last_error",
           "s3r_version", "s3r_built_arch", "s3r_l1_loss", "s3r_set_timing",
           "s3r_kernel_count", "s3r_kernel_name", "s3r_kernel_times", "s3r_select_visible_static",
           "s3r_adam_step", "s3r_set_lod", "s3r_set_counting", "s3r_to_world",
           "s3r_check_wait_timeout", "s3r_set_epoch", "s3r_device_status", "s3r_set_grad_mode",
           "s3r_ode_param_count", "s3r_ode_poses", "s3r_ode_poses_bwd", "s3r_to_world_bwd")

LOD_THRESHOLD = 0
LOD_STOCHASTIC = 1
GRAD_ACCUMULATE = 0
GRAD_OVERWRITE = 1


class S3RError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class Camera(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("height", ctypes.c_int32), ("fx", ctypes.c_float),
                ("fy", ctypes.c_float), ("cx", ctypes.c_float), ("cy", ctypes.c_float),
                ("near_z", ctypes.c_float), ("world_to_cam", ctypes.c_float * 12)]


class Scene(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("means", ctypes.c_void_p), ("log_scales", ctypes.c_void_p),
                ("quats", ctypes.c_void_p), ("opacity_logits", ctypes.c_void_p),
                ("sh", ctypes.c_void_p), ("sh_degree", ctypes.c_int32),
                ("inst_offsets", ctypes.c_void_p), ("n_inst", ctypes.c_int32)]


class Poses(ctypes.Structure):
    _fields_ = [("quat", ctypes.c_void_p), ("trans", ctypes.c_void_p)]


class Grads(ctypes.Structure):
    _fields_ = [("means", ctypes.c_void_p), ("log_scales", ctypes.c_void_p),
                ("quats", ctypes.c_void_p), ("opacity_logits", ctypes.c_void_p),
                ("sh", ctypes.c_void_p), ("inst_quat", ctypes.c_void_p),
                ("inst_trans", ctypes.c_void_p)]


class Capacity(ctypes.Structure):
    _fields_ = [("max_gaussians", ctypes.c_int64), ("max_splats", ctypes.c_int64),
                ("max_duplicates", ctypes.c_int64), ("max_views", ctypes.c_int32),
                ("max_instances", ctypes.c_int32), ("max_tiles", ctypes.c_int64),
                ("max_pixels", ctypes.c_int64), ("max_rows", ctypes.c_int64)]


class AdamTensor(ctypes.Structure):
    _fields_ = [("param", ctypes.c_void_p), ("grad", ctypes.c_void_p), ("exp_avg", ctypes.c_void_p),
                ("exp_avg_sq", ctypes.c_void_p), ("n", ctypes.c_int64)]


class OdeNet(ctypes.Structure):
    _fields_ = [("embed_dim", ctypes.c_int32), ("params", ctypes.c_void_p), ("embed", ctypes.c_void_p)]


class Counts(ctypes.Structure):
    _fields_ = [("n_selected", ctypes.c_int64), ("n_splats", ctypes.c_int64),
                ("n_duplicates", ctypes.c_int64), ("n_frustum", ctypes.c_int64),
                ("n_blend_pairs", ctypes.c_int64), ("device_status", ctypes.c_uint32),
                ("epoch", ctypes.c_uint32), ("n_eval_fwd", ctypes.c_int64),
                ("n_eval_bwd", ctypes.c_int64)]


class LodParams(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("p_max", ctypes.c_float), ("distance", ctypes.c_float),
                ("offset", ctypes.c_float * 3), ("seed", ctypes.c_uint64)]


_lib = None


def load(path: str = LIB_PATH):
    """Load libs3r.so (built by ``paper_2503_08217_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with `python -m paper_2503_08217_gb300.build`"
                           " (the CUDA path has no fallback)")
    L = ctypes.CDLL(path)
    vp, i64, i32, f32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_float
    P = ctypes.POINTER
    L.s3r_workspace_create.argtypes = [P(Capacity), ctypes.c_int, P(vp)]
    L.s3r_workspace_destroy.argtypes = [vp]
    L.s3r_workspace_bytes.argtypes = [vp]
    L.s3r_workspace_bytes.restype = i64
    L.s3r_project.argtypes = [vp, P(Scene), P(Poses), P(Camera), i32, f32, vp, vp, f32, vp]
    L.s3r_sort.argtypes = [vp, vp]
    L.s3r_render_fwd.argtypes = [vp, vp, vp, vp]
    L.s3r_render_bwd.argtypes = [vp, P(Scene), P(Poses), vp, vp, P(Grads), vp]
    L.s3r_update_visibility.argtypes = [i64, f32, vp, vp, vp, i32, vp]
    L.s3r_query_counts.argtypes = [vp, vp, P(Counts)]
    L.s3r_l1_loss.argtypes = [i64, vp, vp, vp, vp, vp]
    L.s3r_set_timing.argtypes = [vp, i32]
    L.s3r_set_lod.argtypes = [vp, P(LodParams)]
    L.s3r_set_counting.argtypes = [vp, i32]
    L.s3r_set_grad_mode.argtypes = [vp, i32]
    L.s3r_ode_param_count.argtypes = [i32]
    L.s3r_ode_param_count.restype = i64
    L.s3r_ode_poses.argtypes = [P(OdeNet), i32, vp, vp, i32, i32, vp, vp, vp, vp]
    L.s3r_ode_poses_bwd.argtypes = [P(OdeNet), i32, vp, i32, i32, vp, vp, vp, vp, vp, vp, vp]
    L.s3r_select_visible_static.argtypes = [i64, f32, vp, vp, vp, vp]
    L.s3r_adam_step.argtypes = [P(AdamTensor), i32, f32, f32, f32, f32, i32, vp, vp]
    L.s3r_device_status.argtypes = [vp]
    L.s3r_device_status.restype = vp
    L.s3r_to_world.argtypes = [P(Scene), P(Poses), vp, vp, vp, vp]
    L.s3r_to_world_bwd.argtypes = [vp, P(Scene), P(Poses), P(Grads), vp]
    L.s3r_check_wait_timeout.argtypes = [vp, i32, vp]
    L.s3r_set_epoch.argtypes = [vp, ctypes.c_uint32, vp]
    L.s3r_kernel_count.restype = i32
    L.s3r_kernel_name.argtypes = [i32]
    L.s3r_kernel_name.restype = ctypes.c_char_p
    L.s3r_kernel_times.argtypes = [vp, P(f32), i32]
    L.s3r_sync_status.argtypes = [vp, vp]
    L.s3r_debug_buffer.argtypes = [vp, ctypes.c_char_p]
    L.s3r_debug_buffer.restype = vp
    L.s3r_last_error.restype = ctypes.c_char_p
    L.s3r_version.restype = i32
    L.s3r_built_arch.restype = i32
    for name in ("s3r_workspace_create", "s3r_workspace_destroy", "s3r_project", "s3r_sort",
                 "s3r_render_fwd", "s3r_render_bwd", "s3r_update_visibility",
                 "s3r_query_counts", "s3r_sync_status", "s3r_l1_loss", "s3r_set_timing",
                 "s3r_kernel_times", "s3r_select_visible_static", "s3r_adam_step", "s3r_set_lod",
                 "s3r_set_counting", "s3r_to_world", "s3r_check_wait_timeout",
                 "s3r_set_epoch", "s3r_set_grad_mode", "s3r_ode_poses", "s3r_ode_poses_bwd", "s3r_to_world_bwd"):
        getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def _check(status: int):
    if status != 0:
        raise S3RError(status, load().s3r_last_error().decode())


def _ptr(t) -> int | None:
    if t is None:
        return None
    if not isinstance(t, torch.Tensor):
        raise TypeError("expected a torch tensor")
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return t.data_ptr()


def _stream(stream=None) -> int:
    s = torch.cuda.current_stream() if stream is None else stream
    return s.cuda_stream


def make_camera(cam) -> Camera:
    """s3r_camera from any object with width, height, fx, fy, cx, cy, near,
    world_to_cam (3x4)."""
    c = Camera()
    c.width, c.height = int(cam.width), int(cam.height)
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    c.near_z = float(getattr(cam, "near", 0.2))
    w = [float(x) for x in list(__import__("numpy").asarray(cam.world_to_cam).reshape(12))]
    c.world_to_cam = (ctypes.c_float * 12)(*w)
    return c


def make_scene(means, log_scales, quats, opacity_logits, sh, inst_offsets, sh_degree: int) -> Scene:
    s = Scene()
    s.n = int(means.shape[0])
    s.means, s.log_scales, s.quats = _ptr(means), _ptr(log_scales), _ptr(quats)
    s.opacity_logits, s.sh = _ptr(opacity_logits), _ptr(sh)
    s.sh_degree = int(sh_degree)
    s.inst_offsets = _ptr(inst_offsets)
    s.n_inst = int(inst_offsets.shape[0]) - 2
    return s


def make_poses(inst_quat, inst_trans) -> Poses:
    p = Poses()
    p.quat, p.trans = _ptr(inst_quat), _ptr(inst_trans)
    return p


class Workspace:
    """Owns an s3r_workspace (device intermediates, allocated once)."""

    def __init__(self, *, max_gaussians: int, max_splats: int, max_duplicates: int,
                 max_views: int, max_instances: int, max_tiles: int, max_pixels: int,
                 max_rows: int = 0, device: int | None = None):
        L = load()
        self.device = torch.cuda.current_device() if device is None else int(device)
        cap = Capacity(max_gaussians, max_splats, max_duplicates, max_views, max_instances,
                       max_tiles, max_pixels, max_rows)
        self.capacity = cap
        h = ctypes.c_void_p()
        _check(L.s3r_workspace_create(ctypes.byref(cap), self.device, ctypes.byref(h)))
        self._h = h
        self.n_views = 0
        self.cams = []

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().s3r_workspace_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    @property
    def nbytes(self) -> int:
        return int(load().s3r_workspace_bytes(self._h))

    def project(self, scene: Scene, poses: Poses, cams, t: float, vis_window, point_life,
                lod_threshold: float, stream=None):
        arr = (Camera * len(cams))(*[make_camera(c) if not isinstance(c, Camera) else c
                                      for c in cams])
        self.cams = list(cams)
        self.n_views = len(cams)
        _check(load().s3r_project(self._h, ctypes.byref(scene), ctypes.byref(poses), arr,
                                  len(cams), float(t), _ptr(vis_window), _ptr(point_life),
                                  float(lod_threshold), _stream(stream)))

    def sort(self, stream=None):
        _check(load().s3r_sort(self._h, _stream(stream)))

    def render_fwd(self, background, out_rgb, stream=None):
        _check(load().s3r_render_fwd(self._h, _ptr(background), _ptr(out_rgb), _stream(stream)))

    def render_bwd(self, scene: Scene, poses: Poses, background, dL_drgb, grads: dict,
                   stream=None):
        g = Grads()
        for k in ("means", "log_scales", "quats", "opacity_logits", "sh", "inst_quat",
                  "inst_trans"):
            setattr(g, k, _ptr(grads.get(k)))
        _check(load().s3r_render_bwd(self._h, ctypes.byref(scene), ctypes.byref(poses),
                                     _ptr(background), _ptr(dL_drgb), ctypes.byref(g),
                                     _stream(stream)))

    def counts(self, stream=None) -> dict:
        c = Counts()
        _check(load().s3r_query_counts(self._h, _stream(stream), ctypes.byref(c)))
        return {"n_selected": c.n_selected, "n_splats": c.n_splats,
                "n_duplicates": c.n_duplicates, "n_frustum": c.n_frustum,
                "n_blend_pairs": c.n_blend_pairs, "device_status": c.device_status,
                "epoch": c.epoch, "n_eval_fwd": c.n_eval_fwd, "n_eval_bwd": c.n_eval_bwd}

    def set_lod(self, mode: int = LOD_THRESHOLD, p_max: float = 0.0, distance: float = 1.0,
                offset=(0.0, 0.0, 0.0), seed: int = 0):
        """LOD of the following projections (Eq. 7 when mode is LOD_STOCHASTIC)."""
        if mode == LOD_THRESHOLD:
            _check(load().s3r_set_lod(self._h, None))
            return
        prm = LodParams(int(mode), float(p_max), float(distance), (ctypes.c_float * 3)(*offset),
                        int(seed) & 0xFFFFFFFFFFFFFFFF)
        _check(load().s3r_set_lod(self._h, ctypes.byref(prm)))

    def set_counting(self, enable: bool):
        """Count the blend kernels' walked and evaluated pairs (see counts())."""
        _check(load().s3r_set_counting(self._h, 1 if enable else 0))

    def set_timing(self, enable: bool):
        _check(load().s3r_set_timing(self._h, 1 if enable else 0))

    def kernel_times(self) -> dict:
        """{kernel name: ms of its last launch} (call after synchronising)."""
        L = load()
        n = L.s3r_kernel_count()
        buf = (ctypes.c_float * n)()
        _check(L.s3r_kernel_times(self._h, buf, n))
        return {L.s3r_kernel_name(i).decode(): float(buf[i]) for i in range(n) if buf[i] >= 0}

    def sync_status(self, stream=None):
        _check(load().s3r_sync_status(self._h, _stream(stream)))

    def to_world_bwd(self, scene: Scene, poses: Poses, grads: dict, stream=None):
        """Backward of to_world in place on grads (see s3r_to_world_bwd)."""
        g = Grads()
        for k in ("means", "log_scales", "quats", "opacity_logits", "sh", "inst_quat",
                  "inst_trans"):
            setattr(g, k, _ptr(grads.get(k)))
        _check(load().s3r_to_world_bwd(self._h, ctypes.byref(scene), ctypes.byref(poses),
                                       ctypes.byref(g), _stream(stream)))

    def set_grad_mode(self, mode: int):
        """GRAD_ACCUMULATE (default): render_bwd adds to the gradient buffers;
        GRAD_OVERWRITE: it writes every element (zeros where no view kept the
        Gaussian), so the buffers need no zeroing."""
        _check(load().s3r_set_grad_mode(self._h, int(mode)))

    def status_word(self) -> int:
        """Device address of the latched status word (adam_step's gate)."""
        return int(load().s3r_device_status(self._h) or 0)

    def set_epoch(self, epoch: int, stream=None):
        """Restore the call counter of a saved run (resume of the Eq. 7 draws)."""
        _check(load().s3r_set_epoch(self._h, int(epoch) & 0xFFFFFFFF, _stream(stream)))

    def check_wait_timeout(self, max_polls: int = 1000, stream=None):
        """Make the bounded look-back waits give up on purpose (failure-detection
        test hook); the next sync_status() raises S3R_ERR_TIMEOUT."""
        _check(load().s3r_check_wait_timeout(self._h, int(max_polls), _stream(stream)))

    def debug(self, name: str, dtype: torch.dtype, count: int) -> torch.Tensor:
        """Copy `count` elements of a workspace intermediate to a new tensor."""
        ptr = load().s3r_debug_buffer(self._h, name.encode())
        if not ptr:
            raise KeyError(name)
        if count == 0:
            return torch.empty(0, dtype=dtype, device=f"cuda:{self.device}")
        view = torch.as_tensor(_DeviceArray(ptr, count, dtype), device=f"cuda:{self.device}")
        return view.clone()


_TYPESTR = {torch.float32: "<f4", torch.int32: "<i4", torch.uint8: "|u1", torch.int64: "<i8"}


class _DeviceArray:
    """A view of device memory for torch.as_tensor (CUDA array interface);
    used only to copy workspace intermediates out, never written through."""

    def __init__(self, ptr: int, count: int, dtype: torch.dtype):
        self.__cuda_array_interface__ = {"shape": (int(count),), "typestr": _TYPESTR[dtype],
                                         "data": (int(ptr), False), "version": 3,
                                         "strides": None}


def l1_loss(pred, target, dL_dpred, loss_out, stream=None):
    """loss_out = mean|pred - target|; dL_dpred = sign(pred - target) / n."""
    _check(load().s3r_l1_loss(int(pred.numel()), _ptr(pred), _ptr(target), _ptr(dL_dpred),
                              _ptr(loss_out), _stream(stream)))


def select_visible_static(vis_window, t: float, out_idx, out_count, stream=None):
    """Temporal selection without any device allocation by the library: the
    ids i with v_s <= t <= v_e go to out_idx (uint32, caller-owned) and their
    number to out_count (one uint32 on the device). For callers that may not
    allocate; see s3r_select_visible_static in include/s3r.h."""
    n = int(vis_window.shape[0]) if vis_window is not None else 0
    _check(load().s3r_select_visible_static(n, float(t), _ptr(vis_window), _ptr(out_idx),
                                            _ptr(out_count), _stream(stream)))


def to_world(c_scene, poses, means_out, quats_out, sh_out=None, stream=None):
    """The conventional local-to-world transform (see s3r_to_world): writes the
    dynamic rows of the world-frame means [n,3], unit quaternions [n,4] and,
    with sh_out, rotated SH [n,K,3]; static rows are left as they are."""
    _check(load().s3r_to_world(ctypes.byref(c_scene), ctypes.byref(poses), _ptr(means_out),
                               _ptr(quats_out), _ptr(sh_out), _stream(stream)))


def adam_step(params, grads, exp_avgs, exp_avg_sqs, lr: float, step: int, beta1: float = 0.9,
              beta2: float = 0.999, eps: float = 1e-8, stream=None, gate: int | None = None):
    """One fused Adam step over up to 8 (param, grad, m, v) tensor groups.
    `gate`: device address of a uint32 (e.g. Workspace.status_word()); the
    step changes nothing unless it reads 0 on the device."""
    if not (len(params) == len(grads) == len(exp_avgs) == len(exp_avg_sqs)):
        raise ValueError("adam_step: one gradient and two moment tensors per parameter")
    arr = (AdamTensor * max(1, len(params)))()
    for i, (p, g, m, v) in enumerate(zip(params, grads, exp_avgs, exp_avg_sqs)):
        for t in (p, g, m, v):
            if t.dtype != torch.float32 or t.numel() != p.numel():
                raise ValueError("adam_step: float32 tensors of equal size required")
        arr[i] = AdamTensor(_ptr(p), _ptr(g), _ptr(m), _ptr(v), int(p.numel()))
    _check(load().s3r_adam_step(arr, len(params), float(lr), float(beta1), float(beta2),
                                float(eps), int(step), ctypes.c_void_p(gate) if gate else None,
                                _stream(stream)))


def update_visibility(n: int, t: float, mask, point_life, vis_window, mode: int, stream=None):
    _check(load().s3r_update_visibility(int(n), float(t), _ptr(mask), _ptr(point_life),
                                        _ptr(vis_window), int(mode), _stream(stream)))


# ---------------------------------------------------------------- NeuralODE poses
def ode_param_count(embed_dim: int) -> int:
    n = int(load().s3r_ode_param_count(int(embed_dim)))
    if n < 0:
        raise ValueError(f"embed_dim {embed_dim} outside [0, 16]")
    return n


def _ode_net(params, embed) -> OdeNet:
    d = int(embed.shape[1]) if embed is not None and embed.dim() == 2 else 0
    return OdeNet(d, _ptr(params), _ptr(embed) if d else None)


def ode_poses(params, embed, z0, times, substeps: int, stream=None):
    """Eq. 4 through the library: returns (states, quat [T, K, 4], trans [T, K, 3])
    as new device tensors (see s3r_ode_poses)."""
    K, T = int(z0.shape[0]), int(times.shape[0])
    dev = z0.device
    states = torch.empty(((T - 1) * substeps + 1, K, 6), device=dev)
    quat = torch.empty((T, K, 4), device=dev)
    trans = torch.empty((T, K, 3), device=dev)
    net = _ode_net(params, embed)
    _check(load().s3r_ode_poses(ctypes.byref(net), K, _ptr(z0), _ptr(times), T, int(substeps),
                                _ptr(states), _ptr(quat), _ptr(trans), _stream(stream)))
    return states, quat, trans


def ode_poses_bwd(params, embed, times, substeps: int, states, g_quat, g_trans, g_params, g_embed,
                  g_z0, stream=None):
    """Reverse mode of ode_poses: adds into g_params, g_embed, g_z0."""
    K, T = int(states.shape[1]), int(times.shape[0])
    net = _ode_net(params, embed)
    _check(load().s3r_ode_poses_bwd(ctypes.byref(net), K, _ptr(times), T, int(substeps), _ptr(states),
                                    _ptr(g_quat), _ptr(g_trans), _ptr(g_params), _ptr(g_embed),
                                    _ptr(g_z0), _stream(stream)))
