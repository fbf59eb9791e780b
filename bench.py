#!/usr/bin/env python
"""Throughput of the per-timestep render-and-backprop path on GB300.

One step = one training step of the batched multi-camera path at one
timestep: temporal selection, instance-matrix projection with EWA covariance,
frustum mask and point-life update (Eq. 5), LOD cull, SH colour, tile|depth
duplication and radix sort, 16x16-tile alpha blending (Eq. 2), an L1
photometric loss against a synthetic target, and the hand-written backward to
every Gaussian parameter and instance pose. All cameras of the rig run in one
call sequence captured as a CUDA graph.

Printed (rank 0, one JSON line): views/s (value), Mpix/s, the plain per-view
comparator (the same library, one camera per call sequence, eager, no graph),
per-kernel device times, the roofline of the dominant kernel, the FP64 CPU
oracle timed on a bounded sample on this host, an end-to-end figure through
the public API with host buffers, and the SM clocks seen while timing.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload rig|mid|large|tiny|small-rig]
  python bench.py --impl reference ...   # the FP64 CPU oracle on this host's cores
  python bench.py --conventional ...     # the Fig. 1(a) pipeline (world transform, no LOD)
  python bench.py --sweep scale          # per-view time against scene size
  python bench.py --sweep lod            # per-view time against the LOD threshold
  python bench.py --workload train       # optimisation steps (forward, backward, Adam)
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "fwd+bwd views/s and Mpix/s vs plain per-view path, same GB300; % HBM roofline"

# DRAM bytes (read + write) per launch of a kernel at the rig workload, from
# one ncu capture (summarised under profiles/), valid only while the kernel's
# source code is the one the counters were taken on: the first 16 hex digits
# of the SHA-256 of the file with its comments and blank lines removed (code
# hash), so that a comment edit keeps the figure and any code edit drops it
# (the roofline line then reports traffic null).
NCU_TRAFFIC = {
    "blend_bwd": {"bytes": 1983235328, "source": "paper_2503_08217_gb300/csrc/k_blend.cu",
                  "code_sha256_16": "9d5f105faa34333b", "profile": "profiles/blend_bwd_traffic_rig.md"},
}


def code_hash(path: str) -> str:
    """SHA-256 (16 hex digits) of a C++/CUDA source without its // and /* */
    comments, trailing blanks and blank lines."""
    import hashlib
    import re
    text = open(path, encoding="utf-8").read()
    out, i, n = [], 0, len(text)
    while i < n:
        c = text[i]
        if c == '"':                               # string literal: kept as is
            j = i + 1
            while j < n and text[j] != '"':
                j += 2 if text[j] == "\\" else 1
            out.append(text[i:j + 1])
            i = j + 1
        elif text.startswith("//", i):
            while i < n and text[i] != "\n":
                i += 1
        elif text.startswith("/*", i):
            j = text.find("*/", i + 2)
            i = n if j < 0 else j + 2
        else:
            out.append(c)
            i += 1
    lines = [ln.rstrip() for ln in "".join(out).split("\n")]
    body = "\n".join(ln for ln in lines if ln)
    return hashlib.sha256(body.encode("utf-8")).hexdigest()[:16]


def launch_shapes() -> dict:
    """The build-time launch shapes of the library this run loads: the source
    defaults (the autotuner's choice) for the default build, else the
    variant's name."""
    lib = os.environ.get("S3R_LIBRARY")
    if lib:
        return {"variant": os.path.basename(os.path.dirname(os.path.abspath(lib)))}
    from paper_2503_08217_gb300 import autotune
    return autotune.source_defaults()


def measured_traffic(kernel: str, workload: str):
    t = NCU_TRAFFIC.get(kernel)
    if t is None or workload != "rig" or os.environ.get("S3R_LIBRARY"):
        return None   # the capture describes the default build at the rig workload
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), t["source"])
    if code_hash(path) != t["code_sha256_16"]:
        return None
    return t["bytes"]

# workload name -> (scene spec, overrides, LOD threshold, description)
WORKLOADS = {
    "rig": ("rig", {}, 1.0, "batched surround rig on the large corridor: 8M static + 80 instances "
            "of U{5k..20k}, SH3, 5x 1920x1080 + 2x 1280x960 cameras at one timestep"),
    "mid": ("mid", {}, 1.0, "mid corridor: 1M static + 20x5k dynamic, SH3, one 1920x1080 camera"),
    "large": ("large", {}, 1.0, "large corridor: 8M static + 80 instances, SH3, one 1920x1280 camera"),
    "tiny": ("tiny", {}, 0.0, "tiny corridor: 20k static + 2x1k dynamic, SH0, one 320x192 camera"),
    "small-rig": ("rig", {"n_static": 1_500_000, "n_inst": 16, "n_steps": 60}, 1.0,
                  "profiling case: the surround rig on a 1.5M-Gaussian corridor"),
    "ode": ("train", {}, 1.0, "NeuralODE poses of the training corridor's 120 instances over its "
            "400 timesteps (embedding width 8, RK4 with 2 substeps): forward and reverse mode"),
    "train": ("train", {}, 1.0, "training steps on the 2 km corridor: 16M static + 120 instances of "
              "U{5k..20k}, SH3, the 7-camera surround rig, Adam on every parameter and pose"),
}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="ours", choices=("ours", "reference"))
    p.add_argument("--workload", default="rig", choices=tuple(WORKLOADS))
    p.add_argument("--seed", type=int, default=0)
    p.add_argument("--no-plain", action="store_true", help="skip the plain per-view comparator")
    p.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-adam", action="store_true", help="skip the optimiser-step timing")
    p.add_argument("--lod-mode", default="threshold", choices=("threshold", "stochastic"),
                   help="LOD of the projection: the threshold cull, or Eq. 7 on the Gaussians below r")
    p.add_argument("--lod-r", type=float, default=None, help="LOD scale r in px (default: the workload's)")
    p.add_argument("--lod-pmax", type=float, default=0.5)
    p.add_argument("--lod-dist", type=float, default=100.0)
    p.add_argument("--lod-offset", type=float, default=0.1)
    p.add_argument("--lod-seed", type=int, default=2025)
    p.add_argument("--no-temporal", action="store_true",
                   help="select every Gaussian (windows [-1, 1]) instead of the recorded windows")
    p.add_argument("--conventional", action="store_true",
                   help="the conventional pipeline of Fig. 1(a): every step moves the dynamic "
                        "Gaussians to the world frame (s3r_to_world) and renders the scene without "
                        "instances, every Gaussian selected and no LOD")
    p.add_argument("--sweep", default=None, choices=("scale", "lod"),
                   help="scale: per-view fwd+bwd time of the large corridor stretched at constant "
                        "density, with the temporal record and with every Gaussian visible; lod: "
                        "per-view fwd+bwd time of the large corridor against the LOD threshold")
    p.add_argument("--sweep-scales", default="0.5,1,2,4")
    p.add_argument("--sweep-lods", default="0,0.5,1,2")
    return p.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(x: float, world: int, device=None) -> float:
    """The largest value of x over all ranks (the slowest rank's time); the
    identity on one rank. The reduction runs on `device` (the GPU under NCCL,
    the CPU under gloo)."""
    if world <= 1:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: float, world: int, slowest_ms: float) -> float:
    """Whole-job rate: the units all ranks processed over the slowest rank's
    time (weak scaling, one timestep per rank)."""
    return world * units_per_rank / (slowest_ms / 1e3)


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d.get("hbm_gbs", 6800.0)), "measured", float(d.get("sm_max_mhz", 2070.0))
    return 6800.0, "fallback", 2070.0


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while timing."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = os.path.join("/tmp", f"s3r_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.strip().lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def make_workload(name: str, seed: int):
    from paper_2503_08217_gb300 import scenegen
    spec, over, lod, desc = WORKLOADS[name]
    scene = scenegen.generate(spec, seed=seed, **over)
    return scene, lod, desc


def step_index(scene, rank: int) -> int:
    return min(scene.n_steps - 1, scene.n_steps // 2 + rank)


def tile_passes(tiles: int) -> int:
    """8-bit radix passes over the view-tile ids (as the library plans them)."""
    bits = 0
    while bits < 32 and (1 << bits) < tiles:
        bits += 1
    return (bits + 7) // 8


def kernel_models(counts, scene, n_kept_gaussians: int, n_pixels: int, tiles: int,
                  tile_passes: int):
    """Algorithmic bytes (or FP32 ops) per launch of each kernel."""
    n, nsel, S, K = scene.n, counts["n_selected"], counts["n_splats"], counts["n_duplicates"]
    nfr = counts["n_frustum"]
    kk = (scene.sh_degree + 1) ** 2 * 3 * 4
    geo = 12 + 12 + 16 + 4
    m = {
        # the visibility windows in, the selected ids and the selection bitmap out
        "temporal_compact": ("hbm", 8 * n + 4 * nsel + n / 8),
        # masks: ids, geometry, two masks out, the life record where in
        # frustum, the (index, id) work list; scan: masks in, offsets out;
        # splats: the work list, mask, offset, geometry and SH in, 61-byte
        # records out (the 32-byte packed record, colour and depth, the
        # rectangle and view, the depth key)
        "project": ("hbm", nsel * (4 + geo + 8) + 8 * nfr + n_kept_gaussians * 8),
        "splat_scan": ("hbm", nsel * 8),
        "project_splats": ("hbm", n_kept_gaussians * (8 + 4 + 4 + geo + kk)
                           + S * (32 + 16 + 8 + 1 + 4)),
        "sort_depth_pass0": ("hbm", S * (4 + 8)),
        "sort_depth_pass1": ("hbm", S * 16),
        "sort_depth_pass2": ("hbm", S * 16),
        "sort_depth_pass3": ("hbm", S * 16),
        # duplication: per splat in depth order, its sorted id and packed
        # 32-byte record in, its tile count and 32-byte expansion record out
        # (row-table entries beyond three rows not counted); the
        # scan reads the counts and writes the offsets; the expansion reads
        # offsets and records and writes the pairs
        "splat_tiles": ("hbm", S * (4 + 32) + S * (4 + 32)),
        "duplicate": ("hbm", S * (4 + 4)),
        "duplicate_expand": ("hbm", S * (4 + 32) + K * 8),   # + tile-digit histograms (on chip)
        # per tile: its range and class slot out (the binary searches' reads
        # are cached); the forward's contributor bits cleared
        "tile_ranges": ("hbm", tiles * (8 + 4) + K / 8 * 2),
        # overwrite mode: kept rows written once (no read), the splat adjoints read
        "project_bwd": ("hbm", n_kept_gaussians * (12 + geo + kk + (geo + kk)) + S * 48),
        # FP32 operations per evaluated (pixel, splat) pair, counted in the code
        # (MUFU ops besides). Forward 17: offset (1, the column's dx shared),
        # quadratic form (5), opacity scale and alpha clamp (2), three tests,
        # transmittance update (2), weight (1), three colour FMAs. Backward 42:
        # the same evaluation and two tests (10), 1 - alpha, T recovery, the
        # colour-behind dot product (3), dL/dalpha (2), weight and Bd update
        # (2), the clamp test, dL/dopacity and dL/dpower (2), the moment sums
        # (4.5 per pixel, column terms shared by its two rows), dL/dopacity and
        # colour sums (4), and the 9 additions per pair of the sums over pixels
        "blend_fwd": ("alu", counts["n_eval_fwd"] * 17),
        "blend_bwd": ("alu", counts["n_eval_bwd"] * 42),
    }
    # the world transform of the dynamic rows (Fig. 1(a)): means, quaternions
    # and SH in and out; its backward reads the parameters and the world-frame
    # adjoints and writes the object-frame adjoints in place
    n_dyn = int(scene.inst_offsets[-1] - scene.inst_offsets[1]) if scene.n_inst else 0
    m["to_world"] = ("hbm", n_dyn * 2 * (12 + 16 + kk))
    m["to_world_bwd"] = ("hbm", n_dyn * 3 * (12 + 16 + kk))
    for p in range(tile_passes):
        m[f"sort_tile_pass{p}"] = ("hbm", K * 16)
    return m


def run_ours(args, rank, world, local):
    import torch
    from paper_2503_08217_gb300 import binding, build
    from paper_2503_08217_gb300.render import DeviceScene, Renderer, pixel_count, tile_count

    build.build()
    binding.load()
    torch.cuda.set_device(local)
    dev_name = f"cuda:{local}"
    scene, lod, desc = make_workload(args.workload, args.seed)
    if args.lod_r is not None:
        lod = float(args.lod_r)
    if args.conventional:
        lod = 0.0
        args.no_temporal = True
    k = step_index(scene, rank)
    cams = scene.cams[k]
    n_views = len(cams)
    P = pixel_count(cams)
    dev = DeviceScene.from_host(scene, dev_name)
    cs = dev.c_scene()
    n = scene.n
    max_splats = max(4096, int(n * min(n_views, 3)))
    r = Renderer(n, scene.n_inst, cams, max_splats=max_splats, max_duplicates=min(2**31 - 1, 6 * max_splats))
    lod_cfg = {"mode": args.lod_mode, "r_px": lod}
    if args.lod_mode == "stochastic":
        r.ws.set_lod(binding.LOD_STOCHASTIC, p_max=args.lod_pmax, distance=args.lod_dist,
                     offset=(args.lod_offset,) * 3, seed=args.lod_seed)
        lod_cfg.update(p_max=args.lod_pmax, distance_m=args.lod_dist, offset_m=args.lod_offset,
                       seed=args.lod_seed)

    # --- first-epoch sweep: Eq. 5 over all timesteps, then Eq. 6
    vis = torch.empty((n, 2), device=dev_name)
    life = torch.empty((n, 2), device=dev_name)
    binding.update_visibility(n, 0.0, None, life, vis, binding.VIS_RESET)
    all_vis = vis.clone()
    bg = torch.zeros(3, device=dev_name)
    sweep_t0 = time.time()
    for kk in range(scene.n_steps):
        iq = torch.from_numpy(scene.inst_quat[kk]).to(dev_name)
        it = torch.from_numpy(scene.inst_trans[kk]).to(dev_name)
        r.ws.project(cs, binding.make_poses(iq, it), scene.cams[kk], float(scene.times[kk]), all_vis,
                     life, lod)
    binding.update_visibility(n, 0.0, None, life, vis, binding.VIS_FINALIZE)
    if args.no_temporal:
        vis = all_vis
    torch.cuda.synchronize()
    sweep_s = time.time() - sweep_t0
    r.counts()  # clears any capacity flag raised while sweeping

    iq = torch.from_numpy(scene.inst_quat[k]).to(dev_name)
    it = torch.from_numpy(scene.inst_trans[k]).to(dev_name)
    t = float(scene.times[k])
    gen = torch.Generator(device=dev_name)
    gen.manual_seed(1234 + rank)
    target = torch.rand(3 * P, device=dev_name, generator=gen)
    out = torch.empty(3 * P, device=dev_name)
    dL = torch.empty(3 * P, device=dev_name)
    loss = torch.zeros(1, device=dev_name)
    grads = {"means": torch.zeros_like(dev.means), "log_scales": torch.zeros_like(dev.log_scales),
             "quats": torch.zeros_like(dev.quats), "opacity_logits": torch.zeros_like(dev.opacity_logits),
             "sh": torch.zeros_like(dev.sh), "inst_quat": torch.zeros_like(iq),
             "inst_trans": torch.zeros_like(it)}

    if args.conventional:
        # Fig. 1(a): the world-frame copy of the scene, rendered without
        # instances; its static rows are copied once (they do not move), its
        # dynamic rows (means, quaternions, rotated SH) rewritten every step
        mw = dev.means.clone()
        qw = dev.quats.clone()
        shw = dev.sh.clone()
        cs_w = binding.make_scene(mw, dev.log_scales, qw, dev.opacity_logits, shw,
                                  torch.tensor([0, n], dtype=torch.int64, device=dev_name),
                                  dev.sh_degree)
        no_q = torch.zeros((0, 4), device=dev_name)
        no_t = torch.zeros((0, 3), device=dev_name)

    def make_step(tgt, iq_, it_):
        def step_fn():
            # the loss and every gradient element are written by the library
            # (L1 loss and the overwrite mode of the backward): no zero fills
            if args.conventional:
                poses_ = binding.make_poses(iq_, it_)
                binding.to_world(cs, poses_, mw, qw, shw)
                r.forward(dev, no_q, no_t, cams, t, vis, life, lod, bg, out=out, c_scene=cs_w)
                binding.l1_loss(out, tgt, dL, loss)
                r.backward(dev, no_q, no_t, bg, dL, grads, c_scene=cs_w, overwrite=True)
                # the world-frame adjoints back to the object frame and the poses
                r.ws.to_world_bwd(cs, poses_, grads)
                return
            r.forward(dev, iq_, it_, cams, t, vis, life, lod, bg, out=out, c_scene=cs)
            binding.l1_loss(out, tgt, dL, loss)
            r.backward(dev, iq_, it_, bg, dL, grads, c_scene=cs, overwrite=True)
        return step_fn

    step = make_step(target, iq, it)

    # one counted eager step (outside the timed region) gives the pair counts
    # of the ALU models; the timed graph runs the uncounted kernels
    r.ws.set_counting(True)
    step()
    torch.cuda.synchronize()
    r.sync_status()
    counts = r.counts()
    r.ws.set_counting(False)
    flush = torch.empty(512 * 1024 * 1024 // 4, device=dev_name)

    # per-kernel times: a graph with the timing hook's event records, replayed
    # with the same protocol as the timed steps (kept apart from them so that
    # the event records are not part of the measured step)
    r.ws.set_timing(True)
    graph_k = r.capture(step)
    for _ in range(args.warmup):
        graph_k.replay()
    torch.cuda.synchronize()
    ktimes = {}
    for i in range(args.steps):
        flush.fill_(float(i))
        graph_k.replay()
        torch.cuda.synchronize()
        for name, ms in r.ws.kernel_times().items():
            ktimes.setdefault(name, []).append(ms)
    r.ws.set_timing(False)
    del graph_k
    if args.conventional:
        # the world transform and its backward are not kernels of the
        # workspace's timing hook: each is captured in a graph of its own and
        # timed by events around the replay (L2 flushed before each), so that
        # no host-side argument marshalling falls inside the events
        poses_ = binding.make_poses(iq, it)
        for name, fn in (("to_world", lambda: binding.to_world(cs, poses_, mw, qw, shw)),
                         ("to_world_bwd", lambda: r.ws.to_world_bwd(cs, poses_, grads))):
            g_ = r.capture(fn)
            evs = []
            for i in range(args.warmup + args.steps):
                flush.fill_(float(i))
                a_, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a_.record()
                g_.replay()
                b_.record()
                evs.append((a_, b_))
            torch.cuda.synchronize()
            ktimes[name] = [a_.elapsed_time(b_) for a_, b_ in evs[args.warmup:]]
            del g_
        step()                                        # the gradients as one step leaves them
        torch.cuda.synchronize()

    # the timed steps: the step as a user captures it
    graph = r.capture(step)
    for _ in range(args.warmup):
        graph.replay()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    with ClockSampler(local) as clocks:
        for i in range(args.steps):
            flush.fill_(float(i))                     # L2 flush, outside the timed events
            ev[i][0].record()
            graph.replay()
            ev[i][1].record()
            torch.cuda.synchronize()                  # spreads the loop over the clock samples
    if world > 1:
        torch.distributed.barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = max_over_ranks(float(sum(step_ms)), world, dev_name)
    r.sync_status()
    clock = clocks.summary()
    ms_per_step = total_ms / args.steps
    views_s = job_throughput(n_views * args.steps, world, total_ms)
    mpix_s = job_throughput(P * args.steps, world, total_ms) / 1e6

    # --- kernel table and roofline of the dominant kernel
    keep = r.ws.debug("keep_mask", torch.int32, counts["n_selected"])
    n_kept_g = int((keep != 0).sum().item())
    kmean = {name: float(np.mean(v)) for name, v in ktimes.items()}
    models = kernel_models(counts, scene, n_kept_g, P, tile_count(cams), tile_passes(tile_count(cams)))
    hbm_peak, peak_kind, sm_max = measured_peaks()
    n_sms = int(torch.cuda.get_device_properties(local).multi_processor_count)
    alu_peak_gops = n_sms * 128 * sm_max * 1e6 / 1e9   # FP32 lanes x clock, one op per lane-cycle
    table = {}
    for name, ms in sorted(kmean.items(), key=lambda kv: -kv[1]):
        row = {"ms": round(ms, 4)}
        if name in models and ms > 0:
            bound, amount = models[name]
            if bound == "hbm":
                gbs = amount / (ms / 1e3) / 1e9
                row.update(bound="hbm", bytes=int(amount), gbs=round(gbs, 1), frac=round(gbs / hbm_peak, 3))
            else:
                gops = amount / (ms / 1e3) / 1e9
                row.update(bound="alu", ops=int(amount), gops=round(gops, 1),
                           frac=round(gops / alu_peak_gops, 3))
        table[name] = row
    if "blend_bwd" in table and kmean.get("blend_bwd", 0) > 0:
        # the backward's CTAs also zero the gradient rows of the overwrite mode
        # once its tile queue is empty (the 44-byte arrays in full, the SH rows
        # of the Gaussians no view kept): the kernel's floor is its ALU work at
        # the ALU peak plus that traffic at the HBM peak
        kk_b = (scene.sh_degree + 1) ** 2 * 3 * 4
        zb = 44 * n + kk_b * (n - n_kept_g)
        floor_ms = (models["blend_bwd"][1] / (alu_peak_gops * 1e9) + zb / (hbm_peak * 1e9)) * 1e3
        table["blend_bwd"].update(zero_bytes=int(zb),
                                  frac_alu_plus_hbm=round(floor_ms / kmean["blend_bwd"], 3))
    if "blend_fwd" in table and kmean.get("blend_fwd", 0) > 0:
        # the usual per-pair estimate of a 3DGS forward (15 FP32 operations
        # per evaluated pair) beside the 17 counted in the code
        g15 = counts["n_eval_fwd"] * 15 / (kmean["blend_fwd"] / 1e3) / 1e9
        table["blend_fwd"]["frac_at_15_ops"] = round(g15 / alu_peak_gops, 3)
    dom = max(kmean, key=kmean.get)
    roof = {"kernel": dom, "bound": None, "achieved": None, "peak": None, "unit": None, "frac": None,
            "traffic": measured_traffic(dom, args.workload)}
    if dom in models:
        bound, amount = models[dom]
        if bound == "hbm":
            roof.update(bound="hbm", achieved=table[dom]["gbs"], peak=hbm_peak, unit="GB/s",
                        frac=table[dom]["frac"], peak_source=f"{peak_kind} hbm_gbs")
        else:
            roof.update(bound="alu", achieved=table[dom]["gops"], peak=round(alu_peak_gops, 1),
                        unit="Gop/s (FP32)", frac=table[dom]["frac"],
                        peak_source=f"{n_sms} SMs (queried) x 128 FP32 lanes x max SM clock "
                                    f"{sm_max:.0f} MHz")
            if "frac_alu_plus_hbm" in table[dom]:
                roof.update(fused_zeroing_bytes=table[dom]["zero_bytes"],
                            frac_alu_plus_hbm=table[dom]["frac_alu_plus_hbm"])
    # the timed kernels, plus untimed ones of ours: the L1 loss and the zeroing
    # of its output and, for the conventional pipeline, the world transform and
    # its backward (two launches)
    launches_per_step = len(kmean) + 2 + (3 if args.conventional else 0)

    # --- plain per-view comparator: the same library, one camera per call, eager
    plain = None
    if not args.no_plain:
        r1 = Renderer(n, scene.n_inst, [max(cams, key=lambda c: c.width * c.height)],
                      max_splats=max(4096, n), max_duplicates=min(2**31 - 1, 6 * max(4096, n)))
        if args.lod_mode == "stochastic":
            r1.ws.set_lod(binding.LOD_STOCHASTIC, p_max=args.lod_pmax, distance=args.lod_dist,
                          offset=(args.lod_offset,) * 3, seed=args.lod_seed)
        offs = np.cumsum([0] + [3 * c.width * c.height for c in cams])

        def plain_sweep():
            # the first view's backward writes the gradients, the others add
            for v, cam in enumerate(cams):
                o = out[offs[v]:offs[v + 1]]
                d = dL[offs[v]:offs[v + 1]]
                r1.forward(dev, iq, it, [cam], t, vis, life, lod, bg, out=o, c_scene=cs)
                binding.l1_loss(o, target[offs[v]:offs[v + 1]], d, loss)
                r1.backward(dev, iq, it, bg, d, grads, c_scene=cs, overwrite=v == 0)

        for _ in range(max(1, args.warmup)):
            plain_sweep()
        torch.cuda.synchronize()
        pev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
        for i in range(args.steps):
            flush.fill_(float(i))
            pev[i][0].record()
            plain_sweep()
            pev[i][1].record()
        torch.cuda.synchronize()
        r1.sync_status()
        pms = float(np.mean([a.elapsed_time(b) for a, b in pev]))
        plain = {"value": round(n_views / (pms / 1e3), 3), "unit": "views/s", "ms_per_step": round(pms, 3),
                 "batched_speedup": round(pms / ms_per_step, 3),
                 "how": "one camera per project/sort/render_fwd/l1/render_bwd sequence, eager launches, no graph"}
        del r1

    # --- end to end through the public API, host buffers in the timed region
    e2e = None
    if not args.no_e2e:
        tgt_host = target.cpu().pin_memory()
        iq_host = iq.cpu().pin_memory()
        it_host = it.cpu().pin_memory()
        loss_host = torch.zeros(1).pin_memory()
        st = torch.cuda.current_stream()
        for _ in range(2):
            target.copy_(tgt_host, non_blocking=True)
            graph.replay()
            loss_host.copy_(loss, non_blocking=True)
        torch.cuda.synchronize()
        # the next step's inputs (target image and poses) are copied host ->
        # device on a second stream while the current step computes, into the
        # other of two input sets, each with its own captured step (no copy on
        # the compute stream, so none waits behind the large one on the copy
        # engine); every step's copies and its loss read-back lie between the
        # two timing events
        cs_ = torch.cuda.Stream()
        tg_b = [torch.empty_like(target) for _ in range(2)]
        iq_b = [torch.empty_like(iq) for _ in range(2)]
        it_b = [torch.empty_like(it) for _ in range(2)]
        for b in range(2):
            tg_b[b].copy_(target)
            iq_b[b].copy_(iq)
            it_b[b].copy_(it)
        graphs = [r.capture(make_step(tg_b[b], iq_b[b], it_b[b])) for b in range(2)]
        ready = [torch.cuda.Event() for _ in range(2)]
        consumed = [torch.cuda.Event() for _ in range(2)]
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

        def h2d(b):
            tg_b[b].copy_(tgt_host, non_blocking=True)
            iq_b[b].copy_(iq_host, non_blocking=True)
            it_b[b].copy_(it_host, non_blocking=True)
            ready[b].record(cs_)

        for _ in range(2):
            for g_ in graphs:
                g_.replay()
        torch.cuda.synchronize()
        e0.record(st)
        cs_.wait_event(e0)
        with torch.cuda.stream(cs_):
            h2d(0)
        for i in range(args.steps):
            b = i & 1
            if i + 1 < args.steps:
                nb = (i + 1) & 1
                with torch.cuda.stream(cs_):
                    if i >= 1:
                        cs_.wait_event(consumed[nb])
                    h2d(nb)
            st.wait_event(ready[b])
            graphs[b].replay()
            consumed[b].record(st)
            loss_host.copy_(loss, non_blocking=True)
        e1.record(st)
        torch.cuda.synchronize()
        ems = max_over_ranks(e0.elapsed_time(e1) / args.steps, world, dev_name)
        bi = tgt_host.numel() * 4 + iq_host.numel() * 4 + it_host.numel() * 4
        e2e = {"value": round(job_throughput(n_views, world, ems), 3), "unit": "views/s",
               "h2d_bytes_per_step": int(bi), "d2h_bytes_per_step": 4, "ms_per_step": round(ems, 3),
               "how": "pinned host target image and poses copied every step on a copy stream into one "
                      "of two input sets (one captured step each), overlapping the previous step; "
                      "loss read back every step"}

    # --- the optimiser step of training: fused Adam over every parameter array
    adam = None
    if not args.no_adam:
        params = [dev.means, dev.log_scales, dev.quats, dev.opacity_logits, dev.sh, iq, it]
        gl = [grads[k2] for k2 in ("means", "log_scales", "quats", "opacity_logits", "sh",
                                    "inst_quat", "inst_trans")]
        ms_ = [torch.zeros_like(x) for x in params]
        vs_ = [torch.zeros_like(x) for x in params]
        n_par = sum(x.numel() for x in params)
        saved = [x.clone() for x in params]
        for i in range(3):
            binding.adam_step(params, gl, ms_, vs_, 1e-4, i + 1)
        aev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(5)]
        for i in range(5):
            flush.fill_(float(i))
            aev[i][0].record()
            binding.adam_step(params, gl, ms_, vs_, 1e-4, i + 4)
            aev[i][1].record()
        torch.cuda.synchronize()
        for x, y in zip(params, saved):
            x.copy_(y)
        del saved, ms_, vs_
        ams = float(np.mean([a.elapsed_time(b) for a, b in aev]))
        abytes = 28 * n_par          # read p, g, m, v; write p, m, v
        agbs = abytes / (ams / 1e3) / 1e9
        adam = {"kernel": "adam", "ms": round(ams, 4), "parameters": int(n_par), "bound": "hbm",
                "bytes": int(abytes), "gbs": round(agbs, 1), "frac": round(agbs / hbm_peak, 3),
                "how": "one launch over all 7 parameter arrays, outside the step, L2 flushed before each"}

    cpu = None
    if rank == 0 and not args.no_cpu:
        cpu = cpu_oracle_sample(scene, k, lod, vis.cpu().numpy())

    if rank == 0:
        # the metric's own comparison first (value, the plain per-view
        # comparator, end to end, roofline), details after
        line = {
            "metric": METRIC, "value": round(views_s, 3), "unit": "views/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_per_step, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "plain_per_view": None if plain is None else {k2: plain[k2] for k2 in
                                                          ("value", "unit", "ms_per_step", "batched_speedup")},
            "mpix_per_s": round(mpix_s, 3),
            "e2e": None if e2e is None else {k2: e2e[k2] for k2 in
                                             ("value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step",
                                              "ms_per_step")},
            "roofline": roof,
            "gpu_launches": launches_per_step * args.steps,
            "clocks": clock,
            "cpu_baseline": cpu,
            "config": {"workload": f"{args.workload}: {desc}", "gaussians": n, "instances": scene.n_inst,
                       "cameras": n_views, "pixels_per_view_batch": P, "timestep": k,
                       "sh_degree": scene.sh_degree, "lod_px": lod, "lod": lod_cfg,
                       "temporal_selection": not args.no_temporal,
                       **({"pipeline": "conventional (Fig. 1(a)): dynamic Gaussians moved to the world "
                                       "frame every step (means, quaternions, SH rotated), rendered "
                                       "without instances, every Gaussian selected, no LOD; the "
                                       "backward maps the world-frame adjoints back to the object "
                                       "frame and the poses"} if args.conventional else {}),
                       "l2": "flushed (512 MiB write) between timed steps, outside the timed events",
                       "graph": "whole step captured as one CUDA graph",
                       "parallelism": f"replicas x{world}, one timestep per rank, no collective"},
            "plain_how": None if plain is None else plain["how"],
            "e2e_how": None if e2e is None else e2e["how"],
            "kernels": table,
            "optimizer": adam,
            "counts": {k2: int(v) for k2, v in counts.items()},
            "visibility_sweep_s": round(sweep_s, 3),
            "workspace_gb": round(r.ws.nbytes / 1e9, 3),
            "launch_shapes": launch_shapes(),
        }
        print(json.dumps(line), flush=True)


def run_train(args, rank, world, local):
    """Optimisation steps of the training configuration: the 2 km corridor
    (16M static Gaussians, 120 instances, SH3) seen by the 7-camera rig,
    each step one timestep (cycling over the sequence) through
    train.Trainer.step: the batched forward, the L1 loss against a synthetic
    target, the backward (overwrite mode) to every parameter and to the
    timestep's poses, and fused Adam on both (gated on the device status, no
    per-step host synchronisation). The visibility record is the first
    epoch's (Eq. 5 over every timestep, then Eq. 6). Reports views/s of whole
    steps, the Adam share, and the peak device memory."""
    import torch
    from paper_2503_08217_gb300 import binding, build, train
    from paper_2503_08217_gb300.render import DeviceScene, pixel_count

    build.build()
    binding.load()
    torch.cuda.set_device(local)
    dev_name = f"cuda:{local}"
    torch.cuda.reset_peak_memory_stats(dev_name)
    scene, lod, desc = make_workload("train", args.seed)
    n, K = scene.n, scene.n_inst
    dev = DeviceScene.from_host(scene, dev_name)
    f = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(dev_name)   # noqa: E731
    vis = torch.empty((n, 2), device=dev_name)
    life = torch.empty((n, 2), device=dev_name)
    binding.update_visibility(n, 0.0, None, life, vis, binding.VIS_RESET)
    state = train.TrainState.initial(dev, f(scene.inst_quat), f(scene.inst_trans), vis, life,
                                     {"mode": "threshold", "r": lod})
    max_splats = max(4096, int(n * 3))
    tr = train.Trainer(state, scene.cams, scene.times, lr=1e-4, pose_lr=1e-5, max_splats=max_splats,
                       max_duplicates=min(2**31 - 1, 6 * max_splats))
    # first epoch: Eq. 5 over every timestep with every window open, then Eq. 6
    all_vis = vis.clone()
    cs = dev.c_scene()
    for kk in range(scene.n_steps):
        tr.renderer.ws.project(cs, binding.make_poses(state.inst_quat[kk], state.inst_trans[kk]),
                               scene.cams[kk], float(scene.times[kk]), all_vis, life, lod)
    binding.update_visibility(n, 0.0, None, life, vis, binding.VIS_FINALIZE)
    del all_vis
    torch.cuda.synchronize()
    tr.renderer.counts()
    P = pixel_count(scene.cams[0])
    gen = torch.Generator(device=dev_name)
    gen.manual_seed(99)
    targets = [torch.rand(3 * P, device=dev_name, generator=gen) for _ in range(4)]
    order = [(i * 37) % scene.n_steps for i in range(args.warmup + args.steps)]
    for i in range(args.warmup):
        tr.step(order[i], targets[i % 4], check=False)
    tr.check()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clocks:
        e0.record()
        for i in range(args.warmup, args.warmup + args.steps):
            tr.step(order[i], targets[i % 4], check=False)
        e1.record()
        torch.cuda.synchronize()
    tr.check()                                    # raises if any step latched a failure
    ms = e0.elapsed_time(e1) / args.steps
    # the optimiser's share: the two Adam launches of a step, timed alone
    s_ = tr.state
    k = order[-1]
    g = [tr.grads[nm] for nm in train.PARAM_NAMES]
    ae = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(5)]
    saved = [x.clone() for x in s_.scene.params()]
    for j in range(5):
        ae[j][0].record()
        binding.adam_step(s_.scene.params(), g, s_.exp_avg, s_.exp_avg_sq, 1e-12, s_.adam_steps + 1)
        ae[j][1].record()
    torch.cuda.synchronize()
    for x, y in zip(s_.scene.params(), saved):
        x.copy_(y)
    del saved
    adam_ms = float(np.mean([a.elapsed_time(b) for a, b in ae]))
    n_par = sum(x.numel() for x in s_.scene.params())
    peak = torch.cuda.max_memory_allocated(dev_name) + tr.renderer.ws.nbytes
    views = len(scene.cams[0])
    if rank == 0:
        print(json.dumps({
            "metric": "training steps (fwd+bwd+Adam) views/s, peak HBM", "value": round(views / (ms / 1e3), 3),
            "unit": "views/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(ms, 4), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"train: {desc}", "gaussians": n, "instances": K, "cameras": views,
                       "pixels_per_view_batch": P, "timesteps": scene.n_steps, "lod_px": lod,
                       "step": "train.Trainer.step: forward, L1, backward (overwrite), Adam on the "
                               "Gaussians and on the timestep's poses; timesteps cycled; no host sync",
                       "l2": "not flushed: the step's inputs (2.2 GB of parameters, moments and "
                             "gradients) exceed L2"},
            "adam": {"ms": round(adam_ms, 4), "share": round(adam_ms / ms, 3), "parameters": int(n_par),
                     "gbs": round(28 * n_par / (adam_ms / 1e3) / 1e9, 1)},
            "peak_hbm_gb": round(peak / 1e9, 3),
            "peak_hbm_how": "torch.cuda.max_memory_allocated (scene, gradients, moments, record, targets) "
                            "+ s3r_workspace_bytes",
            "clocks": clocks.summary(),
        }), flush=True)


def run_ode(args):
    """NeuralODE object poses (Sec. 3.2, Eqs. 3-4) at the training
    configuration's size: 120 instances, 400 output times, embedding width 8,
    two RK4 substeps per interval (798 steps per instance). One step = the
    forward (states, quaternions, translations at every output time) and the
    reverse mode from synthetic pose adjoints, graph-captured; the forward is
    also timed alone. The FP32 operation count is the three matrix products
    of f per stage (FMA = 2 operations) times four stages per step; the
    reverse mode recomputes each step's stages and back-propagates through
    them (about three times the forward's products). One warp per instance
    walks its steps in sequence, so the work is latency-bound, not ALU-bound."""
    import torch
    from paper_2503_08217_gb300 import binding, build, scenegen
    build.build()
    binding.load()
    torch.cuda.set_device(0)
    K, D, T, S, H = 120, 8, 400, 2, 64
    params, embed, z0 = scenegen.ode_model(args.seed, K, D)
    cu = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()   # noqa: E731
    params, embed, z0 = cu(params), cu(embed), cu(z0)
    times = torch.linspace(-1.0, 1.0, T, device="cuda")
    gen = torch.Generator(device="cuda")
    gen.manual_seed(3)
    gq = torch.randn((T, K, 4), device="cuda", generator=gen)
    gt = torch.randn((T, K, 3), device="cuda", generator=gen)
    g_p = torch.zeros_like(params)
    g_e = torch.zeros_like(embed)
    g_z = torch.zeros_like(z0)
    out = {}

    def fwd():
        out["s"] = binding.ode_poses(params, embed, z0, times, S)

    def both():
        fwd()
        binding.ode_poses_bwd(params, embed, times, S, out["s"][0], gq, gt, g_p, g_e, g_z)

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            fn()
        for _ in range(args.warmup):
            g.replay()
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        for a_, b_ in ev:
            a_.record()
            g.replay()
            b_.record()
        torch.cuda.synchronize()
        return float(np.mean([a_.elapsed_time(b_) for a_, b_ in ev]))

    ms_fwd = timed(fwd)
    ms_both = timed(both)
    steps = (T - 1) * S
    f_ops = 2 * (H * (7 + D) + H * H + 6 * H)          # FP32 operations of one evaluation of f
    fwd_ops = K * steps * 4 * f_ops
    ops = 4 * fwd_ops                                    # forward + reverse (recompute + adjoint)
    peak = torch.cuda.get_device_properties(0).multi_processor_count * 128 * measured_peaks()[2] * 1e6
    print(json.dumps({
        "metric": "NeuralODE poses fwd+bwd ms (Eqs. 3-4)", "value": round(ms_both, 4), "unit": "ms",
        "higher_is_better": False, "steps": args.steps, "warmup": args.warmup, "dtype": "f32",
        "data": "synthetic", "forward_ms": round(ms_fwd, 4),
        "config": {"workload": "ode: " + WORKLOADS["ode"][3], "instances": K, "output_times": T,
                   "substeps": S, "rk4_steps_per_instance": steps, "hidden": H, "embed_dim": D},
        "roofline": {"bound": "latency (one warp per instance, sequential steps)",
                     "achieved_gops": round(ops / (ms_both / 1e3) / 1e9, 1),
                     "alu_peak_gops": round(peak / 1e9, 1),
                     "frac": round(ops / (ms_both / 1e3) / peak, 4)},
    }), flush=True)


def cpu_oracle_sample(scene, k, lod, vis_np):
    """The FP64 oracle, as it stands, on a bounded sample of the same
    workload: one camera (the smallest of the rig) at the same timestep over
    the full scene, forward (tiled blend) and backward."""
    import oracle
    cams = scene.cams[k]
    cam = min(cams, key=lambda c: c.width * c.height)
    t0 = time.time()
    f = oracle.step_forward(scene, k, vis_np, None, lod, cams=[cam], tiled=True)
    rng = np.random.default_rng(0)
    dL = [rng.standard_normal((3, cam.height, cam.width))]
    oracle.step_backward(scene, k, f, dL, lod, cams=[cam])
    dt = time.time() - t0
    return {"value": round(1.0 / dt, 5), "unit": "views/s", "cores": oracle.num_threads(),
            "kind": "oracle",
            "sample": f"1 view ({cam.width}x{cam.height}) of the same workload and timestep, fwd+bwd, "
                      f"full scene; {dt:.1f} s"}


def run_reference(args, rank, world, local):
    """The FP64 CPU oracle on this host's cores, each step a bounded sample
    of the workload (one camera, same timestep, full scene)."""
    if rank != 0:
        return
    import oracle
    oracle.build()
    scene, lod, desc = make_workload(args.workload, args.seed)
    k = step_index(scene, 0)
    vis, _ = oracle.vis_reset(scene.n)
    cams = scene.cams[k]
    cam = min(cams, key=lambda c: c.width * c.height)
    rng = np.random.default_rng(0)
    dL = [rng.standard_normal((3, cam.height, cam.width))]

    def one():
        f = oracle.step_forward(scene, k, vis, None, lod, cams=[cam], tiled=True)
        oracle.step_backward(scene, k, f, dL, lod, cams=[cam])

    budget = 150.0
    t_first = time.time()
    one()
    per = time.time() - t_first
    steps = max(1, min(args.steps, int(budget / max(per, 1e-3))))
    warm = min(args.warmup, max(0, int(30.0 / max(per, 1e-3))))
    for _ in range(warm):
        one()
    t0 = time.time()
    for _ in range(steps):
        one()
    dt = (time.time() - t0) / steps
    v = 1.0 / dt
    sample = (f"1 view ({cam.width}x{cam.height}) of the {args.workload} workload at timestep {k}, "
              f"full scene, fwd (tiled blend) + bwd per step; {steps} timed steps")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": round(v, 5), "unit": "views/s", "n_gpus": world,
        "steps": steps, "warmup": warm, "ms_per_step": round(dt * 1e3, 1), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"{args.workload}: {desc}", "timestep": k},
        "cpu_baseline": {"value": round(v, 5), "unit": "views/s", "cores": oracle.num_threads(),
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": round(v, 5), "unit": "views/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def _sweep_prepare(scene, lod_sweep):
    """Device scene, renderer and the first-epoch record of a sweep scene:
    Eq. 5 over every timestep with every window open (at the LOD threshold
    `lod_sweep`; M_t is taken before LOD, so the record does not depend on
    it), then Eq. 6. Returns (dev, c_scene, renderer, vis, all_vis)."""
    import torch
    from paper_2503_08217_gb300 import binding
    from paper_2503_08217_gb300.render import DeviceScene, Renderer
    n = scene.n
    k = scene.n_steps // 2
    dev = DeviceScene.from_host(scene)
    cs = dev.c_scene()
    max_splats = max(4096, n)
    r = Renderer(n, scene.n_inst, scene.cams[k], max_splats=max_splats,
                 max_duplicates=min(2**31 - 1, 6 * max_splats))
    vis = torch.empty((n, 2), device="cuda")
    life = torch.empty((n, 2), device="cuda")
    binding.update_visibility(n, 0.0, None, life, vis, binding.VIS_RESET)
    all_vis = vis.clone()
    for kk in range(scene.n_steps):
        iq = torch.from_numpy(scene.inst_quat[kk]).cuda()
        it = torch.from_numpy(scene.inst_trans[kk]).cuda()
        r.ws.project(cs, binding.make_poses(iq, it), scene.cams[kk], float(scene.times[kk]), all_vis,
                     life, lod_sweep)
    binding.update_visibility(n, 0.0, None, life, vis, binding.VIS_FINALIZE)
    torch.cuda.synchronize()
    r.counts()
    return dev, cs, r, vis, all_vis


def _sweep_time(args, scene, dev, cs, r, v, lod, flush):
    """Graph-captured forward + L1 + backward (overwrite) of the middle
    timestep's cameras with record `v` at LOD threshold `lod`: mean ms per
    step over args.steps replays (L2 flushed between them) and the counts."""
    import torch
    from paper_2503_08217_gb300 import binding
    from paper_2503_08217_gb300.render import pixel_count
    k = scene.n_steps // 2
    cams = scene.cams[k]
    P = pixel_count(cams)
    iq = torch.from_numpy(scene.inst_quat[k]).cuda()
    it = torch.from_numpy(scene.inst_trans[k]).cuda()
    t = float(scene.times[k])
    gen = torch.Generator(device="cuda")
    gen.manual_seed(7)
    target = torch.rand(3 * P, device="cuda", generator=gen)
    out = torch.empty(3 * P, device="cuda")
    dL = torch.empty(3 * P, device="cuda")
    loss = torch.zeros(1, device="cuda")
    bg = torch.zeros(3, device="cuda")
    grads = {"means": torch.empty_like(dev.means), "log_scales": torch.empty_like(dev.log_scales),
             "quats": torch.empty_like(dev.quats), "opacity_logits": torch.empty_like(dev.opacity_logits),
             "sh": torch.empty_like(dev.sh), "inst_quat": torch.empty_like(iq),
             "inst_trans": torch.empty_like(it)}

    def step():
        r.forward(dev, iq, it, cams, t, v, None, lod, bg, out=out, c_scene=cs)
        binding.l1_loss(out, target, dL, loss)
        r.backward(dev, iq, it, bg, dL, grads, c_scene=cs, overwrite=True)
    step()
    torch.cuda.synchronize()
    c = r.counts()
    graph = r.capture(step)
    for _ in range(args.warmup):
        graph.replay()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    for i in range(args.steps):
        flush.fill_(float(i))
        ev[i][0].record()
        graph.replay()
        ev[i][1].record()
    torch.cuda.synchronize()
    r.sync_status()
    ms = float(np.mean([a.elapsed_time(b) for a, b in ev]))
    del graph
    return ms, c


def run_scale_sweep(args):
    """Per-view forward + backward time as the scene grows (the corridor of
    the 'large' workload stretched at constant density: Gaussians, instances,
    length and timesteps scale together; one 1920x1280 camera at the middle
    timestep, LOD 1 px). 'temporal' selects with the visibility windows after a
    first-epoch sweep (Eq. 5, then Eq. 6); 'all_visible' gives every Gaussian
    the window [-1, 1], so every one is compacted and projected."""
    import torch
    from paper_2503_08217_gb300 import binding, build, scenegen
    build.build()
    binding.load()
    torch.cuda.set_device(0)
    rows = []
    flush = torch.empty(512 * 1024 * 1024 // 4, device="cuda")
    for f in [float(x) for x in args.sweep_scales.split(",")]:
        scene = scenegen.generate("large", seed=args.seed, length_scale=f)
        lod = 1.0
        n = scene.n
        dev, cs, r, vis, all_vis = _sweep_prepare(scene, lod)
        cams = scene.cams[scene.n_steps // 2]
        row = {"length_scale": f, "gaussians": n, "instances": scene.n_inst, "timesteps": scene.n_steps,
               "corridor_m": round(float(scene.means[:, 2].max() - scene.means[:, 2].min()), 1)}
        for mode, v in (("temporal", vis), ("all_visible", all_vis)):
            ms, c = _sweep_time(args, scene, dev, cs, r, v, lod, flush)
            row[mode] = {"ms_per_view": round(ms / len(cams), 3), "selected": int(c["n_selected"]),
                         "splats": int(c["n_splats"])}
        rows.append(row)
        del r, dev, vis, all_vis
        torch.cuda.empty_cache()
    print(json.dumps({"sweep": "scale", "metric": "fwd+bwd ms per view vs scene scale",
                      "unit": "ms", "higher_is_better": False, "steps": args.steps, "warmup": args.warmup,
                      "data": "synthetic", "rows": rows}), flush=True)


def run_lod_sweep(args):
    """Per-view forward + backward time against the adaptive-LOD threshold
    (Sec. 3.3): the large corridor (8M static + 80 instances, SH3), one
    1920x1280 camera at the middle timestep, temporal selection after a
    first-epoch sweep, r in --sweep-lods (pixels of the projected 2D scale
    below which a Gaussian is culled; r = 0 culls nothing)."""
    import torch
    from paper_2503_08217_gb300 import binding, build, scenegen
    build.build()
    binding.load()
    torch.cuda.set_device(0)
    flush = torch.empty(512 * 1024 * 1024 // 4, device="cuda")
    scene = scenegen.generate("large", seed=args.seed)
    dev, cs, r, vis, _ = _sweep_prepare(scene, 0.0)
    rows = []
    for lod in [float(x) for x in args.sweep_lods.split(",")]:
        ms, c = _sweep_time(args, scene, dev, cs, r, vis, lod, flush)
        rows.append({"lod_px": lod, "ms_per_view": round(ms, 3), "views_per_s": round(1e3 / ms, 1),
                     "selected": int(c["n_selected"]), "splats": int(c["n_splats"]),
                     "pairs": int(c["n_duplicates"])})
    print(json.dumps({"sweep": "lod", "metric": "fwd+bwd ms per view vs LOD threshold",
                      "unit": "ms", "higher_is_better": False, "steps": args.steps, "warmup": args.warmup,
                      "data": "synthetic", "gaussians": scene.n, "timestep": scene.n_steps // 2,
                      "camera": "1920x1280, f 960", "rows": rows}), flush=True)


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.sweep is not None:
        if rank == 0:
            (run_scale_sweep if args.sweep == "scale" else run_lod_sweep)(args)
        return
    if args.impl == "reference":
        run_reference(args, rank, world, local)
        return
    if args.workload == "train":
        run_train(args, rank, world, local)
        return
    if args.workload == "ode":
        if rank == 0:
            run_ode(args)
        return
    if world > 1:
        import torch
        torch.cuda.set_device(local)
        torch.distributed.init_process_group("nccl")
    try:
        run_ours(args, rank, world, local)
    finally:
        if world > 1:
            import torch
            torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
