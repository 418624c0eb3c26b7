"""Benchmark of the DTSDF render + ICP hot path on the Kinect-shaped workload.

Workload (synthetic, seeded; stands in for the paper's 640x480 indoor RGB-D sequences):
4 x 4 x 3 m room of boxes, cylinders and 3 mm sheets with Perlin colour, 5 mm voxels,
2 cm truncation, colour fused, 300 frames at 640x480 (fx = fy = 525, depth noise
0.0012 z^2 m). The map is built from all 300 frames before timing. One step = one
tracking frame through the whole hot path:
  render depth + normals + colour at the previous estimated pose (640x480),
  current-frame preprocessing and 3-level pyramid,
  coarse-to-fine SE(3) point-to-plane ICP (4 / 5 / 10 iterations) with the
  frame-to-keyframe photometric term (keyframe every 10 frames),
  fusion of the frame (allocation + voxel-projection fusion) at the estimated pose.
Every pose stays on the device; nothing synchronises with the host inside a step.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "render+ICP frames/s @640x480, % HBM roofline; p50/p99 serve latency"
WORKLOAD = ("kinect-shaped FP32: 4x4x3 m synthetic room, 5 mm voxels, tau 2 cm, 6 directions, RGB; 300-frame "
            "map; per frame render 640x480 depth+normal+colour, 3-level SE(3) ICP 4/5/10 it + f2kf photometric, "
            "fusion")
WORKLOAD_FP16 = WORKLOAD.replace("kinect-shaped FP32", "kinect-shaped FP16 storage (half sdf, half weight, u8 colour)")
WORKLOAD_MS = ("multi-sensor Sim(3): map of the 4x4x3 m room from 300 sensor-A frames (640x480, f 525, 5 mm voxels); "
               "per step {n} sensor-B frames 1280x720 (f 910, depth x s, s in U[0.9, 1.1]) with priors perturbed "
               "5 deg / 10 cm: preprocessing + pyramid, one batched render at the priors, one batched Sim(3) ICP "
               "(3 levels x 20 iterations), the step captured in a CUDA graph")
FALLBACK_HBM_GBS = 6800.0

# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one render of the default
# workload (FP32 storage with colour, a render of the timed steps): the march (k_render) and the
# crossing refinement (k_refine), from one ncu capture of
# ``bench.py --steps 2 --warmup 3 --no-e2e --no-cpu --no-serve --no-multi``
# (profiles/k_render_kinect640.md). It belongs to the kernel sources it was taken with: reported
# only while their hash matches.
RENDER_TRAFFIC = {"bytes": 232585984 + 5292032 + 199535104 + 6413568, "sources_sha1_16": "f6187b94391ff767",
                  "files": ("render.cu", "common.cuh", "internal.h")}


def render_traffic():
    """Measured DRAM bytes per render launch, or None once the kernel sources have changed."""
    import hashlib
    h = hashlib.sha1()
    for f in RENDER_TRAFFIC["files"]:
        with open(os.path.join(ROOT, "paper_2301_12796_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return RENDER_TRAFFIC["bytes"] if h.hexdigest()[:16] == RENDER_TRAFFIC["sources_sha1_16"] else None


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--frames", type=int, default=300)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-serve", action="store_true", help="tracking: skip the serving block")
    ap.add_argument("--no-multi", action="store_true", help="tracking: skip the multi-sensor Sim(3) block")
    ap.add_argument("--profile", action="store_true", help="small run for ncu: map of 60 frames, few steps")
    ap.add_argument("--workload", default="tracking", choices=["tracking", "multi_sensor", "serve"],
                    help="tracking: Kinect-shaped tracking frames (default); multi_sensor: batched Sim(3) "
                         "registration of 1280x720 second-sensor frames against the 640x480 map; serve: "
                         "a Poisson stream of render + registration requests of mixed sizes served by the "
                         "continuous-batching server over FP16 maps, against serial FP32 solves")
    ap.add_argument("--render-mode", default="direct", choices=["direct", "combined", "freespace"],
                    help="tracking: direct ray-cast of the six directions (default) or the ray-cast of the "
                         "view-dependent combined TSDF with conditional combination")
    ap.add_argument("--storage", default="fp32", choices=["fp32", "fp16"],
                    help="map storage: FP32 sdf/weight/colour, or FP16 sdf + half weight + u8 colour")
    ap.add_argument("--solver", default="gn", choices=["gn", "lm"],
                    help="tracking: Gauss-Newton or Levenberg-Marquardt (Madsen damping) per level")
    ap.add_argument("--photo", default="f2kf", choices=["f2kf", "f2f"],
                    help="tracking: photometric term against a keyframe every 10 frames, or the previous frame")
    ap.add_argument("--problems", type=int, default=64, help="multi_sensor: registration problems per step")
    ap.add_argument("--requests", type=int, default=512, help="serve: requests in the arrival stream")
    ap.add_argument("--rate", type=float, default=2000.0, help="serve: Poisson arrival rate, requests/s")
    ap.add_argument("--maps", type=int, default=3, help="serve: device-resident maps (seeded rooms)")
    ap.add_argument("--map-frames", type=int, default=100, help="serve: frames fused into each map")
    return ap.parse_args()


# ------------------------------------------------------------------ clocks ---
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = os.environ.get("DTSDF_CLOCKS_CSV") or os.path.join(tempfile.gettempdir(),
                                                                        f"dtsdf_clocks_{os.getpid()}.csv")

    def start(self):
        """Start sampling and return once the first sample is written: nvidia-smi's start-up
        (NVML initialisation, some hundred milliseconds) stays out of the timed region."""
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
            return
        deadline = time.time() + 10.0
        while time.time() < deadline and self.proc.poll() is None:
            if os.path.getsize(self.path) > 0:
                break
            time.sleep(0.02)

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            for n, v in zip(names[1:], p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": float(max(smax)) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_hbm_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "of measured"
    except Exception:
        return FALLBACK_HBM_GBS, "of fallback"


# ------------------------------------------------------------ replicas ---
def max_over_ranks(ms: float, tdist, world: int, dev) -> float:
    """The slowest rank's time: every rank runs its own replica of the workload (the path has
    no exchange step), and the job's time is the maximum over ranks."""
    if world <= 1:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=dev)
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world: int, units_per_rank: float, total_ms: float) -> float:
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return world * units_per_rank / (total_ms / 1000.0)


# ---------------------------------------------------------------- workload ---
def make_workload(n_frames: int):
    import scenes
    s = scenes.kinect_room(1, n_frames=n_frames)
    frames = [s.frame(i) for i in range(s.n_frames)]
    return s, frames


def opts_kinect(dt, solver="gn"):
    return dt.icp_opts(levels=3, iters=(10, 5, 4), eps=(0.005, 0.05, 0.05), photo_thr=(0.05, 0.175, 0.175),
                       lam=0.1, z_min=0.1, stop_norm=1e-6, min_rows=10, lm=solver == "lm")


# kernels per call of the tracking step (counted from the ncu launch list of a step): render =
# depth-range pass + march + refinement; set_frame = outlier filter, normals, depth extraction,
# intensity, two pyramid levels, three intensity normalisations
LAUNCHES = {"render": 3, "set_frame": 9, "set_keyframe": 6, "compose": 1, "solve": 19, "integrate": 9}


class Tracker:
    """Device-resident tracking loop over the frames (map, ICP context, buffers, poses)."""

    def __init__(self, dt, torch, s, frames, dev, map_frames, storage=0, combined=False, max_blocks=1 << 19,
                 solver="gn", photo="f2kf", freespace=False):
        self.dt, self.torch, self.s, self.dev = dt, torch, s, dev
        self.combined = combined
        self.freespace = freespace  # the free-space combination render of Alg. 1 (quality reference)
        self.photo = photo  # "f2kf": keyframe every 10 frames; "f2f": the previous frame, T_rs = I
        K = s.K
        self.K = K
        self.map = dt.Map(dt.params(voxel_size=0.005, truncation=0.02, max_blocks=max_blocks, z_max=s.z_max, color=True,
                                    storage=storage))
        self.icp = dt.Icp(K.width, K.height, 3)
        self.opts = opts_kinect(dt, solver)
        H, W = K.height, K.width
        self.depth = [torch.from_numpy(f.depth).to(dev) for f in frames]
        self.rgb = [torch.from_numpy(f.rgb).to(dev) for f in frames]
        self.gt = torch.from_numpy(np.stack([f.pose for f in frames])).to(dev)
        self.est = self.gt.clone()
        self.ref_d = torch.zeros(H, W, device=dev)
        self.ref_n = torch.zeros(H, W, 4, device=dev)
        self.ref_c = torch.zeros(H, W, 4, device=dev)
        self.dT = torch.eye(4, dtype=torch.float64, device=dev)
        self.eye = torch.eye(4, dtype=torch.float64, device=dev)
        self.T_rs = torch.eye(4, dtype=torch.float64, device=dev)
        self.kf = -1
        self.launches = 0
        for i in map_frames:
            self.map.integrate(self.depth[i], self.rgb[i], K, frames[i].pose)
        torch.cuda.synchronize()
        self.n = len(frames)

    def step(self, i, ev=None):
        """Track frame f = 1 + i mod (n - 1). ev: optional list of 4 events (render, icp, fuse phases)."""
        dt, K = self.dt, self.K
        f = 1 + i % (self.n - 1)
        if f == 1:
            self.est[0].copy_(self.gt[0])
        ref = self.est[f - 1]
        if ev:
            ev[0].record()
        if self.freespace:
            self.map.render_freespace_dev(K, ref, self.ref_d, self.ref_n)
        elif self.combined:
            self.map.render_combined_dev(K, ref, self.ref_d, self.ref_n, self.ref_c)
        else:
            self.map.render_dev(K, ref, self.ref_d, self.ref_n, self.ref_c)
        if ev:
            ev[1].record()
        self.icp.set_frame(self.depth[f], self.rgb[f], K, 0.1, self.s.z_max, 0.01)
        kf = f - 1 if self.photo == "f2f" else 10 * ((f - 1) // 10)
        n = (1 if self.freespace else LAUNCHES["render"] + (2 if self.combined else 0)) + LAUNCHES["set_frame"]
        if kf != self.kf:
            self.icp.set_keyframe(self.rgb[kf], K)
            self.kf = kf
            n += LAUNCHES["set_keyframe"]
        if self.photo == "f2f":
            T_rs = self.eye  # the render camera is the previous frame's camera
            n -= LAUNCHES["compose"]
        else:
            dt.pose_compose(self.est[kf], ref, self.T_rs, invert_a=True)
            T_rs = self.T_rs
        self.dT.copy_(self.eye)
        self.icp.solve(self.ref_d, self.ref_n, K, self.dT, self.opts, T_rs_dev=T_rs)
        dt.pose_compose(ref, self.dT, self.est[f])
        if ev:
            ev[2].record()
        self.map.integrate_dev(self.depth[f], self.rgb[f], K, self.est[f])
        if ev:
            ev[3].record()
        self.launches += n + 2 * LAUNCHES["compose"] + LAUNCHES["solve"] + LAUNCHES["integrate"]


def flush_l2(buf):
    buf.add_(1.0)


# --------------------------------------------------------------- cpu side ---
class OracleFrame:
    """The FP64 oracle on whole tracking frames of the workload: the CPU baseline of the tracking
    line and every step of the reference arm. Its map is fused from the workload's frames (setup,
    untimed); one frame is then, as on the device: the render of every pixel at the previous
    frame's pose (the oracle's own render, which is the registration's reference), the whole
    coarse-to-fine schedule (3 levels, 4/5/10 Gauss-Newton iterations, point-to-plane plus
    frame-to-keyframe photometric rows, keyframe every 10 frames) and the fusion of the frame
    at the pose found. threads sets the OpenMP threads of the C oracle (render, fusion); the
    numpy schedule runs with numpy's own threading."""

    def __init__(self, s, frames, map_frames):
        import oracle
        from oracle import icp as oicp
        self.oracle, self.oicp = oracle, oicp
        self.s, self.frames = s, frames
        oracle.threads(cpu_cores())
        t0 = time.perf_counter()
        P = oracle.Params(voxel_size=0.005, truncation=0.02, z_max=s.z_max, color=True)
        self.om = oracle.OracleMap(P)
        self.map_frames = list(map_frames)
        for i in self.map_frames:
            self.om.integrate(frames[i].depth, frames[i].rgb, s.K, frames[i].pose)
        self.setup_s = time.perf_counter() - t0

    def frame(self, f: int, threads: int):
        """Seconds for whole frame f on `threads` OpenMP threads, and the parts."""
        oracle, oicp, s, frames = self.oracle, self.oicp, self.s, self.frames
        K = s.K
        used = oracle.threads(threads)
        T_ref = frames[f - 1].pose
        kf = 10 * ((f - 1) // 10)
        T_rs = np.linalg.inv(frames[kf].pose) @ T_ref
        t0 = time.perf_counter()
        d, n, _, _ = self.om.render(K, T_ref)
        t1 = time.perf_counter()
        rn = np.zeros(n.shape[:2] + (4,), np.float32)
        rn[..., :3] = n
        rn[..., 3] = d
        pre = oracle.preprocess(frames[f].depth, K, 0.1, s.z_max, 0.01)
        levels = oicp.pyramid(pre["z"], K, 3, frames[f].rgb)
        kI = oicp.pyramid(pre["z"], K, 3, frames[kf].rgb)
        photo = [(kI[l].I, K.scaled(l), T_rs) for l in range(3)]
        st = oicp.Settings(eps=(0.005, 0.05, 0.05), iters=(10, 5, 4), photo_thr=(0.05, 0.175, 0.175), lam=0.1)
        dT, log = oicp.track(levels, d.astype(np.float32), rn, K, np.eye(4), st, photo)
        t2 = time.perf_counter()
        self.om.integrate(frames[f].depth, frames[f].rgb, K, T_ref @ dT)
        t3 = time.perf_counter()
        return t3 - t0, dict(render_s=t1 - t0, icp_s=t2 - t1, fuse_s=t3 - t2, iterations=len(log), threads=used)

    def counts(self, f: int) -> dict:
        """The oracle's count of what the render of frame f reads (all threads)."""
        self.oracle.threads(cpu_cores())
        return self.om.render_count(self.s.K, self.frames[f - 1].pose)

    def describe(self, parts, single=None) -> str:
        out = (f"oracle map fused from {len(self.map_frames)} frames of the workload (setup, {self.setup_s:.0f} s); "
               f"one whole 640x480 frame on {parts['threads']} threads: render of every pixel "
               f"({parts['render_s']:.2f} s), the full f2kf schedule of {parts['iterations']} iterations against "
               f"that render ({parts['icp_s']:.2f} s, numpy), fusion of the frame ({parts['fuse_s']:.2f} s)")
        if single is not None:
            out += (f"; single-threaded: {single['render_s']:.1f} + {single['icp_s']:.1f} + "
                    f"{single['fuse_s']:.1f} s")
        return out


def cpu_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def cpu_model() -> str:
    """The host CPU as /proc/cpuinfo names it (model name, or the Arm implementer / part), else the
    machine type."""
    import platform
    try:
        info = open("/proc/cpuinfo").read().splitlines()
        for key in ("model name", "Model", "CPU part"):
            for line in info:
                if line.split(":")[0].strip() == key:
                    val = line.split(":", 1)[1].strip()
                    return f"{platform.machine()} {key}: {val}"
    except OSError:
        pass
    return platform.machine()


# ---------------------------------------------------------------- reference --
def run_reference(args, rank, world):
    """The oracle as it stands, on the host cores, one whole tracking frame of the workload per
    step (after fusing the map from the workload's frames)."""
    if rank != 0:
        return
    s, frames = make_workload(args.frames)
    ob = OracleFrame(s, frames, range(0, len(frames), 2))
    secs, parts = [], None
    for i in range(args.warmup + args.steps):
        f = 1 + i % (len(frames) - 1)
        dt_s, parts = ob.frame(f, cpu_cores())
        if i >= args.warmup:
            secs.append(dt_s)
    value = len(secs) / float(np.sum(secs))
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 / value, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD},
           "cpu_baseline": {"value": value, "unit": "frames/s", "cores": parts["threads"], "cpu": cpu_model(),
                            "kind": "oracle", "sample": ob.describe(parts)},
           "e2e": {"value": value, "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# --------------------------------------------------------------- tracking --
def voxel_bytes(storage: int) -> tuple[int, int]:
    """Bytes per voxel of a geometry brick and of a colour brick."""
    return (4, 4) if storage == 1 else (8, 16)


def march_bytes(ob, tr, s, frames, args, storage):
    """Algorithmic bytes of one render of the timed loop: the distinct bricks the march reads x
    512 x (8 B FP32 sdf + weight | 4 B FP16 + u16), the distinct allocated block cells whose
    hash entry it reads x 16 B, the colour voxels that enter the outputs x (12 B FP32 RGB |
    3 B u8), and the outputs W H x (4 B depth + 12 B normal + 3 B RGB). The counts are the
    FP64 oracle's (its instrumented render of its own map at the same poses); without the
    oracle (--no-cpu), the device's instrumented march counts the bricks instead."""
    npix = s.K.width * s.K.height
    b_geom, b_col = (4, 3) if storage == 1 else (8, 12)
    fr = [1 + (args.warmup + k) % (tr.n - 1) for k in range(min(4, args.steps))]
    if ob is not None:
        c = [ob.counts(f) for f in fr]
        g, p, cv = (float(np.mean([x[k] for x in c])) for k in ("bricks", "cells", "colour_voxels"))
        b = g * 512 * b_geom + p * 16 + cv * b_col + npix * 19
        return b, (f"oracle count at {len(fr)} timed poses: {g:.0f} bricks x 512 x {b_geom} B + {p:.0f} block "
                   f"cells x 16 B + {cv:.0f} colour voxels x {b_col} B + {npix} x 19 B outputs")
    tb = [tr.map.touched(s.K, frames[f - 1].pose) for f in fr]
    g, cb = float(np.mean([x[0] for x in tb])), float(np.mean([x[1] for x in tb]))
    b = g * 512 * b_geom + cb * 512 * b_col + npix * 19
    return b, (f"device count (instrumented march) at {len(fr)} timed poses: {g:.0f} geometry bricks x 512 x "
               f"{b_geom} B + {cb:.0f} colour bricks x 512 x {b_col} B + {npix} x 19 B outputs")


def icp_algorithmic_bytes(K) -> float:
    """Sum over the pyramid levels of iterations x pixels x bytes per pixel-iteration: 4 B current
    depth, 24 B gathered render point and normal, 4 B current intensity and 48 B of keyframe
    taps (4 bilinear taps x intensity and gradient)."""
    total = 0.0
    for l, it in zip(range(3), (10, 5, 4)):
        total += it * (K.width >> l) * (K.height >> l) * (4 + 24 + 4 + 48)
    return total


def run_tracking(args, dt, torch, tdist, dev, rank, world, local):
    storage = 1 if args.storage == "fp16" else 0
    n_frames = 60 if args.profile else args.frames
    s, frames = make_workload(n_frames)
    combined = args.render_mode == "combined"
    # the profiling case keeps the device footprint to a few GB (60-frame map: 121k bricks)
    tr = Tracker(dt, torch, s, frames, dev, range(n_frames), storage, combined,
                 max_blocks=(1 << 17) if args.profile else (1 << 19), solver=args.solver, photo=args.photo,
                 freespace=args.render_mode == "freespace")
    st = tr.map.stats()
    l2 = torch.empty(128 * 1024 * 1024, dtype=torch.float32, device=dev)  # 512 MB > L2
    flush_l2(l2)  # the flush kernel's first launch loads its module (~0.8 s): keep it out of the timed loop
    for i in range(args.warmup):
        tr.step(i)
    torch.cuda.synchronize()
    # autotuner: launch shape of the render (persistent CTAs, refill group, ray tile) at the pose
    # of the first timed frame's reference, chosen before the timed region
    shape_pose = frames[1 + args.warmup % (tr.n - 1) - 1].pose
    render_shape, render_tune_ms = tr.map.tune_render(s.K, shape_pose, tr.ref_d, tr.ref_n, tr.ref_c)
    torch.cuda.synchronize()
    npix = s.K.width * s.K.height
    # event counts of one render (instrumented build of the march: samples, full combinations,
    # block cells entered, allocated cells, hits, cell jumps)
    march = tr.map.touched(s.K, frames[1 + args.warmup % (tr.n - 1) - 1].pose, counters=True)[2]
    # ---------------- timed region
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
    clk = ClockSampler(local)
    clk.start()
    if world > 1:
        tdist.barrier()
    torch.cuda.synchronize()
    tr.launches = 0
    t_wall = time.perf_counter()
    for k in range(args.steps):
        flush_l2(l2)
        tr.step(args.warmup + k, evs[k])
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall
    if world > 1:
        tdist.barrier()
    clocks = clk.stop()
    ph = np.array([[e[0].elapsed_time(e[1]), e[1].elapsed_time(e[2]), e[2].elapsed_time(e[3])] for e in evs])
    step_ms = ph.sum(1)
    total_ms = max_over_ranks(float(step_ms.sum()), tdist, world, dev)
    ms_per_step = total_ms / args.steps
    value = job_throughput(world, args.steps, total_ms)
    launches = tr.launches
    # pose error of the tracked frames against ground truth (sanity, not a parity claim)
    est = tr.est.cpu().numpy()
    gt = tr.gt.cpu().numpy()
    fr = [1 + (args.warmup + k) % (tr.n - 1) for k in range(args.steps)]
    terr = float(np.median([np.linalg.norm(est[f][:3, 3] - gt[f][:3, 3]) for f in fr]))
    # post-fusion error (Sec. 8.2): the map re-rendered at each tracked frame's estimated pose
    # against that frame's input depth, pixel-wise MAE over pixels where both exist (untimed)
    mae = torch.zeros(2, dtype=torch.float64, device=dev)
    acc = np.zeros(2)
    for f in sorted(set(fr)):
        tr.map.render_dev(tr.K, tr.est[f], tr.ref_d, tr.ref_n)
        dt.depth_mae(tr.ref_d, tr.depth[f], out=mae)
        acc += mae.cpu().numpy()
    post_mae_mm = 1e3 * acc[0] / max(acc[1], 1.0)
    # ---------------- e2e through host buffers (pinned), pose read back every step. The inputs of
    # a step are copied on their own stream while the previous step computes; the host reads each
    # step's pose (device -> pinned host) one step later, so the copies overlap the compute and
    # every copy of every step stays inside the timed region.
    e2e = None
    if not args.no_e2e:
        hd = [torch.from_numpy(frames[i].depth).pin_memory() for i in range(min(tr.n, 64))]
        hc = [torch.from_numpy(frames[i].rgb).pin_memory() for i in range(min(tr.n, 64))]
        host_pose = [torch.empty(4, 4, dtype=torch.float64).pin_memory() for _ in range(2)]
        done = [torch.cuda.Event() for _ in range(2)]
        copy_stream = torch.cuda.Stream()
        compute = torch.cuda.current_stream()
        n_e2e = min(args.steps, 60)
        poses = []
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(n_e2e):
            f = 1 + k % (len(hd) - 1)
            with torch.cuda.stream(copy_stream):
                tr.depth[f].copy_(hd[f], non_blocking=True)  # host -> device, inside the timed region
                tr.rgb[f].copy_(hc[f], non_blocking=True)
                arrived = torch.cuda.Event()
                arrived.record(copy_stream)
            compute.wait_event(arrived)
            tr.step(f - 1)
            host_pose[k % 2].copy_(tr.est[f], non_blocking=True)
            done[k % 2].record(compute)
            if k >= 1:
                done[(k - 1) % 2].synchronize()
                poses.append(host_pose[(k - 1) % 2].clone())
        done[(n_e2e - 1) % 2].synchronize()
        poses.append(host_pose[(n_e2e - 1) % 2].clone())
        e2e_s = time.perf_counter() - t0
        assert len(poses) == n_e2e
        e2e = {"value": world * n_e2e / e2e_s, "unit": "frames/s",
               "h2d_bytes_per_step": int(hd[0].numel() * 4 + hc[0].numel()), "d2h_bytes_per_step": 128,
               "steps": n_e2e}
    # ---------------- roofline of the dominant kernel
    render_ms = float(ph[:, 0].mean())
    comb = None
    if combined:
        # the combine pass alone, forced over the padded frustum (L2 flushed before each run)
        pose = tr.est[1 + args.warmup % (tr.n - 1)]
        tr.map.combine_dev(s.K, pose, force=True)
        torch.cuda.synchronize()
        blocks, cbricks = tr.map.combined_blocks()
        ts = []
        for _ in range(5):
            flush_l2(l2)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            tr.map.combine_dev(s.K, pose, force=True)
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        comb_ms = float(np.mean(ts))
        gvb, cvb = voxel_bytes(storage)
        comb_bytes = cbricks * 512 * (gvb + cvb) + blocks * 729 * (8 + 16)
        comb = {"blocks": int(blocks), "bricks": int(cbricks), "full_combine_ms": comb_ms,
                "algorithmic_bytes": float(comb_bytes)}
    peak, peak_kind = measured_hbm_peak()
    # the FP64 oracle on the host: its count of what the renders read (algorithmic bytes) and the
    # CPU baseline (one whole frame on all cores, one single-threaded)
    ob = None
    if rank == 0 and not args.no_cpu and not args.profile:
        ob = OracleFrame(s, frames, range(0, n_frames, 2))
    render_bytes, bytes_def = march_bytes(ob, tr, s, frames, args, storage)
    icp_ms = float(ph[:, 1].mean())
    icp_bytes = icp_algorithmic_bytes(s.K)
    achieved = render_bytes / (render_ms / 1000.0) / 1e9
    if comb is not None:
        a_c = comb["algorithmic_bytes"] / (comb["full_combine_ms"] / 1000.0) / 1e9
        roof = {"kernel": "k_combine (view-dependent combined TSDF, whole padded frustum)", "bound": "hbm",
                "achieved": a_c, "peak": peak, "unit": "GB/s", "frac": a_c / peak, "peak_kind": peak_kind,
                "traffic": None, "algorithmic_bytes_per_launch": comb["algorithmic_bytes"],
                "launch_ms": comb["full_combine_ms"],
                "bytes_definition": "source (block, direction) bricks' core voxels (geometry + colour) read once, "
                                    "729 combined voxels x 24 B written per block"}
    else:
        roof = None
    if roof is None and args.render_mode == "freespace":
        roof = {"kernel": "k_render_freespace (Alg. 1 free-space combination ray-cast)", "bound": "hbm",
                "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak, "peak_kind": peak_kind,
                "traffic": None, "algorithmic_bytes_per_launch": render_bytes, "launch_ms": render_ms,
                "bytes_definition": bytes_def}
    roof = roof or {"kernel": "k_render + k_refine (direct DTSDF ray-cast: the march, then the crossing refinement)",
            "bound": "hbm", "achieved": achieved, "peak": peak,
            "unit": "GB/s", "frac": achieved / peak, "peak_kind": peak_kind,
            "traffic": render_traffic() if storage == 0 and not args.profile else None,
            "algorithmic_bytes_per_launch": render_bytes, "launch_ms": render_ms, "bytes_definition": bytes_def,
            "render_and_icp": {"bytes": render_bytes + icp_bytes, "icp_bytes": icp_bytes, "ms": render_ms + icp_ms,
                               "achieved": (render_bytes + icp_bytes) / ((render_ms + icp_ms) / 1000.0) / 1e9,
                               "frac": (render_bytes + icp_bytes) / ((render_ms + icp_ms) / 1000.0) / 1e9 / peak,
                               "icp_definition": "sum over levels of iterations x pixels x (4 B depth + 24 B gathered "
                                                 "point and normal + 4 B intensity + 48 B keyframe taps), schedule "
                                                 "4/5/10 at 160x120/320x240/640x480"}}
    serve = multi = None
    if not args.profile and not args.no_serve:
        serve = side_block(run_serve(side_args(args, steps=0), dt, torch, tdist, dev, rank, world, local,
                                     emit=False))
    if not args.profile and not args.no_multi:
        multi = side_block(run_multi_sensor(side_args(args, steps=MS_BLOCK_STEPS), dt, torch, tdist, dev, rank,
                                            world, local, emit=False))
    cpu = None
    if ob is not None and world == 1:
        f = 1 + args.warmup % (len(frames) - 1)
        secs, parts = ob.frame(f, cpu_cores())
        secs1, parts1 = ob.frame(f + 1, 1)
        cpu = {"value": 1.0 / secs, "unit": "frames/s", "cores": parts["threads"], "cpu": cpu_model(),
               "kind": "oracle", "single_thread_value": 1.0 / secs1, "sample": ob.describe(parts, parts1)}
    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
               "vs_baseline": None, "dtype": "f32", "data": "synthetic",
               "config": {"workload": WORKLOAD if not storage else WORKLOAD_FP16, "resolution": "640x480",
                          "storage": args.storage, "map_frames": n_frames, "render_mode": args.render_mode,
                          "solver": args.solver, "photometric": args.photo,
                          "combined": comb,
                          "map_bricks": int(st.bricks), "map_voxels_per_direction_M": [round(x * 512 / 1e6, 2)
                                                                                      for x in st.bricks_per_dir],
                          "l2": "flushed between steps (512 MB write outside the timed events)",
                          "parallelism": f"replicas x{world}",
                          "render_shape": {"ctas": render_shape[0], "refill": render_shape[1],
                                           "tile_w": render_shape[2], "tuned_ms": render_tune_ms},
                          "phase_ms": {"render": render_ms, "preprocess_pyramid_icp": float(ph[:, 1].mean()),
                                       "fusion": float(ph[:, 2].mean())},
                          "rays_per_s": world * npix * args.steps / (total_ms / 1000.0),
                          "frame_ms_p50": float(np.percentile(step_ms, 50)),
                          "frame_ms_p99": float(np.percentile(step_ms, 99)),
                          "march_counts_per_frame": march,
                          "wall_s_timed_loop": t_wall, "median_translation_error_m": terr,
                          "post_fusion_mae_mm": post_mae_mm},
               "serve": serve, "multi_sensor": multi, "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
               "clocks": clocks}
        print(json.dumps(out), flush=True)


# ----------------------------------------------------------- multi-sensor --
MS_ITERS = (20, 20, 20)
MS_EPS = (0.01, 0.1, 0.2)
MS_LAUNCHES_PER_FRAME = 5  # outlier filter, normals, depth extraction, 2 pyramid levels; per batch of 64 also
# the depth-range pass, march and refinement of the batched render and one batched registration


class MultiSensor:
    """Batched Sim(3) registration of second-sensor frames against the first sensor's map."""

    def __init__(self, dt, torch, dev, n_problems, n_frames, storage):
        import scenes
        self.dt, self.torch, self.dev = dt, torch, dev
        self.room = room = scenes.kinect_room(1, n_frames=n_frames)
        self.map = dt.Map(dt.params(voxel_size=0.005, truncation=0.02, max_blocks=1 << 19, z_max=room.z_max,
                                    color=False, storage=storage))
        for i in range(n_frames):
            f = room.frame(i)
            self.map.integrate(torch.from_numpy(f.depth).to(dev), None, room.K, f.pose)
        self.probs = scenes.multi_sensor_problems(room, n_problems, seed=1)
        self.K = self.probs[0]["K"]
        H, W = self.K.height, self.K.width
        n = n_problems
        self.depth = [torch.from_numpy(p["depth"]).to(dev) for p in self.probs]
        self.icps = [dt.Icp(W, H, 3) for _ in range(n)]
        self.ref_d = torch.zeros(n, H, W, device=dev)
        self.ref_n = torch.zeros(n, H, W, 4, device=dev)
        self.prior = torch.from_numpy(np.stack([p["prior"] for p in self.probs])).to(dev)
        self.T = torch.zeros(n, 4, 4, dtype=torch.float64, device=dev)
        self.eye = torch.eye(4, dtype=torch.float64, device=dev).expand(n, 4, 4).contiguous()
        self.stats = torch.zeros(n, dt.STATS_BYTES, dtype=torch.uint8, device=dev)
        self.opts = dt.icp_opts(levels=3, iters=MS_ITERS, eps=MS_EPS, stop_norm=1e-6, min_rows=10)
        self.jobs = [(self.K, self.prior[i], self.ref_d[i], self.ref_n[i], None) for i in range(n)]
        self.items = [(self.icps[i], self.ref_n[i], self.K, self.T[i], True, self.stats[i]) for i in range(n)]
        self.shape = None
        self.n = n

    def preprocess(self, stream=None):
        for i in range(self.n):
            self.icps[i].set_frame(self.depth[i], None, self.K, 0.1, 6.0, 0.01, stream=stream)

    def render(self, stream=None):
        self.map.render_batch(self.jobs, stream=stream)

    def register(self, stream=None):
        self.T.copy_(self.eye)
        self.dt.icp_batch(self.items, self.opts, shape=self.shape, stream=stream)

    def step(self, stream=None):
        self.preprocess(stream)
        self.render(stream)
        self.register(stream)

    def errors(self):
        """Rotation (deg), translation (m) and relative scale errors against the true poses."""
        T = self.T.cpu().numpy()
        rot, tr, sc = [], [], []
        for i, p in enumerate(self.probs):
            E = np.linalg.inv(p["prior"]) @ p["T_true"]  # render camera <- true camera, unscaled
            s_est = np.cbrt(np.linalg.det(T[i][:3, :3]))
            R_est = T[i][:3, :3] / s_est
            ang = np.degrees(np.arccos(np.clip((np.trace(R_est.T @ E[:3, :3]) - 1) / 2, -1, 1)))
            rot.append(ang)
            tr.append(np.linalg.norm(T[i][:3, 3] - E[:3, 3]))
            sc.append(abs(s_est * p["scale"] - 1))
        return np.array(rot), np.array(tr), np.array(sc)


def ms_cpu_baseline(ms, n_frames):
    """The oracle on a bounded sample of one registration problem, scaled to the whole batch."""
    import oracle
    from oracle import icp as oicp
    room, p, K = ms.room, ms.probs[0], ms.K
    P = oracle.Params(voxel_size=0.005, truncation=0.02, z_max=room.z_max, color=False)
    om = oracle.OracleMap(P)
    for i in range(0, n_frames, max(1, n_frames // 6)):
        f = room.frame(i)
        om.integrate(f.depth, None, room.K, f.pose)
    stride = 32
    vv, uu = np.mgrid[0:K.height:stride, 0:K.width:stride]
    pix = np.stack([uu.ravel(), vv.ravel()], 1).astype(np.int32)
    t0 = time.perf_counter()
    om.render(K, p["prior"], pix)
    t_render = (time.perf_counter() - t0) * (K.width * K.height) / len(pix)
    ref = room.render(p["prior"], K=K, noise=False, exact=True)
    rn = np.zeros(ref.normals.shape[:2] + (4,), np.float32)
    rn[..., :3] = ref.normals
    pre = oracle.preprocess(p["depth"], K, 0.1, 6.0, 0.01)
    levels = oicp.pyramid(pre["z"], K, 3)
    st = oicp.Settings(sim3=True, eps=MS_EPS, iters=MS_ITERS)
    t_icp = 0.0
    for l in range(3):
        t0 = time.perf_counter()
        oicp.step(levels[l], ref.depth, rn, K, np.eye(4), st.eps[l], st, level_index=l)
        t_icp += (time.perf_counter() - t0) * MS_ITERS[l]
    per_problem = t_render + t_icp
    sample = (f"one problem: oracle render of 1/{stride * stride} of the 1280x720 pixels scaled up "
              f"({t_render:.1f} s), one Sim(3) iteration per level on the full pyramid scaled to 20 per level "
              f"({t_icp:.1f} s); oracle map fused from 1/50 of the sensor-A frames")
    return 1.0 / per_problem, sample


def run_multi_sensor(args, dt, torch, tdist, dev, rank, world, local, emit=True):
    storage = 1 if args.storage == "fp16" else 0
    n_frames = 60 if args.profile else args.frames
    ms = MultiSensor(dt, torch, dev, args.problems, n_frames, storage)
    stream = torch.cuda.current_stream()
    # autotuner: launch shape of the batched registration on these problems
    ms.preprocess()
    ms.render()
    ms.T.copy_(ms.eye)
    shape, tune_ms = dt.icp_batch_tune(ms.items, ms.opts)
    ms.shape = shape
    for _ in range(2):
        ms.step()
    torch.cuda.synchronize()
    # phase times of one eager step (events on the launching stream)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    ph = []
    for _ in range(3):
        ev[0].record()
        ms.preprocess()
        ev[1].record()
        ms.render()
        ev[2].record()
        ms.register()
        ev[3].record()
        torch.cuda.synchronize()
        ph.append([ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2]), ev[2].elapsed_time(ev[3])])
    ph = np.array(ph).mean(0)
    # one step captured in a CUDA graph
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(stream)
    with torch.cuda.stream(side):
        with torch.cuda.graph(g, stream=side):
            ms.step(side)
    stream.wait_stream(side)
    l2 = torch.empty(128 * 1024 * 1024, dtype=torch.float32, device=dev)
    flush_l2(l2)
    for _ in range(args.warmup):
        g.replay()
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clk = ClockSampler(local)
    clk.start()
    if world > 1:
        tdist.barrier()
    torch.cuda.synchronize()
    for k in range(args.steps):
        flush_l2(l2)
        evs[k][0].record()
        g.replay()
        evs[k][1].record()
    torch.cuda.synchronize()
    if world > 1:
        tdist.barrier()
    clocks = clk.stop()
    total_ms = max_over_ranks(float(sum(a.elapsed_time(b) for a, b in evs)), tdist, world, dev)
    n = ms.n
    value = job_throughput(world, n * args.steps, total_ms)
    rot, tr, sc = ms.errors()
    # e2e through host buffers: sensor-B depth frames from pinned memory, poses read back
    e2e = None
    if not args.no_e2e:
        hd = [torch.from_numpy(p["depth"]).pin_memory() for p in ms.probs]
        host_T = torch.empty(n, 4, 4, dtype=torch.float64).pin_memory()
        n_e2e = min(args.steps, 10)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(n_e2e):
            for i in range(n):
                ms.depth[i].copy_(hd[i], non_blocking=True)
            ms.step()
            host_T.copy_(ms.T, non_blocking=True)
            stream.synchronize()
        e2e_s = time.perf_counter() - t0
        e2e = {"value": world * n * n_e2e / e2e_s, "unit": "registrations/s",
               "h2d_bytes_per_step": int(sum(x.numel() * 4 for x in hd)), "d2h_bytes_per_step": n * 128,
               "steps": n_e2e}
    # roofline of the dominant kernel (the batched render): touched bricks of a sample of problems
    gvb, _ = voxel_bytes(storage)
    sample = list(range(0, n, max(1, n // 8)))
    geom = np.mean([ms.map.touched(ms.K, ms.probs[i]["prior"])[0] for i in sample])
    npix = ms.K.width * ms.K.height
    render_bytes = n * (geom * 512 * gvb + npix * (4 + 16))
    peak, peak_kind = measured_hbm_peak()
    achieved = render_bytes / (ph[1] / 1000.0) / 1e9
    # batched ICP: per pixel-iteration 4 B depth + 16 B gathered render tap (upper bound, L2 reuse lowers it)
    st_all = [dt.stats_from_device(ms.stats[i]) for i in range(n)]
    iters = float(np.mean([x.iterations for x in st_all]))
    roof = {"kernel": "k_render (batched direct DTSDF ray-cast)", "bound": "hbm", "achieved": achieved,
            "peak": peak, "unit": "GB/s", "frac": achieved / peak, "peak_kind": peak_kind, "traffic": None,
            "algorithmic_bytes_per_launch": render_bytes, "geom_bricks_per_problem": geom, "launch_ms": float(ph[1])}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu and not args.profile:
        v, sample_desc = ms_cpu_baseline(ms, n_frames)
        cpu = {"value": v, "unit": "registrations/s", "cores": cpu_cores(), "cpu": cpu_model(), "kind": "oracle", "sample": sample_desc}
    if rank == 0:
        out = {"metric": "multi-sensor Sim(3) registrations/s (1280x720 vs 640x480 map)", "value": value,
               "unit": "registrations/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
               "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
               "vs_baseline": None, "dtype": "f32", "data": "synthetic",
               "config": {"workload": WORKLOAD_MS.format(n=n), "problems": n, "storage": args.storage,
                          "map_frames": n_frames, "map_bricks": int(ms.map.stats().bricks),
                          "l2": "flushed between steps (512 MB write outside the timed events)",
                          "parallelism": f"replicas x{world}", "cuda_graph": True,
                          "batch_shape": {"cluster": shape[0], "threads": shape[1], "tuned_ms": tune_ms},
                          "phase_ms_eager": {"preprocess": float(ph[0]), "render_batch": float(ph[1]),
                                             "icp_batch": float(ph[2])},
                          "icp_iterations_mean": iters,
                          "rays_per_s": world * n * npix * args.steps / (total_ms / 1000.0),
                          "errors_vs_truth": {"rot_deg_median": float(np.median(rot)),
                                              "trans_m_median": float(np.median(tr)),
                                              "scale_median": float(np.median(sc)),
                                              "success_rate": float(np.mean((rot < 1.0) & (tr < 0.02))),
                                              "failed": [{"problem": int(k), "rot_deg": float(rot[k]),
                                                          "trans_m": float(tr[k]), "scale": float(sc[k])}
                                                         for k in np.nonzero(~((rot < 1.0) & (tr < 0.02)))[0]]}},
               "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
               "gpu_launches": n * MS_LAUNCHES_PER_FRAME + 4 * ((n + 63) // 64), "clocks": clocks}
        if emit:
            print(json.dumps(out), flush=True)
        ms.map.close()
        return out
    ms.map.close()
    return None


# ------------------------------------------------------------------ serve --
SERVE_OPTS = dict(levels=3, iters=(10, 10, 10), eps=(0.01, 0.1, 0.2), lam=0.0, stop_norm=1e-6, min_rows=10)
WORKLOAD_SERVE = ("serving: {n} render + registration requests, Poisson arrivals at {rate:g}/s, sensors 320x240 / "
                  "640x480 / 1280x720 (shares 0.3 / 0.5 / 0.2), SE(3):Sim(3) = 3:1 (Sim(3) depth scaled by U[0.9, 1.1]), "
                  "priors 2 deg / 2 cm off; {m} device-resident FP16 maps of seeded 4x4x3 m rooms ({f} frames each, "
                  "5 mm voxels); per request preprocessing + 3-level pyramid, render at the prior, 3-level "
                  "registration (10 iterations per level); continuous batching over 4 streams, admission by a "
                  "{gb:g} GB device budget")


def pose_diff(A, B):
    """(rotation angle rad, translation m, relative scale) between two similarity transforms."""
    sa, sb = np.cbrt(np.linalg.det(A[:3, :3])), np.cbrt(np.linalg.det(B[:3, :3]))
    R = (A[:3, :3] / sa).T @ (B[:3, :3] / sb)
    ang = float(np.arccos(np.clip((np.trace(R) - 1) / 2, -1, 1)))
    return ang, float(np.linalg.norm(A[:3, 3] - B[:3, 3])), float(abs(sa / sb - 1))


def serve_stream(srv, reqs, pinned):
    """Submit each request at its arrival time (server clock), collect every result."""
    out = {}
    t0 = srv.clock() + 0.01
    for i, q in enumerate(reqs):
        while srv.clock() - t0 < q["t"]:
            for r in srv.poll(64, wait_us=0):
                out[r.tag] = r
        srv.submit(q["map"], pinned[i], q["K"], q["prior"], sim3=q["sim3"], tag=i)
    deadline = time.time() + 300
    while len(out) < len(reqs):
        assert time.time() < deadline, "serve: results missing"
        for r in srv.poll(256, wait_us=2000):
            out[r.tag] = r
    return [out[i] for i in range(len(reqs))]


def serial_stream(dt, torch, dev, maps, reqs, pinned, icps):
    """The same arrival stream served one request at a time (synchronous per request)."""
    opts = dt.icp_opts(**SERVE_OPTS)
    bufs = {}
    T = torch.eye(4, dtype=torch.float64, device=dev)
    eye = torch.eye(4, dtype=torch.float64, device=dev)
    prior = torch.empty(4, 4, dtype=torch.float64, device=dev)
    host_T = torch.empty(4, 4, dtype=torch.float64).pin_memory()
    done, res = [], []
    t0 = time.perf_counter() + 0.01
    for i, q in enumerate(reqs):
        while time.perf_counter() - t0 < q["t"]:
            pass
        K = q["K"]
        key = (K.width, K.height)
        if key not in bufs:
            bufs[key] = (torch.empty(K.height, K.width, device=dev), torch.zeros(K.height, K.width, device=dev),
                         torch.zeros(K.height, K.width, 4, device=dev))
        d_in, rd, rn = bufs[key]
        src = pinned[i] if torch.is_tensor(pinned[i]) else torch.from_numpy(pinned[i])
        d_in.copy_(src, non_blocking=True)
        prior.copy_(torch.from_numpy(q["prior"]), non_blocking=True)
        icp = icps[key]
        icp.set_frame(d_in, None, K, 0.1, 6.0, 0.01)
        maps[q["map"]].render_dev(K, prior, rd, rn)
        T.copy_(eye)
        dt.icp_batch([(icp, rn, K, T, q["sim3"])], opts, shape=(8, 256))
        host_T.copy_(T, non_blocking=True)
        torch.cuda.current_stream().synchronize()
        done.append(time.perf_counter() - t0 - q["t"])
        res.append(q["prior"] @ host_T.numpy())
    return np.array(done), res


def serve_cpu_baseline(rooms, q):
    """The oracle on a bounded sample of one 640x480 request, scaled to the whole request."""
    import oracle
    from oracle import icp as oicp
    room, K = rooms[q["map"]], q["K"]
    om = oracle.OracleMap(oracle.Params(voxel_size=0.005, truncation=0.02, z_max=room.z_max, color=False))
    for i in range(0, room.n_frames, max(1, room.n_frames // 6)):
        f = room.frame(i)
        om.integrate(f.depth, None, room.K, f.pose)
    stride = 16
    vv, uu = np.mgrid[0:K.height:stride, 0:K.width:stride]
    pix = np.stack([uu.ravel(), vv.ravel()], 1).astype(np.int32)
    t0 = time.perf_counter()
    om.render(K, q["prior"], pix)
    t_render = (time.perf_counter() - t0) * (K.width * K.height) / len(pix)
    ref = room.render(q["prior"], K=K, noise=False, exact=True)
    rn = np.zeros(ref.normals.shape[:2] + (4,), np.float32)
    rn[..., :3] = ref.normals
    pre = oracle.preprocess(q["depth"], K, 0.1, 6.0, 0.01)
    levels = oicp.pyramid(pre["z"], K, 3)
    st = oicp.Settings(sim3=bool(q["sim3"]), eps=SERVE_OPTS["eps"], iters=SERVE_OPTS["iters"])
    t_icp = 0.0
    for l in range(3):
        t0 = time.perf_counter()
        oicp.step(levels[l], ref.depth, rn, K, np.eye(4), st.eps[l], st, level_index=l)
        t_icp += (time.perf_counter() - t0) * SERVE_OPTS["iters"][l]
    sample = (f"one 640x480 request: oracle render of 1/{stride * stride} of the pixels scaled up ({t_render:.1f} s), "
              f"one registration iteration per level scaled to 10 per level ({t_icp:.1f} s); oracle map fused from "
              f"1/{max(1, room.n_frames // 6)} of the frames")
    return 1.0 / (t_render + t_icp), sample


def run_serve(args, dt, torch, tdist, dev, rank, world, local, emit=True):
    import scenes
    n_frames = 20 if args.profile else args.map_frames
    rooms = [scenes.kinect_room(1 + i, n_frames=n_frames) for i in range(args.maps)]
    maps16, maps32 = [], []
    for room in rooms:
        for store, lst in ((dt.STORE_FP16, maps16), (dt.STORE_FP32, maps32)):
            m = dt.Map(dt.params(voxel_size=0.005, truncation=0.02, max_blocks=1 << 18, z_max=room.z_max,
                                 color=False, storage=store))
            lst.append(m)
        for i in range(room.n_frames):
            f = room.frame(i)
            d = torch.from_numpy(f.depth).to(dev)
            lst16, lst32 = maps16[-1], maps32[-1]
            lst16.integrate(d, None, room.K, f.pose)
            lst32.integrate(d, None, room.K, f.pose)
    torch.cuda.synchronize()
    voxels = [round(m.stats().bricks * 512 / 1e6, 2) for m in maps16]
    n_req = 64 if args.profile else args.requests
    reqs = scenes.serve_requests(rooms, n_req, seed=1, rate=args.rate, pool=min(n_req, 96))
    pinned = [torch.from_numpy(q["depth"]).pin_memory() for q in reqs]
    pinned_np = [p.numpy() for p in pinned]
    budget = 16 << 30
    p = dt.server_params(hbm_budget=budget, max_inflight=128, max_batch=32, streams=4,
                         opts=dt.icp_opts(**SERVE_OPTS), shape=(8, 256))
    srv = dt.Server(maps16, p)
    warm = scenes.serve_requests(rooms, 48, seed=2, rate=args.rate, pool=8)
    serve_stream(srv, warm, [q["depth"] for q in warm])
    clk = ClockSampler(local)
    clk.start()
    if world > 1:
        tdist.barrier()
    torch.cuda.synchronize()
    res = serve_stream(srv, reqs, pinned_np)
    clocks = clk.stop()
    st = srv.stats()
    lat = np.array([r.t_done - r.t_submit for r in res])
    span = max(r.t_done for r in res) - min(r.t_submit for r in res)
    value = world * len(reqs) / span
    # latency below capacity: the same kind of stream at a tenth of the offered rate
    low = serve_requests_low(srv, rooms, max(32, n_req // 4), args.rate / 10.0)
    srv.close()
    # serial plain FP32 solves of the same stream
    icps = {(K.width, K.height): dt.Icp(K.width, K.height, 3) for K, _ in scenes.SERVE_SENSORS}
    serial_stream(dt, torch, dev, maps32, warm[:8], [q["depth"] for q in warm[:8]], icps)
    lat_s, res_s = serial_stream(dt, torch, dev, maps32, reqs, pinned, icps)
    span_s = float(lat_s[-1] + reqs[-1]["t"] - reqs[0]["t"])
    # accuracy: FP16 served vs FP32 serial, and both vs the truth
    d_fp = np.array([pose_diff(np.array(r.T_wc[:]).reshape(4, 4), T) for r, T in zip(res, res_s)])
    d_gt = np.array([pose_diff(np.array(r.T_wc[:]).reshape(4, 4) @ np.diag([q["scale"]] * 3 + [1.0]), q["T_true"])
                     for r, q in zip(res, reqs)])
    # roofline of the dominant kernel: one render launch over a batch of the pool's frames per map (events)
    sample = list(range(0, min(len(reqs), 96)))
    bufs = [(torch.from_numpy(reqs[i]["prior"]).to(dev), torch.zeros(reqs[i]["K"].height, reqs[i]["K"].width,
                                                                     device=dev),
             torch.zeros(reqs[i]["K"].height, reqs[i]["K"].width, 4, device=dev)) for i in sample]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    geom = 0.0
    for mi, m in enumerate(maps16):
        sel = [j for j, i in enumerate(sample) if reqs[i]["map"] == mi][:32]
        for j in sel[:4]:
            geom += m.touched(reqs[sample[j]]["K"], reqs[sample[j]]["prior"])[0] * len(sel) / max(1, min(4, len(sel)))
    rms = 0.0
    pix = 0
    for mi, m in enumerate(maps16):
        sel = [j for j, i in enumerate(sample) if reqs[i]["map"] == mi][:32]
        if not sel:
            continue
        jobs = [(reqs[sample[j]]["K"], bufs[j][0], bufs[j][1], bufs[j][2], None) for j in sel]
        m.render_batch(jobs)
        e0.record()
        m.render_batch(jobs)
        e1.record()
        torch.cuda.synchronize()
        rms += e0.elapsed_time(e1)
        pix += sum(reqs[sample[j]]["K"].width * reqs[sample[j]]["K"].height for j in sel)
    render_bytes = geom * 512 * 4 + pix * (4 + 16)
    peak, peak_kind = measured_hbm_peak()
    achieved = render_bytes / (rms / 1000.0) / 1e9
    roof = {"kernel": "k_render (batched direct DTSDF ray-cast, FP16 storage)", "bound": "hbm", "achieved": achieved,
            "peak": peak, "unit": "GB/s", "frac": achieved / peak, "peak_kind": peak_kind, "traffic": None,
            "algorithmic_bytes_per_launch": render_bytes / max(1, args.maps), "launch_ms": rms / max(1, args.maps)}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu and not args.profile:
        q640 = next(q for q in reqs if q["K"].width == 640)
        v, desc = serve_cpu_baseline(rooms, q640)
        cpu = {"value": v, "unit": "requests/s", "cores": cpu_cores(), "cpu": cpu_model(), "kind": "oracle", "sample": desc}
    h2d = int(np.mean([q["depth"].nbytes for q in reqs]))
    if rank == 0:
        out = {"metric": "served render+ICP requests/s, p50/p99 latency (continuous batching, mixed sizes)",
               "value": value, "unit": "requests/s", "n_gpus": world, "steps": len(reqs), "warmup": len(warm),
               "ms_per_step": 1000.0 / value, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
               "dtype": "f16 storage / f32 compute", "data": "synthetic",
               "config": {"workload": WORKLOAD_SERVE.format(n=len(reqs), rate=args.rate, m=args.maps, f=n_frames,
                                                            gb=budget / 2 ** 30),
                          "map_voxels_M": voxels, "parallelism": f"replicas x{world}",
                          "l2": "inputs (maps 1-2 GB each) larger than L2",
                          "server": {"streams": 4, "max_batch": 32, "batches": int(st.batches),
                                     "mean_batch": len(reqs) / max(1, int(st.batches)),
                                     "peak_inflight": int(st.peak_inflight), "peak_bytes": int(st.peak_bytes)}},
               "latency_ms": {"p50": float(np.percentile(lat, 50) * 1e3), "p99": float(np.percentile(lat, 99) * 1e3),
                              "mean": float(lat.mean() * 1e3)},
               "latency_below_capacity": low,
               "serial_fp32": {"value": len(reqs) / span_s, "unit": "requests/s",
                               "latency_ms": {"p50": float(np.percentile(lat_s, 50) * 1e3),
                                              "p99": float(np.percentile(lat_s, 99) * 1e3)}},
               "accuracy": {"fp16_served_vs_fp32_serial": {
                   "rot_rad_median": float(np.median(d_fp[:, 0])), "rot_rad_max": float(d_fp[:, 0].max()),
                   "trans_m_median": float(np.median(d_fp[:, 1])), "trans_m_max": float(d_fp[:, 1].max()),
                   "scale_max": float(d_fp[:, 2].max()),
                   "within_1e-4_rad_1e-4_m_1e-5_scale": float(np.mean((d_fp[:, 0] <= 1e-4) & (d_fp[:, 1] <= 1e-4) &
                                                                      (d_fp[:, 2] <= 1e-5)))},
                   "vs_truth": {"trans_m_median": float(np.median(d_gt[:, 1])),
                                "rot_rad_median": float(np.median(d_gt[:, 0])),
                                "success_rate_1cm_1deg": float(np.mean((d_gt[:, 1] < 0.01) &
                                                                       (d_gt[:, 0] < np.radians(1.0))))}},
               "roofline": roof, "cpu_baseline": cpu,
               "e2e": {"value": value, "unit": "requests/s", "h2d_bytes_per_step": h2d,
                       "d2h_bytes_per_step": ctypes_result_bytes(dt)},
               "gpu_launches": int(st.batches) * (2 + 3 * args.maps) + 5 * len(reqs), "clocks": clocks}
        if emit:
            print(json.dumps(out), flush=True)
    for m in maps16 + maps32:
        m.close()
    return out if rank == 0 else None


def serve_requests_low(srv, rooms, n, rate):
    """p50/p99 latency and throughput of a stream offered at `rate` (below capacity)."""
    import scenes
    reqs = scenes.serve_requests(rooms, n, seed=3, rate=rate, pool=min(n, 48))
    res = serve_stream(srv, reqs, [q["depth"] for q in reqs])
    lat = np.array([r.t_done - r.t_submit for r in res])
    return {"requests": n, "offered_per_s": rate, "p50_ms": float(np.percentile(lat, 50) * 1e3),
            "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "mean_batch": float(np.mean([r.batch_size for r in res]))}


MS_BLOCK_STEPS = 10


def side_args(args, steps):
    """Arguments of a side workload run inside the tracking line: its own defaults (FP32 maps for
    the multi-sensor batch, 512 requests at 2000/s over 3 FP16 maps for serving), the tracking
    line's warm-up, no oracle leg of its own (the tracking line carries the CPU baseline)."""
    a = argparse.Namespace(**vars(args))
    a.steps = steps or args.steps
    a.no_cpu = True
    a.storage = "fp32"
    return a


def side_block(out):
    """The fields of a side workload's JSON line that the tracking line carries as a block."""
    if out is None:
        return None
    keep = ("metric", "value", "unit", "steps", "ms_per_step", "config", "latency_ms", "latency_below_capacity",
            "serial_fp32", "accuracy", "roofline", "e2e", "gpu_launches", "clocks")
    return {k: out[k] for k in keep if k in out}


def ctypes_result_bytes(dt):
    return 32 * 8 + dt.STATS_BYTES


# --------------------------------------------------------------------- main --
def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    import torch
    import torch.distributed as tdist
    import paper_2301_12796_gb300 as dt
    from paper_2301_12796_gb300 import build as B
    if rank == 0:
        B.build()
    if world > 1:
        tdist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
        tdist.barrier()
        B.build()
    torch.cuda.set_device(local)
    dev = torch.device(f"cuda:{local}")
    assert args.warmup >= 3 or args.profile, "at least 3 warm-up steps"
    if args.workload == "multi_sensor":
        run_multi_sensor(args, dt, torch, tdist, dev, rank, world, local)
    elif args.workload == "serve":
        run_serve(args, dt, torch, tdist, dev, rank, world, local)
    else:
        run_tracking(args, dt, torch, tdist, dev, rank, world, local)
    if world > 1:
        tdist.destroy_process_group()


if __name__ == "__main__":
    main()
