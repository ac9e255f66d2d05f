#!/usr/bin/env python
"""Benchmark: 800x800 SpaRW frames per second (BF16 tensor-core MLP) on the 256^3 FP16 scene.

One step = one SpaRW window (Sec. III-B/C): the reference frame rendered in full, memory-centric
(march, Ray Index Table, per-brick TMA gather + tcgen05 MLP, compositing), then 16 target frames,
each warped from the reference (Eq. 1-3 + depth test + void test) and completed by rendering only
its holes (Eq. 4).  value = 16 target frames x steps x ranks / time.  The plain FP32 full render
of the same frame is measured beside it.  With --gpus N every rank renders its own window
(different orbit azimuth): weak scaling, no collective on the data path.

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle on a bounded sample of
the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

WORKLOAD = "sparw_window_800x800_grid256_fp16_occ32_16targets"
METRIC = "800x800 FPS & Msamples/s, BF16+SpaRW vs plain FP32, at PSNR>=45dB vs oracle"
N_TARGETS = 16
W = H = 800
FLOP_PER_SAMPLE = 2 * (39 * 128 + 128 * 128 + 128 * 3)  # 43,520 MLP FLOP per composited sample
HOLE_RECORDS = 128_000_000  # record capacity of the batched hole render (6.7 GB; ~84 M are used)
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one k_gather_mlp_bf16 launch on the
# 800x800 reference frame, from a one-pass ncu capture of this benchmark, and the SHA-1 of the
# kernel sources it was taken on; the roofline reports it only while those sources are unchanged.
GATHER_TRAFFIC = {"bytes": 2742457856 + 1359033856, "sources_sha1": "9d9cadcd8128ab014fadc07c6f8d80e7c5cd154e"}
GATHER_SOURCES = ("mlp_tc.cu", "common.cuh", "internal.h")
# shared-memory wavefronts per composited sample of the BF16 gather (LSU loads + LSU stores +
# tensor-core operand reads, ncu on the 320x320 case), valid for the sources hashed above
GATHER_SMEM_WAVEFRONTS_PER_SAMPLE = (24302060 + 31859312 + 67379200) / 10312421


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=50)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-extra", action="store_true", help="skip the backward and small-scene SpaRW reports")
    p.add_argument("--cpu-res", type=int, default=100, help="oracle sample resolution (square)")
    p.add_argument("--oracle-full-window", action="store_true",
                   help="reference arm: also time one full-resolution oracle window (minutes on the host)")
    p.add_argument("--case", default="full", choices=["full", "small", "backward"],
                   help="small: one 320x320 reference frame (BF16 and FP32) and two targets, for profilers; "
                        "backward: the differentiation workload alone")
    p.add_argument("--brick", type=int, default=4, help="brick size of the small case")
    return p.parse_args()


def small_case(brick: int = 4):
    """A reduced run of the same kernels for profiler captures (the grid stays 416 MB > L2).

    Kernel launch order: reference frame BF16 twice, FP32 once (one k_march, bucketing, gather
    and composite each), then per target one warp and one hole render, then the frame with a hash
    encoding twice.  No autotuning, so a capture's launch index (-s) does not depend on timing."""
    import torch
    import scenes
    from paper_2404_11852_gb300 import build, cicero as cc
    build.build()
    g_h, m_h = scenes.scene_large(), scenes.make_mlp(12)
    grid, mlp = cc.DeviceGrid.from_host(g_h), cc.DeviceMlp.from_host(m_h)
    n = 320
    cam = scenes.orbit_camera(n, n, sampling=scenes.sampling_march(256, 256))
    sd, cd = cc.sampling_from(cam.sampling), cc.camera_from(cam)
    R = n * n
    rgb, depth = torch.empty(R, 3, device="cuda"), torch.empty(R, device="cuda")
    o16, o32 = cc.options(cc.MLP_BF16, brick), cc.options(cc.MLP_FP32, brick)
    ws = cc.workspace(cc.cicero_render_workspace_size(grid.desc, R, sd, o16))
    for opt in (o16, o16, o32):
        cc.cicero_render(grid.desc, mlp.desc, cd, sd, opt, rgb, depth, None, None, ws)
    cc.cicero_workspace_status(ws)
    active = int(ws[:16].view(torch.int32).cpu().numpy()[2])
    wws = cc.workspace(cc.cicero_warp_workspace_size(cd))
    for k in (-8, 8):
        td = cc.camera_from(scenes.offset_camera(cam, k))
        wr, wd = torch.empty(R, 3, device="cuda"), torch.empty(R, device="cuda")
        mask = torch.empty(R, dtype=torch.uint8, device="cuda")
        hidx = torch.empty(R, dtype=torch.int32, device="cuda")
        nh = torch.empty(1, dtype=torch.int32, device="cuda")
        cc.cicero_warp(rgb, depth, cd, td, 180.0, grid.desc, sd, wr, wd, mask, hidx, nh, wws)
        cc.cicero_render_holes(grid.desc, mlp.desc, td, sd, o16, hidx, nh, R, wr, wd, ws)
    cc.cicero_workspace_status(ws)
    # the hash-encoded frame (8 levels x 2 FP16, 2^19 entries), twice
    h = scenes.make_hash_grid(8, 2, 19, 16, 1024, seed=777)
    hd, md = cc.DeviceHashGrid.from_host(h), cc.DeviceMlp.from_host(scenes.make_mlp(16, seed=778))
    wsh = cc.workspace(cc.cicero_render_hash_workspace_size(grid.desc, hd.desc, R, sd, o16))
    for _ in range(2):
        cc.cicero_render_hash(grid.desc, hd.desc, md.desc, cd, sd, o16, rgb, depth, wsh)
    cc.cicero_workspace_status(wsh)
    torch.cuda.synchronize()
    print(json.dumps({"case": "small", "image": f"{n}x{n}", "brick": brick, "active_samples_reference": active}))


# ---------------------------------------------------------------------------------------------
# multi-rank host logic (one process per GPU, replicas: no collective on the data path)


def rank_azimuth(rank: int) -> float:
    """Each rank renders its own SpaRW window, from its own orbit azimuth."""
    return 30.0 + 20.0 * rank


def max_over_ranks(seconds: float, device=None) -> float:
    """The slowest rank's time: the job ends when it does (a no-op without a process group)."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return seconds
    import torch
    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(units_per_step: int, steps: int, world: int, seconds: float) -> float:
    """Whole-job throughput: the units every rank processed over the slowest rank's time."""
    return units_per_step * steps * world / seconds


def stage_roofline(stages, pk, R, n_holes, ref_samples, hole_samples):
    """Per stage of one SpaRW window: algorithmic bytes (or FLOP), achieved rate over the stage's
    device time, and the fraction of the measured peak of the resource that bounds it.

    Bytes counted: march, per composited sample its record (brick id 4 B + position/weight 16 B)
    and per ray its header and depth (36 B); bucket, per record 20 B read + 32 B written (the Ray
    Index Table payload) + 24 B of ray header per ray; gather + MLP, 43,520 FLOP per sample;
    composite, per sample 16 B read + per ray 28 B; warp splat, per reference pixel 16 B read +
    8 B of depth-key atomic per target; warp resolve, ~29 B per target pixel."""
    rays = R + n_holes
    samples = ref_samples + hole_samples
    work = {
        "march": ("issue", 20.0 * samples + 36.0 * rays),
        "bucket": ("hbm", 52.0 * samples + 24.0 * rays),
        "gather_mlp": ("tensor", float(FLOP_PER_SAMPLE) * samples),
        "composite": ("hbm", 16.0 * samples + 28.0 * rays),
        "warp_splat": ("hbm", (16.0 + 8.0 * N_TARGETS) * R),
        "warp_resolve": ("hbm", 29.0 * N_TARGETS * R),
    }
    out = {}
    for k, (bound, amount) in work.items():
        if k not in stages or stages[k]["ms_per_step"] <= 0:
            continue
        t = stages[k]["ms_per_step"] / 1e3
        if bound == "tensor":
            ach = amount / t / 1e12
            out[k] = {"bound": bound, "algorithmic_tflop": amount / 1e12, "achieved": ach, "unit": "TFLOP/s",
                      "frac": ach / pk["bf16_tflops_sustained"]}
        else:
            ach = amount / t / 1e9
            out[k] = {"bound": bound, "algorithmic_gb": amount / 1e9, "achieved": ach, "unit": "GB/s",
                      "frac_of_hbm": ach / pk["hbm_gbs"]}
    return out


def gather_traffic():
    import hashlib
    h = hashlib.sha1()
    for f in GATHER_SOURCES:
        with open(os.path.join(ROOT, "paper_2404_11852_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    ok = GATHER_TRAFFIC["bytes"] is not None and GATHER_TRAFFIC["sources_sha1"] == h.hexdigest()
    return GATHER_TRAFFIC["bytes"] if ok else None


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            j = json.load(f)
        return {"hbm_gbs": j["hbm_gbs"], "bf16_tflops": j["bf16_tflops"],
                "bf16_tflops_sustained": j.get("bf16_tflops_sustained", j["bf16_tflops"]),
                "sm_max_mhz": j.get("sm_max_mhz", 2070.0), "src": "measured"}
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0,
                "src": "fallback"}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index, self.rows, self.proc = index, [], None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if len(r) > 5 + i and r[5 + i] == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


# ---------------------------------------------------------------------------------------------
# CPU oracle leg (the reference arm and the cpu_baseline object)


def oracle_window(res: int, rank: int = 0, frames: list | None = None):
    """The oracle's SpaRW window at res x res on the same scene, FOV, poses and sampling; returns
    (seconds, cores, hole fraction).  With ``frames``, the 16 target frames are appended to it."""
    import oracle
    import scenes
    g, m = scenes.scene_large(), scenes.make_mlp(12)
    oracle.build()
    cam = scenes.orbit_camera(res, res, az_deg=rank_azimuth(rank), sampling=scenes.sampling_march(256, 256))
    t0 = time.perf_counter()
    ref = oracle.render(g, m, cam.sampling, cam=cam)
    holes = 0
    for k in scenes.SPARW_OFFSETS:
        tgt = scenes.offset_camera(cam, k)
        w = oracle.warp(ref["rgb"].astype(np.float32), ref["depth"].astype(np.float32), cam, tgt, void_grid=g,
                        void_sampling=cam.sampling)
        frame = w["rgb"].astype(np.float64)
        if w["n_holes"]:
            frame[w["hole_idx"]] = oracle.render(g, m, cam.sampling, cam=tgt, pix=w["hole_idx"])["rgb"]
        if frames is not None:
            frames.append(frame)
        holes += w["n_holes"]
    dt = time.perf_counter() - t0
    return dt, oracle.max_threads(), holes / (N_TARGETS * res * res)


def oracle_threads(g, m, cam, R, n_pix=2048):
    """The oracle's full-render throughput on one host thread and on all of them (OpenMP over rays),
    on the same seeded sample of the reference frame's rays (rays/s)."""
    import oracle
    import scenes
    pix = (scenes.splitmix64(4242, n_pix) % np.uint64(R)).astype(np.int32)
    out = {}
    for name, th in (("single", 1), ("all", 0)):
        t0 = time.perf_counter()
        oracle.render(g, m, cam.sampling, cam=cam, pix=pix, threads=th)
        out[name + "_rays_per_s"] = n_pix / (time.perf_counter() - t0)
    out["all_cores"] = oracle.max_threads()
    out["speedup"] = out["all_rays_per_s"] / out["single_rays_per_s"]
    out["sample"] = f"{n_pix} seeded reference-frame rays (FP64, 256 slots)"
    return out


def run_reference(args, rank, world, window=None):
    """The oracle arm: rank 0 alone times the oracle; the other ranks exit without work.  A step is
    the oracle's whole SpaRW window at a reduced resolution (a bounded sample of the workload);
    `ms_per_step` is the time of that sample, `value` the 800x800 rate it extrapolates to by the
    pixel ratio (stated in `sample`).  With --oracle-full-window one full-resolution window is timed
    as well."""
    if rank != 0:
        return None
    window = window or oracle_window
    res = args.cpu_res
    for _ in range(max(0, args.warmup)):
        window(res)
    dts = []
    for _ in range(max(1, args.steps)):
        dt, cores, _ = window(res)
        dts.append(dt)
    scale = (W * H) / (res * res)
    t_sample = float(np.mean(dts))
    t_full = t_sample * scale
    fps = N_TARGETS / t_full
    sample = {"resolution": f"{res}x{res}", "pixels_per_frame": res * res, "full_pixels_per_frame": W * H,
              "scale": scale, "ms_per_full_window_extrapolated": t_full * 1e3,
              "what": "whole SpaRW window (reference render, 16 warps, 16 hole renders), FP64"}
    line = {"impl": "reference", "metric": METRIC, "value": fps, "unit": "frames/s", "n_gpus": args.gpus,
            "steps": len(dts), "warmup": max(0, args.warmup), "ms_per_step": t_sample * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "l2": "n/a (CPU)"}, "sample": sample,
            "cpu_baseline": {"value": fps, "unit": "frames/s", "cores": cores, "kind": "oracle",
                             "sample": f"whole SpaRW window at {res}x{res} ({res * res} of {W * H} pixels per "
                                       f"frame), time x {scale:.0f}"},
            "e2e": {"value": fps, "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    if getattr(args, "oracle_full_window", False):
        dt, _, _ = window(W)
        line["full_window"] = {"resolution": f"{W}x{H}", "ms": dt * 1e3, "frames_per_s": N_TARGETS / dt,
                               "extrapolation_error": t_full / dt - 1.0}
    print(json.dumps(line), flush=True)
    return line


# ---------------------------------------------------------------------------------------------
# one SpaRW window on the device


class SparwWindow:
    """Device buffers and the call sequence of one SpaRW window (Sec. III-B/C): the reference frame
    rendered in full, every target warped from it in one batch, then all targets' holes rendered in
    one batch, written into the warped frames (Eq. 4)."""

    def __init__(self, cc, torch, dev, grid, mlp, cam, targets, opt_ref, opt_holes, ref_ws_bytes=0,
                 max_angle_deg=180.0):
        self.cc, self.grid, self.mlp, self.max_angle = cc, grid, mlp, max_angle_deg
        self.R, self.n = cam.width * cam.height, len(targets)
        R, n = self.R, self.n
        self.sd, self.cd = cc.sampling_from(cam.sampling), cc.camera_from(cam)
        self.tds = [cc.camera_from(t) for t in targets]
        self.opt_ref, self.opt_holes = opt_ref, opt_holes
        self.ref_rgb, self.ref_depth = torch.empty(R, 3, device=dev), torch.empty(R, device=dev)
        self.t_rgb, self.t_depth = torch.empty(n, R, 3, device=dev), torch.empty(n, R, device=dev)
        self.mask = torch.empty(n, R, dtype=torch.uint8, device=dev)
        self.hidx = torch.empty(n, R, dtype=torch.int32, device=dev)
        self.nh = torch.zeros(n, 1, dtype=torch.int32, device=dev)
        ref_bytes = max(ref_ws_bytes, cc.cicero_render_workspace_size(grid.desc, R, self.sd, opt_ref))
        self.ws_r = cc.workspace(ref_bytes, dev)
        self.ws_w = cc.workspace(cc.cicero_warp_batch_workspace_size(self.tds), dev)
        self.ws_h = cc.workspace(cc.cicero_render_workspace_size(grid.desc, n * R, self.sd, opt_holes), dev)
        self.lists = [[x[i] for i in range(n)] for x in (self.t_rgb, self.t_depth, self.mask, self.hidx)]

    def render_reference(self, opt=None):
        self.cc.cicero_render(self.grid.desc, self.mlp.desc, self.cd, self.sd, opt or self.opt_ref, self.ref_rgb,
                              self.ref_depth, None, None, self.ws_r)

    def run(self):
        # No separate void test (void_grid None): a void hole's march in the hole batch finds no
        # occupied slot and writes the background with depth +inf, the frames the test would give
        # (bit for bit; tests/test_gpu_window_full.py), without repeating the start of every real
        # hole's march.
        cc, L = self.cc, self.lists
        self.render_reference()
        cc.cicero_warp_batch(self.ref_rgb, self.ref_depth, self.cd, self.tds, self.max_angle, None, None,
                             L[0], L[1], L[2], L[3], self.nh.view(-1), self.ws_w)
        cc.cicero_render_holes_batch(self.grid.desc, self.mlp.desc, self.tds, self.sd, self.opt_holes, L[3], self.nh,
                                     self.n * self.R, L[0], L[1], self.ws_h)

    def classify(self):
        """Per target, the holes the separate void test would mark as disocclusions (mask 1) and as
        void (mask 2).  Overwrites the target frames."""
        cc, L = self.cc, self.lists
        cc.cicero_warp_batch(self.ref_rgb, self.ref_depth, self.cd, self.tds, self.max_angle, self.grid.desc,
                             self.sd, L[0], L[1], L[2], L[3], self.nh.view(-1), self.ws_w)
        m = self.mask.cpu().numpy()
        return (m == 1).sum(axis=1), (m == 2).sum(axis=1)

    def set_frames(self, t_rgb):
        """Write the target frames into ``t_rgb`` [n, R, 3] from the next run on."""
        self.t_rgb = t_rgb
        self.lists[0] = [t_rgb[i] for i in range(self.n)]

    def check(self):
        """Raise if a kernel reported an error (capacity, timeout, broken invariant)."""
        self.cc.cicero_workspace_status(self.ws_r)
        self.cc.cicero_workspace_status(self.ws_h)

    def header(self, ws):
        return ws[:16].view(self.nh.dtype).cpu().numpy()


def frame_psnr(got, want):
    mse = float(np.mean((np.asarray(got, np.float64) - np.asarray(want, np.float64)) ** 2))
    return 10 * math.log10(1.0 / max(mse, 1e-30))


# ---------------------------------------------------------------------------------------------
# the other measured workloads (rank 0, outside the headline timing)


def event_ms(torch, fn, reps):
    """Average device time of fn() over reps, CUDA events on the current stream."""
    fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def sparw_parity(cc, torch, dev, grid, mlp, res, rank, frames, opt):
    """The device SpaRW window (BF16 MLP) at res x res against the oracle's SpaRW window on the same
    scene and cameras: PSNR and max |rgb error| of every pixel of every target frame."""
    import scenes
    cam = scenes.orbit_camera(res, res, az_deg=rank_azimuth(rank), sampling=scenes.sampling_march(256, 256))
    targets = [scenes.offset_camera(cam, k) for k in scenes.SPARW_OFFSETS]
    win = SparwWindow(cc, torch, dev, grid, mlp, cam, targets, opt, opt)
    win.run()
    win.check()
    got = win.t_rgb.cpu().double().numpy()
    ps = [frame_psnr(got[i], frames[i]) for i in range(len(frames))]
    err = max(float(np.abs(got[i] - frames[i]).max()) for i in range(len(frames)))
    return {"image": f"{res}x{res}", "targets": len(frames), "psnr_db_min": min(ps),
            "psnr_db_mean": float(np.mean(ps)), "max_err": err}


BATCH_GRIDS = (96, 128, 160, 192, 224, 256)
BATCH_SIDES = (256, 384, 512, 640, 768, 896, 1024)
BATCH_SAMPLES = (64, 128, 192, 256)
BATCH_JOBS = 48


def batched_workload(cc, torch, dev, n_check=8, reps=5):
    """48 scene/view pairs of uneven size rendered as one batch (cicero_batch_*), replayed from a
    CUDA graph, against the same jobs rendered one cicero_render call at a time.  Six scenes
    (96^3 .. 256^3 x 12 FP16, 24 blobs, 32^3 occupancy at 15%), each with its own MLP, 8 views
    each; image side (256 .. 1024) and samples per ray (64 .. 256, slots every half voxel) drawn
    per job from a seeded stream.  n_check pixels per job are checked against the FP64 oracle."""
    import oracle
    import scenes
    u = scenes.splitmix64(4321, 2 * BATCH_JOBS)
    sc = []
    for i, N in enumerate(BATCH_GRIDS):
        g = scenes.make_grid(N, 12, 24, seed=700 + i, dtype=np.float16, occ_res=32, occ_frac=0.15)
        m = scenes.make_mlp(12, seed=800 + i)
        sc.append((g, m, cc.DeviceGrid.from_host(g, dev), cc.DeviceMlp.from_host(m, dev)))
    specs, keep, rows, outs = [], [], [], []
    for j in range(BATCH_JOBS):
        si = j % len(BATCH_GRIDS)
        side = BATCH_SIDES[int(u[2 * j] % np.uint64(len(BATCH_SIDES)))]
        S = BATCH_SAMPLES[int(u[2 * j + 1] % np.uint64(len(BATCH_SAMPLES)))]
        cam = scenes.orbit_camera(side, side, az_deg=360.0 * j / BATCH_JOBS, el_deg=10.0 + 20.0 * (j % 3),
                                  sampling=scenes.sampling_march(BATCH_GRIDS[si], S))
        cd, sd = cc.camera_from(cam), cc.sampling_from(cam.sampling)
        R = side * side
        rgb, dep = torch.empty(R, 3, device=dev), torch.empty(R, device=dev)
        specs.append((si, cam, S))
        keep.append((cd, sd))
        outs.append((rgb, dep))
        rows.append((sc[si][2].desc, sc[si][3].desc, cd, sd, rgb, dep))
    jobs = cc.jobs_array(rows)
    rays = sum(c.width * c.height for _, c, _ in specs)
    rs = sum(c.width * c.height * S for _, c, S in specs)
    cap = int(0.45 * rs)  # composited samples are ~35% of the slots here; a shortfall is reported
    opt4 = cc.options(cc.MLP_BF16, 4, max_records=cap)
    ws = cc.workspace(cc.cicero_batch_workspace_size(jobs, opt4), dev)
    tuned, tune = cc.cicero_batch_autotune(jobs, opt4, ws)
    brick, groups = tuned.brick, tuned.mlp_groups
    opt = cc.options(cc.MLP_BF16, brick, max_records=cap, mlp_groups=groups)
    b = cc.Batch(jobs, opt, ws)
    b.launch()  # outside the capture: kernel attributes
    torch.cuda.synchronize()
    b.status()
    samples = int(b.header()[2])
    stream = torch.cuda.Stream(dev)
    stream.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        b.launch()
    t_batch = event_ms(torch, graph.replay, reps)
    b.status()
    # the same jobs one cicero_render at a time (one workspace, sized for the largest job)
    o1 = cc.options(cc.MLP_BF16, brick, mlp_groups=groups)
    big = max(cc.cicero_render_workspace_size(sc[si][2].desc, c.width * c.height, keep[j][1], o1)
              for j, (si, c, _) in enumerate(specs))
    ws1 = cc.workspace(big, dev)

    def one_by_one():
        for j, (si, c, _) in enumerate(specs):
            cd, sd = keep[j]
            cc.cicero_render(sc[si][2].desc, sc[si][3].desc, cd, sd, o1, outs[j][0], outs[j][1], None, None, ws1)

    t_single = event_ms(torch, one_by_one, 2)
    cc.cicero_workspace_status(ws1)
    # where the time goes: per-stage device time of one batch launch and of the 48 single renders
    stage_ms = {}
    for name, fn in (("batch", b.launch), ("one_call_per_job", one_by_one)):
        cc.cicero_profile_begin()
        fn()
        torch.cuda.synchronize()
        stage_ms[name] = {k: round(v[0], 3) for k, v in cc.cicero_profile_end().items() if v[1]}
    # oracle check on sampled pixels of every job (outputs of the last batch replay)
    graph.replay()
    torch.cuda.synchronize()
    oracle.build()
    worst, sq, n = 0.0, 0.0, 0
    for j, (si, c, _) in enumerate(specs):
        R = c.width * c.height
        pix = (scenes.splitmix64(9000 + j, n_check) % np.uint64(R)).astype(np.int32)
        ref = oracle.render(sc[si][0], sc[si][1], c.sampling, cam=c, pix=pix)
        got = outs[j][0].cpu().double().numpy()[pix]
        e = np.where(ref["amb"][:, None], np.minimum(np.abs(got - ref["rgb"]), np.abs(got - ref["rgb_alt"])),
                     np.abs(got - ref["rgb"]))
        worst = max(worst, float(e.max()))
        sq += float((e ** 2).sum())
        n += e.size
    del graph
    b.close()
    return {"workload": f"{BATCH_JOBS} jobs: grids 96^3..256^3 x 12 FP16 (6 scenes, own MLPs), images 256^2..1024^2, "
                        "64..256 samples per ray", "rays": rays, "composited_samples": samples,
            "brick": brick, "mlp_groups": groups,
            "autotune_ms": {f"brick{k[0]}_groups{k[1]}": v for k, v in tune.items() if v > 0},
            "batch_ms": t_batch,
            "jobs_per_s": BATCH_JOBS / (t_batch / 1e3), "msamples_per_s": samples / (t_batch / 1e3) / 1e6,
            "one_call_per_job_ms": t_single, "speedup_vs_one_call_per_job": t_single / t_batch,
            "launch": "one CUDA graph (10 kernels for all jobs)", "record_capacity": cap, "stage_ms": stage_ms,
            "oracle_check": {"pixels": n // 3, "max_err": worst, "psnr_db": 10 * math.log10(1.0 / max(sq / n, 1e-30))}}


SWEEP_WINDOWS = (6, 16, 21, 26, 30)
SWEEP_FRAMES = 120


def window_sweep(cc, torch, dev, grid, mlp, o16, sampling=None, label=None):
    """SpaRW over a 120-frame trajectory on the 800x800 scene (the camera orbits the object at
    0.5 deg of azimuth per frame, looking at it: a 60 deg arc) with the reference of each window
    rendered on a second stream (cicero_pipeline, Sec. III-C), for windows of 6 .. 30 targets (the
    paper's window sizes).  Per window size: frames/s overlapped and serialised, speedup over
    rendering every frame in full (BF16), and PSNR of the frames against those full renders (every
    pixel; a frame identical to its full render counts as 100 dB in the mean)."""
    import scenes
    cam = scenes.orbit_camera(W, H, sampling=sampling or scenes.sampling_march(256, 256))
    traj = [scenes.orbit_camera(W, H, az_deg=30.0 + 0.5 * k, sampling=cam.sampling) for k in range(SWEEP_FRAMES)]
    targets = [cc.camera_from(t) for t in traj]
    R = W * H
    cd, sd = cc.camera_from(cam), cc.sampling_from(cam.sampling)
    # every frame rendered in full: the speed and the image the warped frames are compared with
    full = [torch.empty(R, 3, device=dev) for _ in traj]
    fd = torch.empty(R, device=dev)
    ws_f = cc.workspace(cc.cicero_render_workspace_size(grid.desc, R, sd, o16), dev)

    def render_all():
        for t, out in zip(targets, full):
            cc.cicero_render(grid.desc, mlp.desc, t, sd, o16, out, fd, None, None, ws_f)

    t_full = event_ms(torch, render_all, 1)
    del ws_f
    # DS-2: every frame rendered at half resolution (f, cx, cy halved), then upsampled bilinearly
    w2, h2 = W // 2, H // 2
    half = [cc.camera(w2, h2, t.f / 2, t.cx / 2, t.cy / 2, np.array(t.c2w[:], np.float32).reshape(3, 4))
            for t in targets]
    lo_rgb, lo_d = torch.empty(w2 * h2, 3, device=dev), torch.empty(w2 * h2, device=dev)
    ds2 = [torch.empty(R, 3, device=dev) for _ in traj]
    ws_h2 = cc.workspace(cc.cicero_render_workspace_size(grid.desc, w2 * h2, sd, o16), dev)

    def ds2_all():
        for t, out in zip(half, ds2):
            cc.cicero_render(grid.desc, mlp.desc, t, sd, o16, lo_rgb, lo_d, None, None, ws_h2)
            cc.cicero_upsample_bilinear(lo_rgb, w2, h2, out, W, H)

    t_ds2 = event_ms(torch, ds2_all, 1)
    del ws_h2
    p2 = np.minimum([frame_psnr(a.cpu().numpy(), b.cpu().numpy()) for a, b in zip(ds2, full)], 100.0)
    ds2_res = {"fps": SWEEP_FRAMES / (t_ds2 / 1e3), "speedup_vs_full": t_full / t_ds2,
               "psnr_db_mean": float(np.mean(p2)), "psnr_db_median": float(np.median(p2)),
               "psnr_db_min": float(np.min(p2))}
    del ds2
    frames = [torch.empty(R, 3, device=dev) for _ in traj]
    s_ref = torch.cuda.Stream(dev)
    res = {"frames": SWEEP_FRAMES, "full_render_fps": SWEEP_FRAMES / (t_full / 1e3), "ds2": ds2_res, "windows": []}
    if label:
        res["scene"] = label
    for N, lead in [(n, "centred") for n in SWEEP_WINDOWS] + [(16, "paper")]:
        hole_records = N * R * 40  # ~16% of the window's slots
        ws = cc.workspace(cc.cicero_pipeline_workspace_size(grid.desc, cd, sd, o16, N, hole_records), dev)
        p = cc.Pipeline(grid.desc, mlp.desc, cd, sd, o16, N, hole_records, 180.0, ws)

        def run(overlap):
            cur = torch.cuda.current_stream(dev)
            s_ref.wait_stream(cur)
            p.run(targets, frames, None, lead=lead, stream_tgt=cur, stream_ref=s_ref if overlap else cur)

        t_ov = event_ms(torch, lambda: run(True), 2)
        t_se = event_ms(torch, lambda: run(False), 2)
        p.status()
        ps = np.minimum([frame_psnr(a.cpu().numpy(), b.cpu().numpy()) for a, b in zip(frames, full)], 100.0)
        res["windows"].append({"window": N, "lead": lead, "fps_overlapped": SWEEP_FRAMES / (t_ov / 1e3),
                               "fps_serialised": SWEEP_FRAMES / (t_se / 1e3),
                               "speedup_vs_full": t_full / t_ov, "psnr_db_mean": float(np.mean(ps)),
                               "psnr_db_median": float(np.median(ps)), "psnr_db_min": float(np.min(ps))})
        p.close()
        del ws
    return res


PHI_SWEEP = (180.0, 8.0, 4.0, 2.0, 1.0)


def phi_sweep(cc, torch, dev, grid, o16, ref_samples):
    """The warp-angle heuristic (Sec. III-C "Deciding When to Warp"): a point is warped only when
    the angle between its reference and target rays is below phi.  On the headline window (16
    targets around the reference) with a strongly view-dependent MLP (the weights of the direction
    encoding scaled by 6), per phi: fraction of target rays marched, target frames/s and PSNR of
    the targets against their full renders (every pixel)."""
    import scenes
    m = scenes.make_mlp(12, seed=4242)
    m.w1[:, 12:] *= 6.0
    mlp = cc.DeviceMlp.from_host(m, dev)
    cam = scenes.orbit_camera(W, H, sampling=scenes.sampling_march(256, 256))
    targets = [scenes.offset_camera(cam, k) for k in scenes.SPARW_OFFSETS]
    R, sd = W * H, cc.sampling_from(cam.sampling)
    full = torch.empty(len(targets), R, 3, device=dev)
    fd = torch.empty(R, device=dev)
    ws_f = cc.workspace(cc.cicero_render_workspace_size(grid.desc, R, sd, o16), dev)
    for i, t in enumerate(targets):
        cc.cicero_render(grid.desc, mlp.desc, cc.camera_from(t), sd, o16, full[i], fd, None, None, ws_f)
    del ws_f
    # a small phi turns almost every target pixel into a hole: room for all of them
    ob = cc.options(cc.MLP_BF16, o16.brick, max_records=min(int(1.3 * len(targets) * ref_samples), 4_000_000_000))
    out = []
    for phi in PHI_SWEEP:
        win = SparwWindow(cc, torch, dev, grid, mlp, cam, targets, o16, ob, max_angle_deg=phi)
        t = event_ms(torch, win.run, 3)
        win.check()
        ps = np.minimum([frame_psnr(win.t_rgb[i].cpu().numpy(), full[i].cpu().numpy()) for i in range(len(targets))],
                        100.0)
        out.append({"phi_deg": phi, "fraction_marched": float(win.nh.sum().item()) / (len(targets) * R),
                    "target_fps": len(targets) / (t / 1e3), "psnr_db_mean": float(np.mean(ps)),
                    "psnr_db_min": float(np.min(ps))})
        del win
    return {"mlp": "direction-encoding weights x 6", "window": "16 targets, 1..8 deg yaw + 5 mm steps", "phi": out}


def hash_workload(cc, torch, dev, grid, g_h, reps=5):
    """The hash-grid workload (Sec. IV-A, hierarchical encodings; Instant-NGP-like): the 800x800
    frame of the 256^3 scene (its density and occupancy) with the colour features from a
    multiresolution hash encoding of 8 levels x 2 FP16 features, 2^19 entries per level, 16 .. 1024
    cells per axis; BF16 MLP 43 -> 128 -> 128 -> 3.  Frames/s, Msamples/s, the tensor roofline of
    the gather kernel, and the oracle on 256 sampled pixels."""
    import oracle
    import scenes
    h = scenes.make_hash_grid(8, 2, 19, 16, 1024, seed=777)
    m = scenes.make_mlp(16, seed=778)
    hd, md = cc.DeviceHashGrid.from_host(h, dev), cc.DeviceMlp.from_host(m, dev)
    cam = scenes.orbit_camera(W, H, sampling=scenes.sampling_march(256, 256))
    cd, sd = cc.camera_from(cam), cc.sampling_from(cam.sampling)
    R = W * H
    rgb, dep = torch.empty(R, 3, device=dev), torch.empty(R, device=dev)
    best = None
    for brick in (4, 8):
        opt = cc.options(cc.MLP_BF16, brick)
        ws = cc.workspace(cc.cicero_render_hash_workspace_size(grid.desc, hd.desc, R, sd, opt), dev)
        t = event_ms(torch, lambda: cc.cicero_render_hash(grid.desc, hd.desc, md.desc, cd, sd, opt, rgb, dep, ws), reps)
        cc.cicero_workspace_status(ws)
        if best is None or t < best[0]:
            best = (t, brick, ws, opt)
    t, brick, ws, opt = best
    samples = int(ws[:16].view(torch.int32).cpu().numpy()[2])
    cc.cicero_profile_begin()
    cc.cicero_render_hash(grid.desc, hd.desc, md.desc, cd, sd, opt, rgb, dep, ws)
    torch.cuda.synchronize()
    prof = cc.cicero_profile_end()
    g_ms = prof["gather_mlp"][0] / max(prof["gather_mlp"][1], 1)
    flop = 2 * (m.in_dim * 128 + 128 * 128 + 128 * 3) * samples
    pk = peaks()
    oracle.build()
    pix = (scenes.splitmix64(3131, 256) % np.uint64(R)).astype(np.int32)
    ref = oracle.render(scenes.with_hash(g_h, h), m, cam.sampling, cam=cam, pix=pix)
    got = rgb.cpu().double().numpy()[pix]
    e = np.where(ref["amb"][:, None], np.minimum(np.abs(got - ref["rgb"]), np.abs(got - ref["rgb_alt"])),
                 np.abs(got - ref["rgb"]))
    return {"workload": "800x800, 256^3 density + 32^3 occupancy, hash encoding 8 levels x 2 FP16, 2^19 entries, "
                        "16..1024 cells", "brick": brick, "fps": 1e3 / t, "msamples_per_s": samples / t / 1e3,
            "composited_samples": samples, "stages_ms": {k: round(v[0], 3) for k, v in prof.items() if v[1]},
            "gather_mlp_tflops": flop / (g_ms / 1e3) / 1e12,
            "gather_mlp_frac": flop / (g_ms / 1e3) / 1e12 / pk["bf16_tflops_sustained"],
            "oracle_check": {"pixels": 256, "max_err": float(e.max()),
                             "psnr_db": 10 * math.log10(1.0 / max(float(np.mean(e ** 2)), 1e-30))}}


def backward_workload(cc, torch, dev):
    """Forward + backward over 8192 random rays x 256 samples on the 160^3 x 12 FP32 scene, MSE
    loss against seeded target colours (the differentiation workload)."""
    import scenes
    g, m = scenes.scene_backward(), scenes.make_mlp(12)
    R = 8192
    o, d = scenes.random_rays(R)
    sp = scenes.Sampling(near=0.5, far=2.5, n_samples=256, t_stop=1e-3)
    gd, md, sd = cc.DeviceGrid.from_host(g, dev), cc.DeviceMlp.from_host(m, dev), cc.sampling_from(sp)
    ot, dt = torch.from_numpy(o).to(dev), torch.from_numpy(d).to(dev)
    tgt = torch.from_numpy(scenes.random_targets(R)).to(dev)
    rgb, depth = torch.empty(R, 3, device=dev), torch.empty(R, device=dev)
    d_rgb = torch.empty(R, 3, device=dev)
    dd, df = torch.zeros(g.density.shape, device=dev), torch.zeros(g.features.shape, device=dev)
    opt = cc.options(cc.MLP_FP32, 8)
    ws_f = cc.workspace(cc.cicero_render_workspace_size(gd.desc, R, sd, opt), dev)
    ws_b = cc.workspace(cc.cicero_backward_workspace_size(gd.desc, R, sd), dev)
    # with the MLP weight gradients: the workspace that holds their staged operands (tensor-core
    # GEMMs); the smaller one above takes them on the CUDA cores
    ws_bm = cc.workspace(cc.cicero_backward_mlp_workspace_size(gd.desc, R, sd), dev)

    def fwd(o=opt):
        cc.cicero_render_rays(gd.desc, md.desc, ot, dt, sd, o, rgb, depth, None, None, ws_f)

    dm = torch.zeros(m.flat().size, device=dev)

    def bwd(d_mlp=None, ws=None):
        torch.sub(rgb, tgt, out=d_rgb).mul_(2.0 / rgb.numel())  # dL/drgb of the MSE loss
        cc.cicero_render_backward(gd.desc, md.desc, ot, dt, sd, d_rgb, dd, df, d_mlp, ws_b if ws is None else ws)

    fwd()
    t_f = event_ms(torch, fwd, 5)
    # the same forward with the FP32-class tensor-core MLP (split BF16; bricks of 16, as the
    # backward's plan: its kernels read features from global memory, so bigger bricks only make
    # fuller tiles), then the FP32 one again, whose colours feed the loss gradient
    t_fs = event_ms(torch, lambda: fwd(cc.options(cc.MLP_FP32_SPLIT, 16)), 5)
    fwd()
    t_b = event_ms(torch, bwd, 5)
    t_bm = event_ms(torch, lambda: bwd(dm, ws_bm), 5)
    t_bm_simt = event_ms(torch, lambda: bwd(dm), 5)
    cc.cicero_workspace_status(ws_f)
    cc.cicero_workspace_status(ws_b)
    hdr = ws_b[:32].view(torch.int32).cpu().numpy()
    samples = int(hdr[2])  # composited samples of the recompute
    fixed = int(hdr[4])    # of which recomputed in FP32 (uncertain split-BF16 ReLU decisions)
    # per-stage device time of one backward call without and with the MLP weight gradients
    stage = {}
    for name, arg, ws in (("grid", None, None), ("grid_and_mlp", dm, ws_bm), ("grid_and_mlp_cuda_cores", dm, None)):
        torch.cuda.synchronize()
        cc.cicero_profile_begin()
        for _ in range(5):
            bwd(arg, ws)
        torch.cuda.synchronize()
        p = cc.cicero_profile_end()
        stage[name] = {k: p[k][0] / 5 for k in ("march", "bucket", "gather_mlp", "composite", "bwd_ray", "bwd_brick",
                                                "bwd_weights")}
    # B2 without the weight gradients (k_bwd_brick_tc): the tensor-core GEMMs dL/dh1 = dL/dh2 W2 and
    # dL/dfeatures = dL/dh1 W1[:, :C] per composited sample, algorithmic 2 (H H + C H) FLOP, executed
    # as three split-BF16 products with the feature channels padded to N = 16, against the measured
    # sustained BF16 peak.  With the weight gradients on the CUDA cores (k_bwd_brick): recomputed layers
    # 1-2, dL/dh2, dL/dh1, dL/dfeatures, dW3, dW2, dW1 against the FP32 FFMA peak derived from the
    # SM count, 128 FP32 lanes per SM, 2 FLOP per FMA and the 2070 MHz maximum clock
    C, H, I = 12, 128, m.w1.shape[1]
    pk = peaks()
    flop_tc = 2 * (H * H + C * H)
    flop_tc_exec = 3 * 2 * H * (H + 16)
    flop_w = 2 * (I * H + H * H + 3 * H + H * H + C * H) + 2 * (3 * H + H * H + I * H)
    fp32_peak = torch.cuda.get_device_properties(0).multi_processor_count * 128 * 2 * 2.07e9 / 1e12
    roof = {}
    t = stage["grid"]["bwd_brick"] / 1e3
    ach = flop_tc * samples / t / 1e12 if t > 0 else 0.0
    roof["grid"] = {"kernel": "k_bwd_brick_tc", "bound": "tensor", "flop_per_sample": flop_tc,
                    "executed_mma_flop_per_sample": flop_tc_exec, "achieved": ach,
                    "peak": pk["bf16_tflops_sustained"], "unit": "TFLOP/s", "frac": ach / pk["bf16_tflops_sustained"],
                    "executed_tflops": flop_tc_exec * samples / t / 1e12 if t > 0 else 0.0,
                    "peak_src": "measured (sustained bf16)"}
    # with the weight gradients on the tensor cores: k_bwd_brick_tc also stages dL/dh2, dL/dh1 and dL/dz3
    # (same FLOPs, tensor roofline), then k_dw reads every staged block once (per 16 samples 36,352
    # bytes of split-BF16 operand rows: x, h1, h2 written by the recompute, the three gradients by the
    # grid kernel) and forms the weight gradients (dW2 | db2, dW1 | db1, dW3 | db3) as tensor-core GEMMs
    # over the samples: HBM roofline on the staged bytes against the measured copy bandwidth, the
    # GEMMs' algorithmic rate beside it
    t = stage["grid_and_mlp"]["bwd_brick"] / 1e3
    ach = flop_tc * samples / t / 1e12 if t > 0 else 0.0
    roof["grid_staging"] = {"kernel": "k_bwd_brick_tc (staging the weight-gradient operands)", "bound": "tensor",
                            "flop_per_sample": flop_tc, "achieved": ach, "peak": pk["bf16_tflops_sustained"],
                            "unit": "TFLOP/s", "frac": ach / pk["bf16_tflops_sustained"],
                            "peak_src": "measured (sustained bf16)"}
    flop_dw = 2 * (H * (H + 1) + H * (I + 1) + 3 * H)
    stage_bytes = 36352 / 16
    t = stage["grid_and_mlp"]["bwd_weights"] / 1e3
    ach = stage_bytes * samples / t / 1e9 if t > 0 else 0.0
    roof["weights"] = {"kernel": "k_dw", "bound": "hbm", "bytes_per_sample": stage_bytes, "achieved": ach,
                       "peak": pk["hbm_gbs"], "unit": "GB/s", "frac": ach / pk["hbm_gbs"],
                       "peak_src": "measured (copy)", "flop_per_sample": flop_dw,
                       "tflops": flop_dw * samples / t / 1e12 if t > 0 else 0.0}
    t = stage["grid_and_mlp_cuda_cores"]["bwd_brick"] / 1e3
    ach = flop_w * samples / t / 1e12 if t > 0 else 0.0
    roof["grid_and_mlp_cuda_cores"] = {"kernel": "k_bwd_brick (weight gradients, CUDA cores)", "bound": "alu",
                                       "flop_per_sample": flop_w, "achieved": ach, "peak": fp32_peak,
                                       "unit": "TFLOP/s", "frac": ach / fp32_peak,
                                       "peak_src": "derived: SMs x 128 FP32 lanes x 2 x 2070 MHz"}
    return {"workload": "8192 rays x 256 samples, 160^3 x 12 FP32 grid, MSE loss", "forward_ms": t_f,
            "forward_split_bf16_ms": t_fs, "backward_ms": t_b, "backward_with_mlp_weights_ms": t_bm,
            "backward_with_mlp_weights_cuda_cores_ms": t_bm_simt,
            "rays_per_s_fwd_bwd": R / ((t_f + t_b) / 1e3),
            "rays_per_s_fwd_bwd_split_forward": R / ((t_fs + t_b) / 1e3), "composited_samples": samples,
            "fp32_recomputed_samples": fixed,
            "stage_ms": stage, "k_bwd_brick_roofline": roof,
            "grad_bytes": int(dd.numel() * 4 + df.numel() * 4)}


def plain_small(cc, torch, dev):
    """Config 1: a plain render of the 64^3 scene, 64x64 pixels, 64 uniform samples, FP32 and BF16
    MLP; device ms per frame (CUDA events, 20 renders) and the error of every pixel against the FP64
    oracle (the better outcome on the rays whose early stop is ambiguous)."""
    import oracle
    import scenes
    g, m = scenes.scene_small(), scenes.make_mlp(12)
    cam = scenes.orbit_camera(64, 64, sampling=scenes.sampling_uniform(64))
    gd, md = cc.DeviceGrid.from_host(g, dev), cc.DeviceMlp.from_host(m, dev)
    sd, cd = cc.sampling_from(cam.sampling), cc.camera_from(cam)
    R = 64 * 64
    t0 = time.perf_counter()
    ref = oracle.render(g, m, cam.sampling, cam=cam)
    t_oracle = time.perf_counter() - t0
    out = {"workload": "64^3 x 12 FP32 scene (8 blobs), 64x64, 64 uniform samples in [0.5, 2.5], t_stop 1e-3",
           "ambiguous_rays": int(ref["amb"].sum()),
           "oracle": {"ms": t_oracle * 1e3, "cores": oracle.max_threads(), "kind": "FP64, every pixel"}}
    for name, prec in (("fp32", cc.MLP_FP32), ("bf16", cc.MLP_BF16)):
        opt = cc.options(prec, 8)
        ws = cc.workspace(cc.cicero_render_workspace_size(gd.desc, R, sd, opt), dev)
        rgb, depth = torch.empty(R, 3, device=dev), torch.empty(R, device=dev)

        def render():
            cc.cicero_render(gd.desc, md.desc, cd, sd, opt, rgb, depth, None, None, ws)

        ms = event_ms(torch, render, 20)
        cc.cicero_workspace_status(ws)
        got = rgb.cpu().double().numpy()
        e = np.where(ref["amb"][:, None], np.minimum(np.abs(got - ref["rgb"]), np.abs(got - ref["rgb_alt"])),
                     np.abs(got - ref["rgb"]))
        out[name] = {"ms": ms, "max_err": float(e.max()),
                     "psnr_db": 10 * math.log10(1.0 / max(float(np.mean(e ** 2)), 1e-30))}
    return out


def tuned_bf16_brick(cc, torch, dev, gd, md, cam):
    """The BF16 brick the library's autotuner picks for this scene's reference frame (timed renders),
    with the times it measured per brick."""
    R = cam.width * cam.height
    sd, cd = cc.sampling_from(cam.sampling), cc.camera_from(cam)
    ws = cc.workspace(cc.cicero_render_workspace_size(gd.desc, R, sd, cc.options(cc.MLP_BF16, 4)), dev)
    rgb, depth = torch.empty(R, 3, device=dev), torch.empty(R, device=dev)
    b, tune = cc.cicero_autotune_brick(gd.desc, md.desc, cd, sd, cc.MLP_BF16, rgb, depth, ws)
    del ws, rgb, depth
    return b, tune


def sparw_small_scene(cc, torch, dev, n_pix=1024, opaque=False):
    """SpaRW on the 64^3 scene: reference 800x800 at the orbit pose (64 uniform samples), 16 targets
    warped and hole-rendered (BF16 MLP).  Per target: fraction of rays marched and PSNR against
    the FP64 oracle's full render of the target on n_pix sampled pixels (SpaRW's approximation
    error, not gated); the window's device time.  opaque: the blobs scaled to opaque surfaces."""
    import oracle
    import scenes
    g = scenes.scene_small_opaque() if opaque else scenes.scene_small()
    m = scenes.make_mlp(12)
    cam = scenes.orbit_camera(W, H, sampling=scenes.sampling_uniform(64))
    targets = [scenes.offset_camera(cam, k) for k in scenes.SPARW_OFFSETS]
    R, n_t = W * H, len(targets)
    gd, md = cc.DeviceGrid.from_host(g, dev), cc.DeviceMlp.from_host(m, dev)
    brick, tune = tuned_bf16_brick(cc, torch, dev, gd, md, cam)
    opt = cc.options(cc.MLP_BF16, brick)
    opt_h = cc.options(cc.MLP_BF16, brick, max_records=120_000_000)  # holes are ~10% of the pixels
    win = SparwWindow(cc, torch, dev, gd, md, cam, targets, opt, opt_h)
    t_win = event_ms(torch, win.run, 5)
    win.check()
    t_rgb, nh = win.t_rgb, win.nh
    oracle.build()
    holes = nh.view(-1).cpu().numpy()
    per = []
    for i, tgt in enumerate(targets):
        pix = (scenes.splitmix64(5000 + i, n_pix) % np.uint64(R)).astype(np.int32)
        ref = oracle.render(g, m, cam.sampling, cam=tgt, pix=pix)
        got = t_rgb[i].cpu().double().numpy()[pix]
        e = np.where(ref["amb"][:, None], np.minimum(np.abs(got - ref["rgb"]), np.abs(got - ref["rgb_alt"])),
                     np.abs(got - ref["rgb"]))
        mse = float(np.mean(e ** 2))
        per.append({"k": scenes.SPARW_OFFSETS[i], "fraction_marched": float(holes[i]) / R,
                    "psnr_db": 10 * math.log10(1.0 / max(mse, 1e-30)), "max_err": float(e.max())})
    disocc, void = win.classify()
    for i, p in enumerate(per):
        p.update({"disocclusion_holes": int(disocc[i]), "void_holes": int(void[i]),
                  "fraction_void": float(void[i]) / R})
    scene = (f"opaque surfaces (blob amplitudes x {scenes.OPAQUE_AMP_SCALE:g}: rays stop within a sample or two "
             f"of a blob, the expected depth is a surface)" if opaque
             else "fog-like blobs (amplitudes U[10, 40]: ~50 composited samples per ray)")
    return {"workload": "64^3 x 12 FP32 scene, 800x800, 64 samples, 16 targets (1 deg yaw + 5 mm apart)",
            "scene": scene, "brick": brick, "autotune_ms": tune,
            "window_ms": t_win, "target_fps": n_t / (t_win / 1e3), "psnr_pixels_per_target": n_pix,
            "psnr_db_min": min(p["psnr_db"] for p in per), "fraction_marched_mean": float(holes.sum()) / (n_t * R),
            "marched": "disocclusion and void holes (a void hole's march composites nothing)", "targets": per}


# ---------------------------------------------------------------------------------------------
# GPU leg


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.case == "small":
        return small_case(args.brick)
    if args.case == "backward":
        import torch
        from paper_2404_11852_gb300 import build, cicero as cc
        build.build()
        cc.lib()
        print(json.dumps({"case": "backward", **backward_workload(cc, torch, "cuda")}), flush=True)
        return None

    import torch
    import torch.distributed as dist
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    import scenes
    from paper_2404_11852_gb300 import build, cicero as cc
    build.build()

    g_h, m_h = scenes.scene_large(), scenes.make_mlp(12)
    grid = cc.DeviceGrid.from_host(g_h)
    mlp = cc.DeviceMlp.from_host(m_h)
    cam = scenes.orbit_camera(W, H, az_deg=rank_azimuth(rank), sampling=scenes.sampling_march(256, 256))
    targets = [scenes.offset_camera(cam, k) for k in scenes.SPARW_OFFSETS]
    R = W * H
    sd = cc.sampling_from(cam.sampling)
    cd = cc.camera_from(cam)
    dev = torch.device("cuda", local)
    # brick size per precision, picked by the library's autotuner (timed renders of this frame)
    tune_bytes = cc.cicero_render_workspace_size(grid.desc, R, sd, cc.options(cc.MLP_BF16, 4))
    ws_t = cc.workspace(tune_bytes, dev)
    ref_rgb, ref_depth = torch.empty(R, 3, device=dev), torch.empty(R, device=dev)
    b16, tune16 = cc.cicero_autotune_brick(grid.desc, mlp.desc, cd, sd, cc.MLP_BF16, ref_rgb, ref_depth, ws_t)
    b32, tune32 = cc.cicero_autotune_brick(grid.desc, mlp.desc, cd, sd, cc.MLP_FP32, ref_rgb, ref_depth, ws_t)
    bsp, tunesp = cc.cicero_autotune_brick(grid.desc, mlp.desc, cd, sd, cc.MLP_FP32_SPLIT, ref_rgb, ref_depth, ws_t)
    del ws_t, ref_rgb, ref_depth
    o16, o32 = cc.options(cc.MLP_BF16, b16), cc.options(cc.MLP_FP32, b32)
    o_split = cc.options(cc.MLP_FP32_SPLIT, bsp)  # FP32-class MLP on the tensor cores (split BF16)
    # all targets' holes are rendered in one batched pass; records are capped well above need
    ob = cc.options(cc.MLP_BF16, b16, max_records=HOLE_RECORDS)
    win = SparwWindow(cc, torch, dev, grid, mlp, cam, targets, o16, ob,
                      ref_ws_bytes=cc.cicero_render_workspace_size(grid.desc, R, sd, o32))
    t_rgb, nh = win.t_rgb, win.nh
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)  # > 129 MB L2
    step = win.run

    def full(opt):
        win.render_reference(opt)

    def timed(fn, steps, warmup, host_io=None):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        total = 0.0
        for _ in range(steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            fn()
            if host_io:
                host_io()
            e1.record()
            torch.cuda.synchronize()
            total += e0.elapsed_time(e1) / 1e3
        return max_over_ranks(total, dev)

    # headline: SpaRW windows, device-resident inputs
    launches0 = cc.cicero_launch_count()
    with ClockSampler(local) as clk:
        t_main = timed(step, args.steps, args.warmup)
    launches = (cc.cicero_launch_count() - launches0) / (args.steps + args.warmup)
    win.check()
    hole_hdr = win.header(win.ws_h)
    value = job_value(N_TARGETS, args.steps, world, t_main)
    holes = nh.sum().item()

    # end to end: the same step with its result (16 target frames) read back to pinned host memory
    host_out = torch.empty(N_TARGETS, R, 3, dtype=torch.float32, pin_memory=True)
    pose_h = torch.from_numpy(np.stack([t.c2w for t in targets] + [cam.c2w]).astype(np.float32)).pin_memory()

    def d2h():
        host_out.copy_(t_rgb, non_blocking=True)

    def step_e2e():
        # poses come from pinned host memory (they are passed to the kernels by value)
        p = pose_h.numpy()
        for i, td in enumerate(win.tds):
            td.c2w[:] = [float(v) for v in p[i].reshape(-1)]
        step()

    t_e2e_serial = timed(step_e2e, args.steps, 1, host_io=d2h)

    # the same windows streamed: window i's frames are copied to pinned host memory on a copy
    # stream while window i+1 computes into the other frame buffer; every window's result is read
    # back inside the timed region (no L2 flush between windows: the grid and the records they
    # stream are larger than L2)
    frames = [t_rgb, torch.empty_like(t_rgb)]
    hosts = [host_out, torch.empty(N_TARGETS, R, 3, dtype=torch.float32, pin_memory=True)]
    copier = torch.cuda.Stream(dev)

    def streamed(steps):
        done = [None, None]
        for i in range(steps):
            b = i & 1
            if done[b] is not None:
                torch.cuda.current_stream().wait_event(done[b])  # window i-2's copy has read this buffer
            win.set_frames(frames[b])
            step_e2e()
            ready = torch.cuda.Event()
            ready.record()
            copier.wait_event(ready)
            with torch.cuda.stream(copier):
                hosts[b].copy_(frames[b], non_blocking=True)
            done[b] = torch.cuda.Event()
            done[b].record(copier)
        for ev in done:
            if ev is not None:
                torch.cuda.current_stream().wait_event(ev)

    streamed(2)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    streamed(args.steps)
    e1.record()
    torch.cuda.synchronize()
    t_e2e = max_over_ranks(e0.elapsed_time(e1) / 1e3, dev)
    win.set_frames(frames[0])
    e2e_value = job_value(N_TARGETS, args.steps, world, t_e2e)
    e2e_serial = job_value(N_TARGETS, args.steps, world, t_e2e_serial)

    # the plain FP32 full render and the BF16 full render of the same frame
    n_fp = max(2, args.steps)
    t_fp32 = timed(lambda: full(o32), n_fp, 1)
    hdr = win.header(win.ws_r)
    active = int(hdr[2])
    t_bf16 = timed(lambda: full(o16), n_fp, 1)
    t_split = timed(lambda: full(o_split), n_fp, 1)
    # marched slots of the frame: per pixel, the slot where its march stopped (or its last valid
    # slot), from one more render outside the timed regions
    n_steps = torch.empty(R, dtype=torch.int32, device=dev)
    cc.cicero_render(grid.desc, mlp.desc, cd, sd, o16, win.ref_rgb, win.ref_depth, None, n_steps, win.ws_r)
    marched = int(n_steps.sum().item())
    del n_steps

    # per-stage device time (CUDA events on the launching stream) over two profiled windows
    cc.cicero_profile_begin()
    for _ in range(2):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    prof = cc.cicero_profile_end()
    cc.cicero_profile_begin()
    full(o16)
    torch.cuda.synchronize()
    prof_ref = cc.cicero_profile_end()

    pk = peaks()
    g_ms, g_n = prof_ref["gather_mlp"]
    t_launch = g_ms / max(g_n, 1) / 1e3
    achieved = FLOP_PER_SAMPLE * active / t_launch / 1e12
    roof = {"kernel": "k_gather_mlp_bf16 (reference frame)", "bound": "tensor", "achieved": achieved,
            "peak": pk["bf16_tflops_sustained"], "unit": "TFLOP/s", "frac": achieved / pk["bf16_tflops_sustained"],
            "traffic": gather_traffic(), "peak_src": f"{pk['src']} (sustained bf16)",
            "flop_per_launch": FLOP_PER_SAMPLE * active}
    if gather_traffic() is not None:
        # the shared-memory bound: one 128-byte wavefront per clock per SM
        n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
        t_smem = GATHER_SMEM_WAVEFRONTS_PER_SAMPLE * active / (n_sm * pk["sm_max_mhz"] * 1e6)
        roof["shared_memory"] = {"wavefronts_per_sample": GATHER_SMEM_WAVEFRONTS_PER_SAMPLE,
                                 "bound_ms": t_smem * 1e3, "frac": t_smem / t_launch}
        # the same launch against the HBM roofline: its DRAM bytes (ncu, above) over its event time
        hbm = gather_traffic() / t_launch / 1e9
        roof["hbm"] = {"achieved": hbm, "peak": pk["hbm_gbs"], "unit": "GB/s", "frac": hbm / pk["hbm_gbs"]}
    stages = {k: {"ms_per_step": v[0] / 2, "launches_per_step": v[1] / 2} for k, v in prof.items() if v[1]}
    stage_roof = stage_roofline(stages, pk, R, int(holes), active, int(hole_hdr[2]))

    # quality: reference frame (BF16) vs the FP64 oracle on sampled pixels, and the cpu baseline
    cpu = None
    quality = {}
    if rank == 0 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        pix = (scenes.splitmix64(777, 256) % np.uint64(R)).astype(np.int32)
        full(o16)
        got = win.ref_rgb.cpu().double().numpy()[pix]
        ref = oracle.render(g_h, m_h, cam.sampling, cam=cam, pix=pix)
        e = np.where(ref["amb"][:, None], np.minimum(np.abs(got - ref["rgb"]), np.abs(got - ref["rgb_alt"])),
                     np.abs(got - ref["rgb"]))
        quality = {"ref_bf16_max_err": float(e.max()),
                   "ref_bf16_psnr_db": float(10 * math.log10(1.0 / max(float(np.mean(e ** 2)), 1e-30))),
                   "sample_pixels": int(len(pix))}
        full(o32)
        got = win.ref_rgb.cpu().double().numpy()[pix]
        e = np.where(ref["amb"][:, None], np.minimum(np.abs(got - ref["rgb"]), np.abs(got - ref["rgb_alt"])),
                     np.abs(got - ref["rgb"]))
        quality["ref_fp32_max_err"] = float(e.max())
        full(o_split)
        got = win.ref_rgb.cpu().double().numpy()[pix]
        e = np.where(ref["amb"][:, None], np.minimum(np.abs(got - ref["rgb"]), np.abs(got - ref["rgb_alt"])),
                     np.abs(got - ref["rgb"]))
        quality["ref_fp32_split_max_err"] = float(e.max())
        frames = []
        dt, cores, _ = oracle_window(args.cpu_res, rank, frames)
        quality["sparw_bf16_vs_oracle_sparw"] = sparw_parity(cc, torch, dev, grid, mlp, args.cpu_res, rank, frames,
                                                             o16)
        scale = R / (args.cpu_res ** 2)
        cpu = {"value": N_TARGETS / (dt * scale), "unit": "frames/s", "cores": cores, "kind": "oracle",
               "sample": f"whole SpaRW window at {args.cpu_res}x{args.cpu_res} ({args.cpu_res**2} of {R} pixels "
                         f"per frame, FP64), time x {scale:.0f}",
               "threads": oracle_threads(g_h, m_h, cam, R)}

    others = {}
    if rank == 0 and not args.no_extra:
        others["config_backward"] = backward_workload(cc, torch, dev)
        others["config_plain_64"] = plain_small(cc, torch, dev)
        others["config_sparw_small_scene"] = sparw_small_scene(cc, torch, dev)
        others["config_sparw_opaque_scene"] = sparw_small_scene(cc, torch, dev, opaque=True)
        others["config_batched"] = batched_workload(cc, torch, dev)
        others["sparw_window_sweep"] = window_sweep(cc, torch, dev, grid, mlp, o16)
        g_op = cc.DeviceGrid.from_host(scenes.scene_small_opaque(), dev)
        m_op = cc.DeviceMlp.from_host(scenes.make_mlp(12), dev)
        b_op, _ = tuned_bf16_brick(cc, torch, dev, g_op, m_op,
                                   scenes.orbit_camera(W, H, sampling=scenes.sampling_uniform(64)))
        others["sparw_window_sweep_opaque_scene"] = window_sweep(
            cc, torch, dev, g_op, m_op, cc.options(cc.MLP_BF16, b_op),
            sampling=scenes.sampling_uniform(64), label=f"64^3 opaque-surface scene, 64 uniform samples, brick {b_op}")
        del g_op, m_op
        others["sparw_phi_sweep"] = phi_sweep(cc, torch, dev, grid, o16, active)
        others["config_hash_grid"] = hash_workload(cc, torch, dev, grid, g_h)

    # the holes the separate void test would classify (outside every timed region)
    disocc, void = win.classify()
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_main / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16 (MLP), f16 grid, f32 march/composite/warp",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "image": f"{W}x{H}", "grid": "256^3 x 12 fp16 + 32^3 occupancy (15%)",
                       "targets_per_reference": N_TARGETS, "samples": "<=256 per ray, step 0.5 voxel",
                       "brick": "autotuned per precision (cicero_autotune_brick)",
                       "l2": "flushed (256 MB write) between timed steps (value, serialised e2e); the streamed "
                             "e2e runs windows back to back, each streaming inputs larger than L2 (416 MB grid, GBs "
                             "of records)", "parallelism": f"replicas x{world}"},
            "plain_fp32_fps": n_fp * world / t_fp32,
            "bf16_full_fps": n_fp * world / t_bf16,
            "msamples_per_s_bf16_full": active * n_fp * world / t_bf16 / 1e6,
            "marched_slots_per_frame": marched,
            "mslots_marched_per_s_bf16_full": marched * n_fp * world / t_bf16 / 1e6,
            "mslots_marched_per_s_fp32_full": marched * n_fp * world / t_fp32 / 1e6,
            "msamples_per_s_fp32_full": active * n_fp * world / t_fp32 / 1e6,
            "fp32_split_full_fps": n_fp * world / t_split,
            "msamples_per_s_fp32_split_full": active * n_fp * world / t_split / 1e6,
            "active_samples_per_frame": active,
            "autotune_ms_by_brick": {"bf16": tune16, "fp32": tune32, "fp32_split": tunesp},
            "brick": {"bf16": b16, "fp32": b32, "fp32_split": bsp},
            "fraction_rays_marched_targets": holes / (N_TARGETS * R),
            "hole_batch": {"rays": holes / 1, "disocclusion_rays": int(disocc.sum()), "void_rays": int(void.sum()),
                           "composited_samples": int(hole_hdr[2]),
                           "records_reserved": int(np.uint32(hole_hdr[3])), "record_capacity": HOLE_RECORDS},
            "roofline": roof, "stages": stages, "stage_roofline": stage_roof, "quality": quality, "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": "frames/s", "h2d_bytes_per_step": int(pose_h.numel() * 4),
                    "d2h_bytes_per_step": int(host_out.numel() * 4),
                    "mode": "windows streamed: each window's 16 frames read back to pinned host memory on a copy "
                            "stream while the next window computes (double-buffered frames)",
                    "serialised_value": e2e_serial,
                    "serialised_mode": "one window at a time: compute, then read back, then synchronise"},
            "gpu_launches": int(round(launches)) * args.steps,
            "clocks": clk.summary(),
            **others,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
