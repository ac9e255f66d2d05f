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
HOLE_RECORDS = 320_000_000  # record capacity of the batched hole render (19 GB)
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one k_gather_mlp_bf16 launch on the
# 800x800 reference frame, from a one-pass ncu capture of this benchmark, and the SHA-1 of the
# kernel sources it was taken on; the roofline reports it only while those sources are unchanged.
GATHER_TRAFFIC = {"bytes": 2499950080 + 1201474304, "sources_sha1": "6879172ada0c195223960e350463f4a7892a192e"}
GATHER_SOURCES = ("mlp_tc.cu", "common.cuh", "internal.h")


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=50)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cpu-res", type=int, default=100, help="oracle sample resolution (square)")
    p.add_argument("--case", default="full", choices=["full", "small"],
                   help="small: one 320x320 reference frame (BF16 and FP32) and two targets, for profilers")
    p.add_argument("--brick", type=int, default=4, help="brick size of the small case")
    return p.parse_args()


def small_case(brick: int = 4):
    """A reduced run of the same kernels for profiler captures (the grid stays 416 MB > L2).

    Kernel launch order: reference frame BF16 twice, FP32 once (one k_march, bucketing, gather
    and composite each), then per target one warp and one hole render.  No autotuning, so a
    capture's launch index (-s) does not depend on timing."""
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
                "bf16_tflops_sustained": j.get("bf16_tflops_sustained", j["bf16_tflops"]), "src": "measured"}
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "src": "fallback"}


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


def oracle_window(res: int, rank: int = 0):
    """The oracle's SpaRW window at res x res on the same scene, FOV, poses and sampling; returns
    (seconds, cores, hole fraction)."""
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
        if w["n_holes"]:
            oracle.render(g, m, cam.sampling, cam=tgt, pix=w["hole_idx"])
        holes += w["n_holes"]
    dt = time.perf_counter() - t0
    return dt, oracle.max_threads(), holes / (N_TARGETS * res * res)


def run_reference(args, rank, world, window=None):
    """The oracle arm: rank 0 alone times the oracle; the other ranks exit without work."""
    if rank != 0:
        return None
    window = window or oracle_window
    dts = []
    for _ in range(max(1, args.steps)):
        dt, cores, _ = window(args.cpu_res)
        dts.append(dt)
    scale = (W * H) / (args.cpu_res * args.cpu_res)
    t_step = float(np.mean(dts)) * scale
    fps = N_TARGETS / t_step
    line = {"impl": "reference", "metric": METRIC, "value": fps, "unit": "frames/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": 0, "ms_per_step": t_step * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": fps, "unit": "frames/s", "cores": cores, "kind": "oracle",
                             "sample": f"whole SpaRW window at {args.cpu_res}x{args.cpu_res} "
                                       f"({args.cpu_res**2} of {W*H} pixels per frame), time x {scale:.0f}"},
            "e2e": {"value": fps, "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return line


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
    tds = [cc.camera_from(t) for t in targets]
    dev = torch.device("cuda", local)
    # brick size per precision, picked by the library's autotuner (timed renders of this frame)
    ws_r = cc.workspace(cc.cicero_render_workspace_size(grid.desc, R, sd, cc.options(cc.MLP_BF16, 4)), dev)
    ref_rgb = torch.empty(R, 3, device=dev)
    ref_depth = torch.empty(R, device=dev)
    b16, tune16 = cc.cicero_autotune_brick(grid.desc, mlp.desc, cd, sd, cc.MLP_BF16, ref_rgb, ref_depth, ws_r)
    b32, tune32 = cc.cicero_autotune_brick(grid.desc, mlp.desc, cd, sd, cc.MLP_FP32, ref_rgb, ref_depth, ws_r)
    o16, o32 = cc.options(cc.MLP_BF16, b16), cc.options(cc.MLP_FP32, b32)
    ws_w = cc.workspace(cc.cicero_warp_workspace_size(tds[0]), dev)
    t_rgb = torch.empty(N_TARGETS, R, 3, device=dev)
    t_depth = torch.empty(N_TARGETS, R, device=dev)
    mask = torch.empty(N_TARGETS, R, dtype=torch.uint8, device=dev)
    hidx = torch.empty(N_TARGETS, R, dtype=torch.int32, device=dev)
    nh = torch.zeros(N_TARGETS, 1, dtype=torch.int32, device=dev)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)  # > 129 MB L2

    # all targets' holes are rendered in one batched pass; records are capped well above need
    ob = cc.options(cc.MLP_BF16, b16, max_records=HOLE_RECORDS)
    ws_h = cc.workspace(cc.cicero_render_workspace_size(grid.desc, N_TARGETS * R, sd, ob), dev)
    hidx_l = [hidx[i] for i in range(N_TARGETS)]
    trgb_l = [t_rgb[i] for i in range(N_TARGETS)]
    tdep_l = [t_depth[i] for i in range(N_TARGETS)]

    ws_wb = cc.workspace(cc.cicero_warp_batch_workspace_size(tds), dev)
    mask_l = [mask[i] for i in range(N_TARGETS)]
    nh_flat = nh.view(-1)

    def step():
        cc.cicero_render(grid.desc, mlp.desc, cd, sd, o16, ref_rgb, ref_depth, None, None, ws_r)
        cc.cicero_warp_batch(ref_rgb, ref_depth, cd, tds, 180.0, grid.desc, sd, trgb_l, tdep_l, mask_l, hidx_l, nh_flat,
                             ws_wb)
        cc.cicero_render_holes_batch(grid.desc, mlp.desc, tds, sd, ob, hidx_l, nh, N_TARGETS * R, trgb_l, tdep_l,
                                     ws_h)

    def full(opt):
        cc.cicero_render(grid.desc, mlp.desc, cd, sd, opt, ref_rgb, ref_depth, None, None, ws_r)

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
    cc.cicero_workspace_status(ws_r)
    cc.cicero_workspace_status(ws_h)
    hole_hdr = ws_h[:16].view(torch.int32).cpu().numpy()
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
        for i, td in enumerate(tds):
            td.c2w[:] = [float(v) for v in p[i].reshape(-1)]
        step()

    t_e2e = timed(step_e2e, args.steps, 1, host_io=d2h)
    e2e_value = job_value(N_TARGETS, args.steps, world, t_e2e)

    # the plain FP32 full render and the BF16 full render of the same frame
    n_fp = max(2, args.steps)
    t_fp32 = timed(lambda: full(o32), n_fp, 1)
    hdr = ws_r[:16].view(torch.int32).cpu().numpy()
    active = int(hdr[2])
    t_bf16 = timed(lambda: full(o16), n_fp, 1)

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
    stages = {k: {"ms_per_step": v[0] / 2, "launches_per_step": v[1] / 2} for k, v in prof.items() if v[1]}

    # quality: reference frame (BF16) vs the FP64 oracle on sampled pixels, and the cpu baseline
    cpu = None
    quality = {}
    if rank == 0 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        pix = (scenes.splitmix64(777, 256) % np.uint64(R)).astype(np.int32)
        full(o16)
        got = ref_rgb.cpu().double().numpy()[pix]
        ref = oracle.render(g_h, m_h, cam.sampling, cam=cam, pix=pix)
        e = np.where(ref["amb"][:, None], np.minimum(np.abs(got - ref["rgb"]), np.abs(got - ref["rgb_alt"])),
                     np.abs(got - ref["rgb"]))
        quality = {"ref_bf16_max_err": float(e.max()),
                   "ref_bf16_psnr_db": float(10 * math.log10(1.0 / max(float(np.mean(e ** 2)), 1e-30))),
                   "sample_pixels": int(len(pix))}
        dt, cores, _ = oracle_window(args.cpu_res, rank)
        scale = R / (args.cpu_res ** 2)
        cpu = {"value": N_TARGETS / (dt * scale), "unit": "frames/s", "cores": cores, "kind": "oracle",
               "sample": f"whole SpaRW window at {args.cpu_res}x{args.cpu_res} ({args.cpu_res**2} of {R} pixels "
                         f"per frame, FP64), time x {scale:.0f}"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_main / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16 (MLP), f16 grid, f32 march/composite/warp",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "image": f"{W}x{H}", "grid": "256^3 x 12 fp16 + 32^3 occupancy (15%)",
                       "targets_per_reference": N_TARGETS, "samples": "<=256 per ray, step 0.5 voxel",
                       "brick": "autotuned per precision (cicero_autotune_brick)",
                       "l2": "flushed (256 MB write) between timed steps", "parallelism": f"replicas x{world}"},
            "plain_fp32_fps": n_fp * world / t_fp32,
            "bf16_full_fps": n_fp * world / t_bf16,
            "msamples_per_s_bf16_full": active * n_fp * world / t_bf16 / 1e6,
            "msamples_per_s_fp32_full": active * n_fp * world / t_fp32 / 1e6,
            "active_samples_per_frame": active,
            "autotune_ms_by_brick": {"bf16": tune16, "fp32": tune32}, "brick": {"bf16": b16, "fp32": b32},
            "fraction_rays_marched_targets": holes / (N_TARGETS * R),
            "hole_batch": {"rays": holes / 1, "composited_samples": int(hole_hdr[2]),
                           "records_reserved": int(np.uint32(hole_hdr[3])), "record_capacity": HOLE_RECORDS},
            "roofline": roof, "stages": stages, "quality": quality, "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": "frames/s", "h2d_bytes_per_step": int(pose_h.numel() * 4),
                    "d2h_bytes_per_step": int(host_out.numel() * 4)},
            "gpu_launches": int(round(launches)) * args.steps,
            "clocks": clk.summary(),
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
