"""The bench's multi-rank host logic on CPU: two gloo ranks, as torchrun would launch them.

Rendering shards by frames (each rank renders its own SpaRW window), so the only cross-rank step
is the timing reduction: the job's time is the slowest rank's, and the reported throughput counts
the frames of every rank.  The reference arm runs on rank 0 alone.
"""
import json
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    import bench

    res = {}
    # each rank measured a different time; every rank must see the slowest
    res["max"] = bench.max_over_ranks(1.0 + 0.5 * rank)
    res["value"] = bench.job_value(bench.N_TARGETS, 5, world, res["max"])
    res["azimuth"] = bench.rank_azimuth(rank)

    class Args:
        steps, warmup, cpu_res, gpus = 2, 1, 8, world

    calls = []

    def fake_window(res_px, r=0):
        calls.append(res_px)
        return 0.25, 3, 0.1

    res["reference"] = bench.run_reference(Args, rank, world, window=fake_window)
    res["reference_calls"] = len(calls)
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump(res, f)


def test_two_gloo_ranks(tmp_path, capfd):
    mp = pytest.importorskip("torch.multiprocessing")
    world, port = 2, _free_port()
    mp.start_processes(_worker, args=(world, port, str(tmp_path)), nprocs=world, join=True, start_method="spawn")
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]
    # the timing reduction: both ranks see the slowest rank's time
    assert res[0]["max"] == res[1]["max"] == 1.5
    # whole-job throughput: 16 frames x 5 steps x 2 ranks over the slowest time
    assert res[0]["value"] == pytest.approx(16 * 5 * 2 / 1.5)
    # weak scaling: the ranks render different windows
    assert res[0]["azimuth"] != res[1]["azimuth"]
    # reference arm: rank 0 times the oracle and prints one line, rank 1 does no work
    assert res[0]["reference_calls"] == 3 and res[1]["reference_calls"] == 0  # 1 warm-up + 2 timed

    assert res[1]["reference"] is None
    line = res[0]["reference"]
    assert line["impl"] == "reference" and line["cpu_baseline"]["kind"] == "oracle"
    scale = (800 * 800) / (8 * 8)
    assert line["value"] == pytest.approx(16 / (0.25 * scale))
    # the steps and their time are what ran (the sample); the extrapolation is stated beside them
    assert line["steps"] == 2 and line["warmup"] == 1 and line["ms_per_step"] == pytest.approx(250.0)
    assert line["sample"]["scale"] == pytest.approx(scale) and line["sample"]["resolution"] == "8x8"
    assert line["sample"]["ms_per_full_window_extrapolated"] == pytest.approx(250.0 * scale)
    assert line["e2e"]["h2d_bytes_per_step"] == 0
    printed = [l for l in capfd.readouterr().out.splitlines() if l.startswith("{")]
    assert len(printed) == 1 and json.loads(printed[0])["impl"] == "reference"


def test_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(2.5) == 2.5
    assert bench.job_value(16, 10, 1, 2.0) == 80.0
