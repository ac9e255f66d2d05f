"""Batched rendering of uneven scene/view pairs (cicero_batch_*): every job must come out exactly as
its own cicero_render would (same kernels' arithmetic per record and per ray, whatever the work
split), match the FP64 oracle within the BF16 tolerance, and replay unchanged from a CUDA graph."""
import numpy as np
import pytest

import scenes
from helpers import psnr, rgb_errors

pytestmark = pytest.mark.gpu

TOL16, PSNR16 = 2e-2, 45.0


@pytest.fixture(scope="module")
def cc():
    from paper_2404_11852_gb300 import cicero
    cicero.lib()
    return cicero


def _specs():
    """Four jobs of uneven size: grids 40^3..72^3 (two with occupancy masks), images 21x33..80x50,
    uniform and box-march sampling, each scene with its own MLP."""
    f16 = np.float16
    return [
        (scenes.make_grid(48, 12, 8, seed=201, dtype=f16), scenes.make_mlp(12, seed=301, random_bias=True),
         scenes.orbit_camera(48, 40, az_deg=10.0, sampling=scenes.sampling_uniform(64))),
        (scenes.make_grid(72, 12, 10, seed=202, dtype=f16, occ_res=16, occ_frac=0.3),
         scenes.make_mlp(12, seed=302, random_bias=True),
         scenes.orbit_camera(64, 64, az_deg=120.0, sampling=scenes.sampling_march(72, 160))),
        (scenes.make_grid(40, 12, 6, seed=203, dtype=f16), scenes.make_mlp(12, seed=303, random_bias=True),
         scenes.orbit_camera(33, 21, az_deg=250.0, el_deg=-15.0, sampling=scenes.sampling_uniform(32))),
        (scenes.make_grid(64, 12, 8, seed=204, dtype=f16, occ_res=32, occ_frac=0.15),
         scenes.make_mlp(12, seed=304, random_bias=True),
         scenes.orbit_camera(80, 50, az_deg=300.0, sampling=scenes.sampling_march(64, 128))),
    ]


@pytest.fixture(scope="module")
def batch(cc):
    import torch
    specs = _specs()
    dev = [(cc.DeviceGrid.from_host(g), cc.DeviceMlp.from_host(m), cc.camera_from(cam), cc.sampling_from(cam.sampling))
           for g, m, cam in specs]
    outs = [(torch.full((cam.width * cam.height, 3), -1.0, device="cuda"),
             torch.full((cam.width * cam.height,), -1.0, device="cuda")) for _, _, cam in specs]
    jobs = cc.jobs_array([(gd.desc, md.desc, cd, sd, rgb, dep) for (gd, md, cd, sd), (rgb, dep) in zip(dev, outs)])
    return specs, dev, outs, jobs


def _individual(cc, gd, md, cd, sd, R, brick):
    import torch
    opt = cc.options(cc.MLP_BF16, brick)
    rgb, dep = torch.empty(R, 3, device="cuda"), torch.empty(R, device="cuda")
    ws = cc.workspace(cc.cicero_render_workspace_size(gd.desc, R, sd, opt))
    cc.cicero_render(gd.desc, md.desc, cd, sd, opt, rgb, dep, None, None, ws)
    cc.cicero_workspace_status(ws)
    return rgb, dep


@pytest.mark.parametrize("brick", [4, 8])
def test_batch_equals_individual_renders(cc, batch, brick):
    import torch
    specs, dev, outs, jobs = batch
    opt = cc.options(cc.MLP_BF16, brick)
    ws = cc.workspace(cc.cicero_batch_workspace_size(jobs, opt))
    b = cc.Batch(jobs, opt, ws)
    b.launch()
    b.status()
    for (g, m, cam), (gd, md, cd, sd), (rgb, dep) in zip(specs, dev, outs):
        want_rgb, want_dep = _individual(cc, gd, md, cd, sd, cam.width * cam.height, brick)
        assert torch.equal(rgb, want_rgb)
        assert torch.equal(dep, want_dep)
    b.close()


def test_batch_matches_oracle(cc, orc, batch):
    specs, dev, outs, jobs = batch
    opt = cc.options(cc.MLP_BF16, 8)
    ws = cc.workspace(cc.cicero_batch_workspace_size(jobs, opt))
    b = cc.Batch(jobs, opt, ws)
    b.launch()
    b.status()
    for (g, m, cam), (rgb, dep) in zip(specs, outs):
        ref = orc.render(g, m, cam.sampling, cam=cam)
        got = rgb.cpu().double().numpy()
        err, amb = rgb_errors(got, ref)
        assert amb.sum() <= max(2, 1e-3 * len(err))
        assert err.max() <= TOL16
        best = np.where(amb[:, None], ref["rgb_alt"], ref["rgb"])
        best = np.where(np.abs(got - ref["rgb"]).max(1, keepdims=True) <= np.abs(got - best).max(1, keepdims=True),
                        ref["rgb"], best)
        assert psnr(got, best) >= PSNR16
        # depth: finite exactly where the oracle's is (away from the void threshold), close where both are
        d = dep.cpu().double().numpy()
        sure = ~amb & (np.abs(ref["acc"] - cam.sampling.void_acc) > 1e-3)
        assert (np.isfinite(d[sure]) == np.isfinite(ref["depth"][sure])).all()
        both = sure & np.isfinite(d) & np.isfinite(ref["depth"])
        assert np.abs(d[both] - ref["depth"][both]).max(initial=0) <= 20 * 1e-4


def test_batch_graph_replay(cc, batch):
    import torch
    specs, dev, outs, jobs = batch
    opt = cc.options(cc.MLP_BF16, 8)
    ws = cc.workspace(cc.cicero_batch_workspace_size(jobs, opt))
    b = cc.Batch(jobs, opt, ws)
    b.launch()  # first launch outside the capture (kernel attributes)
    torch.cuda.synchronize()
    want = [(rgb.clone(), dep.clone()) for rgb, dep in outs]
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        b.launch()
    for _ in range(2):
        for rgb, dep in outs:
            rgb.fill_(-2.0)
            dep.fill_(-2.0)
        graph.replay()
        torch.cuda.synchronize()
        b.status()
        for (rgb, dep), (wr, wd) in zip(outs, want):
            assert torch.equal(rgb, wr) and torch.equal(dep, wd)
    b.close()


def test_batch_autotune(cc, batch):
    specs, dev, outs, jobs = batch
    opt = cc.options(cc.MLP_BF16, 4)
    ws = cc.workspace(cc.cicero_batch_workspace_size(jobs, opt))
    best, ms = cc.cicero_batch_autotune(jobs, opt, ws)
    assert best.brick in (4, 8, 16) and 1 <= best.mlp_groups <= 4
    assert ms[(best.brick, best.mlp_groups)] > 0 and all(v == -1.0 or v > 0 for v in ms.values())
    assert min(v for v in ms.values() if v > 0) == ms[(best.brick, best.mlp_groups)]


def test_batch_record_capacity_overflow_reported(cc, batch):
    specs, dev, outs, jobs = batch
    opt = cc.options(cc.MLP_BF16, 8, max_records=1000)
    ws = cc.workspace(cc.cicero_batch_workspace_size(jobs, opt))
    b = cc.Batch(jobs, opt, ws)
    b.launch()
    with pytest.raises(cc.CiceroError) as e:
        b.status()
    assert e.value.status == cc.ERR_WORKSPACE
    b.close()
