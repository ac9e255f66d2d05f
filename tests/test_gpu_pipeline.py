"""SpaRW over a trajectory (cicero_pipeline_*): reference frames rendered on a second stream while
the previous window's targets are warped and hole-rendered.  The overlap must not change a single
pixel: the pipeline equals the same schedule done call by call on one stream, and follows the
oracle's SpaRW chain on every frame."""
import numpy as np
import pytest

import scenes
from helpers import psnr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cc():
    from paper_2404_11852_gb300 import cicero
    cicero.lib()
    return cicero


@pytest.fixture(scope="module")
def setup(cc):
    g, m = scenes.scene_small(), scenes.make_mlp(12)
    cam = scenes.orbit_camera(64, 48, sampling=scenes.sampling_uniform(64))
    traj = [scenes.offset_camera(cam, k, yaw_deg=1.5, shift=0.01) for k in range(10)]
    gd, md = cc.DeviceGrid.from_host(g), cc.DeviceMlp.from_host(m)
    return g, m, cam, traj, gd, md


def _run_pipeline(cc, setup, window, precision, two_streams=True, hole_records=0):
    import torch
    g, m, cam, traj, gd, md = setup
    cd, sd = cc.camera_from(cam), cc.sampling_from(cam.sampling)
    targets = [cc.camera_from(t) for t in traj]
    refs = cc.reference_poses(targets, window)
    opt = cc.options(precision, 8)
    ws = cc.workspace(cc.cicero_pipeline_workspace_size(gd.desc, cd, sd, opt, window, hole_records))
    p = cc.Pipeline(gd.desc, md.desc, cd, sd, opt, window, hole_records, 180.0, ws)
    R = cam.width * cam.height
    rgb = [torch.full((R, 3), -1.0, device="cuda") for _ in traj]
    dep = [torch.full((R,), -1.0, device="cuda") for _ in traj]
    s_ref = torch.cuda.Stream() if two_streams else None
    p.run(targets, refs, rgb, dep, stream_ref=s_ref)
    torch.cuda.synchronize()
    p.status()
    p.close()
    return refs, rgb, dep


@pytest.mark.parametrize("window", [4, 3])
def test_pipeline_equals_call_by_call(cc, setup, window):
    import torch
    g, m, cam, traj, gd, md = setup
    refs, rgb, dep = _run_pipeline(cc, setup, window, cc.MLP_BF16, hole_records=200_000)
    sd, opt = cc.sampling_from(cam.sampling), cc.options(cc.MLP_BF16, 8)
    R = cam.width * cam.height
    ws_r = cc.workspace(cc.cicero_render_workspace_size(gd.desc, R, sd, opt))
    ws_h = cc.workspace(cc.cicero_render_workspace_size(gd.desc, R, sd, opt))
    for i, t in enumerate(traj):
        w = i // window
        rr, rd = torch.empty(R, 3, device="cuda"), torch.empty(R, device="cuda")
        cc.cicero_render(gd.desc, md.desc, refs[w], sd, opt, rr, rd, None, None, ws_r)
        tc = cc.camera_from(t)
        wr, wd = torch.empty(R, 3, device="cuda"), torch.empty(R, device="cuda")
        mask = torch.empty(R, dtype=torch.uint8, device="cuda")
        hidx = torch.empty(R, dtype=torch.int32, device="cuda")
        nh = torch.empty(1, dtype=torch.int32, device="cuda")
        ws_w = cc.workspace(cc.cicero_warp_workspace_size(tc))
        cc.cicero_warp(rr, rd, refs[w], tc, 180.0, gd.desc, sd, wr, wd, mask, hidx, nh, ws_w)
        cc.cicero_render_holes(gd.desc, md.desc, tc, sd, opt, hidx, nh, R, wr, wd, ws_h)
        cc.cicero_workspace_status(ws_h)
        assert torch.equal(rgb[i], wr), i
        assert torch.equal(dep[i], wd), i


def test_pipeline_overlap_changes_nothing(cc, setup):
    import torch
    _, a, da = _run_pipeline(cc, setup, 4, cc.MLP_BF16, two_streams=True)
    _, b, db = _run_pipeline(cc, setup, 4, cc.MLP_BF16, two_streams=False)
    for x, y in zip(a + da, b + db):
        assert torch.equal(x, y)


def test_pipeline_follows_oracle_chain(cc, orc, setup):
    """FP32 pipeline against the oracle running the same chain (its own reference renders at the
    same extrapolated poses, its warp and hole renders) on every frame."""
    g, m, cam, traj, gd, md = setup
    refs, rgb, dep = _run_pipeline(cc, setup, 4, cc.MLP_FP32)
    worst = 1e9
    for w, rc in enumerate(refs):
        ref_cam = scenes.Camera(rc.width, rc.height, rc.f, rc.cx, rc.cy, np.array(rc.c2w[:], np.float32).reshape(3, 4),
                                cam.sampling)
        oref = orc.render(g, m, cam.sampling, cam=ref_cam)
        for i in range(w * 4, min(len(traj), w * 4 + 4)):
            o_w = orc.warp(oref["rgb"].astype(np.float32), oref["depth"].astype(np.float32), ref_cam, traj[i],
                           void_grid=g, void_sampling=cam.sampling)
            o_rgb = o_w["rgb"].astype(np.float64)
            if o_w["n_holes"]:
                o_rgb[o_w["hole_idx"]] = orc.render(g, m, cam.sampling, cam=traj[i], pix=o_w["hole_idx"])["rgb"]
            worst = min(worst, psnr(rgb[i].cpu().double().numpy(), o_rgb))
    print(f"pipeline vs oracle chain: worst frame {worst:.1f} dB")
    assert worst >= 40.0
