"""SpaRW over a trajectory (cicero_pipeline_*): reference frames rendered on a second stream while
the previous window's targets are warped and hole-rendered.  The overlap must not change a single
pixel: the pipeline equals the same schedule done call by call on one stream, and follows the
oracle's SpaRW chain on every frame, with the oracle fed the GPU's reference frames."""
import numpy as np
import pytest

import scenes
from helpers import check_render, psnr

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
    refs = cc.cicero_reference_poses(targets, window)
    opt = cc.options(precision, 8)
    ws = cc.workspace(cc.cicero_pipeline_workspace_size(gd.desc, cd, sd, opt, window, hole_records))
    p = cc.Pipeline(gd.desc, md.desc, cd, sd, opt, window, hole_records, 180.0, ws)
    R = cam.width * cam.height
    rgb = [torch.full((R, 3), -1.0, device="cuda") for _ in traj]
    dep = [torch.full((R,), -1.0, device="cuda") for _ in traj]
    s_ref = torch.cuda.Stream() if two_streams else None
    p.run(targets, rgb, dep, stream_ref=s_ref)
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
    """FP32 pipeline against the oracle's SpaRW chain on every frame.  The oracle is fed the GPU's
    reference frame of each window (rendered by cicero_render at the pose the pipeline derives,
    the same bits as the pipeline's own reference, see test_pipeline_equals_call_by_call), so both
    sides warp the same points: the warped pixels equal the oracle's warp bit for bit, and the
    hole pixels, rendered in FP32, are within 1e-4 of the oracle's render of the same pixels."""
    import torch
    g, m, cam, traj, gd, md = setup
    refs, rgb, dep = _run_pipeline(cc, setup, 4, cc.MLP_FP32)
    sd, opt = cc.sampling_from(cam.sampling), cc.options(cc.MLP_FP32, 8)
    R = cam.width * cam.height
    ws_r = cc.workspace(cc.cicero_render_workspace_size(gd.desc, R, sd, opt))
    n_holes = 0
    for w, rc in enumerate(refs):
        ref_cam = scenes.Camera(rc.width, rc.height, rc.f, rc.cx, rc.cy, np.array(rc.c2w[:], np.float32).reshape(3, 4),
                                cam.sampling)
        rr, rd = torch.empty(R, 3, device="cuda"), torch.empty(R, device="cuda")
        acc, ns = torch.empty(R, device="cuda"), torch.empty(R, dtype=torch.int32, device="cuda")
        cc.cicero_render(gd.desc, md.desc, rc, sd, opt, rr, rd, acc, ns, ws_r)
        cc.cicero_workspace_status(ws_r)
        g_ref = {"rgb": rr.cpu().double().numpy(), "depth": rd.cpu().double().numpy(),
                 "acc": acc.cpu().double().numpy(), "n_steps": ns.cpu().numpy()}
        check_render(g_ref, orc.render(g, m, cam.sampling, cam=ref_cam), 1e-4)
        for i in range(w * 4, min(len(traj), w * 4 + 4)):
            o_w = orc.warp(rr.cpu().numpy(), rd.cpu().numpy(), ref_cam, traj[i], void_grid=g,
                           void_sampling=cam.sampling)
            out_rgb, out_dep = rgb[i].cpu().double().numpy(), dep[i].cpu().double().numpy()
            holes = o_w["hole_idx"]
            keep = np.ones(R, bool)
            keep[holes] = False
            # void holes (mask 2) are rendered by the pipeline's hole pass: background, depth +inf
            void = o_w["mask"] == 2
            np.testing.assert_array_equal(out_rgb[keep & ~void], o_w["rgb"][keep & ~void].astype(np.float64))
            np.testing.assert_array_equal(out_dep[keep & ~void], o_w["depth"][keep & ~void].astype(np.float64))
            np.testing.assert_array_equal(out_rgb[void], np.tile(np.asarray(cam.sampling.bg, np.float64), (void.sum(), 1)))
            assert np.isinf(out_dep[void]).all()
            if len(holes):
                ref = orc.render(g, m, cam.sampling, cam=traj[i], pix=holes)
                check_render({"rgb": out_rgb[holes], "depth": out_dep[holes], "acc": ref["acc"]}, ref, 1e-4)
            n_holes += len(holes)
    assert n_holes > 0
