"""GPU parity of rendering (Sec. II-B stages run memory-centric, Sec. IV-A) against the FP64
oracle: FP32 path within 1e-4, BF16 tensor-core path within 2e-2 and PSNR >= 45 dB; the Ray
Index Table (samples grouped by brick) bit-exact; the MLP alone against the oracle's MLP."""
import numpy as np
import pytest

import scenes
from helpers import check_render, gpu_render, psnr

pytestmark = pytest.mark.gpu

TOL32, TOL16, PSNR16 = 1e-4, 2e-2, 45.0


@pytest.fixture(scope="module")
def cc():
    import torch
    assert torch.cuda.is_available()
    from paper_2404_11852_gb300 import cicero
    cicero.lib()
    return cicero


@pytest.fixture(scope="module")
def small():
    return scenes.scene_small(), scenes.make_mlp(12)


@pytest.fixture(scope="module")
def occ_scene():
    g = scenes.make_grid(96, 12, 10, seed=77, dtype=np.float16, occ_res=32, occ_frac=0.15)
    return g, scenes.make_mlp(12, seed=78, random_bias=True)


@pytest.mark.parametrize("brick", [8, 4, 16])
def test_fp32_small_scene(cc, orc, small, brick):
    g, m = small
    cam = scenes.orbit_camera(64, 64, sampling=scenes.sampling_uniform(64))
    ref = orc.render(g, m, cam.sampling, cam=cam)
    if brick == 16:
        pytest.skip("16^3 bricks of 12 FP32 channels exceed shared memory in the FP32 kernel")
    out = gpu_render(cc, g, m, cam, cam.sampling, 0, brick)
    check_render(out, ref, TOL32)


def test_fp32_ragged_image_and_slots(cc, orc, small):
    g, m = small
    cam = scenes.orbit_camera(37, 23, az_deg=75.0, el_deg=-10.0,
                              sampling=scenes.Sampling(near=0.4, far=2.6, n_samples=45, t_stop=1e-3,
                                                       bg=(0.2, 0.4, 0.9)))
    ref = orc.render(g, m, cam.sampling, cam=cam)
    out = gpu_render(cc, g, m, cam, cam.sampling, 0, 8)
    check_render(out, ref, TOL32)


def test_fp32_no_early_stop(cc, orc, small):
    g, m = small
    cam = scenes.orbit_camera(32, 32, az_deg=200.0, sampling=scenes.sampling_uniform(96, t_stop=0.0))
    ref = orc.render(g, m, cam.sampling, cam=cam)
    out = gpu_render(cc, g, m, cam, cam.sampling, 0, 8)
    check_render(out, ref, TOL32)


def test_fp16_grid_occupancy_march_fp32(cc, orc, occ_scene):
    g, m = occ_scene
    cam = scenes.orbit_camera(48, 48, az_deg=120.0, sampling=scenes.sampling_march(96, 160))
    ref = orc.render(g, m, cam.sampling, cam=cam)
    out = gpu_render(cc, g, m, cam, cam.sampling, 0, 8)
    check_render(out, ref, TOL32)
    assert (ref["acc"] > 0.5).mean() > 0.05  # the view hits the occupied cells


@pytest.mark.parametrize("brick", [4, 8, 16])
def test_fp32_split_small_scene(cc, orc, small, brick):
    """The FP32-class tensor-core MLP (split-BF16 products) at the FP32 tolerance."""
    g, m = small
    cam = scenes.orbit_camera(64, 64, az_deg=60.0, sampling=scenes.sampling_uniform(64))
    ref = orc.render(g, m, cam.sampling, cam=cam)
    out = gpu_render(cc, g, m, cam, cam.sampling, cc.MLP_FP32_SPLIT, brick)
    err, _ = check_render(out, ref, TOL32)
    print(f"split-BF16 small scene, brick {brick}: max|drgb| {err:.3g}")


def test_fp32_split_fp16_grid_occupancy(cc, orc, occ_scene):
    g, m = occ_scene
    cam = scenes.orbit_camera(48, 48, az_deg=120.0, sampling=scenes.sampling_march(96, 160))
    ref = orc.render(g, m, cam.sampling, cam=cam)
    out = gpu_render(cc, g, m, cam, cam.sampling, cc.MLP_FP32_SPLIT, 8)
    check_render(out, ref, TOL32)


def test_fp32_split_channel_limit(cc):
    """More than 16 feature channels: the split-BF16 MLP refuses (CICERO_ERR_UNSUPPORTED)."""
    g = scenes.make_grid(16, 20, 2, seed=5)
    m = scenes.make_mlp(20, seed=6)
    cam = scenes.orbit_camera(8, 8, sampling=scenes.sampling_uniform(16))
    with pytest.raises(cc.CiceroError) as ei:
        gpu_render(cc, g, m, cam, cam.sampling, cc.MLP_FP32_SPLIT, 8)
    assert ei.value.status == 2


def test_fp32_split_sixteen_channels(cc, orc):
    """C = 16, the widest grid the split-BF16 MLP takes (input row 43 of 48 columns): FP32 tolerance."""
    g = scenes.make_grid(32, 16, 4, seed=61)
    m = scenes.make_mlp(16, seed=62)
    cam = scenes.orbit_camera(40, 40, sampling=scenes.sampling_uniform(48))
    ref = orc.render(g, m, cam.sampling, cam=cam)
    out = gpu_render(cc, g, m, cam, cam.sampling, cc.MLP_FP32_SPLIT, 8)
    check_render(out, ref, TOL32)


def test_brick_box_beyond_shared_memory(cc):
    """An FP32 feature grid at bricks of 16 needs a staged box of 17^3 vertices x 12 x 4 B (235 KB),
    more than shared memory holds: the BF16 and FP32 renders refuse with CICERO_ERR_UNSUPPORTED,
    while the split-BF16 MLP, which stages no brick, renders it."""
    g = scenes.make_grid(32, 12, 2, seed=5)
    m = scenes.make_mlp(12, seed=6)
    cam = scenes.orbit_camera(8, 8, sampling=scenes.sampling_uniform(16))
    for prec in (cc.MLP_BF16, cc.MLP_FP32):
        with pytest.raises(cc.CiceroError) as ei:
            gpu_render(cc, g, m, cam, cam.sampling, prec, 16)
        assert ei.value.status == 2, prec
    gpu_render(cc, g, m, cam, cam.sampling, cc.MLP_FP32_SPLIT, 16)


def test_bf16_small_scene(cc, orc, small):
    g, m = small
    cam = scenes.orbit_camera(64, 64, sampling=scenes.sampling_uniform(64))
    ref = orc.render(g, m, cam.sampling, cam=cam)
    out = gpu_render(cc, g, m, cam, cam.sampling, 1, 8)
    err, p = check_render(out, ref, TOL16, psnr_min=PSNR16)
    print(f"BF16 small scene: max|drgb| {err:.3g}, PSNR {p:.1f} dB")


@pytest.mark.parametrize("brick", [4, 8, 16])
def test_bf16_fp16_grid_occupancy(cc, orc, occ_scene, brick):
    g, m = occ_scene
    cam = scenes.orbit_camera(40, 40, az_deg=300.0, sampling=scenes.sampling_march(96, 160))
    ref = orc.render(g, m, cam.sampling, cam=cam)
    out = gpu_render(cc, g, m, cam, cam.sampling, 1, brick)
    check_render(out, ref, TOL16, psnr_min=PSNR16)


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_degenerate_sizes(cc, orc, small, precision):
    import torch
    g, m = small
    tol = TOL16 if precision == 1 else TOL32
    cam = scenes.orbit_camera(1, 1, sampling=scenes.sampling_uniform(64))
    check_render(gpu_render(cc, g, m, cam, cam.sampling, precision), orc.render(g, m, cam.sampling, cam=cam), tol)
    # zero rays: a valid call that writes nothing
    gd, md = cc.DeviceGrid.from_host(g), cc.DeviceMlp.from_host(m)
    sd = cc.sampling_from(cam.sampling)
    o = torch.zeros(0, 3, device="cuda")
    ws = cc.workspace(cc.cicero_render_workspace_size(gd.desc, 0, sd))
    ws.fill_(0xFF)  # whatever the workspace held, the call leaves a clear status word
    cc.cicero_render_rays(gd.desc, md.desc, o, o, sd, None, o, None, None, None, ws)
    cc.cicero_workspace_status(ws)
    # a camera that misses the box entirely renders the background
    far = scenes.Camera(8, 8, 10.0, 4.0, 4.0, scenes.look_at_c2w([5.0, 5.0, 5.0], target=[10.0, 10.0, 10.0]).astype(np.float32),
                        scenes.Sampling(bg=(0.3, 0.2, 0.1)))
    out = gpu_render(cc, g, m, far, far.sampling, precision)
    np.testing.assert_allclose(out["rgb"], np.tile([0.3, 0.2, 0.1], (64, 1)), atol=1e-7)
    assert np.isinf(out["depth"]).all() and (out["acc"] == 0).all()


def test_explicit_rays_fp32(cc, orc, small):
    import torch
    g, m = small
    o, d = scenes.random_rays(777, seed=5)
    sp = scenes.sampling_uniform(64)
    ref = orc.render(g, m, sp, rays=(o, d))
    gd, md = cc.DeviceGrid.from_host(g), cc.DeviceMlp.from_host(m)
    sd = cc.sampling_from(sp)
    ot, dt = torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda()
    rgb = torch.empty(777, 3, device="cuda")
    depth, acc = torch.empty(777, device="cuda"), torch.empty(777, device="cuda")
    ns = torch.empty(777, dtype=torch.int32, device="cuda")
    ws = cc.workspace(cc.cicero_render_workspace_size(gd.desc, 777, sd))
    cc.cicero_render_rays(gd.desc, md.desc, ot, dt, sd, None, rgb, depth, acc, ns, ws)
    cc.cicero_workspace_status(ws)
    out = {"rgb": rgb.cpu().double().numpy(), "depth": depth.cpu().double().numpy(),
           "acc": acc.cpu().double().numpy(), "n_steps": ns.cpu().numpy()}
    check_render(out, ref, TOL32)


# ---------------------------------------------------------------------------------------------
# Ray Index Table: bit-exact grouping of samples by brick


def _axis_camera(axis):
    """A camera looking along +z (axis 2) or +x (axis 0) with a long focal length, so that its rays
    are axis-parallel (the centre pixel exactly) or nearly so, its origin on occupancy cell
    boundaries of the 96^3 scene (cells of 1/16 of the box)."""
    R = np.eye(3) if axis == 2 else np.array([[0.0, 0.0, 1.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0]])
    pos = np.array([-0.6875, 0.0625, -1.5]) if axis == 2 else np.array([-1.5, 0.0, 0.125])
    c2w = np.concatenate([R, pos[:, None]], 1).astype(np.float32)
    return scenes.Camera(33, 33, 4000.0, 16.5, 16.5, c2w, scenes.sampling_march(96, 160))


@pytest.mark.parametrize("which,brick", [("small", 8), ("small", 4), ("occ", 8), ("occ", 16), ("axis_z", 8),
                                         ("axis_x", 4)])
def test_ray_index_table_bit_exact(cc, orc, small, occ_scene, which, brick):
    """The samples that reach Feature Gathering, grouped by brick, bit-exact against the oracle's
    slot-by-slot classification.  The axis cases put rays parallel or nearly parallel to an axis
    and start them on occupancy cell boundaries, where the march's per-ray mask of active slots
    (found from cell boundary crossings) is most easily wrong."""
    import torch
    if which == "small":
        g, _ = small
        cam = scenes.orbit_camera(48, 40, sampling=scenes.sampling_uniform(64))
    elif which == "occ":
        g, _ = occ_scene
        cam = scenes.orbit_camera(40, 40, az_deg=120.0, sampling=scenes.sampling_march(96, 160))
    else:
        g, _ = occ_scene
        cam = _axis_camera(2 if which == "axis_z" else 0)
    S = cam.sampling.n_samples
    R = cam.width * cam.height
    want = orc.active_samples(g, cam.sampling, brick, cam=cam)
    gd = cc.DeviceGrid.from_host(g)
    sd, cd, opt = cc.sampling_from(cam.sampling), cc.camera_from(cam), cc.options(0, brick)
    nb = int(np.prod([(n - 2) // brick + 1 for n in g.n]))
    offs = torch.empty(nb + 1, dtype=torch.int32, device="cuda")
    samples = torch.empty(R * S, dtype=torch.int32, device="cuda")
    ws = cc.workspace(cc.cicero_build_rit_workspace_size(gd.desc, cd, sd, opt))
    n_b = cc.cicero_build_rit(gd.desc, cd, sd, opt, offs, samples, ws)
    cc.cicero_workspace_status(ws)
    assert n_b == nb
    offs = offs.cpu().numpy().astype(np.int64)
    total = int(offs[-1])
    smp = samples.cpu().numpy()[:total].astype(np.int64)
    brick_of = np.repeat(np.arange(nb), np.diff(offs))
    amb = want["amb"]
    keep_g = ~amb[smp // S]
    keep_o = ~amb[want["ray"]]
    got = np.stack([brick_of[keep_g], smp[keep_g]], 1)
    exp = np.stack([want["brick"][keep_o].astype(np.int64),
                    want["ray"][keep_o].astype(np.int64) * S + want["slot"][keep_o]], 1)
    assert len(got) == len(exp) > 0
    got = got[np.lexsort((got[:, 1], got[:, 0]))]
    exp = exp[np.lexsort((exp[:, 1], exp[:, 0]))]
    np.testing.assert_array_equal(got, exp)
    assert amb.sum() <= max(2, 1e-3 * R)
    # inside each brick the samples come octant by octant (x, y, z halves of the brick as bits
    # 0, 1, 2), in the order the library exports them
    vox = dict(zip((want["ray"].astype(np.int64) * S + want["slot"]).tolist(), want["voxel"].tolist()))
    nx, ny = g.n[0], g.n[1]
    v = np.array([vox[i] for i in smp[keep_g].tolist()], dtype=np.int64)
    i0 = np.stack([v % nx, (v // nx) % ny, v // (nx * ny)], 1)
    octant = (((i0 % brick) >= brick // 2) * np.array([1, 2, 4])).sum(1)
    b_of = brick_of[keep_g]
    same = b_of[1:] == b_of[:-1]
    assert (octant[1:][same] >= octant[:-1][same]).all()


# ---------------------------------------------------------------------------------------------
# Feature Computation alone


@pytest.mark.parametrize("M", [1, 128, 300])
def test_mlp_eval(cc, orc, M):
    import torch
    m = scenes.make_mlp(12, seed=99, random_bias=True)
    x = scenes.uniform(100 + M, M * m.in_dim, -1.5, 1.5).reshape(M, m.in_dim).astype(np.float32)
    want = orc.mlp_eval(m, x)
    md = cc.DeviceMlp.from_host(m)
    xt = torch.from_numpy(x).cuda()
    ws = cc.workspace(cc.cicero_mlp_eval_workspace_size(M))
    for prec, tol in ((cc.MLP_FP32, 1e-5), (cc.MLP_BF16, 2e-2)):
        c = torch.empty(M, 3, device="cuda")
        cc.cicero_mlp_eval(md.desc, xt, prec, c, ws)
        cc.cicero_workspace_status(ws)
        err = np.abs(c.cpu().double().numpy() - want).max()
        assert err <= tol, (prec, err)


# ---------------------------------------------------------------------------------------------
# the large single frame (800x800, 256^3 FP16 grid with a 32^3 occupancy mask) on sampled pixels


@pytest.fixture(scope="module")
def large():
    return scenes.scene_large(), scenes.make_mlp(12)


@pytest.mark.parametrize("precision,brick", [(0, 8), (1, 4), (1, 8), (2, 8)])  # the benchmark's bricks: FP32 8, BF16 4
def test_large_frame_sampled(cc, orc, large, precision, brick):
    g, m = large
    cam = scenes.orbit_camera(800, 800, sampling=scenes.sampling_march(256, 256))
    out = gpu_render(cc, g, m, cam, cam.sampling, precision, brick)
    pix = (scenes.splitmix64(4242, 400) % np.uint64(800 * 800)).astype(np.int32)
    ref = orc.render(g, m, cam.sampling, cam=cam, pix=pix)
    sub = {k: v[pix] for k, v in out.items()}
    tol = TOL16 if precision == 1 else TOL32
    err, p = check_render(sub, ref, tol, psnr_min=PSNR16 if precision == 1 else None)
    assert (ref["acc"] > 0.5).mean() > 0.05
    print(f"800x800 precision {precision} brick {brick}: max|drgb| {err:.3g} PSNR {p}")
