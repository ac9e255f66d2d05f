"""The hash-grid workload: colour features from a multiresolution hash encoding (dense and hashed
levels), density from the dense grid, BF16 tensor-core MLP; against the FP64 oracle."""
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


def _render(cc, g, m, cam, brick=8):
    import torch
    gd, md = cc.DeviceGrid.from_host(g), cc.DeviceMlp.from_host(m)
    hd = cc.DeviceHashGrid.from_host(g.hash)
    cd, sd, opt = cc.camera_from(cam), cc.sampling_from(cam.sampling), cc.options(cc.MLP_BF16, brick)
    R = cam.width * cam.height
    ws = cc.workspace(cc.cicero_render_hash_workspace_size(gd.desc, hd.desc, R, sd, opt))
    rgb, dep = torch.empty(R, 3, device="cuda"), torch.empty(R, device="cuda")
    cc.cicero_render_hash(gd.desc, hd.desc, md.desc, cd, sd, opt, rgb, dep, ws)
    cc.cicero_workspace_status(ws)
    return rgb.cpu().double().numpy(), dep.cpu().double().numpy()


@pytest.mark.parametrize("levels,log2_size,base,top,dtype,brick", [
    (8, 14, 4, 96, np.float16, 8),     # dense coarse levels, hashed fine levels
    (4, 12, 6, 40, np.float32, 4),     # FP32 table, generic level count
    (8, 19, 16, 512, np.float16, 16),  # the benchmark's encoding
])
def test_hash_render_matches_oracle(cc, orc, levels, log2_size, base, top, dtype, brick):
    h = scenes.make_hash_grid(levels, 2, log2_size, base, top, seed=55 + levels, dtype=dtype)
    g = scenes.with_hash(scenes.make_grid(64, 12, 8, seed=56, dtype=np.float16, occ_res=16, occ_frac=0.3), h)
    m = scenes.make_mlp(2 * levels, seed=57, random_bias=True)
    cam = scenes.orbit_camera(56, 40, az_deg=210.0, sampling=scenes.sampling_march(64, 128))
    dense = [(r + 1) ** 3 <= (1 << log2_size) for r in h.res]
    assert any(dense) and not all(dense)  # both kinds of level are exercised
    got, dep = _render(cc, g, m, cam, brick)
    ref = orc.render(g, m, cam.sampling, cam=cam)
    err, amb = rgb_errors(got, ref)
    assert amb.sum() <= max(2, 1e-3 * len(err))
    assert err.max() <= TOL16, err.max()
    best = np.where(amb[:, None], ref["rgb_alt"], ref["rgb"])
    assert psnr(got, best) >= PSNR16
    sure = ~amb & (np.abs(ref["acc"] - 0.5) > 1e-3)
    assert (np.isfinite(dep[sure]) == np.isfinite(ref["depth"][sure])).all()
    assert (ref["acc"] > 0.5).mean() > 0.05


def test_hash_render_rejects_bad_arguments(cc):
    import torch
    h = scenes.make_hash_grid(3, 2, 10, 4, 16, dtype=np.float16)
    g = scenes.with_hash(scenes.scene_fd().astype(np.float16), h)
    m = scenes.make_mlp(6)
    gd, md, hd = cc.DeviceGrid.from_host(g), cc.DeviceMlp.from_host(m), cc.DeviceHashGrid.from_host(h)
    cam = scenes.orbit_camera(8, 8)
    cd, sd = cc.camera_from(cam), cc.sampling_from(cam.sampling)
    x = torch.empty(64, 3, device="cuda")
    ws = cc.workspace(1 << 20)
    with pytest.raises(cc.CiceroError) as e:  # the FP32 MLP path is not offered for hash encodings
        cc.cicero_render_hash(gd.desc, hd.desc, md.desc, cd, sd, cc.options(cc.MLP_FP32, 8), x, None, ws)
    assert e.value.status == cc.ERR_UNSUPPORTED
    bad = scenes.make_mlp(12)  # in_dim does not match 3 levels x 2 features
    with pytest.raises(cc.CiceroError):
        cc.cicero_render_hash(gd.desc, hd.desc, cc.DeviceMlp.from_host(bad).desc, cd, sd, cc.options(cc.MLP_BF16, 8),
                              x, None, ws)
