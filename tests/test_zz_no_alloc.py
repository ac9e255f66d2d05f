"""The allocation-free warp entry point (cicero_warp_noalloc) against cicero_warp.

cicero_warp_noalloc exists for callers that cannot allocate device memory (real-time loops that
must not enter an allocator, host programs without a device allocator of their own).  Its scratch
is a fixed array inside the library, so this test checks, through the C ABI, that two calls in a row each give exactly what cicero_warp
gives with a workspace (the warp is bit-exact, so the tolerance of the other warp tests is zero),
and that a target larger than the built-in scratch is refused before any GPU work.
"""
import numpy as np
import pytest

import scenes

pytestmark = pytest.mark.gpu


def _buffers(torch, n):
    return (torch.empty(n, 3, device="cuda"), torch.empty(n, device="cuda"),
            torch.empty(n, dtype=torch.uint8, device="cuda"), torch.empty(n, dtype=torch.int32, device="cuda"),
            torch.empty(1, dtype=torch.int32, device="cuda"))


def test_noalloc_warp_matches_workspace_warp():
    import torch
    from paper_2404_11852_gb300 import cicero as cc
    g = scenes.scene_small()
    cam = scenes.orbit_camera(96, 80, sampling=scenes.sampling_uniform(64))
    n = cam.width * cam.height
    rgb = torch.from_numpy(scenes.uniform(3, n * 3).astype(np.float32).reshape(n, 3)).cuda()
    depth_h = scenes.uniform(4, n, 1.0, 2.2).astype(np.float32)
    depth_h[scenes.uniform(5, n) < 0.3] = np.inf
    depth = torch.from_numpy(depth_h).cuda()
    gd = cc.DeviceGrid.from_host(g)
    sd, rc = cc.sampling_from(cam.sampling), cc.camera_from(cam)
    for k in (3, -6):  # two calls in a row, different targets
        tc = cc.camera_from(scenes.offset_camera(cam, k, yaw_deg=1.5, shift=0.01))
        a = _buffers(torch, n)
        ws = cc.workspace(cc.cicero_warp_workspace_size(tc))
        cc.cicero_warp(rgb, depth, rc, tc, 180.0, gd.desc, sd, *a, ws)
        b = _buffers(torch, n)
        cc.cicero_warp_noalloc(rgb, depth, rc, tc, 180.0, gd.desc, sd, *b)
        torch.cuda.synchronize()
        nh = int(a[4].item())
        assert nh == int(b[4].item()) and nh > 0
        for x, y in zip(a[:3], b[:3]):
            assert torch.equal(x, y)
        assert torch.equal(a[3][:nh], b[3][:nh])


def test_noalloc_warp_rejects_oversize_target():
    import torch
    from paper_2404_11852_gb300 import cicero as cc
    big = cc.camera(1025, 1024, 800.0, 512.0, 512.0, np.eye(3, 4))
    x = torch.empty(4, device="cuda")
    m = torch.empty(4, dtype=torch.uint8, device="cuda")
    i = torch.empty(4, dtype=torch.int32, device="cuda")
    with pytest.raises(cc.CiceroError) as e:
        cc.cicero_warp_noalloc(x, x, big, big, 180.0, None, None, x, x, m, i, i)
    assert e.value.status == cc.ERR_UNSUPPORTED
