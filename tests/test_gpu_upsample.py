"""The bilinear resampling of the DS-2 comparator against the oracle's definition."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("w,h,W,H,C", [(400, 400, 800, 800, 3), (37, 23, 80, 50, 3), (5, 3, 5, 3, 1),
                                       (1, 1, 7, 7, 3), (64, 48, 33, 17, 1)])
def test_upsample_matches_oracle(orc, w, h, W, H, C):
    import torch
    from paper_2404_11852_gb300 import cicero as cc
    img = np.random.default_rng(w * 131 + W).random((h, w, C)).astype(np.float32)
    src = torch.from_numpy(img).cuda().reshape(h * w, C)
    dst = torch.empty(H * W, C, device="cuda")
    cc.cicero_upsample_bilinear(src, w, h, dst, W, H)
    want = orc.upsample_bilinear(img, W, H).reshape(H * W, C)
    # the kernel forms the sampling coordinate in FP32: one ulp of u (< 64 here: 8e-6) moves the
    # interpolation weight by as much, and values in [0, 1] by at most that
    np.testing.assert_allclose(dst.cpu().double().numpy(), want, atol=1e-5)
