"""GPU parity of the hand-written backward (grid gradients of an rgb loss) against the FP64
oracle's analytic gradient, itself pinned to FP64 central differences: relative inf-norm
error <= 1e-3."""
import numpy as np
import pytest

import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cc():
    from paper_2404_11852_gb300 import cicero
    cicero.lib()
    return cicero


def gpu_grads(cc, g32, m, o, d, sp, grad, with_mlp=False, feat_offset=0, mlp_path="tc", fill=None):
    """feat_offset > 0 places d_features that many floats into a larger buffer (an address that
    is not 16-byte aligned when feat_offset % 4 != 0).  With the MLP weight gradients, mlp_path
    "tc" sizes the workspace for their tensor-core GEMMs, "simt" for the CUDA-core path.  fill:
    a byte written over the whole workspace first (0xFF makes every unwritten BF16 value a NaN)."""
    import torch
    gd, md = cc.DeviceGrid.from_host(g32), cc.DeviceMlp.from_host(m)
    sd = cc.sampling_from(sp)
    ot, dt = torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda()
    gr = torch.from_numpy(grad.astype(np.float32)).cuda()
    dd = torch.zeros(g32.density.shape, device="cuda")
    df = torch.zeros(g32.features.size + feat_offset, device="cuda")[feat_offset:].view(g32.features.shape)
    dm = torch.zeros(m.flat().size, device="cuda") if with_mlp else None
    size = cc.cicero_backward_mlp_workspace_size if with_mlp and mlp_path == "tc" else cc.cicero_backward_workspace_size
    ws = cc.workspace(size(gd.desc, o.shape[0], sd))
    if fill is not None:
        ws.fill_(fill)
    cc.cicero_render_backward(gd.desc, md.desc, ot, dt, sd, gr, dd, df, dm, ws)
    cc.cicero_workspace_status(ws)
    out = dd.cpu().double().numpy(), df.cpu().double().numpy()
    return out + (dm.cpu().double().numpy(),) if with_mlp else out


def mlp_parts(m, flat):
    """Split a flat [W1, b1, W2, b2, W3, b3] vector into its six pieces."""
    parts, k = [], 0
    for a in (m.w1, m.b1, m.w2, m.b2, m.w3, m.b3):
        parts.append(flat[k:k + a.size])
        k += a.size
    return parts


def rel_inf(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-30)


def test_backward_fd_scene(cc, orc):
    g = scenes.scene_fd().astype(np.float32)
    m = scenes.make_mlp(4, random_bias=True)
    o, d = scenes.random_rays(32)
    tgt = scenes.random_targets(32).astype(np.float64)
    sp = scenes.Sampling(near=0.5, far=2.5, n_samples=32, t_stop=0.0)
    out = orc.render(g, m, sp, rays=(o, d))
    grad = 2.0 * (out["rgb"] - tgt) / tgt.size
    wd, wf, _ = orc.backward(g, m, sp, grad, rays=(o, d))
    dd, df = gpu_grads(cc, g, m, o, d, sp, grad)
    assert rel_inf(dd, wd) <= 1e-3, rel_inf(dd, wd)
    assert rel_inf(df, wf) <= 1e-3, rel_inf(df, wf)


@pytest.mark.parametrize("brick_scene", ["small", "occ"])
def test_backward_larger_scene(cc, orc, brick_scene):
    if brick_scene == "small":
        g = scenes.make_grid(48, 12, 8, seed=31)
        sp = scenes.Sampling(near=0.5, far=2.5, n_samples=96, t_stop=1e-3)
    else:
        g = scenes.make_grid(64, 12, 8, seed=32, dtype=np.float16, occ_res=16, occ_frac=0.3)
        sp = scenes.sampling_march(64, 128)
    m = scenes.make_mlp(12, seed=33, random_bias=True)
    o, d = scenes.random_rays(300, seed=34)
    out = orc.render(g, m, sp, rays=(o, d))
    keep = ~out["amb"]
    tgt = scenes.random_targets(300, seed=35).astype(np.float64)
    grad = 2.0 * (out["rgb"] - tgt) / tgt.size
    grad[~keep] = 0.0  # ambiguous early stops contribute nothing on either side
    wd, wf, _ = orc.backward(g, m, sp, grad, rays=(o, d))
    dd, df = gpu_grads(cc, g, m, o, d, sp, grad)
    assert rel_inf(dd, wd) <= 1e-3, rel_inf(dd, wd)
    assert rel_inf(df, wf) <= 1e-3, rel_inf(df, wf)


@pytest.mark.parametrize("C, feat_offset", [(6, 0), (12, 1), (12, 4), (20, 0)])
def test_backward_channel_layouts(cc, orc, C, feat_offset):
    """The trilinear adjoint adds four channels per 16-byte atomic when C % 4 == 0 and d_features
    is 16-byte aligned, one channel per atomic otherwise: both paths against the oracle.  C = 20
    is beyond the tensor-core kernels (at most 16 channels): the FP32 recompute and the CUDA-core
    grid-gradient kernel run instead."""
    g = scenes.make_grid(40, C, 6, seed=41)
    m = scenes.make_mlp(C, seed=42, random_bias=True)
    o, d = scenes.random_rays(200, seed=43)
    sp = scenes.Sampling(near=0.5, far=2.5, n_samples=64, t_stop=1e-3)
    out = orc.render(g, m, sp, rays=(o, d))
    tgt = scenes.random_targets(200, seed=44).astype(np.float64)
    grad = 2.0 * (out["rgb"] - tgt) / tgt.size
    grad[out["amb"]] = 0.0
    wd, wf, _ = orc.backward(g, m, sp, grad, rays=(o, d))
    dd, df = gpu_grads(cc, g, m, o, d, sp, grad, feat_offset=feat_offset)
    assert rel_inf(dd, wd) <= 1e-3, rel_inf(dd, wd)
    assert rel_inf(df, wf) <= 1e-3, rel_inf(df, wf)


@pytest.mark.parametrize("with_mlp", [False, True])
def test_backward_config4_grid(cc, orc, with_mlp):
    """The differentiation workload's configuration (160^3 x 12 FP32 grid, 256 slots in [0.5, 2.5],
    t_stop 1e-3, bricks of 8, the MSE loss against seeded targets) on every 16th of its 8192 rays:
    grid (and MLP weight) gradients against the oracle.  Gradients are sums over rays, so the rays
    are subset rather than the outputs sampled."""
    g = scenes.scene_backward()
    m = scenes.make_mlp(12)
    o, d = scenes.random_rays(8192)
    sel = np.arange(0, 8192, 16)
    o, d = o[sel], d[sel]
    sp = scenes.Sampling(near=0.5, far=2.5, n_samples=256, t_stop=1e-3)
    out = orc.render(g, m, sp, rays=(o, d))
    tgt = scenes.random_targets(8192)[sel].astype(np.float64)
    grad = 2.0 * (out["rgb"] - tgt) / (8192 * 3)
    grad[out["amb"]] = 0.0
    wd, wf, wm = orc.backward(g, m, sp, grad, rays=(o, d), with_mlp=with_mlp)
    res = gpu_grads(cc, g, m, o, d, sp, grad, with_mlp=with_mlp)
    assert rel_inf(res[0], wd) <= 1e-3, rel_inf(res[0], wd)
    assert rel_inf(res[1], wf) <= 1e-3, rel_inf(res[1], wf)
    if with_mlp:
        for name, a, b in zip(("w1", "b1", "w2", "b2", "w3", "b3"), mlp_parts(m, res[2]), mlp_parts(m, wm)):
            assert rel_inf(a, b) <= 1e-3, (name, rel_inf(a, b))


def test_backward_degenerate(cc, orc):
    """No rays: a valid call that adds nothing.  Rays that miss the box, or whose loss gradient is
    zero, add nothing either, and rays beside them keep their oracle gradient."""
    import torch
    g = scenes.scene_fd().astype(np.float32)
    m = scenes.make_mlp(4, random_bias=True)
    gd, md = cc.DeviceGrid.from_host(g), cc.DeviceMlp.from_host(m)
    sp = scenes.Sampling(near=0.5, far=2.5, n_samples=32, t_stop=0.0)
    sd = cc.sampling_from(sp)
    z = torch.zeros(0, 3, device="cuda")
    dd = torch.zeros(g.density.shape, device="cuda")
    df = torch.zeros(g.features.shape, device="cuda")
    ws = cc.workspace(cc.cicero_backward_workspace_size(gd.desc, 0, sd))
    ws.fill_(0xFF)  # whatever the workspace held, the call leaves a clear status word
    cc.cicero_render_backward(gd.desc, md.desc, z, z, sd, z, dd, df, None, ws)
    cc.cicero_workspace_status(ws)
    assert float(dd.abs().max()) == 0.0 and float(df.abs().max()) == 0.0
    # 16 rays: 4 miss the box (origin far away, pointing away), 4 have a zero loss gradient
    o, d = scenes.random_rays(16, seed=9)
    o[:4] = np.array([5.0, 5.0, 5.0], dtype=o.dtype)
    d[:4] = np.array([1.0, 0.0, 0.0], dtype=d.dtype)
    tgt = scenes.random_targets(16, seed=10).astype(np.float64)
    out = orc.render(g, m, sp, rays=(o, d))
    grad = 2.0 * (out["rgb"] - tgt) / tgt.size
    grad[4:8] = 0.0
    wd, wf, _ = orc.backward(g, m, sp, grad, rays=(o, d))
    gd_, gf_ = gpu_grads(cc, g, m, o, d, sp, grad)
    assert rel_inf(gd_, wd) <= 1e-3, rel_inf(gd_, wd)
    assert rel_inf(gf_, wf) <= 1e-3, rel_inf(gf_, wf)


def test_autograd_function_matches_backward(cc, orc):
    import torch
    from paper_2404_11852_gb300.autograd import render_rays
    g = scenes.scene_fd().astype(np.float32)
    m = scenes.make_mlp(4, random_bias=True)
    o, d = scenes.random_rays(64, seed=3)
    sp = scenes.Sampling(near=0.5, far=2.5, n_samples=48, t_stop=0.0)
    dens = torch.from_numpy(g.density).cuda().requires_grad_(True)
    feat = torch.from_numpy(g.features).cuda().requires_grad_(True)
    md = cc.DeviceMlp.from_host(m)
    rgb = render_rays(dens, feat, md, torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda(), sp)
    tgt = torch.from_numpy(scenes.random_targets(64, seed=4)).cuda()
    loss = ((rgb - tgt) ** 2).mean()
    loss.backward()
    ref = orc.render(g, m, sp, rays=(o, d))
    np.testing.assert_allclose(rgb.detach().cpu().double().numpy(), ref["rgb"], atol=1e-4)
    grad = 2.0 * (ref["rgb"] - tgt.cpu().double().numpy()) / (64 * 3)
    wd, wf, _ = orc.backward(g, m, sp, grad, rays=(o, d))
    assert rel_inf(dens.grad.cpu().double().numpy(), wd) <= 1e-3
    assert rel_inf(feat.grad.cpu().double().numpy(), wf) <= 1e-3


@pytest.mark.parametrize("path", ["tc", "simt"])
@pytest.mark.parametrize("case", ["fd", "occ", "few"])
def test_backward_mlp_weights(cc, orc, case, path):
    """dL/d(W1, b1, W2, b2, W3, b3) against the oracle, per tensor (relative inf-norm <= 1e-3),
    together with the grid gradients of the same call (which must not change with d_mlp).  "few":
    two rays, under 16 composited samples (one partial block of the staged operands, every other
    CTA of the weight-gradient kernel idle), in a workspace of NaN bytes."""
    fill = None
    if case == "few":
        g = scenes.scene_fd().astype(np.float32)
        m = scenes.make_mlp(4, random_bias=True)
        o, d = scenes.random_rays(2, seed=5)
        sp = scenes.Sampling(near=0.5, far=2.5, n_samples=6, t_stop=0.0)
        fill = 0xFF
    elif case == "fd":
        g = scenes.scene_fd().astype(np.float32)
        m = scenes.make_mlp(4, random_bias=True)
        o, d = scenes.random_rays(64, seed=5)
        sp = scenes.Sampling(near=0.5, far=2.5, n_samples=48, t_stop=0.0)
    else:
        g = scenes.make_grid(64, 12, 8, seed=32, dtype=np.float16, occ_res=16, occ_frac=0.3)
        m = scenes.make_mlp(12, seed=33, random_bias=True)
        o, d = scenes.random_rays(400, seed=36)
        sp = scenes.sampling_march(64, 128)
    R = o.shape[0]
    out = orc.render(g, m, sp, rays=(o, d))
    tgt = scenes.random_targets(R, seed=37).astype(np.float64)
    grad = 2.0 * (out["rgb"] - tgt) / tgt.size
    grad[out["amb"]] = 0.0  # ambiguous early stops contribute nothing on either side
    wd, wf, wm = orc.backward(g, m, sp, grad, rays=(o, d), with_mlp=True)
    dd, df, dm = gpu_grads(cc, g, m, o, d, sp, grad, with_mlp=True, mlp_path=path, fill=fill)
    assert rel_inf(dd, wd) <= 1e-3, rel_inf(dd, wd)
    assert rel_inf(df, wf) <= 1e-3, rel_inf(df, wf)
    names = ("w1", "b1", "w2", "b2", "w3", "b3")
    for name, a, b in zip(names, mlp_parts(m, dm), mlp_parts(m, wm)):
        assert np.abs(b).max() > 0.0, name
        assert rel_inf(a, b) <= 1e-3, (name, rel_inf(a, b))


def test_backward_mlp_weights_degenerate(cc, orc):
    """With d_mlp and the tensor-core workspace: no rays, and rays that all miss the box, add
    nothing to any gradient and leave a clear status word (workspace of NaN bytes)."""
    import torch
    g = scenes.scene_fd().astype(np.float32)
    m = scenes.make_mlp(4, random_bias=True)
    sp = scenes.Sampling(near=0.5, far=2.5, n_samples=32, t_stop=0.0)
    for R in (0, 8):
        o, d = scenes.random_rays(max(R, 1), seed=9)
        o, d = o[:R].copy(), d[:R].copy()
        o[:] = np.array([5.0, 5.0, 5.0], dtype=o.dtype)
        d[:] = np.array([1.0, 0.0, 0.0], dtype=d.dtype)
        grad = np.ones((R, 3))
        dd, df, dm = gpu_grads(cc, g, m, o, d, sp, grad, with_mlp=True, mlp_path="tc", fill=0xFF)
        assert np.abs(dd).max() == 0.0 and np.abs(df).max() == 0.0 and np.abs(dm).max() == 0.0, R


def test_backward_weight_path_dispatch(cc, orc):
    """The weight gradients run as the staged tensor-core GEMMs (one weight-gradient launch per
    call) when the workspace is cicero_backward_mlp_workspace_size, and on the CUDA cores (no such
    launch) when it is only cicero_backward_workspace_size; both give the same gradients (each path
    is within 1e-3 of the oracle elsewhere, so within 2e-3 of the other)."""
    import torch
    g = scenes.scene_fd().astype(np.float32)
    m = scenes.make_mlp(4, random_bias=True)
    o, d = scenes.random_rays(64, seed=5)
    sp = scenes.Sampling(near=0.5, far=2.5, n_samples=48, t_stop=0.0)
    grad = np.random.default_rng(3).standard_normal((64, 3)) * 1e-2
    out = {}
    for path in ("tc", "simt"):
        torch.cuda.synchronize()
        cc.cicero_profile_begin()
        out[path] = gpu_grads(cc, g, m, o, d, sp, grad, with_mlp=True, mlp_path=path)
        torch.cuda.synchronize()
        prof = cc.cicero_profile_end()
        assert prof["bwd_weights"][1] == (1 if path == "tc" else 0), (path, prof["bwd_weights"])
        assert prof["bwd_brick"][1] == 1, (path, prof["bwd_brick"])
    for a, b in zip(out["tc"], out["simt"]):
        assert rel_inf(a, b) <= 2e-3, rel_inf(a, b)


@pytest.mark.parametrize("C, path", [(16, "tc"), (16, "simt"), (20, "tc")])
def test_backward_sixteen_channels(cc, orc, C, path):
    """C = 16, the widest grid the tensor-core kernels take (dL/dfeatures fills the N = 16 MMA, the
    input row 16 + 27 = 43 of 48 columns): grid and all six MLP gradients against the oracle, with
    the weight gradients on the tensor cores and on the CUDA cores.  C = 20 with the tensor-core
    workspace: beyond that width the backward takes the FP32 recompute and the CUDA-core kernel."""
    g = scenes.make_grid(40, C, 6, seed=51)
    m = scenes.make_mlp(C, seed=52, random_bias=True)
    o, d = scenes.random_rays(200, seed=53)
    sp = scenes.Sampling(near=0.5, far=2.5, n_samples=64, t_stop=1e-3)
    out = orc.render(g, m, sp, rays=(o, d))
    tgt = scenes.random_targets(200, seed=54).astype(np.float64)
    grad = 2.0 * (out["rgb"] - tgt) / tgt.size
    grad[out["amb"]] = 0.0
    wd, wf, wm = orc.backward(g, m, sp, grad, rays=(o, d), with_mlp=True)
    dd, df, dm = gpu_grads(cc, g, m, o, d, sp, grad, with_mlp=True, mlp_path=path)
    assert rel_inf(dd, wd) <= 1e-3, rel_inf(dd, wd)
    assert rel_inf(df, wf) <= 1e-3, rel_inf(df, wf)
    for name, a, b in zip(("w1", "b1", "w2", "b2", "w3", "b3"), mlp_parts(m, dm), mlp_parts(m, wm)):
        assert rel_inf(a, b) <= 1e-3, (name, rel_inf(a, b))


def test_autograd_mlp_weights(cc, orc):
    """The autograd wrapper's MLP gradients (tensors with requires_grad) against the oracle."""
    import torch
    from paper_2404_11852_gb300.autograd import render_rays
    g = scenes.scene_fd().astype(np.float32)
    m = scenes.make_mlp(4, random_bias=True)
    o, d = scenes.random_rays(64, seed=6)
    sp = scenes.Sampling(near=0.5, far=2.5, n_samples=48, t_stop=0.0)
    dens = torch.from_numpy(g.density).cuda()
    feat = torch.from_numpy(g.features).cuda()
    params = [torch.from_numpy(a).cuda().float().requires_grad_(True) for a in (m.w1, m.b1, m.w2, m.b2, m.w3, m.b3)]
    md = cc.DeviceMlp(*params, n_freq=m.n_freq)
    rgb = render_rays(dens, feat, md, torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda(), sp)
    tgt = torch.from_numpy(scenes.random_targets(64, seed=7)).cuda()
    ((rgb - tgt) ** 2).mean().backward()
    ref = orc.render(g, m, sp, rays=(o, d))
    grad = 2.0 * (ref["rgb"] - tgt.cpu().double().numpy()) / (64 * 3)
    _, _, wm = orc.backward(g, m, sp, grad, rays=(o, d), with_mlp=True)
    for p, b in zip(params, mlp_parts(m, wm)):
        assert p.grad is not None and p.grad.shape == p.shape
        assert rel_inf(p.grad.cpu().double().numpy().ravel(), b) <= 1e-3
