"""Shared helpers of the GPU parity tests: run the CUDA path through the C ABI and compare it
with the oracle, accepting either outcome on rays whose early-stop decision is ambiguous."""
import numpy as np

AMBIG_MAX_FRAC = 1e-3


def gpu_render(cc, grid_h, mlp_h, cam, sp, precision=0, brick=8, dev_grid=None, dev_mlp=None):
    import torch
    g = dev_grid or cc.DeviceGrid.from_host(grid_h)
    m = dev_mlp or cc.DeviceMlp.from_host(mlp_h)
    cd, sd, opt = cc.camera_from(cam), cc.sampling_from(sp), cc.options(precision, brick)
    R = cam.width * cam.height
    ws = cc.workspace(cc.cicero_render_workspace_size(g.desc, R, sd, opt))
    rgb = torch.empty(R, 3, device="cuda")
    depth = torch.empty(R, device="cuda")
    acc = torch.empty(R, device="cuda")
    ns = torch.empty(R, dtype=torch.int32, device="cuda")
    cc.cicero_render(g.desc, m.desc, cd, sd, opt, rgb, depth, acc, ns, ws)
    cc.cicero_workspace_status(ws)
    return {"rgb": rgb.cpu().numpy().astype(np.float64), "depth": depth.cpu().numpy().astype(np.float64),
            "acc": acc.cpu().numpy().astype(np.float64), "n_steps": ns.cpu().numpy()}


def rgb_errors(out_rgb, ref, idx=None):
    """Per-ray max |rgb error|, taking the better outcome on ambiguous rays."""
    r, ra, amb = ref["rgb"], ref["rgb_alt"], ref["amb"]
    if idx is not None:
        r, ra, amb = r[idx], ra[idx], amb[idx]
    e = np.abs(out_rgb - r).max(axis=1)
    ea = np.abs(out_rgb - ra).max(axis=1)
    return np.where(amb, np.minimum(e, ea), e), amb


def psnr(a, b):
    mse = float(np.mean((np.asarray(a, np.float64) - np.asarray(b, np.float64)) ** 2))
    return float("inf") if mse == 0 else 10 * np.log10(1.0 / mse)


def check_render(out, ref, tol, void_acc=0.5, psnr_min=None):
    err, amb = rgb_errors(out["rgb"], ref)
    n = len(err)
    assert amb.sum() <= max(2, AMBIG_MAX_FRAC * n), f"{amb.sum()} ambiguous rays of {n}"
    assert err.max() <= tol, f"max |rgb err| {err.max():.3g} > {tol}"
    # accumulated opacity and depth on non-ambiguous rays
    ok = ~amb
    assert np.abs(out["acc"][ok] - ref["acc"][ok]).max(initial=0) <= tol
    sure = ok & (np.abs(ref["acc"] - void_acc) > 1e-3)
    fin_g, fin_o = np.isfinite(out["depth"][sure]), np.isfinite(ref["depth"][sure])
    assert (fin_g == fin_o).all()
    both = np.isfinite(out["depth"]) & np.isfinite(ref["depth"]) & sure
    if both.any():
        assert np.abs(out["depth"][both] - ref["depth"][both]).max() <= 20 * tol
    if "n_steps" in out:
        assert (out["n_steps"][ok] == ref["n_steps"][ok]).all()
    if psnr_min is not None:
        best = np.where(amb[:, None], np.where(
            np.abs(out["rgb"] - ref["rgb"]).max(1, keepdims=True) <= np.abs(out["rgb"] - ref["rgb_alt"]).max(1, keepdims=True),
            ref["rgb"], ref["rgb_alt"]), ref["rgb"])
        p = psnr(out["rgb"], best)
        assert p >= psnr_min, f"PSNR {p:.2f} dB < {psnr_min}"
        return err.max(), p
    return err.max(), None
