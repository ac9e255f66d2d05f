"""torch.autograd.Function around the FP32 renderer and its hand-written backward.

Forward: ``cicero_render_rays`` (FP32 MLP).  Backward: ``cicero_render_backward``, which
recomputes each ray's forward pass and returns the gradients of the density and feature grids
and, when any of the MLP's tensors requires a gradient, of the MLP's six tensors
(w1, b1, w2, b2, w3, b3).  Only argument marshalling happens here.
"""
from __future__ import annotations

import torch

from . import cicero as cc


class RenderRays(torch.autograd.Function):
    @staticmethod
    def forward(ctx, density, features, ray_o, ray_d, mlp, sp, aabb_min, aabb_max, act_shift, occ, *mlp_params):
        grid = cc.DeviceGrid(density.detach(), features.detach(), aabb_min, aabb_max, act_shift, occ)
        sd = cc.sampling_from(sp)
        R = ray_o.shape[0]
        rgb = torch.empty(R, 3, device=ray_o.device, dtype=torch.float32)
        ws = cc.workspace(cc.cicero_render_workspace_size(grid.desc, R, sd), ray_o.device)
        cc.cicero_render_rays(grid.desc, mlp.desc, ray_o, ray_d, sd, None, rgb, None, None, None, ws)
        ctx.save_for_backward(density, features, ray_o, ray_d)
        ctx.mlp, ctx.sp, ctx.meta = mlp, sp, (aabb_min, aabb_max, act_shift, occ)
        ctx.mlp_shapes = [p.shape for p in mlp_params]
        return rgb

    @staticmethod
    def backward(ctx, d_rgb):
        density, features, ray_o, ray_d = ctx.saved_tensors
        aabb_min, aabb_max, act_shift, occ = ctx.meta
        grid = cc.DeviceGrid(density.detach(), features.detach(), aabb_min, aabb_max, act_shift, occ)
        sd = cc.sampling_from(ctx.sp)
        dd = torch.zeros(density.shape, device=density.device, dtype=torch.float32)
        df = torch.zeros(features.shape, device=features.device, dtype=torch.float32)
        want_mlp = any(ctx.needs_input_grad[10:])
        n_mlp = sum(int(torch.Size(s).numel()) for s in ctx.mlp_shapes)
        dm = torch.zeros(n_mlp, device=density.device, dtype=torch.float32) if want_mlp else None
        # with MLP gradients, a workspace that holds their staged operands (tensor-core GEMMs)
        size = cc.cicero_backward_mlp_workspace_size if want_mlp else cc.cicero_backward_workspace_size
        ws = cc.workspace(size(grid.desc, ray_o.shape[0], sd), ray_o.device)
        cc.cicero_render_backward(grid.desc, ctx.mlp.desc, ray_o, ray_d, sd, d_rgb.contiguous().float(), dd, df,
                                  dm, ws)
        mlp_grads = [None] * len(ctx.mlp_shapes)
        if want_mlp:
            mlp_grads = list(torch.split(dm, [int(torch.Size(s).numel()) for s in ctx.mlp_shapes]))
            mlp_grads = [g.view(s) for g, s in zip(mlp_grads, ctx.mlp_shapes)]
        return (dd.to(density.dtype), df.to(features.dtype), None, None, None, None, None, None, None, None,
                *mlp_grads)


def render_rays(density, features, mlp, ray_o, ray_d, sp, aabb_min=(-1.0, -1.0, -1.0), aabb_max=(1.0, 1.0, 1.0),
                act_shift: float = -4.0, occ=None):
    """rgb [R, 3] of explicit rays, differentiable with respect to ``density``, ``features`` and the
    tensors of ``mlp`` (a ``DeviceMlp``; float32 contiguous tensors are used as given, so their
    ``requires_grad`` carries through)."""
    return RenderRays.apply(density, features, ray_o, ray_d, mlp, sp, aabb_min, aabb_max, act_shift, occ, *mlp.t)
