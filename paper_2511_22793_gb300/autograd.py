"""torch.autograd.Function over the hand-written forward and backward kernels.

Forward: gsparc_project -> gsparc_bin_sort -> gsparc_attr_mlp ->
gsparc_render_fwd.  Backward: gsparc_render_bwd (per-pixel state recomputed
from the stored final log-transmittance and contributor count) ->
gsparc_attr_mlp_bwd and gsparc_project_bwd.  Binning and sorting are not
differentiated (the ordering is piecewise constant).
"""
from __future__ import annotations

import torch

from . import gsparc as G
from .pipeline import DeviceMLP, DeviceScene, Renderer


class SplatFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, renderer: Renderer, tx, means, log_scales, quats, opacity_logit, latent,
                W1, b1, W2, b2, W3, b3):
        scene = DeviceScene(means, log_scales, quats, opacity_logit, latent)
        mlp = DeviceMLP(int(W2.shape[0]), W1, b1, W2, b2, W3, b3)
        renderer.geometry(scene)
        attr = renderer.attributes(scene, mlp, tx)
        spec, logT, nc = renderer.render(attr)
        ctx.renderer = renderer
        ctx.save_for_backward(tx, means, log_scales, quats, opacity_logit, latent, W1, b1, W2, b2,
                              W3, b3, attr, logT, nc)
        ctx.mark_non_differentiable(logT, nc)
        return spec

    @staticmethod
    def backward(ctx, d_spec):
        r: Renderer = ctx.renderer
        (tx, means, log_scales, quats, ologit, latent, W1, b1, W2, b2, W3, b3, attr, logT,
         nc) = ctx.saved_tensors
        scene = DeviceScene(means, log_scales, quats, ologit, latent)
        mlp = DeviceMLP(int(W2.shape[0]), W1, b1, W2, b2, W3, b3)
        d_spec = d_spec.contiguous()
        d_attr = torch.zeros_like(attr)
        d_proj = torch.zeros_like(r.proj)
        r.render_backward(attr, logT, nc, d_spec, d_attr, d_proj)
        d_means = torch.zeros_like(means)
        d_ls = torch.zeros_like(log_scales)
        d_q = torch.zeros_like(quats)
        d_ol = torch.zeros_like(ologit)
        d_lat = torch.zeros_like(latent)
        d_w = [torch.zeros_like(t) for t in (W1, b1, W2, b2, W3, b3)]
        r.attributes_backward(scene, mlp, tx, d_attr, d_means, d_ol, d_lat, d_w)
        r.project_backward(scene, d_proj, d_means, d_ls, d_q)
        return (None, None, d_means, d_ls, d_q, d_ol, d_lat, *d_w)


def splat(renderer: Renderer, tx, scene_params, mlp_params):
    """Differentiable spectrum [B, K, H, W, 2] for transmitters tx [B, 3]."""
    return SplatFunction.apply(renderer, tx, *scene_params, *mlp_params)
