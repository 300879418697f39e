"""Oracle forward pass, L2 loss and full FP64 gradient.

TEST INFRASTRUCTURE (see the package docstring).

Forward (Algorithm 1, forward half, with the transmitter as the query and
the receiver fixed): project every Gaussian (projection.py), evaluate the
attribute network for each transmitter (attributes.py), render every
requested pixel with the per-pixel FP64 renderer (render_oracle.c).

Loss: mean over transmitters, pixels and subcarriers of |z - z_target|^2
(complex L2; the workloads use it in place of the paper's L1+SSIM, Eq. 4), or
the channel loss of the spatial-mean CSI head (Eq. 2, Eq. 3; csi.py).

Gradient: the renderer's analytic FP64 gradient (render_oracle.c) chained by
autograd through the float64 projection and attribute network.
"""
from __future__ import annotations

import numpy as np
import torch

from . import attributes as _attr
from . import csi as _csi
from . import projection as _proj
from . import render as _render


def _t(a, grad=False):
    t = torch.tensor(np.asarray(a), dtype=torch.float64)
    if grad:
        t.requires_grad_(True)
    return t


def _geo_np(geo):
    return {k: geo[k].detach().numpy() for k in ("px", "py", "cxx", "cxy", "cyy", "r", "valid")}


def _attr_np(at):
    return {k: at[k].detach().numpy() for k in ("sigma", "a", "phi0", "L")}


def forward(scene, mlp, view, band, tx, pixels=None, exact=False, threads=0):
    """Spectra for every transmitter in tx [B, 3].

    Returns dict: z [B, npix, K] complex128, T [B, npix], n_used [B, npix],
    geo (projection dict), attrs (list of attribute dicts).
    """
    means, log_scales, quats, ologit, latent = [_t(a) for a in scene.arrays()]
    weights = [_t(a) for a in mlp.arrays()]
    with torch.no_grad():
        geo = _proj.project(means, log_scales, quats, view)
        attrs = [_attr.attributes(means, ologit, latent, weights, t, view.rx)
                 for t in np.asarray(tx, dtype=np.float64)]
    zs, Ts, ns = [], [], []
    g = _geo_np(geo)
    for at in attrs:
        z, T, n = _render.render_fwd(g, _attr_np(at), view.H, view.W, band.K, band.f_c, band.df,
                                     pixels=pixels, exact=exact, threads=threads)
        zs.append(z)
        Ts.append(T)
        ns.append(n)
    return dict(z=np.stack(zs), T=np.stack(Ts), n_used=np.stack(ns), geo=geo, attrs=attrs)


def loss_and_grad(scene, mlp, view, band, tx, target, pixels=None, threads=0, loss_kind="l2"):
    """L2 loss against target [B, npix, K] complex and the FP64 gradient.

    loss_kind "csi": the channel loss (Eq. 3) of the spatial-mean estimate (Eq. 2) against
    target [B, K] complex (full images only); grads['h'] holds the estimate.

    Returns (loss, grads) with grads a dict keyed like the inputs: means,
    log_scales, quats, opacity_logit, latent, W1, b1, W2, b2, W3, b3.
    Also returns the spectrum under grads['z'].
    """
    names = ["means", "log_scales", "quats", "opacity_logit", "latent"]
    wnames = ["W1", "b1", "W2", "b2", "W3", "b3"]
    params = [_t(a, grad=True) for a in scene.arrays()]
    weights = [_t(a, grad=True) for a in mlp.arrays()]
    means, log_scales, quats, ologit, latent = params
    geo = _proj.project(means, log_scales, quats, view)
    tx = np.asarray(tx, dtype=np.float64)
    attrs = [_attr.attributes(means, ologit, latent, weights, t, view.rx) for t in tx]
    g = _geo_np(geo)
    target = np.asarray(target)
    B = tx.shape[0]
    zs = []
    for b in range(B):
        z, _, _ = _render.render_fwd(g, _attr_np(attrs[b]), view.H, view.W, band.K, band.f_c,
                                     band.df, pixels=pixels, threads=threads)
        zs.append(z)
    z = np.stack(zs)
    h_hat = None
    if loss_kind == "csi":
        assert pixels is None
        h_hat = _csi.csi_head(z, view.H, view.W)
        loss, d_h = _csi.channel_loss(h_hat, target)
        gz = _csi.csi_head_bwd(d_h, view.H, view.W)
    else:
        M = z.size
        diff = z - target
        loss = float(np.sum(diff.real ** 2 + diff.imag ** 2) / M)
        gz = 2.0 * diff / M
    d_geo = np.zeros((len(g["px"]), 5))
    outs, grads_out = [], []
    for b in range(B):
        gr = _render.render_bwd(g, _attr_np(attrs[b]), view.H, view.W, band.K, band.f_c,
                                band.df, gz[b], pixels=pixels, threads=threads)
        d_geo += gr[:, 0:5]
        for j, k in zip(range(5, 9), ("sigma", "a", "phi0", "L")):
            outs.append(attrs[b][k])
            grads_out.append(torch.tensor(gr[:, j]))
    for j, k in enumerate(("px", "py", "cxx", "cxy", "cyy")):
        outs.append(geo[k])
        grads_out.append(torch.tensor(d_geo[:, j]))
    torch.autograd.backward(outs, grads_out)
    grads = {}
    for nm, p in zip(names + wnames, params + weights):
        grads[nm] = p.grad.numpy().copy() if p.grad is not None else np.zeros(p.shape)
    grads["z"] = z
    if h_hat is not None:
        grads["h"] = h_hat
    return loss, grads


def loss_only(scene, mlp, view, band, tx, target, pixels=None, threads=0):
    out = forward(scene, mlp, view, band, tx, pixels=pixels, threads=threads)
    diff = out["z"] - np.asarray(target)
    return float(np.sum(diff.real ** 2 + diff.imag ** 2) / diff.size)
