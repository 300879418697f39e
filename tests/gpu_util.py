"""Helpers shared by the GPU parity tests: run the CUDA path through the C ABI
on seeded synthetic inputs, run the FP64 oracle on the same inputs, compare."""
from __future__ import annotations

import numpy as np
import torch

from oracle import attributes as oattr
from oracle import projection as oproj
from oracle import render as orender
from paper_2511_22793_gb300 import gsparc as G
from paper_2511_22793_gb300 import synth
from paper_2511_22793_gb300.pipeline import DeviceMLP, DeviceScene, Renderer

DEV = "cuda"


def rel_l2(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    den = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (den if den > 0 else 1.0))


def spectrum_to_complex(spec):
    """[B, K, H, W, 2] float32 tensor -> [B, H*W, K] complex128 (oracle layout)."""
    z = spec.detach().cpu().numpy().astype(np.float64)
    B, K, H, W, _ = z.shape
    return (z[..., 0] + 1j * z[..., 1]).transpose(0, 2, 3, 1).reshape(B, H * W, K)


def oracle_geo_attr(sc, mlp, view, tx):
    """FP64 projection (dict of numpy) and attributes (list of dicts) of the oracle."""
    f64 = lambda a: torch.tensor(np.asarray(a), dtype=torch.float64)
    geo = oproj.project(f64(sc.means), f64(sc.log_scales), f64(sc.quats), view)
    weights = [f64(a) for a in mlp.arrays()]
    attrs = []
    for t in np.asarray(tx, dtype=np.float64):
        at = oattr.attributes(f64(sc.means), f64(sc.opacity_logit), f64(sc.latent), weights, t, view.rx)
        attrs.append({k: at[k].numpy() for k in ("sigma", "a", "phi0", "L")})
    g = {k: geo[k].numpy() for k in ("px", "py", "cxx", "cxy", "cyy", "r", "valid", "ext_x", "ext_y",
                                     "sxx", "sxy", "syy")}
    return g, attrs


def oracle_render(g, attrs, view, band, pixels=None):
    zs, Ts, ns = [], [], []
    for at in attrs:
        z, T, n = orender.render_fwd(g, at, view.H, view.W, band.K, band.f_c, band.df, pixels=pixels)
        zs.append(z)
        Ts.append(T)
        ns.append(n)
    return np.stack(zs), np.stack(Ts), np.stack(ns)


def gpu_forward(sc, mlp, H, W, K, tx, precision=G.GSPARC_FP32, capacity=None):
    r = Renderer(H, W, K, sc.n, pair_capacity=capacity, device=DEV)
    ds = DeviceScene.from_host(sc, DEV)
    dm = DeviceMLP.from_host(mlp, DEV)
    txd = torch.tensor(np.asarray(tx, dtype=np.float32), device=DEV)
    r.geometry(ds)
    attr = r.attributes(ds, dm, txd, precision)
    spec, logT, nc = r.render(attr)
    torch.cuda.synchronize()
    assert r.check() == 0
    return r, ds, dm, txd, attr, spec, logT, nc
