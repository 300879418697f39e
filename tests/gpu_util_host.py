"""Host-only helpers shared by the CPU (host shim) and GPU tests: the oracle's per-Gaussian
values for a seeded scene, rounded to FP32, as the projection records and attributes both sides
consume."""
import numpy as np
import torch

from oracle import attributes as oattr
from oracle import projection as oproj
from paper_2511_22793_gb300 import synth


def oracle_inputs_fp32(n, view, B, seed, hidden=32):
    """(g32, at32, proj [n,8] f32, attr [B,n,4] f32): the oracle's projection and attributes of a
    seeded n-Gaussian scene seen from B seeded transmitters, rounded to FP32; g32 / at32 hold the
    same values in float64 for the oracle's renderer."""
    sc = synth.make_scene(n, seed=seed)
    mlp = synth.make_mlp(hidden, seed=3)
    tx = synth.make_tx(B, seed=seed + 1)
    f64 = lambda a: torch.tensor(np.asarray(a), dtype=torch.float64)
    geo = oproj.project(f64(sc.means), f64(sc.log_scales), f64(sc.quats), view)
    g = {k: geo[k].numpy() for k in ("px", "py", "cxx", "cxy", "cyy", "r", "valid", "sxx", "syy")}
    weights = [f64(a) for a in mlp.arrays()]
    attrs = []
    for t in np.asarray(tx, dtype=np.float64):
        at = oattr.attributes(f64(sc.means), f64(sc.opacity_logit), f64(sc.latent), weights, t, view.rx)
        attrs.append({k: at[k].numpy() for k in ("sigma", "a", "phi0", "L")})
    g32 = {k: (v.astype(np.float32).astype(np.float64) if v.dtype != bool else v) for k, v in g.items()}
    at32 = [{k: v.astype(np.float32).astype(np.float64) for k, v in at.items()} for at in attrs]
    proj = np.zeros((n, 8), np.float32)
    proj[:, 0], proj[:, 1] = g32["px"], g32["py"]
    proj[:, 2] = np.where(g["valid"], np.sqrt(2 * np.log(255) * g["sxx"]), -1)
    proj[:, 3] = np.where(g["valid"], np.sqrt(2 * np.log(255) * g["syy"]), -1)
    proj[:, 4], proj[:, 5], proj[:, 6], proj[:, 7] = g32["cxx"], g32["cxy"], g32["cyy"], g32["r"]
    attr = np.stack([np.stack([at["a"], at["phi0"], at["sigma"], at["L"]], -1) for at in at32]).astype(np.float32)
    return g32, at32, proj, attr
