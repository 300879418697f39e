"""Oracle adaptive density control (Algorithm 1, densification branch; Sec. 4.2 "Densification,
Pruning, and Implementation").

TEST INFRASTRUCTURE (see the package docstring).  float64 NumPy; the rotation matrix comes from
the oracle's projection module.

What the paper states: while the step count i is below T_densify, per-Gaussian positional
gradient norms are accumulated; every Delta_densify steps each Gaussian whose accumulated norm
reaches tau_grad is cloned in place when max(Sigma_i) <= eps * r_scene, and otherwise split into N
children whose scale is Sigma_i / (0.8 N); Gaussians with opacity below sigma_min or a screen
footprint above r_max are pruned; every Delta_reset steps every opacity becomes min(sigma_i, 0.01).

Readings (the paper gives none of the thresholds and leaves the details open):
  - the statistic is the mean of ||dL/dmu_i|| over the steps since the last densification in
    which Gaussian i was visible, i.e. its projection was not culled (footprint radius > 0); a
    Gaussian never visible is not a candidate;
  - max(Sigma_i) is the largest per-axis scale exp(l_i); the scale rule divides the per-axis
    scales by 0.8 N, i.e. log-scales minus ln(0.8 N);
  - a child of a split sits at mu_i + R_i diag(exp(l_i)) xi, xi ~ N(0, I_3) drawn from the
    parent's own distribution; the draws are inputs [N, n_split, 3], row i serving Gaussian i
    if it splits (a row per Gaussian keeps the draws independent of the decisions); a child copies the parent's
    rotation, opacity and per-Gaussian payload (latent or emission buffer); the parent goes;
  - a clone is an exact copy;
  - output order: parents in index order, each emitting in place its kept self, then its
    clone, or its N children; pruning then removes entries without reordering;
  - pruning by opacity, sigmoid(logit) < sigma_min (strict), applies to every output; pruning by
    footprint, radius > r_max (strict, the largest projected half-extent in pixels of the last
    step), applies to the Gaussians that existed before this densification (clones and children
    have no footprint yet);
  - the opacity reset acts on the logit: logit <- min(logit, logit(0.01));
  - schedule: steps count from 1; accumulate while i < T_densify; densify when also
    i mod Delta_densify == 0; reset when also i mod Delta_reset == 0 (both inside the
    i < T_densify branch, as Algorithm 1 nests them); statistics restart after a densification;
  - proposed values (3D Gaussian Splatting conventions where it has one): tau_grad = 2e-4,
    eps = 0.01, r_scene = 5 sqrt(3) m (the half-diagonal of the 10 m scene cube), N = 2,
    sigma_min = 0.005, r_max = 20 px, Delta_densify = 100, Delta_reset = 3000,
    T_densify = 15000.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import torch

from . import projection as P

RESET_OPACITY = 0.01


@dataclass
class Thresholds:
    tau_grad: float = 2e-4
    eps: float = 0.01
    r_scene: float = 5.0 * math.sqrt(3.0)
    n_split: int = 2
    sigma_min: float = 0.005
    r_max: float = 20.0
    densify_every: int = 100
    reset_every: int = 3000
    densify_until: int = 15000


def schedule(i: int, th: Thresholds):
    """(accumulate, densify, reset) flags of step i (1-based)."""
    acc = i < th.densify_until
    return acc, acc and i % th.densify_every == 0, acc and i % th.reset_every == 0


def accumulate(norm_sum, count, grad_means, visible):
    """Adds ||dL/dmu_i|| to norm_sum and 1 to count for every visible Gaussian."""
    vis = np.asarray(visible, dtype=bool)
    g = np.linalg.norm(np.asarray(grad_means, dtype=np.float64), axis=1)
    return norm_sum + np.where(vis, g, 0.0), count + vis.astype(np.int64)


def decide(norm_sum, count, log_scales, th: Thresholds):
    """Per-Gaussian action: 0 keep, 1 clone, 2 split."""
    count = np.asarray(count)
    avg = np.where(count > 0, norm_sum / np.maximum(count, 1), 0.0)
    cand = (count > 0) & (avg >= th.tau_grad)
    small = np.exp(np.asarray(log_scales, dtype=np.float64)).max(axis=1) <= th.eps * th.r_scene
    return np.where(cand, np.where(small, 1, 2), 0)


def densify_and_prune(g, radius, action, xi, th: Thresholds):
    """One densification of the Gaussian set g (dict of float64 arrays: means [N,3], log_scales
    [N,3], quats [N,4], opacity_logit [N], payload [N,P]) given each Gaussian's last footprint
    radius [N] in pixels, its action from `decide`, and the split draws xi [N, n_split, 3] (row i
    used if Gaussian i splits).  Returns the new set and, for each output, the index of its
    parent."""
    n = g["means"].shape[0]
    R = P.quat_to_rotmat(torch.tensor(g["quats"], dtype=torch.float64)).numpy() if n else np.zeros((0, 3, 3))
    scale = np.exp(g["log_scales"])
    rows, parent, fresh = [], [], []
    for i in range(n):
        one = {key: g[key][i] for key in g}
        if action[i] == 2:
            for c in range(th.n_split):
                child = dict(one)
                child["means"] = g["means"][i] + R[i] @ (scale[i] * xi[i, c])
                child["log_scales"] = g["log_scales"][i] - math.log(0.8 * th.n_split)
                rows.append(child)
                parent.append(i)
                fresh.append(True)
            continue
        rows.append(one)
        parent.append(i)
        fresh.append(False)
        if action[i] == 1:
            rows.append(dict(one))
            parent.append(i)
            fresh.append(True)
    keep = []
    for j, row in enumerate(rows):
        sigma = 1.0 / (1.0 + math.exp(-float(row["opacity_logit"])))
        too_faint = sigma < th.sigma_min
        too_wide = (not fresh[j]) and radius[parent[j]] > th.r_max
        keep.append(not (too_faint or too_wide))
    out = {}
    for key in g:
        kept = [row[key] for j, row in enumerate(rows) if keep[j]]
        out[key] = np.array(kept, dtype=np.float64).reshape((len(kept),) + g[key].shape[1:])
    return out, np.array([p for j, p in enumerate(parent) if keep[j]], dtype=np.int64)


def reset_opacity(opacity_logit):
    """sigma <- min(sigma, 0.01), on the logits."""
    cap = math.log(RESET_OPACITY / (1.0 - RESET_OPACITY))
    return np.minimum(np.asarray(opacity_logit, dtype=np.float64), cap)
