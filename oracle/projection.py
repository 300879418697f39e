"""Oracle projection: receiver-centric transform, equirectangular map, 2D covariance.

TEST INFRASTRUCTURE (see the package docstring).  Plain PyTorch CPU ops in
float64; autograd on these ops supplies the oracle's projection gradient.

Follows Sec. 4.2 ("Directional Projection and Splatting"):
  x' = V (mu - x_rx)
  p_x = (atan2(x', z') / pi + 1) W / 2
  p_y = 2 asin(y' / |x'|) H / pi
  Sigma' = J V Sigma V^T J^T  (depth dropped)
and Sec. 3.2 for Sigma = R S S^T R^T with R from a quaternion and S the
diagonal of scales.

Readings (the paper is silent on these):
  - quaternion order (w, x, y, z), normalised before use;
  - scales are exp(log_scale), so S S^T = diag(exp(2 log_scale));
  - J is the Jacobian of the map above, except that in the azimuth row the
    factor 1/rho (rho = sqrt(x'^2 + z'^2)) is capped at 1/max(rho, 1e-3 |x'|)
    while the row keeps its direction (z'/rho, 0, -x'/rho); exactly at the
    zenith that direction is taken as (1, 0, 0).  The elevation row is exact.
    Near the zenith the azimuth of a direction changes faster than any
    footprint the linearisation can describe, and this keeps the footprint
    wide in azimuth (every column) instead of collapsing it;
  - 0.3 px^2 is added to the diagonal of Sigma' (3D Gaussian Splatting
    practice, on which the paper builds);
  - a Gaussian closer than r_near to the receiver is culled;
  - the footprint's half extents are sqrt(q_max Sigma'_xx) and
    sqrt(q_max Sigma'_yy) with q_max = 2 ln 255, the level at which the
    kernel falls to 1/255.
"""
from __future__ import annotations

import math

import torch

Q_MAX = 2.0 * math.log(255.0)
DILATION = 0.3
RHO_FLOOR = 1e-3


def quat_to_rotmat(q: torch.Tensor) -> torch.Tensor:
    """Rotation matrix of the unit quaternion q/|q|, q = (w, x, y, z) (Hamilton)."""
    q = q / torch.linalg.norm(q, dim=-1, keepdim=True)
    w, x, y, z = q.unbind(-1)
    rows = [
        torch.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], -1),
        torch.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], -1),
        torch.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], -1),
    ]
    return torch.stack(rows, -2)


def covariance3d(log_scales: torch.Tensor, quats: torch.Tensor) -> torch.Tensor:
    """Sigma = R S S^T R^T (Sec. 3.2)."""
    R = quat_to_rotmat(quats)
    S2 = torch.diag_embed(torch.exp(2.0 * log_scales))
    return R @ S2 @ R.transpose(-1, -2)


def equirect_map(xp: torch.Tensor, H: int, W: int):
    """Pixel coordinates of receiver-frame points (Sec. 4.2 map)."""
    x, y, z = xp.unbind(-1)
    r = torch.linalg.norm(xp, dim=-1)
    px = (torch.atan2(x, z) / math.pi + 1.0) * (W / 2.0)
    py = 2.0 * torch.asin(torch.clamp(y / r, -1.0, 1.0)) * (H / math.pi)
    return px, py, r


def map_jacobian(xp: torch.Tensor, H: int, W: int) -> torch.Tensor:
    """d(p_x, p_y)/d(x', y', z'), a [.., 2, 3] matrix, with the zenith cap on 1/rho."""
    x, y, z = xp.unbind(-1)
    r2 = (xp * xp).sum(-1)
    r = torch.sqrt(r2)
    rho = torch.sqrt(x * x + z * z)
    pos = rho > 0
    safe = torch.where(pos, rho, torch.ones_like(rho))
    cx = torch.where(pos, x / safe, torch.zeros_like(x))     # sin(azimuth)
    cz = torch.where(pos, z / safe, torch.ones_like(z))      # cos(azimuth)
    rho_cap = torch.maximum(rho, RHO_FLOOR * r)
    sx = W / (2.0 * math.pi)
    sy = 2.0 * H / math.pi
    zero = torch.zeros_like(x)
    row0 = torch.stack([sx * cz / rho_cap, zero, -sx * cx / rho_cap], -1)
    row1 = torch.stack([-sy * y * cx / r2, sy * rho / r2, -sy * y * cz / r2], -1)
    return torch.stack([row0, row1], -2)


def project(means, log_scales, quats, view):
    """Project every Gaussian.  Inputs are float64 tensors (or arrays).

    Returns a dict of float64 tensors: px, py, cxx, cxy, cyy (the conic, i.e.
    the inverse of Sigma'), sxx, sxy, syy (Sigma'), r (receiver distance),
    ext_x, ext_y (footprint half extents) and a bool tensor valid.
    """
    means = torch.as_tensor(means, dtype=torch.float64)
    log_scales = torch.as_tensor(log_scales, dtype=torch.float64)
    quats = torch.as_tensor(quats, dtype=torch.float64)
    V = torch.tensor(view.V, dtype=torch.float64).reshape(3, 3)
    rx = torch.tensor(view.rx, dtype=torch.float64)

    xp = (means - rx) @ V.T
    px, py, r = equirect_map(xp, view.H, view.W)
    J = map_jacobian(xp, view.H, view.W)
    Sigma = covariance3d(log_scales, quats)
    M = J @ V                                   # J V
    S2 = M @ Sigma @ M.transpose(-1, -2)        # J V Sigma V^T J^T
    sxx = S2[:, 0, 0] + DILATION
    sxy = S2[:, 0, 1]
    syy = S2[:, 1, 1] + DILATION
    det = sxx * syy - sxy * sxy
    cxx = syy / det
    cxy = -sxy / det
    cyy = sxx / det
    ext_x = torch.sqrt(Q_MAX * sxx)
    ext_y = torch.sqrt(Q_MAX * syy)
    valid = r >= view.near
    return dict(px=px, py=py, cxx=cxx, cxy=cxy, cyy=cyy, sxx=sxx, sxy=sxy, syy=syy,
                r=r, ext_x=ext_x, ext_y=ext_y, valid=valid)
