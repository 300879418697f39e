"""CSI head and channel loss (Sec. 4.2 "Rendered Spectrum", Eq. 2; Sec. 5 training
objective, Eq. 3).

TEST INFRASTRUCTURE (see the package docstring).

Eq. 2: the complex channel estimate is the spatial mean of the rendered spectrum over the
H x W grid, h_hat = (1 / HW) sum_{u,v} z[u, v]; with several subcarriers, one estimate per
subcarrier k.

Eq. 3: the channel loss is the squared error of the real and imaginary parts,
(h_re - h_hat_re)^2 + (h_im - h_hat_im)^2.  Reading for several transmitters and
subcarriers: the mean of that squared error over all (transmitter, subcarrier) entries
(a complex MSE, which is Eq. 3 itself for one transmitter and one subcarrier).

NMSE = sum |h_hat - h|^2 / sum |h|^2 (Sec. 5.3, the Argos evaluation).
"""
from __future__ import annotations

import numpy as np


def csi_head(z: np.ndarray, H: int, W: int) -> np.ndarray:
    """Eq. 2.  z [..., H*W, K] complex (pixels row-major) -> h_hat [..., K]."""
    z = np.asarray(z)
    assert z.shape[-2] == H * W
    return z.sum(axis=-2) / (H * W)


def channel_loss(h_hat: np.ndarray, h: np.ndarray):
    """Eq. 3 averaged over the entries.  Returns (loss, dL/dh_hat) with the gradient as a
    complex array g = dL/dRe + j dL/dIm."""
    d = np.asarray(h_hat) - np.asarray(h)
    m = d.size
    loss = float(np.sum(d.real ** 2 + d.imag ** 2) / m)
    return loss, 2.0 * d / m


def csi_head_bwd(d_h: np.ndarray, H: int, W: int) -> np.ndarray:
    """Gradient of Eq. 2: every pixel of plane k receives d_h[..., k] / HW.
    d_h [..., K] -> [..., H*W, K]."""
    d_h = np.asarray(d_h)
    return np.broadcast_to(d_h[..., None, :] / (H * W), d_h.shape[:-1] + (H * W, d_h.shape[-1])).copy()


def nmse(h_hat: np.ndarray, h: np.ndarray) -> float:
    d = np.asarray(h_hat) - np.asarray(h)
    return float(np.sum(np.abs(d) ** 2) / np.sum(np.abs(np.asarray(h)) ** 2))
