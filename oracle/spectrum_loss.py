"""Oracle magnitude-spectrum loss (Eq. 4): L = (1 - lam) L1(|z|, y) + lam (1 - SSIM(|z|, y)).

TEST INFRASTRUCTURE (see the package docstring).  Plain PyTorch CPU ops in float64; autograd
on them supplies the gradient with respect to the magnitudes, chained to the complex spectrum
by hand (d|z|/dz = z / |z|).

Readings (the paper names the loss and lambda_1 = 0.2 but not the SSIM details):
  - the rendered complex spectrum z enters through its magnitude x = |z| (the target is a
    magnitude spectrum y, the RFID/BLE case the paper names), and the gradient of x at z = 0
    is taken as 0;
  - L1 is the mean absolute error over every (transmitter, subcarrier, pixel);
  - SSIM is computed per (transmitter, subcarrier) plane with the conventions of the 3D
    Gaussian splatting code the method builds on: an 11 x 11 Gaussian window with sigma 1.5,
    normalised to sum 1, zero padding with the output the size of the plane, constants
    C1 = 0.01^2 and C2 = 0.03^2; the plane's SSIM is the mean of its SSIM map and the loss
    takes the mean over planes;
  - lam = 0.2.
"""
from __future__ import annotations

import numpy as np
import torch

WINDOW = 11
SIGMA = 1.5
C1 = 0.01 ** 2
C2 = 0.03 ** 2
LAMBDA = 0.2


def window_1d(size=WINDOW, sigma=SIGMA):
    t = np.arange(size, dtype=np.float64) - (size - 1) / 2.0
    g = np.exp(-t * t / (2.0 * sigma * sigma))
    return g / g.sum()


def window_2d(size=WINDOW, sigma=SIGMA):
    g = window_1d(size, sigma)
    return np.outer(g, g)


def _filter(img):
    """'same' zero-padded correlation of every [H, W] plane of img [P, H, W] with the window."""
    w = torch.tensor(window_2d(), dtype=torch.float64).reshape(1, 1, WINDOW, WINDOW)
    return torch.nn.functional.conv2d(img.unsqueeze(1), w, padding=WINDOW // 2).squeeze(1)


def ssim_map(x, y):
    """SSIM map of planes x, y [P, H, W] (float64 tensors)."""
    mx, my = _filter(x), _filter(y)
    sxx = _filter(x * x) - mx * mx
    syy = _filter(y * y) - my * my
    sxy = _filter(x * y) - mx * my
    return ((2 * mx * my + C1) * (2 * sxy + C2)) / ((mx * mx + my * my + C1) * (sxx + syy + C2))


def loss_from_magnitude(x, y, lam=LAMBDA):
    """x, y [P, H, W] float64 tensors -> scalar tensor."""
    l1 = (x - y).abs().mean()
    ssim = ssim_map(x, y).mean(dim=(1, 2)).mean()
    return (1.0 - lam) * l1 + lam * (1.0 - ssim)


def loss_and_grad(z, y, lam=LAMBDA):
    """z [B, K, H, W] complex (numpy), y [B, K, H, W] real -> (loss, dL/dRe z, dL/dIm z)."""
    z = np.asarray(z)
    B, K, H, W = z.shape
    mag = np.abs(z).astype(np.float64)
    x = torch.tensor(mag.reshape(B * K, H, W), dtype=torch.float64, requires_grad=True)
    yt = torch.tensor(np.asarray(y, dtype=np.float64).reshape(B * K, H, W))
    L = loss_from_magnitude(x, yt, lam)
    (gx,) = torch.autograd.grad(L, [x])
    gx = gx.numpy().reshape(B, K, H, W)
    safe = np.where(mag > 0, mag, 1.0)
    unit = np.where(mag > 0, z / safe, 0.0)
    return float(L.detach()), gx * unit.real, gx * unit.imag
