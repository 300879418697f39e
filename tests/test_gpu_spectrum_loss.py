"""Magnitude-spectrum loss (gsparc_spectrum_loss, Eq. 4: L1 + SSIM) against the FP64 oracle
(oracle/spectrum_loss.py): the loss and dL/dz, planes smaller than the window, the full
64-subcarrier 360x90 size, the identity case and zero spectrum values."""
import numpy as np
import pytest
import torch

from gpu_util import DEV, rel_l2
from oracle import spectrum_loss as S
from paper_2511_22793_gb300 import gsparc as G

pytestmark = pytest.mark.gpu


def _case(B, K, H, W, seed):
    """Magnitudes in [0.1, 1.1) and targets 6-36% above or below them: the L1 term's sign is the
    same in FP32 and FP64 (a target within rounding of its magnitude would flip it, and one
    flip among 2 million pixels moves the gradient by ~1e-3 relative L2)."""
    rng = np.random.default_rng(seed)
    mag = 0.1 + rng.uniform(size=(B, K, H, W))
    z = mag * np.exp(2j * np.pi * rng.uniform(size=(B, K, H, W)))
    y = mag * (1.0 + 0.3 * np.sign(rng.normal(size=mag.shape)) * (0.2 + rng.uniform(size=mag.shape)))
    return z, y


def _gpu(z, y, lam=0.2, grad=True):
    B, K, H, W = z.shape
    zd = torch.tensor(np.stack([z.real, z.imag], -1).astype(np.float32), device=DEV)
    yd = torch.tensor(y.astype(np.float32), device=DEV)
    ws = torch.empty(G.gsparc_spectrum_loss_workspace(B, K, H, W), dtype=torch.uint8, device=DEV)
    loss = torch.zeros(1, device=DEV)
    dz = torch.empty_like(zd) if grad else None
    G.gsparc_spectrum_loss(zd, yd, ws, loss, dz, lam=lam)
    torch.cuda.synchronize()
    return float(loss), (dz.cpu().numpy().astype(np.float64) if grad else None)


@pytest.mark.parametrize("B,K,H,W", [(1, 1, 16, 16), (2, 3, 45, 180), (1, 2, 7, 9), (1, 64, 90, 360)])
def test_loss_and_gradient_match_oracle(B, K, H, W):
    z, y = _case(B, K, H, W, 7 + H)
    # the FP32 values the GPU sees feed the oracle too
    z = (np.stack([z.real, z.imag], -1).astype(np.float32).astype(np.float64) @ np.array([1.0, 1j]))
    y = y.astype(np.float32).astype(np.float64)
    L, gre, gim = S.loss_and_grad(z, y)
    Lg, dz = _gpu(z, y)
    assert abs(Lg - L) <= 1e-5 * abs(L)
    assert rel_l2(dz[..., 0], gre) <= 1e-4
    assert rel_l2(dz[..., 1], gim) <= 1e-4
    Lg2, _ = _gpu(z, y, grad=False)
    assert abs(Lg2 - L) <= 1e-5 * abs(L)


def test_identity_gives_zero_loss():
    """y = |z|: zero loss, and a gradient no larger than the L1 term's subgradient (1 - lam) / M
    (the FP32 magnitude may sit an ulp off its target, on either side), the SSIM part vanishing."""
    z, _ = _case(1, 4, 30, 60, 3)
    z = (np.stack([z.real, z.imag], -1).astype(np.float32).astype(np.float64) @ np.array([1.0, 1j]))
    y = np.abs(z).astype(np.float32).astype(np.float64)
    L, dz = _gpu(z, y)
    assert abs(L) <= 1e-5
    assert np.abs(dz).max() <= (1.0 - 0.2) / z.size * (1.0 + 1e-3) + 1e-6


def test_zero_spectrum_values_get_zero_gradient():
    z, y = _case(1, 1, 20, 20, 5)
    z[0, 0, 10, 10] = 0.0
    z[0, 0, 3, 17] = 0.0
    _, dz = _gpu(z, y)
    assert np.all(dz[0, 0, 10, 10] == 0.0) and np.all(dz[0, 0, 3, 17] == 0.0)
