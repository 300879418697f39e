"""Oracle attribute network: per-Gaussian emission from a transmitter query.

TEST INFRASTRUCTURE (see the package docstring).  Plain PyTorch CPU ops in
float64; autograd on these ops supplies the oracle's gradient.

Follows Eq. 1 (s_i = sigmoid(f(x) - log d_i), d_i = |x_tx - mu_i|) and the
compositing rule of Sec. 4.2, whose s_i/d_i term adds free-space attenuation.

Readings (the paper is silent or not self-consistent on these):
  - one network is shared by all Gaussians; its input is the transmitter
    position (3), the Gaussian's 16-dim latent and log d_i; two hidden layers
    with ReLU; three outputs o = (o_0, o_1, o_2);
  - amplitude a_i = sigmoid(o_0 - log d_i) / d_i (the Eq. 1 bias and the 1/d_i
    of the compositing rule), phase offset phi0_i = o_1 in radians, opacity
    sigma_i = sigmoid(opacity_logit_i + o_2);
  - d_i is clamped below at 0.01 m;
  - the subcarrier enters as the delay of the path transmitter -> Gaussian ->
    receiver, L_i = d_i + |mu_i - x_rx| (Sec. 3.1 channel model, phase
    e^{-j 2 pi f tau});
  - the query is the transmitter with the receiver fixed (the paper's RFID
    setting, Sec. 5), so d_i is measured from the transmitter.
"""
from __future__ import annotations

import torch

D_MIN = 0.01


def mlp_outputs(tx, latent, logd, W1, b1, W2, b2, W3, b3):
    """o = W3^T relu(W2^T relu(W1^T h0 + b1) + b2) + b3, h0 = [tx, latent, log d]."""
    n = latent.shape[0]
    h0 = torch.cat([tx.reshape(1, 3).expand(n, 3), latent, logd.reshape(n, 1)], dim=1)
    h1 = torch.relu(h0 @ W1 + b1)
    h2 = torch.relu(h1 @ W2 + b2)
    return h2 @ W3 + b3


def attributes(means, opacity_logit, latent, weights, tx, rx):
    """Per-Gaussian (a, phi0, sigma, L) for one transmitter position tx.

    weights = (W1, b1, W2, b2, W3, b3) as float64 tensors with W stored
    input-major ([fan_in, fan_out]).  Returns a dict of [N] tensors.
    """
    tx = torch.as_tensor(tx, dtype=torch.float64)
    rx = torch.as_tensor(rx, dtype=torch.float64)
    d = torch.clamp(torch.linalg.norm(means - tx, dim=1), min=D_MIN)
    logd = torch.log(d)
    o = mlp_outputs(tx, latent, logd, *weights)
    a = torch.sigmoid(o[:, 0] - logd) / d
    phi0 = o[:, 1]
    sigma = torch.sigmoid(opacity_logit + o[:, 2])
    L = d + torch.linalg.norm(means - rx, dim=1)
    return dict(a=a, phi0=phi0, sigma=sigma, L=L, d=d, o=o)
