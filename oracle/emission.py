"""Oracle per-Gaussian emission network (the paper's own form of Eq. 1).

TEST INFRASTRUCTURE (see the package docstring).  Plain PyTorch CPU ops in
float64; autograd on these ops supplies the oracle's gradient.

Follows Eq. 1, s_i = sigmoid(f_i(x) - log d_i) with the sigmoid applied to the
real and imaginary parts separately, the Sec. 4.2 implementation notes (every
Gaussian carries its own network R^3 -> R^2 with 16 hidden units, stored in a
flat per-Gaussian buffer; widths 8, 16 and 64 in the Sec. 7 ablation) and the
s_i / d_i term of the Sec. 4.2 compositing rule, which the Sec. 7 ablation
switches on and off.

Readings (the paper is silent on these):
  - the network's input is the query position, here the transmitter (the
    receiver is fixed, as in the shared-network form), one hidden layer with
    ReLU (the activation is unstated), outputs (o_0, o_1);
  - s_i = sigmoid(o_0 - log d_i) + j sigmoid(o_1 - log d_i), d_i = max(|x_tx -
    mu_i|, 0.01 m);
  - the renderer's attributes: amplitude a_i = |s_i| / d_i (|s_i| with the
    1/d term off), phase offset phi0_i = arg s_i, opacity sigma_i =
    sigmoid(opacity_logit_i) (this network has no opacity output), path length
    L_i = d_i + |mu_i - x_rx|, so that a_i e^{j phi0_i} = s_i / d_i;
  - flat buffer of Gaussian i, hidden width h: W1 [3, h] (input-major), b1 [h],
    W2 [h, 2] (input-major), b2 [2]: 6h + 2 values.
"""
from __future__ import annotations

import torch

D_MIN = 0.01


def n_params(hidden: int) -> int:
    """Values in one Gaussian's flat buffer."""
    return 6 * hidden + 2


def unpack(flat, hidden: int):
    """[N, >= 6h+2] flat buffers -> (W1 [N,3,h], b1 [N,h], W2 [N,h,2], b2 [N,2])."""
    h = hidden
    n = flat.shape[0]
    W1 = flat[:, 0:3 * h].reshape(n, 3, h)
    b1 = flat[:, 3 * h:4 * h]
    W2 = flat[:, 4 * h:6 * h].reshape(n, h, 2)
    b2 = flat[:, 6 * h:6 * h + 2]
    return W1, b1, W2, b2


def network(flat, hidden: int, tx):
    """o_i = W2_i^T relu(W1_i^T x + b1_i) + b2_i for every Gaussian i: [N, 2]."""
    W1, b1, W2, b2 = unpack(flat, hidden)
    x = torch.as_tensor(tx, dtype=torch.float64)
    hid = torch.relu(torch.einsum("k,nkj->nj", x, W1) + b1)
    return torch.einsum("nj,njc->nc", hid, W2) + b2


def attributes(means, opacity_logit, flat, hidden, tx, rx, inv_d=True):
    """Per-Gaussian (a, phi0, sigma, L) for one transmitter position tx.

    Returns a dict of [N] tensors plus the complex emission s (re, im) and d.
    """
    tx = torch.as_tensor(tx, dtype=torch.float64)
    rx = torch.as_tensor(rx, dtype=torch.float64)
    d = torch.clamp(torch.linalg.norm(means - tx, dim=1), min=D_MIN)
    logd = torch.log(d)
    o = network(flat, hidden, tx)
    re = torch.sigmoid(o[:, 0] - logd)
    im = torch.sigmoid(o[:, 1] - logd)
    mag = torch.sqrt(re * re + im * im)
    a = mag / d if inv_d else mag
    phi0 = torch.atan2(im, re)
    sigma = torch.sigmoid(opacity_logit)
    L = d + torch.linalg.norm(means - rx, dim=1)
    return dict(a=a, phi0=phi0, sigma=sigma, L=L, d=d, re=re, im=im, o=o)


def attributes_vjp(means, opacity_logit, flat, hidden, tx_all, rx, d_attr, inv_d=True):
    """Gradients of sum_b sum_i <attr[b,i], d_attr[b,i]> (attr = (a, phi0, sigma, L)) with respect
    to the means [N,3], the opacity logits [N] and the flat buffers [N, P] (FP64 autograd)."""
    means = torch.as_tensor(means, dtype=torch.float64).clone().requires_grad_(True)
    ologit = torch.as_tensor(opacity_logit, dtype=torch.float64).clone().requires_grad_(True)
    flat = torch.as_tensor(flat, dtype=torch.float64).clone().requires_grad_(True)
    d_attr = torch.as_tensor(d_attr, dtype=torch.float64)
    total = torch.zeros((), dtype=torch.float64)
    for b, tx in enumerate(tx_all):
        at = attributes(means, ologit, flat, hidden, tx, rx, inv_d=inv_d)
        stacked = torch.stack([at["a"], at["phi0"], at["sigma"], at["L"]], -1)
        total = total + (stacked * d_attr[b]).sum()
    gm, go, gf = torch.autograd.grad(total, [means, ologit, flat])
    return gm.numpy(), go.numpy(), gf.numpy()
