"""Oracle Adam update (Algorithm 1, "Adam" step; Sec. 4.2 optimisation).

TEST INFRASTRUCTURE (see the package docstring).  float64 NumPy.

Kingma & Ba's update, as 3D Gaussian Splatting uses it:
  m <- b1 m + (1 - b1) g
  v <- b2 v + (1 - b2) g^2
  p <- p - lr * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps)
Readings: b1 = 0.9, b2 = 0.999, eps = 1e-15 (the paper gives the learning
rates, Table of hyperparameters, but not these).
"""
from __future__ import annotations

import numpy as np


def adam_step(p, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-15):
    """One step at 1-based step count t.  Returns new (p, m, v) as float64."""
    p = np.asarray(p, dtype=np.float64)
    g = np.asarray(g, dtype=np.float64)
    m = b1 * np.asarray(m, dtype=np.float64) + (1.0 - b1) * g
    v = b2 * np.asarray(v, dtype=np.float64) + (1.0 - b2) * g * g
    mhat = m / (1.0 - b1 ** t)
    vhat = v / (1.0 - b2 ** t)
    return p - lr * mhat / (np.sqrt(vhat) + eps), m, v


def position_lr(step, total, lr_init=1.6e-4, lr_final=1.6e-7):
    """Exponential anneal of the position learning rate from lr_init to
    lr_final over `total` steps (Table of hyperparameters)."""
    if total <= 1:
        return lr_init
    t = min(max(step / (total - 1), 0.0), 1.0)
    return float(np.exp(np.log(lr_init) * (1.0 - t) + np.log(lr_final) * t))
