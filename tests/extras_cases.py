"""Seeded cases and FP64 oracle results shared by the host-shim and GPU tests of the training
extras (the confidence objective of Eq. 5, adaptive density control)."""
import math

import numpy as np
import torch

from oracle import confidence as CF


def conf_case(B, hidden, seed):
    rng = np.random.default_rng(seed)
    pos = rng.uniform(-5, 5, size=(B, 3)).astype(np.float32)
    L = rng.uniform(0.01, 0.6, size=B).astype(np.float32)
    w = np.concatenate([rng.normal(size=3 * hidden) / math.sqrt(3) * 0.5, 0.3 * rng.normal(size=hidden),
                        rng.normal(size=hidden) / math.sqrt(hidden), [0.1]]).astype(np.float32)
    return pos, L, w


def conf_oracle(pos, L, w, hidden, alpha=0.3):
    h = hidden
    t = [torch.tensor(w[0:3 * h].reshape(3, h).astype(np.float64), requires_grad=True),
         torch.tensor(w[3 * h:4 * h].astype(np.float64), requires_grad=True),
         torch.tensor(w[4 * h:5 * h].reshape(h, 1).astype(np.float64), requires_grad=True),
         torch.tensor(w[5 * h:5 * h + 1].astype(np.float64), requires_grad=True)]
    P = torch.tensor(pos.astype(np.float64))
    Lt = torch.tensor(L.astype(np.float64), requires_grad=True)
    obj = CF.objective(P, t, Lt, alpha=alpha)
    grads = torch.autograd.grad(obj, t + [Lt])
    C = CF.confidence(P, [x.detach() for x in t])
    dw = np.concatenate([g.reshape(-1).numpy() for g in grads[:4]])
    pre = (P @ t[0] + t[1]).detach().numpy()
    return float(obj.detach()), C.numpy(), grads[4].numpy(), dw, np.abs(pre).min()
