"""GPU loss and Adam kernels against the oracle."""
import numpy as np
import pytest
import torch

from gpu_util import DEV
from oracle import adam as oadam
from paper_2511_22793_gb300 import gsparc as G

pytestmark = pytest.mark.gpu


def test_l2_loss_and_gradient():
    rng = np.random.default_rng(41)
    z = rng.normal(size=(3, 5, 7, 11, 2)).astype(np.float32)
    t = rng.normal(size=(3, 5, 7, 11, 2)).astype(np.float32)
    zd, td = torch.tensor(z, device=DEV), torch.tensor(t, device=DEV)
    loss = torch.zeros(1, device=DEV)
    dz = torch.empty_like(zd)
    G.gsparc_l2_loss(zd, td, loss, dz)
    torch.cuda.synchronize()
    d = z.astype(np.float64) - t
    M = d.size // 2
    np.testing.assert_allclose(loss.item(), np.sum(d * d) / M, rtol=1e-5)
    np.testing.assert_allclose(dz.cpu().numpy(), 2 * d / M, rtol=1e-5, atol=1e-9)


def test_adam_matches_oracle():
    rng = np.random.default_rng(42)
    n = 10_001
    p = rng.normal(size=n).astype(np.float32)
    pd = torch.tensor(p, device=DEV)
    m = torch.zeros_like(pd)
    v = torch.zeros_like(pd)
    q, mm, vv = p.astype(np.float64), np.zeros(n), np.zeros(n)
    for step in range(1, 6):
        g = rng.normal(size=n).astype(np.float32)
        G.gsparc_adam(pd, torch.tensor(g, device=DEV), m, v, 5e-3, step, eps=1e-15)
        q, mm, vv = oadam.adam_step(q, g, mm, vv, step, 5e-3, eps=1e-15)
    torch.cuda.synchronize()
    np.testing.assert_allclose(pd.cpu().numpy(), q, rtol=1e-5, atol=1e-6)
