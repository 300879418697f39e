"""Pin for the oracle's Adam update against torch.optim.Adam (a library routine)."""
import numpy as np
import torch

from oracle import adam


def test_adam_matches_torch_fp64():
    rng = np.random.default_rng(61)
    p0 = rng.normal(size=257)
    p = torch.tensor(p0.copy(), requires_grad=True)
    opt = torch.optim.Adam([p], lr=5e-3, betas=(0.9, 0.999), eps=1e-15)
    q, m, v = p0.copy(), np.zeros(257), np.zeros(257)
    for t in range(1, 8):
        g = rng.normal(size=257)
        p.grad = torch.tensor(g)
        opt.step()
        q, m, v = adam.adam_step(q, g, m, v, t, 5e-3)
    np.testing.assert_allclose(q, p.detach().numpy(), rtol=1e-13, atol=1e-15)


def test_position_lr_anneal_endpoints():
    assert np.isclose(adam.position_lr(0, 100), 1.6e-4, rtol=1e-14)
    assert np.isclose(adam.position_lr(99, 100), 1.6e-7, rtol=1e-14)
    mid = adam.position_lr(49.5, 100)
    assert np.isclose(mid, np.sqrt(1.6e-4 * 1.6e-7), rtol=1e-12)
