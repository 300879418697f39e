"""Pins of the oracle's confidence-weighted objective (Eq. 5): C > 1, a hand-worked value, the
optimum the paper derives (C* = alpha / L_task for L_task < alpha, C -> 1 otherwise), central
differences of the gradient and the min-max normalisation."""
import math

import numpy as np
import torch

from oracle import confidence as CF


def _weights(seed, hidden=32, scale=1.0):
    rng = np.random.default_rng(seed)
    f = lambda *s: torch.tensor(rng.normal(size=s) * scale, dtype=torch.float64)
    return [f(3, hidden) / math.sqrt(3), f(hidden), f(hidden, 1) / math.sqrt(hidden), f(1)]


def _constant(g, hidden=32):
    """A network whose output is g everywhere (zero weights, output bias g)."""
    z = lambda *s: torch.zeros(*s, dtype=torch.float64)
    return [z(3, hidden), z(hidden), z(hidden, 1), torch.tensor([g], dtype=torch.float64)]


def test_confidence_exceeds_one():
    """C - 1 = exp(g) > 0: strictly above 1 for moderate g, never below 1 (for very negative g
    the sum 1 + exp(g) rounds to 1 in floating point)."""
    pos = torch.tensor(np.random.default_rng(0).uniform(-5, 5, size=(500, 3)))
    w = _weights(1)
    C = CF.confidence(pos, w)
    g = CF.network(pos, *w)
    assert float(g.abs().max()) < 30.0 and float(C.min()) > 1.0
    assert np.allclose((C - 1.0).numpy(), torch.exp(g).numpy(), rtol=1e-12, atol=0)
    wide = CF.confidence(pos, _weights(1, scale=3.0))
    assert float(wide.min()) >= 1.0


def test_constant_network_by_hand():
    """g = ln 2 gives C = 3 and the objective mean(3 L - 0.3 ln 3)."""
    pos = torch.zeros((4, 3), dtype=torch.float64)
    L = torch.tensor([0.1, 0.2, 0.05, 1.0], dtype=torch.float64)
    val = float(CF.objective(pos, _constant(math.log(2.0)), L))
    assert abs(val - float(np.mean(3.0 * L.numpy() - 0.3 * math.log(3.0)))) < 1e-15


def test_optimum_matches_the_derivation():
    """For L_task < alpha the objective is stationary in g at C = alpha / L_task (g = ln(alpha /
    L - 1)) and larger on either side; for L_task >= alpha its derivative in g is positive, so
    the optimum lies at C -> 1."""
    pos = torch.zeros((1, 3), dtype=torch.float64)
    for L in (0.01, 0.1, 0.25):
        g_star = math.log(CF.ALPHA / L - 1.0)
        w = _constant(g_star)
        w[3].requires_grad_(True)
        val = CF.objective(pos, w, torch.tensor([L], dtype=torch.float64))
        (gb,) = torch.autograd.grad(val, [w[3]])
        assert abs(float(gb)) < 1e-12
        for dg in (-0.3, 0.3):
            other = float(CF.objective(pos, _constant(g_star + dg), torch.tensor([L], dtype=torch.float64)))
            assert other > float(val.detach())
    for L in (0.3, 0.5, 2.0):
        for g in (-4.0, 0.0, 3.0):
            w = _constant(g)
            w[3].requires_grad_(True)
            val = CF.objective(pos, w, torch.tensor([L], dtype=torch.float64))
            (gb,) = torch.autograd.grad(val, [w[3]])
            assert float(gb) > 0.0


def test_gradient_against_central_differences():
    rng = np.random.default_rng(3)
    pos = torch.tensor(rng.uniform(-5, 5, size=(6, 3)))
    L = torch.tensor(rng.uniform(0.01, 0.5, size=6))
    w = _weights(4, hidden=8)
    # keep every hidden pre-activation away from the ReLU kink
    assert float((pos @ w[0] + w[1]).abs().min()) > 1e-3
    params = [t.clone().requires_grad_(True) for t in w] + [L.clone().requires_grad_(True)]
    val = CF.objective(pos, params[:4], params[4])
    grads = torch.autograd.grad(val, params)
    h = 1e-6
    for k, p in enumerate(params):
        base = [t.detach().clone() for t in params]
        num = np.zeros(p.shape)
        for idx in np.ndindex(*p.shape):
            hi = [t.clone() for t in base]
            lo = [t.clone() for t in base]
            hi[k][idx] += h
            lo[k][idx] -= h
            num[idx] = (float(CF.objective(pos, hi[:4], hi[4])) - float(CF.objective(pos, lo[:4], lo[4]))) / (2 * h)
        assert np.allclose(grads[k].numpy(), num, rtol=1e-6, atol=1e-9)


def test_normalisation():
    C = torch.tensor([1.5, 3.0, 1.2, 2.1], dtype=torch.float64)
    n = CF.normalised(C).numpy()
    assert n.min() == 0.0 and n.max() == 1.0
    assert np.allclose(n, (C.numpy() - 1.2) / 1.8, rtol=0, atol=1e-15)
