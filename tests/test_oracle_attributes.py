"""Pins for the oracle's attribute network (Eq. 1 and the 1/d of the Sec. 4.2 rule)."""
import math

import numpy as np
import torch

from oracle import attributes as A


def _weights(hidden, fill=None):
    W1 = torch.zeros(20, hidden, dtype=torch.float64)
    b1 = torch.zeros(hidden, dtype=torch.float64)
    W2 = torch.zeros(hidden, hidden, dtype=torch.float64)
    b2 = torch.zeros(hidden, dtype=torch.float64)
    W3 = torch.zeros(hidden, 3, dtype=torch.float64)
    b3 = torch.zeros(3, dtype=torch.float64)
    return [W1, b1, W2, b2, W3, b3]


def _scene(n, seed=0):
    rng = np.random.default_rng(seed)
    means = torch.tensor(rng.uniform(-5, 5, (n, 3)))
    ologit = torch.tensor(rng.normal(size=n))
    latent = torch.tensor(rng.normal(size=(n, 16)))
    return means, ologit, latent


def test_constant_network_closed_form():
    """All weights zero: o = b3, so a = sigmoid(b3_0 - ln d)/d = 1/(d (1 + d e^{-b3_0})),
    phi0 = b3_1, sigma = sigmoid(logit + b3_2)."""
    means, ologit, latent = _scene(64)
    w = _weights(8)
    w[5] = torch.tensor([0.7, -1.3, 0.4], dtype=torch.float64)
    tx = torch.tensor([0.5, 1.0, -2.0], dtype=torch.float64)
    out = A.attributes(means, ologit, latent, w, tx, torch.zeros(3, dtype=torch.float64))
    d = np.linalg.norm(means.numpy() - tx.numpy(), axis=1)
    np.testing.assert_allclose(out["a"].numpy(), 1.0 / (d * (1.0 + d * math.exp(-0.7))), rtol=1e-13)
    np.testing.assert_allclose(out["phi0"].numpy(), -1.3, rtol=0, atol=0)
    np.testing.assert_allclose(out["sigma"].numpy(), 1.0 / (1.0 + np.exp(-(ologit.numpy() + 0.4))),
                               rtol=1e-14)
    r = np.linalg.norm(means.numpy(), axis=1)
    np.testing.assert_allclose(out["L"].numpy(), d + r, rtol=1e-14)


def test_log_distance_feature_wiring():
    """Route only the log-distance input (feature 19) through one hidden unit
    into o_0: o_0 = relu(ln d), so a = 1/(2d) for d > 1 and 1/(d (1 + d)) for d < 1."""
    means, ologit, latent = _scene(256, seed=1)
    w = _weights(4)
    w[0][19, 0] = 1.0
    w[2][0, 0] = 1.0
    w[4][0, 0] = 1.0
    tx = torch.zeros(3, dtype=torch.float64)
    out = A.attributes(means, ologit, latent, w, tx, torch.zeros(3, dtype=torch.float64))
    d = np.linalg.norm(means.numpy(), axis=1)
    expect = np.where(d > 1.0, 1.0 / (2.0 * d), 1.0 / (d * (1.0 + d)))
    np.testing.assert_allclose(out["a"].numpy(), expect, rtol=1e-13)


def test_transmitter_and_latent_wiring():
    """Feature 0 is tx_x and feature 3 + j is latent_j: route tx_x into o_1 and
    latent_5 into o_2 through separate hidden units."""
    means, ologit, latent = _scene(32, seed=2)
    w = _weights(4)
    w[0][0, 1] = 1.0          # tx_x -> h1_1
    w[0][3 + 5, 2] = 1.0      # latent_5 -> h1_2
    w[2][1, 1] = 1.0
    w[2][2, 2] = 1.0
    w[4][1, 1] = 1.0          # h2_1 -> o_1 (phase)
    w[4][2, 2] = 1.0          # h2_2 -> o_2 (opacity offset)
    tx = torch.tensor([2.5, 0.0, 0.0], dtype=torch.float64)
    out = A.attributes(means, ologit, latent, w, tx, torch.zeros(3, dtype=torch.float64))
    np.testing.assert_allclose(out["phi0"].numpy(), 2.5, atol=0)
    lat5 = np.maximum(latent[:, 5].numpy(), 0.0)
    np.testing.assert_allclose(out["sigma"].numpy(), 1.0 / (1.0 + np.exp(-(ologit.numpy() + lat5))),
                               rtol=1e-14)


def test_distance_clamp():
    means = torch.tensor([[1.0, 2.0, 3.0]], dtype=torch.float64)
    w = _weights(2)
    out = A.attributes(means, torch.zeros(1, dtype=torch.float64), torch.zeros(1, 16, dtype=torch.float64),
                       w, means[0], torch.zeros(3, dtype=torch.float64))
    assert out["d"].item() == A.D_MIN
    # o = 0: a = sigmoid(-ln 0.01)/0.01 = (1/(1 + 0.01))/0.01
    np.testing.assert_allclose(out["a"].item(), 1.0 / (1.01 * 0.01), rtol=1e-13)


def test_relu_blocks_negative_preactivations():
    means, ologit, latent = _scene(16, seed=3)
    w = _weights(2)
    w[1][:] = -1.0            # b1 < 0 with zero W1: h1 = 0
    w[2][:] = 5.0
    w[3][:] = -0.25           # h2 = relu(-0.25) = 0
    w[4][:] = 9.0
    out = A.attributes(means, ologit, latent, w, torch.zeros(3, dtype=torch.float64),
                       torch.zeros(3, dtype=torch.float64))
    np.testing.assert_array_equal(out["o"].numpy(), 0.0)
