"""Pins of the oracle's per-Gaussian emission network (Eq. 1 per Gaussian, Sec. 4.1 and 4.2):
closed forms worked by hand, the 1/d toggle, the distance clamp, independence of the
Gaussians, and central finite differences of its FP64 gradient."""
import math

import numpy as np
import torch

from oracle import emission as E


def _sig(x):
    return 1.0 / (1.0 + math.exp(-x))


def _t(a):
    return torch.tensor(np.asarray(a, dtype=np.float64))


def test_zero_output_weights_closed_form():
    """W2 = 0: o = b2, so s = sigmoid(b2 - ln d).  Mean at (3, 4, 0), transmitter at the
    origin: d = 5; b2 = (ln 5, ln 15) gives s = sigmoid(0) + j sigmoid(ln 3) = 1/2 + 3j/4."""
    h = 4
    flat = np.zeros((1, E.n_params(h)))
    flat[0, :3 * h] = np.arange(3 * h) * 0.1          # W1, irrelevant once W2 = 0
    flat[0, 6 * h:] = [math.log(5.0), math.log(15.0)]
    at = E.attributes(_t([[3.0, 4.0, 0.0]]), _t([0.3]), _t(flat), h, (0.0, 0.0, 0.0), (0.0, 0.0, 1.0))
    mag = math.sqrt(0.25 + 0.5625)
    assert abs(float(at["re"][0]) - 0.5) < 1e-15 and abs(float(at["im"][0]) - 0.75) < 1e-15
    assert abs(float(at["a"][0]) - mag / 5.0) < 1e-15
    assert abs(float(at["phi0"][0]) - math.atan(1.5)) < 1e-15
    assert abs(float(at["sigma"][0]) - _sig(0.3)) < 1e-15
    assert abs(float(at["L"][0]) - (5.0 + math.sqrt(9 + 16 + 1))) < 1e-14


def test_width_one_network_by_hand():
    """h = 1, W1 = (1, 2, 3), b1 = -1, W2 = (2, -1), b2 = 0, transmitter (1, 1, 1), mean one metre
    away (ln d = 0): pre-activation 1 + 2 + 3 - 1 = 5, o = (10, -5); with b1 = -10 the unit is
    off and o = b2 = 0."""
    flat = np.array([[1.0, 2.0, 3.0, -1.0, 2.0, -1.0, 0.0, 0.0]])
    means = _t([[2.0, 1.0, 1.0]])
    at = E.attributes(means, _t([0.0]), _t(flat), 1, (1.0, 1.0, 1.0), (0.0, 0.0, 0.0), inv_d=False)
    re, im = _sig(10.0), _sig(-5.0)
    assert np.allclose(at["o"].numpy(), [[10.0, -5.0]], rtol=0, atol=1e-15)
    assert abs(float(at["a"][0]) - math.hypot(re, im)) < 1e-15
    assert abs(float(at["phi0"][0]) - math.atan2(im, re)) < 1e-15
    flat[0, 3] = -10.0
    at = E.attributes(means, _t([0.0]), _t(flat), 1, (1.0, 1.0, 1.0), (0.0, 0.0, 0.0), inv_d=False)
    assert np.allclose(at["o"].numpy(), [[0.0, 0.0]], rtol=0, atol=0)
    assert abs(float(at["a"][0]) - math.hypot(0.5, 0.5)) < 1e-15
    assert abs(float(at["phi0"][0]) - math.pi / 4) < 1e-15


def _random_case(n, h, seed):
    rng = np.random.default_rng(seed)
    means = rng.uniform(-5, 5, size=(n, 3))
    ologit = rng.normal(size=n)
    flat = rng.normal(size=(n, E.n_params(h))) / 2.0
    return means, ologit, flat


def test_inverse_distance_toggle_and_clamp():
    """a with the 1/d term equals a without it divided by d, the other outputs unchanged; a mean
    at the transmitter has d = 0.01 m."""
    means, ologit, flat = _random_case(64, 16, 1)
    means[5] = [0.5, -1.0, 2.0]
    tx, rx = (0.5, -1.0, 2.0), (0.0, 0.0, 0.0)
    on = E.attributes(_t(means), _t(ologit), _t(flat), 16, tx, rx, inv_d=True)
    off = E.attributes(_t(means), _t(ologit), _t(flat), 16, tx, rx, inv_d=False)
    assert np.allclose((on["a"] * on["d"]).numpy(), off["a"].numpy(), rtol=1e-15, atol=0)
    for k in ("phi0", "sigma", "L"):
        assert np.array_equal(on[k].numpy(), off[k].numpy())
    assert float(on["d"][5]) == E.D_MIN


def test_gaussians_are_independent():
    """Each Gaussian has its own network: permuting the Gaussians permutes the outputs (to
    rounding: the batched contraction may order its three-term sums by position)."""
    means, ologit, flat = _random_case(50, 8, 2)
    perm = np.random.default_rng(3).permutation(50)
    a = E.attributes(_t(means), _t(ologit), _t(flat), 8, (1.0, 2.0, -1.0), (0.0, 0.0, 0.0))
    b = E.attributes(_t(means[perm]), _t(ologit[perm]), _t(flat[perm]), 8, (1.0, 2.0, -1.0), (0.0, 0.0, 0.0))
    for k in ("a", "phi0", "sigma", "L"):
        assert np.allclose(a[k].numpy()[perm], b[k].numpy(), rtol=1e-13, atol=1e-15)


def test_gradient_against_central_differences():
    """attributes_vjp against central differences of sum <attr, g> in means, logits and flat
    buffers (h = 1e-6 relative; ReLU pre-activations kept away from zero)."""
    n, h = 6, 4
    means, ologit, flat = _random_case(n, h, 12)   # a case whose pre-activations avoid the kink
    txs = [(1.0, -2.0, 0.5), (-3.0, 1.0, 2.0)]
    rx = (0.2, 0.1, -0.3)
    g = np.random.default_rng(5).normal(size=(2, n, 4))

    def f(m, o, fl):
        tot = 0.0
        for b, tx in enumerate(txs):
            at = E.attributes(_t(m), _t(o), _t(fl), h, tx, rx)
            tot += float((torch.stack([at["a"], at["phi0"], at["sigma"], at["L"]], -1).numpy() * g[b]).sum())
        return tot

    # keep every hidden pre-activation at least 0.05 from the ReLU kink
    for tx in txs:
        W1, b1, _, _ = E.unpack(_t(flat), h)
        pre = torch.einsum("k,nkj->nj", _t(tx), W1) + b1
        assert float(pre.abs().min()) > 0.05
    gm, go, gf = E.attributes_vjp(means, ologit, flat, h, txs, rx, g)
    for arr, grad in ((means, gm), (ologit, go), (flat, gf)):
        num = np.zeros_like(arr)
        it = np.nditer(arr, flags=["multi_index"])
        for _ in it:
            idx = it.multi_index
            step = 1e-6 * max(1.0, abs(arr[idx]))
            hi = arr.copy()
            lo = arr.copy()
            hi[idx] += step
            lo[idx] -= step
            args_hi = [means, ologit, flat]
            args_lo = [means, ologit, flat]
            k = [id(means), id(ologit), id(flat)].index(id(arr))
            args_hi[k], args_lo[k] = hi, lo
            num[idx] = (f(*args_hi) - f(*args_lo)) / (2 * step)
        assert np.allclose(grad, num, rtol=1e-6, atol=1e-8)
