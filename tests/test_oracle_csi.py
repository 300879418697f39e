"""Pins of the oracle's CSI head (Eq. 2), channel loss (Eq. 3) and the chained gradient of
the channel loss, against closed forms and central differences."""
import math

import numpy as np
import pytest

from oracle import csi as C
from oracle import pipeline as PL
from oracle import render as R
from paper_2511_22793_gb300 import synth

C_LIGHT = 299792458.0


def test_csi_head_closed_forms():
    H, W, K = 6, 10, 3
    c = np.array([1.5 - 2j, 0.25j, -3.0])
    z = np.broadcast_to(c, (2, H * W, K)).copy()
    assert np.allclose(C.csi_head(z, H, W), np.broadcast_to(c, (2, K)), rtol=0, atol=1e-15)
    # alternating signs over an even number of pixels average to zero
    sign = np.where(np.arange(H * W) % 2 == 0, 1.0, -1.0)
    assert np.allclose(C.csi_head(sign[None, :, None] * z, H, W), 0.0, atol=1e-15)
    # the gradient of the mean is 1/HW at every pixel
    d = C.csi_head_bwd(np.array([[2.0 + 4.0j]]), H, W)
    assert d.shape == (1, H * W, 1) and np.allclose(d, (2.0 + 4.0j) / (H * W))


def test_channel_loss_closed_forms_and_gradient():
    rng = np.random.default_rng(3)
    h = rng.normal(size=(2, 5)) + 1j * rng.normal(size=(2, 5))
    assert C.channel_loss(h, h)[0] == 0.0
    # Eq. 3 for one entry: (h_re - hh_re)^2 + (h_im - hh_im)^2
    l1, _ = C.channel_loss(np.array([1.0 + 2.0j]), np.array([-0.5 + 4.0j]))
    assert l1 == pytest.approx(1.5 ** 2 + 2.0 ** 2, rel=1e-15)
    hh = h + (1.0 + 1.0j)
    assert C.channel_loss(hh, h)[0] == pytest.approx(2.0, rel=1e-15)
    _, g = C.channel_loss(hh, h)
    for idx in [(0, 0), (1, 3)]:
        for unit in (1.0, 1.0j):
            e = 1e-6
            p = hh.copy()
            p[idx] += e * unit
            m = hh.copy()
            m[idx] -= e * unit
            fd = (C.channel_loss(p, h)[0] - C.channel_loss(m, h)[0]) / (2 * e)
            an = g[idx].real if unit == 1.0 else g[idx].imag
            assert fd == pytest.approx(an, rel=1e-7)
    assert C.nmse(h, h) == 0.0 and C.nmse(np.zeros_like(h), h) == pytest.approx(1.0)


def test_single_gaussian_csi_phase_and_magnitude(oracle_lib):
    """One Gaussian: every pixel carries the same phase e^{j(phi0 - 2 pi f_k L / c)}, so the
    spatial mean over subcarriers advances by exactly e^{-j 2 pi df L / c}, and its magnitude
    is a/HW times the sum over pixels of alpha (T = 1 in front of the only Gaussian)."""
    H, W, K = 20, 40, 5
    f_c, df = 2.4e9, 312.5e3
    g = dict(px=np.array([17.3]), py=np.array([9.6]), cxx=np.array([0.12]), cxy=np.array([0.03]),
             cyy=np.array([0.2]), r=np.array([3.0]), valid=np.array([True]))
    at = dict(sigma=np.array([0.7]), a=np.array([0.4]), phi0=np.array([0.9]), L=np.array([7.25]))
    z, _, _ = R.render_fwd(g, at, H, W, K, f_c, df)
    h = C.csi_head(z, H, W)
    ratio = h[1:] / h[:-1]
    assert np.allclose(ratio, np.exp(-2j * math.pi * df * 7.25 / C_LIGHT), rtol=0, atol=1e-12)
    # alpha of every pixel from the compositing rule (q from the conic, 3-sigma-style cut-offs)
    ys, xs = np.divmod(np.arange(H * W), W)
    dx = xs + 0.5 - 17.3
    dx = dx - W * np.floor(dx / W + 0.5)
    dy = ys + 0.5 - 9.6
    q = 0.12 * dx * dx + 2 * 0.03 * dx * dy + 0.2 * dy * dy
    alpha = np.minimum(0.99, 0.7 * np.exp(-0.5 * q))
    alpha[(q > 2 * math.log(255.0)) | (alpha < 1.0 / 255.0)] = 0.0
    f0 = f_c - (K // 2) * df
    expect0 = 0.4 * alpha.sum() / (H * W) * np.exp(1j * (0.9 - 2 * math.pi * f0 * 7.25 / C_LIGHT))
    assert abs(h[0] - expect0) <= 1e-12 * abs(expect0)


def test_channel_loss_gradient_vs_central_differences(oracle_lib):
    """Channel loss of the spatial mean through projection, attribute network and renderer;
    FD on 16 sampled scene and network parameters."""
    H, W, K = 18, 72, 3
    sc = synth.make_scene(60, seed=61)
    sc.log_scales = sc.log_scales + np.float32(1.2)
    mlp = synth.make_mlp(8, seed=62)
    view = synth.View(H=H, W=W)
    band = synth.Band(K=K)
    tx = synth.make_tx(2, seed=63).astype(np.float64)
    rng = np.random.default_rng(64)
    target = 0.01 * (rng.normal(size=(2, K)) + 1j * rng.normal(size=(2, K)))
    scd = synth.Scene(*[np.asarray(a, dtype=np.float64).copy() for a in sc.arrays()])
    mld = synth.MLPWeights(8, *[np.asarray(a, dtype=np.float64).copy() for a in mlp.arrays()])
    loss, grads = PL.loss_and_grad(scd, mld, view, band, tx, target, loss_kind="csi")
    assert loss == pytest.approx(C.channel_loss(grads["h"], target)[0])

    def eval_loss():
        out = PL.forward(scd, mld, view, band, tx)
        sigs = []
        for at in out["attrs"]:
            gg = {k: out["geo"][k].numpy() for k in ("px", "py", "cxx", "cxy", "cyy", "r", "valid")}
            a = {k: at[k].numpy() for k in ("sigma", "a", "phi0", "L")}
            sigs.append(R.render_fwd(gg, a, H, W, K, band.f_c, band.df, signature=True)[3])
        return C.channel_loss(C.csi_head(out["z"], H, W), target)[0], np.stack(sigs)

    _, s0 = eval_loss()
    names = ["means", "log_scales", "quats", "opacity_logit", "latent", "W1", "b1", "W2", "b2",
             "W3", "b3"]
    holders = {nm: arr for nm, arr in zip(names[:5], scd.arrays())}
    holders.update({nm: arr for nm, arr in zip(names[5:], mld.arrays())})
    checked, tries = 0, 0
    while checked < 16 and tries < 200:
        tries += 1
        nm = names[int(rng.integers(len(names)))]
        flat = holders[nm].reshape(-1)
        j = int(rng.integers(flat.size))
        x0 = flat[j]
        h = 1e-6 * max(1.0, abs(x0))
        flat[j] = x0 + h
        lp, sp = eval_loss()
        flat[j] = x0 - h
        lm, sm = eval_loss()
        flat[j] = x0
        if not (np.array_equal(sp, s0) and np.array_equal(sm, s0)):
            continue
        fd = (lp - lm) / (2 * h)
        an = grads[nm].reshape(-1)[j]
        if abs(fd) < 1e-13 and abs(an) < 1e-13:
            continue
        assert abs(fd - an) <= 1e-5 * max(abs(fd), abs(an)) + 1e-13, (nm, j, fd, an)
        checked += 1
    assert checked >= 16
