"""Pins for the oracle's per-pixel compositing (Sec. 4.2 rule, Algorithm 1 inner loop)."""
import math

import numpy as np
import pytest
import torch

from oracle import attributes as A
from oracle import pipeline as PL
from oracle import projection as P
from oracle import render as R
from paper_2511_22793_gb300 import synth

C = 299792458.0


def _geo(n, px, py, cxx, cxy, cyy, r, valid=None):
    f = lambda v: np.broadcast_to(np.asarray(v, dtype=np.float64), (n,)).copy()
    return dict(px=f(px), py=f(py), cxx=f(cxx), cxy=f(cxy), cyy=f(cyy), r=f(r),
                valid=np.ones(n, dtype=bool) if valid is None else np.asarray(valid))


def _att(n, sigma, a, phi0, L):
    f = lambda v: np.broadcast_to(np.asarray(v, dtype=np.float64), (n,)).copy()
    return dict(sigma=f(sigma), a=f(a), phi0=f(phi0), L=f(L))


def _pix(H, W, xs, ys):
    return np.array([y * W + x for x, y in zip(xs, ys)], dtype=np.int32)


def test_single_gaussian_closed_form(oracle_lib):
    """One Gaussian: z_k(u) = sigma e^{-q/2} a e^{j(phi0 - 2 pi f_k L / c)} wherever
    alpha = sigma e^{-q/2} passes the cut-offs, and 0 elsewhere."""
    H, W, K = 20, 40, 5
    f_c, df = 2.4e9, 312.5e3
    g = _geo(1, 10.3, 7.8, 0.21, -0.05, 0.33, 2.0)
    at = _att(1, 0.8, 0.37, 0.9, 6.25)
    z, T, n = R.render_fwd(g, at, H, W, K, f_c, df)
    xs, ys = np.meshgrid(np.arange(W) + 0.5, np.arange(H) + 0.5)
    dx = (xs - 10.3).ravel()
    dx = dx - W * np.floor(dx / W + 0.5)
    dy = (ys - 7.8).ravel()
    q = 0.21 * dx * dx + 2 * (-0.05) * dx * dy + 0.33 * dy * dy
    alpha = np.minimum(0.99, 0.8 * np.exp(-q / 2))
    keep = (q <= 2 * math.log(255)) & (alpha >= 1 / 255)
    fk = f_c + (np.arange(K) - K // 2) * df
    ph = 0.37 * np.exp(1j * (0.9 - 2 * math.pi * fk * 6.25 / C))
    expect = np.where(keep[:, None], alpha[:, None] * ph[None, :], 0)
    np.testing.assert_allclose(z, expect, rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(T, np.where(keep, 1 - alpha, 1.0), rtol=1e-14)


def test_mean_on_pixel_centre_through_projection(oracle_lib):
    """A Gaussian whose mean projects onto the centre of pixel (x, y) renders
    z = sigma a e^{j psi} there (G = 1)."""
    H, W = 90, 360
    x, y = 123, 40
    phi = ((x + 0.5) * 2.0 / W - 1.0) * math.pi
    th = (y + 0.5) * math.pi / (2.0 * H)
    r = 3.0
    mu = np.array([[r * math.cos(th) * math.sin(phi), r * math.sin(th), r * math.cos(th) * math.cos(phi)]])
    geo = P.project(torch.tensor(mu), torch.full((1, 3), math.log(0.2), dtype=torch.float64),
                    torch.tensor([[1.0, 0, 0, 0]], dtype=torch.float64), synth.View(H=H, W=W))
    assert abs(geo["px"].item() - (x + 0.5)) < 1e-9 and abs(geo["py"].item() - (y + 0.5)) < 1e-9
    g = {k: geo[k].numpy() for k in ("px", "py", "cxx", "cxy", "cyy", "r", "valid")}
    at = _att(1, 0.6, 0.25, -0.4, 7.0)
    z, _, _ = R.render_fwd(g, at, H, W, 1, 2.4e9, 312.5e3, pixels=_pix(H, W, [x], [y]))
    psi = -0.4 - 2 * math.pi * 2.4e9 * 7.0 / C
    np.testing.assert_allclose(z[0, 0], 0.6 * 0.25 * np.exp(1j * psi), rtol=1e-12)


def test_coincident_gaussians_geometric_series(oracle_lib):
    """n identical Gaussians at one spot: composited count m is the largest with
    (1-alpha)^m >= 1e-4, T = (1-alpha)^m and z = a e^{j psi} (1 - (1-alpha)^m)."""
    for alpha, n in ((0.3, 10), (0.3, 40), (0.75, 12), (0.99, 5)):
        g = _geo(n, 5.5, 5.5, 0.5, 0.0, 0.5, np.linspace(1.0, 2.0, n))
        at = _att(n, alpha, 0.4, 0.2, 3.0)
        z, T, m = R.render_fwd(g, at, 12, 12, 1, 2.4e9, 1e6, pixels=_pix(12, 12, [5], [5]))
        mm = 0
        while mm < n and (1 - alpha) ** (mm + 1) >= 1e-4:
            mm += 1
        assert m[0] == mm
        np.testing.assert_allclose(T[0], (1 - alpha) ** mm, rtol=1e-12)
        psi = 0.2 - 2 * math.pi * 2.4e9 * 3.0 / C
        np.testing.assert_allclose(z[0, 0], 0.4 * np.exp(1j * psi) * (1 - (1 - alpha) ** mm), rtol=1e-12)


def test_subcarrier_ratio_single_gaussian(oracle_lib):
    H, W, K = 16, 32, 64
    g = _geo(1, 12.0, 8.0, 0.1, 0.0, 0.1, 2.0)
    at = _att(1, 0.7, 1.3, 0.5, 11.7)
    z, _, _ = R.render_fwd(g, at, H, W, K, 2.4e9, 312.5e3, pixels=_pix(H, W, [12], [8]))
    ratio = z[0, 1:] / z[0, :-1]
    np.testing.assert_allclose(ratio, np.exp(-2j * math.pi * 312.5e3 * 11.7 / C), rtol=1e-11)
    # K = 1 renders the carrier f_c itself
    z1, _, _ = R.render_fwd(g, at, H, W, 1, 2.4e9, 312.5e3, pixels=_pix(H, W, [12], [8]))
    np.testing.assert_allclose(z1[0, 0], z[0, K // 2], rtol=1e-13)


def _random_render_inputs(n, H, W, seed):
    rng = np.random.default_rng(seed)
    g = dict(px=rng.uniform(0, W, n), py=rng.uniform(-2, H + 2, n),
             cxx=rng.uniform(0.05, 0.6, n), cyy=rng.uniform(0.05, 0.6, n),
             r=rng.uniform(0.5, 8, n), valid=rng.uniform(size=n) > 0.05)
    g["cxy"] = rng.uniform(-0.8, 0.8, n) * np.sqrt(g["cxx"] * g["cyy"])
    at = dict(sigma=rng.uniform(0.02, 0.99, n), a=rng.uniform(0.01, 0.3, n),
              phi0=rng.normal(size=n), L=rng.uniform(1, 15, n))
    return g, at


def test_input_order_invariance_bit_exact(oracle_lib):
    H, W, K = 18, 36, 3
    g, at = _random_render_inputs(300, H, W, seed=41)
    z0, T0, n0 = R.render_fwd(g, at, H, W, K, 2.4e9, 312.5e3)
    perm = np.random.default_rng(42).permutation(300)
    g2 = {k: np.asarray(v)[perm] for k, v in g.items()}
    at2 = {k: np.asarray(v)[perm] for k, v in at.items()}
    z1, T1, n1 = R.render_fwd(g2, at2, H, W, K, 2.4e9, 312.5e3)
    assert np.array_equal(z0, z1) and np.array_equal(T0, T1) and np.array_equal(n0, n1)


def test_transmittance_monotone(oracle_lib):
    """T_final lies in [1e-4, 1]; in exact mode adding a Gaussian never raises it."""
    H, W, K = 18, 36, 1
    g, at = _random_render_inputs(200, H, W, seed=43)
    _, T, _ = R.render_fwd(g, at, H, W, K, 2.4e9, 312.5e3)
    assert np.all(T <= 1.0) and np.all(T >= 1e-4)
    _, Te, _ = R.render_fwd(g, at, H, W, K, 2.4e9, 312.5e3, exact=True)
    g2 = {k: np.asarray(v)[:150] for k, v in g.items()}
    at2 = {k: np.asarray(v)[:150] for k, v in at.items()}
    _, Te2, _ = R.render_fwd(g2, at2, H, W, K, 2.4e9, 312.5e3, exact=True)
    assert np.all(Te <= Te2 * (1 + 1e-15))


def test_mpmath_bruteforce_tiny(oracle_lib):
    """<= 4 Gaussians x 16 pixels at 50 digits straight from the definition."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    H, W, K = 4, 8, 3
    f_c, df = 2.4e9, 312.5e3
    rng = np.random.default_rng(44)
    n = 4
    g = dict(px=rng.uniform(0, W, n), py=rng.uniform(0, H, n), cxx=rng.uniform(0.2, 0.9, n),
             cyy=rng.uniform(0.2, 0.9, n), r=rng.uniform(1, 3, n), valid=np.ones(n, bool))
    g["cxy"] = rng.uniform(-0.5, 0.5, n) * np.sqrt(g["cxx"] * g["cyy"])
    at = dict(sigma=rng.uniform(0.3, 0.95, n), a=rng.uniform(0.1, 1, n), phi0=rng.normal(size=n),
              L=rng.uniform(2, 9, n))
    z, _, _ = R.render_fwd(g, at, H, W, K, f_c, df)
    for p in range(H * W):
        x, y = p % W, p // W
        hits = []
        for i in range(n):
            dx = mp.mpf(x) + mp.mpf("0.5") - mp.mpf(float(g["px"][i]))
            dx = dx - W * mp.floor(dx / W + mp.mpf("0.5"))
            dy = mp.mpf(y) + mp.mpf("0.5") - mp.mpf(float(g["py"][i]))
            q = (mp.mpf(float(g["cxx"][i])) * dx * dx + 2 * mp.mpf(float(g["cxy"][i])) * dx * dy
                 + mp.mpf(float(g["cyy"][i])) * dy * dy)
            if q > 2 * mp.log(255):
                continue
            al = min(mp.mpf("0.99"), mp.mpf(float(at["sigma"][i])) * mp.exp(-q / 2))
            if al < mp.mpf(1) / 255:
                continue
            hits.append((float(g["r"][i]), i, al))
        hits.sort()
        T = mp.mpf(1)
        zz = [mp.mpc(0)] * K
        for _, i, al in hits:
            if T * (1 - al) < mp.mpf("1e-4"):
                break
            for k in range(K):
                fk = mp.mpf(f_c) + (k - K // 2) * mp.mpf(df)
                psi = mp.mpf(float(at["phi0"][i])) - 2 * mp.pi * fk * mp.mpf(float(at["L"][i])) / C
                zz[k] += T * al * mp.mpf(float(at["a"][i])) * mp.expjpi(psi / mp.pi)
            T = T * (1 - al)
        for k in range(K):
            assert abs(complex(zz[k]) - z[p, k]) <= 1e-13 * max(1.0, abs(complex(zz[k])))


def test_zenith_rotation_shifts_columns(oracle_lib):
    """Rotating scene and transmitter by m * 2 pi / W about the vertical axis
    through the receiver shifts the spectrum by m columns (network blind to the
    transmitter's coordinates so the attributes are rotation invariant)."""
    H, W, K = 18, 72, 2
    sc = synth.make_scene(150, seed=45)
    sc.log_scales = sc.log_scales + np.float32(1.0)   # wider footprints on the 5-degree grid
    mlp = synth.make_mlp(8, seed=46)
    mlp.W1[0:3, :] = 0.0
    tx = np.array([[1.5, 2.0, -0.5]])
    view = synth.View(H=H, W=W)
    band = synth.Band(K=K)
    z0 = PL.forward(sc, mlp, view, band, tx)["z"][0].reshape(H, W, K)
    Rot = pytest.importorskip("scipy.spatial.transform").Rotation
    for m in (18, 7):
        ang = m * 360.0 / W
        R_ = Rot.from_euler("y", ang, degrees=True)
        sc2 = synth.Scene(means=R_.apply(sc.means.astype(np.float64)),
                          log_scales=sc.log_scales,
                          quats=(R_ * Rot.from_quat(sc.quats.astype(np.float64)[:, [1, 2, 3, 0]])).as_quat()[:, [3, 0, 1, 2]],
                          opacity_logit=sc.opacity_logit, latent=sc.latent)
        z1 = PL.forward(sc2, mlp, view, band, R_.apply(tx))["z"][0].reshape(H, W, K)
        np.testing.assert_allclose(z1, np.roll(z0, m, axis=1), rtol=1e-8, atol=1e-9 * np.abs(z0).max())


def test_exact_mode_close_to_cutoff_mode(oracle_lib):
    """The 3DGS cut-offs (q_max, alpha >= 1/255, T >= 1e-4) change the spectrum by
    a small amount relative to the exact compositing sum."""
    H, W, K = 18, 36, 4
    g, at = _random_render_inputs(400, H, W, seed=47)
    z, _, _ = R.render_fwd(g, at, H, W, K, 2.4e9, 312.5e3)
    ze, _, _ = R.render_fwd(g, at, H, W, K, 2.4e9, 312.5e3, exact=True)
    rel = np.linalg.norm(z - ze) / np.linalg.norm(ze)
    assert rel < 2e-2
