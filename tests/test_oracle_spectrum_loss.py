"""Pins of the oracle's magnitude-spectrum loss (Eq. 4, L1 + SSIM): SSIM of a plane with itself,
the closed form of constant planes, the window, a brute-force SSIM from its definition, L1 by
hand, and central differences of the complex gradient."""
import math

import numpy as np
import torch

from oracle import spectrum_loss as S


def test_window():
    g = S.window_1d()
    assert abs(g.sum() - 1.0) < 1e-15 and np.allclose(g, g[::-1], rtol=0, atol=0)
    assert abs(g[5] / g[6] - math.exp(1.0 / (2 * S.SIGMA ** 2))) < 1e-12
    assert abs(S.window_2d().sum() - 1.0) < 1e-14


def test_identical_planes_give_ssim_one_and_zero_loss():
    rng = np.random.default_rng(0)
    z = rng.normal(size=(2, 3, 12, 20)) + 1j * rng.normal(size=(2, 3, 12, 20))
    x = torch.tensor(np.abs(z).reshape(6, 12, 20))
    assert np.allclose(S.ssim_map(x, x).numpy(), 1.0, rtol=0, atol=1e-12)
    L, gre, gim = S.loss_and_grad(z, np.abs(z))
    assert abs(L) < 1e-12


def test_constant_planes_closed_form():
    """x = a and y = b everywhere: away from the zero padding mu_x = a, mu_y = b and every
    variance is 0, so S = (2ab + C1) / (a^2 + b^2 + C1)."""
    a, b = 0.7, 0.3
    x = torch.full((1, 30, 40), a, dtype=torch.float64)
    y = torch.full((1, 30, 40), b, dtype=torch.float64)
    m = S.ssim_map(x, y).numpy()[0]
    want = (2 * a * b + S.C1) / (a * a + b * b + S.C1)
    assert np.allclose(m[5:-5, 5:-5], want, rtol=1e-12, atol=0)


def _ssim_brute(x, y):
    """SSIM map of one [H, W] plane from the definition: windowed moments with zero padding."""
    H, W = x.shape
    g = S.window_2d()
    r = S.WINDOW // 2
    out = np.zeros((H, W))
    for i in range(H):
        for j in range(W):
            mx = my = exx = eyy = exy = 0.0
            for di in range(-r, r + 1):
                for dj in range(-r, r + 1):
                    ii, jj = i + di, j + dj
                    if 0 <= ii < H and 0 <= jj < W:
                        wv = g[di + r, dj + r]
                        mx += wv * x[ii, jj]
                        my += wv * y[ii, jj]
                        exx += wv * x[ii, jj] ** 2
                        eyy += wv * y[ii, jj] ** 2
                        exy += wv * x[ii, jj] * y[ii, jj]
            sxx, syy, sxy = exx - mx * mx, eyy - my * my, exy - mx * my
            out[i, j] = ((2 * mx * my + S.C1) * (2 * sxy + S.C2)) / ((mx * mx + my * my + S.C1) * (sxx + syy + S.C2))
    return out


def test_ssim_map_against_brute_force():
    rng = np.random.default_rng(1)
    x = rng.uniform(0, 1, size=(7, 13))
    y = np.clip(x + 0.2 * rng.normal(size=(7, 13)), 0, None)
    got = S.ssim_map(torch.tensor(x[None]), torch.tensor(y[None])).numpy()[0]
    assert np.allclose(got, _ssim_brute(x, y), rtol=1e-12, atol=1e-14)


def test_l1_part_by_hand():
    """With lam = 0 the loss is the mean absolute error of the magnitudes: |3+4j| = 5 against
    2, |1| against 1.5, |-2j| against 2, |0| against 0.25: (3 + 0.5 + 0 + 0.25) / 4."""
    z = np.array([3 + 4j, 1, -2j, 0]).reshape(1, 1, 2, 2)
    y = np.array([2.0, 1.5, 2.0, 0.25]).reshape(1, 1, 2, 2)
    L, _, _ = S.loss_and_grad(z, y, lam=0.0)
    assert abs(L - 3.75 / 4) < 1e-15


def test_gradient_against_central_differences():
    """dL/dRe z and dL/dIm z against central differences (step 1e-6), magnitudes kept away from
    0 and from the target (the L1 kink)."""
    rng = np.random.default_rng(2)
    z = (0.5 + rng.uniform(size=(1, 2, 8, 9))) * np.exp(2j * np.pi * rng.uniform(size=(1, 2, 8, 9)))
    y = np.abs(z) * (1 + 0.3 * np.sign(rng.normal(size=z.shape)) * (0.2 + rng.uniform(size=z.shape)))
    L, gre, gim = S.loss_and_grad(z, y)
    h = 1e-6
    for part, grad in ((1.0, gre), (1j, gim)):
        num = np.zeros(z.shape)
        for idx in np.ndindex(z.shape):
            zp, zm = z.copy(), z.copy()
            zp[idx] += h * part
            zm[idx] -= h * part
            num[idx] = (S.loss_and_grad(zp, y)[0] - S.loss_and_grad(zm, y)[0]) / (2 * h)
        assert np.allclose(grad, num, rtol=1e-5, atol=1e-9)


def test_zero_spectrum_value_has_zero_gradient():
    z = np.ones((1, 1, 12, 12), complex)
    z[0, 0, 6, 6] = 0
    _, gre, gim = S.loss_and_grad(z, np.full(z.shape, 0.5))
    assert gre[0, 0, 6, 6] == 0 and gim[0, 0, 6, 6] == 0
