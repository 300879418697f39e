"""Finite-difference pins for the oracle's analytic gradient.

The renderer's hand-derived FP64 gradient (render_oracle.c) is checked
against central differences of its own forward; the chained gradient
(projection and attribute network by autograd) against central differences
of the whole loss.  Parameters whose +-h changes the composited set (a
cut-off or the termination point moved) are resampled.
"""
import math

import numpy as np
import pytest

from oracle import pipeline as PL
from oracle import render as R
from paper_2511_22793_gb300 import synth

COLS = ("px", "py", "cxx", "cxy", "cyy", "sigma", "a", "phi0", "L")


def _inputs(n, H, W, seed):
    rng = np.random.default_rng(seed)
    g = dict(px=rng.uniform(0, W, n), py=rng.uniform(-1, H + 1, n),
             cxx=rng.uniform(0.05, 0.5, n), cyy=rng.uniform(0.05, 0.5, n),
             r=rng.uniform(0.5, 8, n), valid=np.ones(n, bool))
    g["cxy"] = rng.uniform(-0.7, 0.7, n) * np.sqrt(g["cxx"] * g["cyy"])
    at = dict(sigma=rng.uniform(0.05, 0.9, n), a=rng.uniform(0.05, 0.5, n),
              phi0=rng.normal(size=n), L=rng.uniform(1, 15, n))
    return g, at


def _loss(g, at, H, W, K, target, exact):
    z, _, _, sig = R.render_fwd(g, at, H, W, K, 2.4e9, 312.5e3, exact=exact, signature=True)
    d = z - target
    return float(np.sum(d.real ** 2 + d.imag ** 2)), sig


@pytest.mark.parametrize("exact", [True, False])
def test_render_gradient_vs_central_differences(oracle_lib, exact):
    H, W, K, n = 16, 32, 6, 60
    g, at = _inputs(n, H, W, seed=51)
    rng = np.random.default_rng(52)
    target = rng.normal(size=(H * W, K)) * 0.05 + 1j * rng.normal(size=(H * W, K)) * 0.05
    z, _, _ = R.render_fwd(g, at, H, W, K, 2.4e9, 312.5e3, exact=exact)
    grad = R.render_bwd(g, at, H, W, K, 2.4e9, 312.5e3, 2.0 * (z - target), exact=exact)
    checked = 0
    tries = 0
    while checked < 32 and tries < 400:
        tries += 1
        i = int(rng.integers(n))
        c = int(rng.integers(9))
        src = g if COLS[c] in g else at
        x0 = src[COLS[c]][i]
        h = 1e-6 * max(1.0, abs(x0))
        src[COLS[c]][i] = x0 + h
        lp, sp = _loss(g, at, H, W, K, target, exact)
        src[COLS[c]][i] = x0 - h
        lm, sm = _loss(g, at, H, W, K, target, exact)
        src[COLS[c]][i] = x0
        _, s0 = _loss(g, at, H, W, K, target, exact)
        if not (np.array_equal(sp, s0) and np.array_equal(sm, s0)):
            continue           # composited set changed: not differentiable here
        fd = (lp - lm) / (2 * h)
        an = grad[i, c]
        if abs(fd) < 1e-9 and abs(an) < 1e-9:
            continue
        assert abs(fd - an) <= 1e-5 * max(abs(fd), abs(an)) + 1e-10, (COLS[c], i, fd, an)
        checked += 1
    assert checked >= 32


def test_full_loss_gradient_vs_central_differences(oracle_lib):
    """Loss through projection, attribute network and renderer; FD on 32 sampled
    scene and network parameters."""
    H, W, K = 18, 72, 4
    sc = synth.make_scene(80, seed=53)
    sc.log_scales = sc.log_scales + np.float32(1.2)
    mlp = synth.make_mlp(8, seed=54)
    view = synth.View(H=H, W=W)
    band = synth.Band(K=K)
    tx = synth.make_tx(2, seed=55).astype(np.float64)
    rng = np.random.default_rng(56)
    target = 0.02 * (rng.normal(size=(2, H * W, K)) + 1j * rng.normal(size=(2, H * W, K)))
    scd = synth.Scene(*[np.asarray(a, dtype=np.float64).copy() for a in sc.arrays()])
    mld = synth.MLPWeights(8, *[np.asarray(a, dtype=np.float64).copy() for a in mlp.arrays()])
    loss, grads = PL.loss_and_grad(scd, mld, view, band, tx, target)

    def sig_of():
        out = PL.forward(scd, mld, view, band, tx)
        from oracle import render as RR
        sigs = []
        for at in out["attrs"]:
            g = {k: out["geo"][k].numpy() for k in ("px", "py", "cxx", "cxy", "cyy", "r", "valid")}
            a = {k: at[k].numpy() for k in ("sigma", "a", "phi0", "L")}
            sigs.append(RR.render_fwd(g, a, H, W, K, band.f_c, band.df, signature=True)[3])
        return np.stack(sigs), out

    s0, _ = sig_of()
    names = ["means", "log_scales", "quats", "opacity_logit", "latent", "W1", "b1", "W2", "b2",
             "W3", "b3"]
    holders = {nm: arr for nm, arr in zip(names[:5], scd.arrays())}
    holders.update({nm: arr for nm, arr in zip(names[5:], mld.arrays())})
    checked, tries = 0, 0
    while checked < 32 and tries < 300:
        tries += 1
        nm = names[int(rng.integers(len(names)))]
        arr = holders[nm]
        flat = arr.reshape(-1)
        j = int(rng.integers(flat.size))
        x0 = flat[j]
        h = 1e-6 * max(1.0, abs(x0))
        flat[j] = x0 + h
        sp, op = sig_of()
        lp = float(np.sum(np.abs(op["z"] - target) ** 2) / target.size)
        flat[j] = x0 - h
        sm, om = sig_of()
        lm = float(np.sum(np.abs(om["z"] - target) ** 2) / target.size)
        flat[j] = x0
        if not (np.array_equal(sp, s0) and np.array_equal(sm, s0)):
            continue
        fd = (lp - lm) / (2 * h)
        an = grads[nm].reshape(-1)[j]
        if abs(fd) < 1e-12 and abs(an) < 1e-12:
            continue
        assert abs(fd - an) <= 1e-5 * max(abs(fd), abs(an)) + 1e-12, (nm, j, fd, an)
        checked += 1
    assert checked >= 32
