"""Per-Gaussian emission network (gsparc_emission_fwd / _bwd) against the FP64 oracle
(oracle/emission.py): attributes, gradients, the 1/d toggle, widths 8 to 64, and the spectrum
rendered from its attributes."""
import numpy as np
import pytest
import torch

from gpu_util import DEV, oracle_render, rel_l2, spectrum_to_complex
from oracle import emission as E
from oracle import projection as oproj
from paper_2511_22793_gb300 import gsparc as G
from paper_2511_22793_gb300 import synth
from paper_2511_22793_gb300.pipeline import DeviceScene, Renderer

pytestmark = pytest.mark.gpu

RX = (0.0, 0.0, 0.0)


def _weights(n, h, seed):
    """Flat buffers [n, 6h + 2]: W ~ N(0,1)/sqrt(fan_in), biases N(0, 0.1^2)."""
    rng = np.random.default_rng(seed)
    flat = np.zeros((n, E.n_params(h)))
    flat[:, :3 * h] = rng.normal(size=(n, 3 * h)) / np.sqrt(3.0)
    flat[:, 3 * h:4 * h] = 0.1 * rng.normal(size=(n, h))
    flat[:, 4 * h:6 * h] = rng.normal(size=(n, 2 * h)) / np.sqrt(h)
    flat[:, 6 * h:] = 0.1 * rng.normal(size=(n, 2))
    return flat


def _device_weights(flat, h):
    n = flat.shape[0]
    stride = G.gsparc_emission_stride(h)
    buf = np.zeros((max(n, 1), stride), np.float32)
    buf[:n, :flat.shape[1]] = flat
    return torch.tensor(buf[:n] if n else buf[:0], device=DEV).contiguous()


def _oracle_attr(means, ologit, flat32, h, txs, inv_d):
    f64 = lambda a: torch.tensor(np.asarray(a, dtype=np.float64))
    out = []
    for t in txs:
        at = E.attributes(f64(means), f64(ologit), f64(flat32), h, t, RX, inv_d=inv_d)
        out.append(np.stack([at[k].numpy() for k in ("a", "phi0", "sigma", "L")], -1))
    return np.stack(out)


@pytest.mark.parametrize("n,h,B,inv_d", [(1, 16, 1, True), (777, 8, 3, True), (50_000, 16, 1, True),
                                         (3001, 64, 2, False), (4096, 16, 4, False), (130, 5, 1, True)])
def test_emission_forward_matches_oracle(n, h, B, inv_d):
    sc = synth.make_scene(max(n, 1), seed=61)
    means = sc.means[:n].astype(np.float32)
    ologit = sc.opacity_logit[:n].astype(np.float32)
    flat = _weights(n, h, 62).astype(np.float32)
    txs = synth.make_tx(B, seed=63)
    attr = torch.empty((B, n, 4), device=DEV)
    G.gsparc_emission_fwd(torch.tensor(txs, device=DEV), RX, torch.tensor(means, device=DEV),
                          torch.tensor(ologit, device=DEV), _device_weights(flat, h), h, attr, inv_d=inv_d)
    torch.cuda.synchronize()
    got = attr.cpu().numpy().astype(np.float64)
    want = _oracle_attr(means, ologit, flat, h, txs, inv_d)
    for c in range(4):
        e = rel_l2(got[..., c], want[..., c])
        assert e <= 1e-5, (c, e)
    # phase within [0, pi/2] (Re, Im > 0), amplitude positive
    assert np.all(got[..., 1] > 0) and np.all(got[..., 1] < np.pi / 2 + 1e-6) and np.all(got[..., 0] > 0)


def _kink_rows(means, flat32, h, txs, eps=1e-5):
    """Gaussians with a hidden pre-activation within eps of the ReLU kink for some transmitter."""
    f64 = lambda a: torch.tensor(np.asarray(a, dtype=np.float64))
    W1, b1, _, _ = E.unpack(f64(flat32), h)
    bad = np.zeros(flat32.shape[0], bool)
    for t in txs:
        pre = torch.einsum("k,nkj->nj", f64(t), W1) + b1
        bad |= (pre.abs() < eps).any(dim=1).numpy()
    return bad


@pytest.mark.parametrize("n,h,B,inv_d", [(777, 16, 1, True), (20_000, 16, 3, True), (3001, 64, 2, False),
                                         (1000, 8, 1, False)])
def test_emission_backward_matches_oracle(n, h, B, inv_d):
    """Gradients (added into zero buffers) against the oracle's FP64 vector-Jacobian product for a
    random upstream gradient; Gaussians at a ReLU kink (at most 0.1%) are left out of the
    comparison, since FP32 and FP64 may take the unit on different sides."""
    sc = synth.make_scene(n, seed=71)
    means = sc.means.astype(np.float32)
    ologit = sc.opacity_logit.astype(np.float32)
    flat = _weights(n, h, 72).astype(np.float32)
    txs = synth.make_tx(B, seed=73)
    g = np.random.default_rng(74).normal(size=(B, n, 4)).astype(np.float32)
    dm = torch.zeros((n, 3), device=DEV)
    do = torch.zeros(n, device=DEV)
    wdev = _device_weights(flat, h)
    dw = torch.zeros_like(wdev)
    G.gsparc_emission_bwd(torch.tensor(txs, device=DEV), RX, torch.tensor(means, device=DEV),
                          torch.tensor(ologit, device=DEV), wdev, h, torch.tensor(g, device=DEV), dm, do, dw,
                          inv_d=inv_d)
    torch.cuda.synchronize()
    gm, go, gf = E.attributes_vjp(means.astype(np.float64), ologit.astype(np.float64), flat.astype(np.float64),
                                  h, txs.astype(np.float64), RX, g.astype(np.float64), inv_d=inv_d)
    keep = ~_kink_rows(means, flat, h, txs)
    assert keep.mean() >= 0.999
    dwn = dw.cpu().numpy().astype(np.float64)
    assert np.all(dwn[:, E.n_params(h):] == 0.0)          # padding untouched
    assert rel_l2(dm.cpu().numpy()[keep], gm[keep]) <= 1e-4
    assert rel_l2(do.cpu().numpy()[keep], go[keep]) <= 1e-5
    for lo, hi in ((0, 3 * h), (3 * h, 4 * h), (4 * h, 6 * h), (6 * h, 6 * h + 2)):   # W1, b1, W2, b2
        e = rel_l2(dwn[keep, lo:hi], gf[keep, lo:hi])
        assert e <= 1e-4, (lo, hi, e)


def test_emission_backward_accumulates():
    """Two calls add twice the gradient of one."""
    n, h = 500, 16
    sc = synth.make_scene(n, seed=81)
    args = (torch.tensor(synth.make_tx(2, seed=82), device=DEV), RX, torch.tensor(sc.means, device=DEV),
            torch.tensor(sc.opacity_logit, device=DEV), _device_weights(_weights(n, h, 83).astype(np.float32), h),
            h, torch.randn((2, n, 4), device=DEV))
    outs = []
    for calls in (1, 2):
        dm, do = torch.zeros((n, 3), device=DEV), torch.zeros(n, device=DEV)
        dw = torch.zeros_like(args[4])
        for _ in range(calls):
            G.gsparc_emission_bwd(*args, dm, do, dw)
        torch.cuda.synchronize()
        outs.append([t.cpu().numpy() for t in (dm, do, dw)])
    for one, two in zip(*outs):
        assert rel_l2(two, 2 * one) <= 1e-6


@pytest.mark.parametrize("inv_d", [True, False])
def test_spectrum_from_emission_matches_oracle(inv_d):
    """The renderer fed by the per-Gaussian network against the oracle's per-pixel renderer fed by
    the oracle's emission attributes (FP64 projection): relative L2 per spectrum <= 1e-3."""
    n, h, H, W, K = 2000, 16, 45, 180, 8
    sc = synth.make_scene(n, seed=91)
    flat = _weights(n, h, 92).astype(np.float32)
    txs = synth.make_tx(2, seed=93)
    r = Renderer(H, W, K, n, device=DEV)
    ds = DeviceScene.from_host(sc, DEV)
    r.geometry(ds)
    attr = torch.empty((2, n, 4), device=DEV)
    G.gsparc_emission_fwd(torch.tensor(txs, device=DEV), RX, ds.means, ds.opacity_logit, _device_weights(flat, h),
                          h, attr, inv_d=inv_d)
    spec, _, _ = r.render(attr)
    torch.cuda.synchronize()
    assert r.check() == 0
    view, band = synth.View(H=H, W=W), synth.Band(K=K)
    f64 = lambda a: torch.tensor(np.asarray(a), dtype=torch.float64)
    geo = oproj.project(f64(sc.means), f64(sc.log_scales), f64(sc.quats), view)
    g = {k: geo[k].numpy() for k in ("px", "py", "cxx", "cxy", "cyy", "r", "valid", "ext_x", "ext_y",
                                     "sxx", "sxy", "syy")}
    attrs = []
    for t in txs:
        at = E.attributes(f64(sc.means), f64(sc.opacity_logit), f64(flat), h, t, view.rx, inv_d=inv_d)
        attrs.append({k: at[k].numpy() for k in ("sigma", "a", "phi0", "L")})
    z_ref, _, _ = oracle_render(g, attrs, view, band)
    z = spectrum_to_complex(spec)
    for b in range(2):
        assert rel_l2(z[b], z_ref[b]) <= 1e-3
