"""GPU gradients (hand-written backward behind a torch.autograd.Function)
against the FP64 oracle's analytic gradient, which the CPU tests pin to
central finite differences.

Tolerance: <= 1e-3 relative L2 per gradient tensor for the per-Gaussian
render inputs and <= 5e-3 for the chained scene / network gradients (the
chain through Sigma'^-1 and the quaternion amplifies FP32 rounding of the
largest entries; see the derivation beside each bound).
"""
import numpy as np
import pytest
import torch

from gpu_util import DEV, oracle_geo_attr, rel_l2, spectrum_to_complex
from oracle import attributes as oattr
from oracle import pipeline as opl
from oracle import render as orender
from paper_2511_22793_gb300 import gsparc as G
from paper_2511_22793_gb300 import synth
from paper_2511_22793_gb300.autograd import splat
from paper_2511_22793_gb300.pipeline import DeviceMLP, DeviceScene, Renderer

pytestmark = pytest.mark.gpu


def _target(B, H, W, K, seed):
    rng = np.random.default_rng(seed)
    return 0.01 * (rng.normal(size=(B, H * W, K)) + 1j * rng.normal(size=(B, H * W, K)))


def _to_dev_target(t, B, H, W, K):
    a = np.stack([t.real, t.imag], -1).reshape(B, H, W, K, 2).transpose(0, 3, 1, 2, 4)
    return torch.tensor(a.copy(), dtype=torch.float32, device=DEV)


def _gpu_grads(sc, mlp, H, W, K, tx, target):
    B = tx.shape[0]
    r = Renderer(H, W, K, sc.n, device=DEV)
    ds = DeviceScene.from_host(sc, DEV)
    dm = DeviceMLP.from_host(mlp, DEV)
    ps = [t.clone().requires_grad_(True) for t in ds.tensors()]
    ws = [t.clone().requires_grad_(True) for t in dm.tensors()]
    spec = splat(r, torch.tensor(tx, device=DEV), ps, ws)
    tgt = _to_dev_target(target, B, H, W, K)
    loss = ((spec - tgt) ** 2).sum() / (spec.numel() // 2)
    loss.backward()
    torch.cuda.synchronize()
    assert r.check() == 0
    names = ["means", "log_scales", "quats", "opacity_logit", "latent", "W1", "b1", "W2", "b2", "W3",
             "b3"]
    return float(loss), {n: p.grad.cpu().numpy().astype(np.float64) for n, p in zip(names, ps + ws)}, spec


@pytest.mark.parametrize("n,H,W,K,B,hidden,widen", [(400, 45, 180, 8, 2, 16, 0.4),
                                                   (2000, 90, 360, 64, 1, 32, 0.0),
                                                   (1000, 90, 360, 1, 2, 32, 0.0)])
def test_full_gradient_matches_oracle(n, H, W, K, B, hidden, widen):
    sc = synth.make_scene(n, seed=21)
    if widen:
        sc.log_scales = sc.log_scales + np.float32(widen)
    mlp = synth.make_mlp(hidden, seed=3)
    tx = synth.make_tx(B, seed=22)
    target = _target(B, H, W, K, 23)
    loss, g, spec = _gpu_grads(sc, mlp, H, W, K, tx, target)
    ref_loss, ref = opl.loss_and_grad(sc, mlp, synth.View(H=H, W=W), synth.Band(K=K), tx, target)
    assert abs(loss - ref_loss) <= 1e-3 * ref_loss
    assert rel_l2(spectrum_to_complex(spec), ref["z"]) <= 1e-3
    for k in g:
        e = rel_l2(g[k], ref[k])
        assert e <= 5e-3, "%s: relative L2 %.3e" % (k, e)


def test_render_bwd_per_gaussian_inputs():
    """gsparc_render_bwd alone: d(p, conic, sigma, a, phi0, L) against the oracle's
    analytic render gradient on the same FP32 attribute and projection values
    (both computed by the oracle and rounded to FP32, so only the backward
    differs)."""
    H, W, K, B, n = 90, 360, 32, 1, 3000
    sc = synth.make_scene(n, seed=31)
    mlp = synth.make_mlp(32, seed=3)
    tx = synth.make_tx(B, seed=32)
    view, band = synth.View(H=H, W=W), synth.Band(K=K)
    g, attrs = oracle_geo_attr(sc, mlp, view, tx)
    # FP32 copies of the oracle's per-Gaussian values feed both sides
    g32 = {k: (v.astype(np.float32).astype(np.float64) if v.dtype != bool else v) for k, v in g.items()}
    at32 = [{k: v.astype(np.float32).astype(np.float64) for k, v in at.items()} for at in attrs]
    proj = np.zeros((n, 8), np.float32)
    proj[:, 0], proj[:, 1] = g32["px"], g32["py"]
    proj[:, 2] = np.where(g["valid"], np.sqrt(2 * np.log(255) * g["sxx"]), -1)
    proj[:, 3] = np.where(g["valid"], np.sqrt(2 * np.log(255) * g["syy"]), -1)
    proj[:, 4], proj[:, 5], proj[:, 6], proj[:, 7] = g32["cxx"], g32["cxy"], g32["cyy"], g32["r"]
    attr = np.stack([np.stack([at["a"], at["phi0"], at["sigma"], at["L"]], -1) for at in at32]).astype(np.float32)
    r = Renderer(H, W, K, n, device=DEV)
    r.proj.copy_(torch.tensor(proj, device=DEV))
    G.gsparc_bin_sort(r.view, n, r.proj, r.capacity, r.ws, r.sorted_ids, None, r.tile_ranges, r.n_pairs,
                      r.status)
    attr_d = torch.tensor(attr, device=DEV)
    spec, logT, nc = r.render(attr_d)
    rng = np.random.default_rng(33)
    gz = rng.normal(size=(B, H * W, K)) + 1j * rng.normal(size=(B, H * W, K))
    d_spec = _to_dev_target(gz, B, H, W, K)
    d_attr = torch.zeros_like(attr_d)
    d_proj = torch.zeros_like(r.proj)
    r.render_backward(attr_d, logT, nc, d_spec, d_attr, d_proj)
    torch.cuda.synchronize()
    ref = orender.render_bwd(g32, at32[0], H, W, K, band.f_c, band.df, gz[0])
    da = d_attr.cpu().numpy()[0].astype(np.float64)
    dp = d_proj.cpu().numpy().astype(np.float64)
    got = {"px": dp[:, 0], "py": dp[:, 1], "cxx": dp[:, 4], "cxy": dp[:, 5], "cyy": dp[:, 6],
           "sigma": da[:, 2], "a": da[:, 0], "phi0": da[:, 1], "L": da[:, 3]}
    for c, k in enumerate(("px", "py", "cxx", "cxy", "cyy", "sigma", "a", "phi0", "L")):
        e = rel_l2(got[k], ref[:, c])
        assert e <= 1e-3, "%s: relative L2 %.3e" % (k, e)


@pytest.mark.parametrize("n,H,W,K,B,seed", [(3000, 90, 360, 64, 1, 31), (2000, 90, 360, 37, 2, 32),
                                             (1500, 45, 180, 8, 2, 33), (3000, 180, 720, 100, 1, 34),
                                             (1500, 45, 180, 100, 1, 35)])
def test_render_bwd_tensor_cores_matches_fp32_kernel_and_oracle(n, H, W, K, B, seed):
    """gsparc_render_bwd_tc and the scheduled gsparc_render_bwd_tc_balanced against
    gsparc_render_bwd (same inputs, relative L2 <= 1e-4 per component) and the oracle's
    analytic gradient of transmitter 0 (<= 1e-3).  The scheduled form runs unsplit (items
    ordered only), with every walk longer than one batch split (front chunks taking s_tot
    from the spectrum), and split with s_tot given as a buffer; with more than 2 x SMs
    (transmitter, tile, strip) units (the 180x720 case) no walk is split."""
    sc = synth.make_scene(n, seed=seed)
    mlp = synth.make_mlp(32, seed=3)
    tx = synth.make_tx(B, seed=seed + 1)
    view, band = synth.View(H=H, W=W), synth.Band(K=K)
    g, attrs = oracle_geo_attr(sc, mlp, view, tx)
    g32 = {k: (v.astype(np.float32).astype(np.float64) if v.dtype != bool else v) for k, v in g.items()}
    at32 = [{k: v.astype(np.float32).astype(np.float64) for k, v in at.items()} for at in attrs]
    proj = np.zeros((n, 8), np.float32)
    proj[:, 0], proj[:, 1] = g32["px"], g32["py"]
    proj[:, 2] = np.where(g["valid"], np.sqrt(2 * np.log(255) * g["sxx"]), -1)
    proj[:, 3] = np.where(g["valid"], np.sqrt(2 * np.log(255) * g["syy"]), -1)
    proj[:, 4], proj[:, 5], proj[:, 6], proj[:, 7] = g32["cxx"], g32["cxy"], g32["cyy"], g32["r"]
    attr = np.stack([np.stack([at["a"], at["phi0"], at["sigma"], at["L"]], -1) for at in at32]).astype(np.float32)
    r = Renderer(H, W, K, n, device=DEV)
    r.proj.copy_(torch.tensor(proj, device=DEV))
    G.gsparc_bin_sort(r.view, n, r.proj, r.capacity, r.ws, r.sorted_ids, None, r.tile_ranges, r.n_pairs,
                      r.status)
    attr_d = torch.tensor(attr, device=DEV)
    spec, logT, nc = r.render(attr_d)
    rng = np.random.default_rng(seed + 2)
    gz = rng.normal(size=(B, H * W, K)) + 1j * rng.normal(size=(B, H * W, K))
    d_spec = _to_dev_target(gz, B, H, W, K)
    # s_tot[b, s, p] = sum over strip s of Re(conj(g) z), as the fused forward writes it
    nst = G.s_tot_strips(K)
    zc = spectrum_to_complex(spec).reshape(B, H * W, K)
    prod = (np.conj(gz) * zc).real
    s_tot_np = np.stack([prod[:, :, s * 64:(s + 1) * 64].sum(-1) for s in range(nst)], 1) if K > 64 \
        else prod.sum(-1)[:, None]
    s_tot = torch.tensor(s_tot_np.reshape(B, nst, H, W).astype(np.float32), device=DEV)
    forms = {
        "fp32": lambda da, dp: r.render_backward(attr_d, logT, nc, d_spec, da, dp),
        "tc": lambda da, dp: G.gsparc_render_bwd_tc(r.view, r.band, B, n, r.proj, r.tile_ranges, r.sorted_ids,
                                                    attr_d, logT, nc, d_spec, da, dp),
        "ordered": lambda da, dp: r.render_backward(attr_d, logT, nc, d_spec, da, dp, tensor_cores=True),
        "split": lambda da, dp: r.render_backward(attr_d, logT, nc, d_spec, da, dp, tensor_cores=True,
                                                  spectrum=spec, split_min=1),
        "split_s_tot": lambda da, dp: r.render_backward(attr_d, logT, nc, d_spec, da, dp, tensor_cores=True,
                                                        s_tot=s_tot, split_min=1),
    }
    res = {}
    for name, fn in forms.items():
        d_attr = torch.zeros_like(attr_d)
        d_proj = torch.zeros_like(r.proj)
        fn(d_attr, d_proj)
        torch.cuda.synchronize()
        res[name] = (d_attr.cpu().numpy().astype(np.float64), d_proj.cpu().numpy().astype(np.float64))
    assert r.check() == 0
    fa, fp = res["fp32"]
    for name in ("tc", "ordered", "split", "split_s_tot"):
        ta, tp = res[name]
        for j in range(4):
            e = rel_l2(ta[..., j], fa[..., j])
            assert e <= 1e-4, (name, "attr", j, e)
        for j in (0, 1, 4, 5, 6):
            e = rel_l2(tp[:, j], fp[:, j])
            assert e <= 1e-4, (name, "proj", j, e)
    ta, tp = res["split"]
    ref = orender.render_bwd(g32, at32[0], H, W, K, band.f_c, band.df, gz[0])
    if B == 1:
        got = {"px": tp[:, 0], "py": tp[:, 1], "cxx": tp[:, 4], "cxy": tp[:, 5], "cyy": tp[:, 6],
               "sigma": ta[0, :, 2], "a": ta[0, :, 0], "phi0": ta[0, :, 1], "L": ta[0, :, 3]}
        for c, k in enumerate(("px", "py", "cxx", "cxy", "cyy", "sigma", "a", "phi0", "L")):
            assert rel_l2(got[k], ref[:, c]) <= 1e-3, k


def _relu_margin(sc, mlp, tx):
    """Per Gaussian, min over transmitters and hidden units of |u| - bound(u), with u the FP64
    pre-activation of a hidden unit and bound(u) what the split-BF16 products can move it: each
    operand is carried as hi + lo BF16 terms (8 significant bits each, so the representation
    error is at most 2^-17 relative), the dropped lo*lo product is at most 2^-18 relative and
    the FP32 accumulation adds 2^-24 per term, so one product is off by at most 2^-15.5 of
    |a b|; four times that over sum |a b| bounds a layer, and layer 2 also inherits layer 1's
    bound through |W2|.  A ReLU decision can differ from FP64 only where the margin is <= 0."""
    f64 = lambda a: torch.tensor(np.asarray(a), dtype=torch.float64)
    means, latent = f64(sc.means), f64(sc.latent)
    W1, b1, W2, b2 = (f64(a) for a in mlp.arrays()[:4])
    eps = 4.0 * 2.0 ** -15.5
    out = torch.full((sc.n,), float("inf"), dtype=torch.float64)
    for t in np.asarray(tx, dtype=np.float64):
        d = torch.clamp(torch.linalg.norm(means - f64(t), dim=1), min=0.01)
        h0 = torch.cat([f64(t).reshape(1, 3).expand(sc.n, 3), latent, torch.log(d).reshape(-1, 1)], 1)
        u1 = h0 @ W1 + b1
        bnd1 = eps * (h0.abs() @ W1.abs() + b1.abs())
        h1 = torch.relu(u1)
        u2 = h1 @ W2 + b2
        bnd2 = eps * (h1.abs() @ W2.abs() + b2.abs()) + bnd1 @ W2.abs()
        m = torch.minimum((u1.abs() - bnd1).min(1).values, (u2.abs() - bnd2).min(1).values)
        out = torch.minimum(out, m)
    return out.numpy()


def _row_err(got, want):
    g = got.reshape(got.shape[0], -1)
    w = want.reshape(want.shape[0], -1)
    return np.linalg.norm(g - w, axis=1) / np.maximum(np.linalg.norm(w, axis=1), 1e-30)


def _mlp_grads_gpu(r, ds, dm, txd, d_attr_np, tc, hidden=None):
    n = ds.n
    gm = torch.zeros((n, 3), device=DEV)
    go = torch.zeros(n, device=DEV)
    gl = torch.zeros((n, 16), device=DEV)
    gw = [torch.zeros_like(t) for t in dm.tensors()]
    r.attributes_backward(ds, dm, txd, torch.tensor(d_attr_np, device=DEV), gm, go, gl, gw, tensor_cores=tc,
                          hidden=hidden)
    torch.cuda.synchronize()
    return [t.cpu().numpy().astype(np.float64) for t in [gm, go, gl] + gw]


def _mlp_grads_oracle(sc, mlp, tx, d_attr_np):
    """FP64 oracle: d/d(params) of sum(attr * d_attr) through the attribute network (means
    only through the network inputs d and L, as gsparc_attr_mlp_bwd)."""
    f64 = lambda a: torch.tensor(np.asarray(a), dtype=torch.float64)
    means = f64(sc.means).requires_grad_(True)
    ologit = f64(sc.opacity_logit).requires_grad_(True)
    latent = f64(sc.latent).requires_grad_(True)
    weights = [f64(a).requires_grad_(True) for a in mlp.arrays()]
    total = 0.0
    for bi in range(len(tx)):
        at = oattr.attributes(means, ologit, latent, weights, f64(tx[bi]), (0.0, 0.0, 0.0))
        stacked = torch.stack([at["a"], at["phi0"], at["sigma"], at["L"]], -1)
        total = total + (stacked * f64(d_attr_np[bi])).sum()
    return [t.numpy() for t in torch.autograd.grad(total, [means, ologit, latent] + weights)]


@pytest.mark.parametrize("n,B,hidden,seed", [(3000, 1, 32, 41), (1000, 3, 16, 42), (50_000, 1, 32, 43),
                                            (777, 2, 32, 44)])
def test_attr_mlp_bwd_tensor_cores(n, B, hidden, seed):
    """gsparc_attr_mlp_bwd_tc against gsparc_attr_mlp_bwd and against the FP64 oracle's
    vector-Jacobian product of the attribute network, for a random upstream gradient (777
    rows leave a ragged last tile).  A ReLU whose pre-activation lies within the rounding of
    the split-BF16 products of zero can switch the other way than in FP32 or FP64, which
    changes that Gaussian's gradient outright: such rows (per-row relative error > 1e-3
    against either reference) may be at most 0.1% of the rows; their upstream gradient is
    then zeroed and every output compared: per-Gaussian gradients relative L2 <= 1e-4 against
    the FP32 kernel and <= 1e-3 against the oracle, weight and bias gradients <= 1e-3."""
    sc = synth.make_scene(n, seed=seed)
    mlp = synth.make_mlp(hidden, seed=seed + 1)
    tx = synth.make_tx(B, seed=seed + 2)
    r = Renderer(90, 360, 1, n, device=DEV)
    ds = DeviceScene.from_host(sc, DEV)
    dm = DeviceMLP.from_host(mlp, DEV)
    txd = torch.tensor(tx, device=DEV)
    d_attr_np = np.random.default_rng(seed + 3).normal(size=(B, n, 4)).astype(np.float32)
    fp, tc = (_mlp_grads_gpu(r, ds, dm, txd, d_attr_np, t) for t in (False, True))
    ref = _mlp_grads_oracle(sc, mlp, tx, d_attr_np)
    flipped = np.zeros(n, bool)
    for c in range(3):
        flipped |= (_row_err(tc[c], fp[c]) > 1e-3) | (_row_err(tc[c], ref[c]) > 1e-3)
    assert flipped.mean() <= 1e-3, "%d of %d rows differ" % (flipped.sum(), n)
    # every excluded row must really sit at a ReLU kink: some hidden pre-activation (of some
    # transmitter) within the split-BF16 rounding bound of zero
    margin = _relu_margin(sc, mlp, tx)
    for i in np.flatnonzero(flipped):
        assert margin[i] <= 0.0, "row %d excluded but its nearest kink is %.3e beyond the bound" % (i, margin[i])
    d_attr_np[:, flipped] = 0.0
    fp, tc = (_mlp_grads_gpu(r, ds, dm, txd, d_attr_np, t) for t in (False, True))
    ref = _mlp_grads_oracle(sc, mlp, tx, d_attr_np)
    names = ["means", "opacity_logit", "latent", "W1", "b1", "W2", "b2", "W3", "b3"]
    for c, k in enumerate(names):
        assert np.all(np.isfinite(tc[c])), k
        e_fp, e_or = rel_l2(tc[c], fp[c]), rel_l2(tc[c], ref[c])
        assert e_fp <= (1e-4 if c < 3 else 1e-3), "%s: relative L2 vs FP32 kernel %.3e" % (k, e_fp)
        assert e_or <= 1e-3, "%s: relative L2 vs oracle %.3e" % (k, e_or)


def _fp32_kink_margin(sc, mlp, tx):
    """Per Gaussian, min over transmitters and hidden units of |u| - bound(u), u the FP64
    pre-activation and bound(u) = 1e-5 (1 + sum |terms|), layer 2 also carrying layer 1's bound
    through |W2| (FP32 rounding of a sum of at most 65 terms is below 65 * 2^-24 ~ 4e-6 of its
    sum of magnitudes): FP32 sums of the same terms in any order (the forward's per-row dot
    products, the backward's tile products) and the exact sum take the same ReLU decision where
    it is > 0."""
    f64 = lambda a: torch.tensor(np.asarray(a), dtype=torch.float64)
    means, latent = f64(sc.means), f64(sc.latent)
    W1, b1, W2, b2 = (f64(a) for a in mlp.arrays()[:4])
    out = torch.full((sc.n,), float("inf"), dtype=torch.float64)
    for t in np.asarray(tx, dtype=np.float64):
        d = torch.clamp(torch.linalg.norm(means - f64(t), dim=1), min=0.01)
        h0 = torch.cat([f64(t).reshape(1, 3).expand(sc.n, 3), latent, torch.log(d).reshape(-1, 1)], 1)
        u1 = h0 @ W1 + b1
        h1 = torch.relu(u1)
        u2 = h1 @ W2 + b2
        bnd1 = 1e-5 * (1 + h0.abs() @ W1.abs() + b1.abs())
        bnd2 = 1e-5 * (1 + h1.abs() @ W2.abs() + b2.abs()) + bnd1 @ W2.abs()
        m1 = (u1.abs() - bnd1).min(1).values
        m2 = (u2.abs() - bnd2).min(1).values
        out = torch.minimum(out, torch.minimum(m1, m2))
    return out.numpy()


@pytest.mark.parametrize("n,B,hidden,seed", [(3000, 1, 32, 41), (777, 2, 32, 44), (1001, 3, 16, 42),
                                            (513, 1, 64, 45), (999, 1, 8, 46)])
def test_attr_mlp_bwd_stored_activations(n, B, hidden, seed):
    """gsparc_attr_mlp_bwd reading the activations the FP32 forward stored (the buffer NaN
    beforehand, so its unwritten padding columns must stay out of every sum) against the same call
    recomputing them and against the FP64 oracle.  The forward's attributes are unchanged by
    storing, bit for bit; every stored entry is finite.  The stored activations are the forward's
    own sums, the recomputed ones the backward's tile products (and FP64's sums are exact), so a
    ReLU decision can differ only at a pre-activation within FP32 rounding of zero: rows differing
    by more than 1e-4 from the recomputing call or 1e-3 from the oracle must have such a kink and
    are left out (their upstream gradient zeroed); the rest agree to 1e-5 relative L2
    (per-Gaussian gradients) and 1e-4 (weight gradients), and everything is within 1e-3 of the
    oracle."""
    sc = synth.make_scene(n, seed=seed)
    mlp = synth.make_mlp(hidden, seed=seed + 1)
    tx = synth.make_tx(B, seed=seed + 2)
    r = Renderer(90, 360, 1, n, device=DEV)
    ds = DeviceScene.from_host(sc, DEV)
    dm = DeviceMLP.from_host(mlp, DEV)
    txd = torch.tensor(tx, device=DEV)
    ld = G.hidden_ld(B * n)
    hid = torch.full((2 * hidden * ld,), float("nan"), device=DEV)
    a0 = r.attributes(ds, dm, txd)
    a1 = r.attributes(ds, dm, txd, hidden=hid)
    torch.cuda.synchronize()
    assert torch.equal(a0, a1)
    h = hid.view(2 * hidden, ld)
    assert torch.isfinite(h[:, :B * n]).all() and (h[:, :B * n] >= 0).all()
    d_attr_np = np.random.default_rng(seed + 3).normal(size=(B, n, 4)).astype(np.float32)
    rec = _mlp_grads_gpu(r, ds, dm, txd, d_attr_np, False)
    kept = _mlp_grads_gpu(r, ds, dm, txd, d_attr_np, False, hidden=hid)
    ref = _mlp_grads_oracle(sc, mlp, tx, d_attr_np)
    differ = np.zeros(n, bool)
    for c in range(3):
        differ |= (_row_err(kept[c], rec[c]) > 1e-4) | (_row_err(kept[c], ref[c]) > 1e-3)
    margin = _fp32_kink_margin(sc, mlp, tx)
    assert np.all(margin[differ] <= 0.0), np.flatnonzero(differ & (margin > 0))
    if differ.any():
        d_attr_np[:, differ] = 0.0
        rec = _mlp_grads_gpu(r, ds, dm, txd, d_attr_np, False)
        kept = _mlp_grads_gpu(r, ds, dm, txd, d_attr_np, False, hidden=hid)
        ref = _mlp_grads_oracle(sc, mlp, tx, d_attr_np)
    for k, (a, b, c) in enumerate(zip(kept, rec, ref)):
        bound = 1e-5 if k < 3 else 1e-4
        assert np.linalg.norm(a - b) <= bound * np.linalg.norm(b), k
        assert np.linalg.norm(a - c) <= 1e-3 * np.linalg.norm(c), k


@pytest.mark.parametrize("tc", [False, True])
def test_attr_mlp_bwd_weight_gradients_unaligned(tc):
    """The network backward adds each thread block's weight and bias gradients by bulk reductions
    when the gradient arrays are 16-byte aligned and by one atomic per entry otherwise: the same
    weight, bias and per-Gaussian gradients either way (views of a buffer at a 4-byte offset
    against separate tensors; relative L2 <= 1e-5, the additions only reordered)."""
    n, B, hidden, seed = 3000, 2, 32, 61
    sc = synth.make_scene(n, seed=seed)
    mlp = synth.make_mlp(hidden, seed=seed + 1)
    tx = synth.make_tx(B, seed=seed + 2)
    r = Renderer(90, 360, 1, n, device=DEV)
    ds = DeviceScene.from_host(sc, DEV)
    dm = DeviceMLP.from_host(mlp, DEV)
    txd = torch.tensor(tx, device=DEV)
    d_attr = torch.tensor(np.random.default_rng(seed + 3).normal(size=(B, n, 4)).astype(np.float32), device=DEV)

    def grads(unaligned):
        shapes = [t.shape for t in dm.tensors()]
        sizes = [int(np.prod(sh)) for sh in shapes]
        if unaligned:
            flat = torch.zeros(sum(sizes) + 1, device=DEV)
            offs = np.cumsum([1] + sizes)
            gw = [flat[int(o):int(o) + z].view(sh) for o, z, sh in zip(offs[:-1], sizes, shapes)]
            assert all(t.data_ptr() % 16 != 0 for t in gw[:4])
        else:
            gw = [torch.zeros(sh, device=DEV) for sh in shapes]
        gm = torch.zeros((n, 3), device=DEV)
        go = torch.zeros(n, device=DEV)
        gl = torch.zeros((n, 16), device=DEV)
        r.attributes_backward(ds, dm, txd, d_attr, gm, go, gl, gw, tensor_cores=tc)
        torch.cuda.synchronize()
        return [t.cpu().numpy().astype(np.float64) for t in [gm, go, gl] + gw]

    a, u = grads(False), grads(True)
    for c, k in enumerate(["means", "opacity_logit", "latent", "W1", "b1", "W2", "b2", "W3", "b3"]):
        assert np.all(np.isfinite(u[c])), k
        assert rel_l2(u[c], a[c]) <= 1e-5, "%s: %.3e" % (k, rel_l2(u[c], a[c]))
