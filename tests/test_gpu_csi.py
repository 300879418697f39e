"""CSI head (Eq. 2), channel loss (Eq. 3) and their gradient on the GPU against the FP64
oracle (the CPU tests pin the oracle's head, loss and chained gradient)."""
import numpy as np
import pytest
import torch

from gpu_util import DEV, oracle_geo_attr, oracle_render, rel_l2, spectrum_to_complex
from oracle import csi as ocsi
from oracle import pipeline as opl
from paper_2511_22793_gb300 import gsparc as G
from paper_2511_22793_gb300 import synth
from paper_2511_22793_gb300.pipeline import DeviceMLP, DeviceScene, Renderer

pytestmark = pytest.mark.gpu


def _setup(n, H, W, K, B, seed, hidden=32):
    sc = synth.make_scene(n, seed=seed)
    mlp = synth.make_mlp(hidden, seed=3)
    tx = synth.make_tx(B, seed=seed + 1)
    r = Renderer(H, W, K, n, device=DEV)
    ds = DeviceScene.from_host(sc, DEV)
    dm = DeviceMLP.from_host(mlp, DEV)
    r.geometry(ds)
    attr = r.attributes(ds, dm, torch.tensor(tx, device=DEV))
    return sc, mlp, tx, r, ds, dm, attr


def _c(t):
    a = t.cpu().numpy().astype(np.float64)
    return a[..., 0] + 1j * a[..., 1]


@pytest.mark.parametrize("n,H,W,K,B,seed", [(2000, 90, 360, 16, 2, 71), (3000, 45, 180, 1, 1, 72),
                                             (1500, 90, 360, 37, 1, 73), (2500, 180, 720, 64, 1, 74)])
def test_csi_head_and_fused_forward_match_oracle(n, H, W, K, B, seed):
    """gsparc_csi_head of the FP32 spectrum, and gsparc_render_csi_tc with and without the
    spectrum, against the oracle's spatial mean (relative L2 <= 2e-4 over the B x K
    estimates); the fused call's spectrum and per-pixel state are bit-identical to
    gsparc_render_fwd_tc's and its estimate agrees with the head of that spectrum to 1e-5."""
    sc, mlp, tx, r, ds, dm, attr = _setup(n, H, W, K, B, seed)
    view, band = synth.View(H=H, W=W), synth.Band(K=K)
    g, attrs = oracle_geo_attr(sc, mlp, view, tx)
    zo, _, _ = oracle_render(g, attrs, view, band)
    h_ref = ocsi.csi_head(zo, H, W)
    csi = torch.empty((B, K, 2), device=DEV)
    spec, logT, nc = r.render(attr)
    G.gsparc_csi_head(spec, csi, 1.0 / (H * W))
    torch.cuda.synchronize()
    assert rel_l2(_c(csi), h_ref) <= 2e-4
    spec_tc, logT_tc, nc_tc = r.render(attr, tensor_cores=True)
    G.gsparc_csi_head(spec_tc, csi, 1.0 / (H * W))
    h_tc_head = _c(csi)
    fused_out = r.alloc_outputs(B)
    h_fused = _c(r.render_csi(attr, out=fused_out))
    h_nospec = _c(r.render_csi(attr))
    torch.cuda.synchronize()
    assert r.check() == 0
    assert torch.equal(fused_out[0], spec_tc)
    assert torch.equal(fused_out[1], logT_tc) and torch.equal(fused_out[2], nc_tc)
    for h in (h_fused, h_nospec):
        assert rel_l2(h, h_tc_head) <= 1e-5
        assert rel_l2(h, h_ref) <= 2e-4


def test_csi_loss_and_head_gradient():
    rng = np.random.default_rng(75)
    B, K, H, W = 3, 7, 9, 20
    h = rng.normal(size=(B, K)) + 1j * rng.normal(size=(B, K))
    t = rng.normal(size=(B, K)) + 1j * rng.normal(size=(B, K))
    to = lambda z: torch.tensor(np.stack([z.real, z.imag], -1), dtype=torch.float32, device=DEV)
    loss = torch.zeros(1, device=DEV)
    d = torch.empty((B, K, 2), device=DEV)
    G.gsparc_csi_loss(to(h), to(t), loss, d)
    d_spec = torch.empty((B, K, H, W, 2), device=DEV)
    G.gsparc_csi_head_bwd(d, d_spec, 1.0 / (H * W))
    torch.cuda.synchronize()
    ref_loss, ref_d = ocsi.channel_loss(h.astype(np.complex64).astype(np.complex128),
                                        t.astype(np.complex64).astype(np.complex128))
    assert float(loss) == pytest.approx(ref_loss, rel=1e-5)
    assert rel_l2(_c(d), ref_d) <= 1e-6
    ref_spec = ocsi.csi_head_bwd(_c(d), H, W)                       # [B, H*W, K]
    got = _c(d_spec).reshape(B, K, H * W).transpose(0, 2, 1)
    assert np.array_equal(got, ref_spec.astype(np.complex64).astype(np.complex128)) or \
        rel_l2(got, ref_spec) <= 1e-7


@pytest.mark.parametrize("n,H,W,K,B", [(600, 45, 180, 8, 2), (2000, 90, 360, 16, 1)])
def test_channel_loss_gradient_chain_matches_oracle(n, H, W, K, B):
    """Channel loss of the fused estimate through the whole backward (head gradient, the
    tensor-core compositing backward, attribute network, projection) against the oracle's
    FP64 gradient (pinned to central differences): relative L2 <= 5e-3 per parameter
    tensor, as the spectrum-loss gradient test."""
    seed = 76
    sc, mlp, tx, r, ds, dm, attr = _setup(n, H, W, K, B, seed)
    if n == 600:
        sc.log_scales = sc.log_scales + np.float32(0.4)
        ds = DeviceScene.from_host(sc, DEV)
        r.geometry(ds)
        attr = r.attributes(ds, dm, torch.tensor(tx, device=DEV))
    rng = np.random.default_rng(seed + 5)
    target = 1e-3 * (rng.normal(size=(B, K)) + 1j * rng.normal(size=(B, K)))
    tgt = torch.tensor(np.stack([target.real, target.imag], -1), dtype=torch.float32, device=DEV)
    out = r.alloc_outputs(B)
    csi = r.render_csi(attr, out=out)
    loss = torch.zeros(1, device=DEV)
    d_csi = torch.empty_like(csi)
    G.gsparc_csi_loss(csi, tgt, loss, d_csi)
    d_spec = torch.empty_like(out[0])
    G.gsparc_csi_head_bwd(d_csi, d_spec, 1.0 / (H * W))
    d_attr = torch.zeros_like(attr)
    d_proj = torch.zeros_like(r.proj)
    r.render_backward(attr, out[1], out[2], d_spec, d_attr, d_proj, tensor_cores=True)
    gm = torch.zeros_like(ds.means)
    gls = torch.zeros_like(ds.log_scales)
    gq = torch.zeros_like(ds.quats)
    go = torch.zeros_like(ds.opacity_logit)
    gl = torch.zeros_like(ds.latent)
    gw = [torch.zeros_like(t) for t in dm.tensors()]
    r.attributes_backward(ds, dm, torch.tensor(tx, device=DEV), d_attr, gm, go, gl, gw)
    r.project_backward(ds, d_proj, gm, gls, gq)
    torch.cuda.synchronize()
    assert r.check() == 0
    ref_loss, ref = opl.loss_and_grad(sc, mlp, synth.View(H=H, W=W), synth.Band(K=K), tx, target,
                                      loss_kind="csi")
    assert abs(float(loss) - ref_loss) <= 1e-3 * ref_loss
    assert rel_l2(_c(csi), ref["h"]) <= 2e-4
    got = dict(means=gm, log_scales=gls, quats=gq, opacity_logit=go, latent=gl,
               **dict(zip(["W1", "b1", "W2", "b2", "W3", "b3"], gw)))
    for k, v in got.items():
        e = rel_l2(v.cpu().numpy().astype(np.float64), ref[k])
        assert e <= 5e-3, "%s: relative L2 %.3e" % (k, e)
