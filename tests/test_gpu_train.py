"""GPU loss and Adam kernels against the oracle."""
import numpy as np
import pytest
import torch

from gpu_util import DEV
from oracle import adam as oadam
from paper_2511_22793_gb300 import gsparc as G
from paper_2511_22793_gb300 import synth
from paper_2511_22793_gb300.pipeline import DeviceMLP, DeviceScene, Renderer

pytestmark = pytest.mark.gpu


def test_l2_loss_and_gradient():
    rng = np.random.default_rng(41)
    z = rng.normal(size=(3, 5, 7, 11, 2)).astype(np.float32)
    t = rng.normal(size=(3, 5, 7, 11, 2)).astype(np.float32)
    zd, td = torch.tensor(z, device=DEV), torch.tensor(t, device=DEV)
    loss = torch.zeros(1, device=DEV)
    dz = torch.empty_like(zd)
    G.gsparc_l2_loss(zd, td, loss, dz)
    torch.cuda.synchronize()
    d = z.astype(np.float64) - t
    M = d.size // 2
    np.testing.assert_allclose(loss.item(), np.sum(d * d) / M, rtol=1e-5)
    np.testing.assert_allclose(dz.cpu().numpy(), 2 * d / M, rtol=1e-5, atol=1e-9)


def test_adam_matches_oracle():
    rng = np.random.default_rng(42)
    n = 10_001
    p = rng.normal(size=n).astype(np.float32)
    pd = torch.tensor(p, device=DEV)
    m = torch.zeros_like(pd)
    v = torch.zeros_like(pd)
    q, mm, vv = p.astype(np.float64), np.zeros(n), np.zeros(n)
    for step in range(1, 6):
        g = rng.normal(size=n).astype(np.float32)
        G.gsparc_adam(pd, torch.tensor(g, device=DEV), m, v, 5e-3, step, eps=1e-15)
        q, mm, vv = oadam.adam_step(q, g, mm, vv, step, 5e-3, eps=1e-15)
    torch.cuda.synchronize()
    np.testing.assert_allclose(pd.cpu().numpy(), q, rtol=1e-5, atol=1e-6)


def _s_tot_buffer(r, B, form):
    strips = G.s_tot_strips(r.K) if form == "tc" else G.fp32_strips(r.K)
    return torch.empty((B, strips, r.H, r.W), dtype=torch.float32, device=DEV)


@pytest.mark.parametrize("form", ["tc", "fp32"])
@pytest.mark.parametrize("n,H,W,K,B", [(3000, 90, 360, 64, 1), (2000, 45, 180, 37, 2)])
def test_fused_l2_loss_forward_matches_unfused(n, H, W, K, B, form):
    """gsparc_render_fwd_l2_tc / gsparc_render_fwd_l2: the gradient is bit-identical to
    gsparc_l2_loss on the spectrum of gsparc_render_fwd_tc / gsparc_render_fwd, the loss agrees
    to 1e-5 relative (summation order), the state buffers are identical, s_tot is the strip sum
    of Re(conj(dL/dz) z), and without a spectrum buffer nothing else changes."""
    tc = form == "tc"
    sc = synth.make_scene(n, seed=91)
    mlp = synth.make_mlp(32, seed=92)
    tx = synth.make_tx(B, seed=93)
    r = Renderer(H, W, K, n, device=DEV)
    ds, dm = DeviceScene.from_host(sc, DEV), DeviceMLP.from_host(mlp, DEV)
    r.geometry(ds)
    attr = r.attributes(ds, dm, torch.tensor(tx, device=DEV))
    spec, logT, nc = r.render(attr, tensor_cores=tc)
    target = torch.randn_like(spec) * 0.01
    loss = torch.zeros(1, device=DEV)
    d_ref = torch.empty_like(spec)
    G.gsparc_l2_loss(spec, target, loss, d_ref)
    # s_tot[b, s, p] = sum over the strip's subcarriers of Re(conj(dL/dz) z)
    z64, g64 = spec.double(), d_ref.double()
    prod = (z64 * g64).sum(-1)                                     # [B, K, H, W]
    mag = (z64.abs() * g64.abs()).sum(-1)
    nst = G.s_tot_strips(K) if tc else G.fp32_strips(K)
    width = (K if K <= 64 else 64) if tc else (K if K <= 32 else 32)
    want = torch.stack([prod[:, s * width:(s + 1) * width].sum(1) for s in range(nst)], 1)
    scale = torch.stack([mag[:, s * width:(s + 1) * width].sum(1) for s in range(nst)], 1)
    for with_spec in (True, False):
        out = r.alloc_outputs(B)
        loss2 = torch.full((1,), 7.0, device=DEV)
        d2 = torch.empty_like(spec)
        s_tot = _s_tot_buffer(r, B, form)
        fn = G.gsparc_render_fwd_l2_tc if tc else G.gsparc_render_fwd_l2
        fn(r.view, r.band, B, n, r.proj, r.tile_ranges, r.sorted_ids, attr, target, loss2, d2,
           out[0] if with_spec else None, out[1], out[2], s_tot=s_tot)
        torch.cuda.synchronize()
        assert torch.equal(d2, d_ref)
        # the blocks' partial sums are added atomically in FP32, in no fixed order
        assert abs(float(loss2) - float(loss)) <= 1e-5 * float(loss)
        assert torch.equal(out[1], logT) and torch.equal(out[2], nc)
        if with_spec:
            assert torch.equal(out[0], spec)
        assert float(((s_tot.double() - want).abs() - 1e-5 * scale).max()) <= 0.0


@pytest.mark.parametrize("form", ["tc", "fp32"])
@pytest.mark.parametrize("n,H,W,K,B,split_min", [(50_000, 90, 360, 64, 1, 0), (3000, 45, 180, 100, 2, 1),
                                                   (4000, 90, 360, 16, 1, 2)])
def test_scheduled_backward_training_path(n, H, W, K, B, split_min, form):
    """The training step's backward: fused-loss forward writing s_tot, then the scheduled
    backward (gsparc_render_bwd_tc_balanced / gsparc_render_bwd_balanced: long walks split,
    front chunks fed by s_tot) against the unscheduled call of the same form
    (gsparc_render_bwd_tc / gsparc_render_bwd) on the same inputs (relative L2 <= 1e-4 per
    gradient component).  The first case is the 50k-Gaussian, 64-subcarrier, 360x90 training
    workload with the default split rule; the schedule splits some walks there (checked on the
    host from n_contrib)."""
    tc = form == "tc"
    sc = synth.make_scene(n, seed=95)
    mlp = synth.make_mlp(32, seed=96)
    tx = synth.make_tx(B, seed=97)
    r = Renderer(H, W, K, n, device=DEV)
    ds, dm = DeviceScene.from_host(sc, DEV), DeviceMLP.from_host(mlp, DEV)
    r.geometry(ds)
    attr = r.attributes(ds, dm, torch.tensor(tx, device=DEV), G.GSPARC_BF16X2 if tc else G.GSPARC_FP32)
    _, logT, nc = r.alloc_outputs(B)
    target = torch.randn((B, K, H, W, 2), device=DEV) * 0.01
    loss = torch.zeros(1, device=DEV)
    d_spec = torch.empty_like(target)
    s_tot, tile_walk = _s_tot_buffer(r, B, form), r.walk_buffer(B)
    fwd = G.gsparc_render_fwd_l2_tc if tc else G.gsparc_render_fwd_l2
    fwd(r.view, r.band, B, n, r.proj, r.tile_ranges, r.sorted_ids, attr, target, loss, d_spec, None, logT, nc,
        s_tot=s_tot, tile_walk=tile_walk)
    res = []
    for kind in ("plain", "balanced", "balanced_walks"):
        d_attr = torch.zeros_like(attr)
        d_proj = torch.zeros_like(r.proj)
        if kind == "plain":
            bwd = G.gsparc_render_bwd_tc if tc else G.gsparc_render_bwd
            bwd(r.view, r.band, B, n, r.proj, r.tile_ranges, r.sorted_ids, attr, logT, nc, d_spec, d_attr, d_proj)
        else:
            r.render_backward(attr, logT, nc, d_spec, d_attr, d_proj, tensor_cores=tc, s_tot=s_tot,
                              split_min=split_min, tile_walk=tile_walk if kind == "balanced_walks" else None)
        torch.cuda.synchronize()
        res.append((d_attr.cpu().numpy().astype(np.float64), d_proj.cpu().numpy().astype(np.float64)))
    assert r.check() == 0
    ua, up = res[0]
    for ba, bp in res[1:]:
        for j in range(4):
            e = np.linalg.norm(ba[..., j] - ua[..., j]) / np.linalg.norm(ua[..., j])
            assert e <= 1e-4, ("attr", j, e)
        for j in (0, 1, 4, 5, 6):
            e = np.linalg.norm(bp[:, j] - up[:, j]) / np.linalg.norm(up[:, j])
            assert e <= 1e-4, ("proj", j, e)
    # the forward's tile walks: min(largest n_contrib of the tile's pixels, list length), bit-exact
    TH, TW = (H + 15) // 16, (W + 15) // 16
    pad = np.zeros((B, TH * 16, TW * 16), np.int64)
    pad[:, :H, :W] = nc.cpu().numpy()
    walks = pad.reshape(B, TH, 16, TW, 16).max(axis=(2, 4)).reshape(B, -1)
    rng_ = r.tile_ranges.cpu().numpy().astype(np.int64)
    want = np.minimum(walks, (rng_[:, 1] - rng_[:, 0])[None, :])
    assert np.array_equal(tile_walk.cpu().numpy().astype(np.int64), want)
    # the schedule had walks to split: some tile's walk spans more than split_min batches
    smin = 3 if split_min == 0 else split_min
    assert int(((want + 15) // 16 > smin).sum()) > 0


def test_packed_inputs_upload_and_alignment():
    """PackedInputs: every view starts 256-byte aligned inside one allocation, holds its array
    after one upload, and writing one view leaves the others unchanged."""
    from paper_2511_22793_gb300.pipeline import PackedInputs
    rng = np.random.default_rng(7)
    arrays = [rng.normal(size=sh).astype(np.float32) for sh in [(1001, 3), (7,), (5, 16), (1,), (2, 3, 4, 5, 2)]]
    p = PackedInputs([a.shape for a in arrays], DEV)
    for i, a in enumerate(arrays):
        p.set_host(i, a)
    p.upload()
    torch.cuda.synchronize()
    base = p.flat.data_ptr()
    for v, a in zip(p.views, arrays):
        assert (v.data_ptr() - base) % 256 == 0
        assert v.data_ptr() + v.numel() * 4 <= base + p.nbytes
        assert torch.equal(v.cpu(), torch.from_numpy(a))
    p.views[2].fill_(3.0)
    torch.cuda.synchronize()
    for i, (v, a) in enumerate(zip(p.views, arrays)):
        if i != 2:
            assert torch.equal(v.cpu(), torch.from_numpy(a))
