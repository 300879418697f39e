"""GPU parity of the whole forward path (project -> bin/sort -> attribute
network -> compositing) against the FP64 per-pixel oracle.

Tolerance: <= 1e-3 relative L2 per spectrum (one transmitter, all subcarriers
and pixels) against the FP64 oracle, the bound stated for the FP32 path.
"""
import numpy as np
import pytest
import torch

from gpu_util import (DEV, gpu_forward, oracle_geo_attr, oracle_render, rel_l2,
                      spectrum_to_complex)
from paper_2511_22793_gb300 import gsparc as G
from paper_2511_22793_gb300 import synth

pytestmark = pytest.mark.gpu
TOL = 1e-3


def _check(n, H, W, K, B, hidden, seed, pixels=None, widen=0.0):
    sc = synth.make_scene(n, seed=seed)
    if widen:
        sc.log_scales = sc.log_scales + np.float32(widen)
    mlp = synth.make_mlp(hidden, seed=3)
    tx = synth.make_tx(B, seed=2 + seed)
    r, ds, dm, txd, attr, spec, logT, nc = gpu_forward(sc, mlp, H, W, K, tx)
    view, band = synth.View(H=H, W=W), synth.Band(K=K)
    g, attrs = oracle_geo_attr(sc, mlp, view, tx)
    zref, Tref, nref = oracle_render(g, attrs, view, band, pixels=pixels)
    z = spectrum_to_complex(spec)
    T = np.exp2(logT.cpu().numpy().astype(np.float64)).reshape(B, H * W)
    if pixels is not None:
        z = z[:, pixels]
        T = T[:, pixels]
    for b in range(B):
        e = rel_l2(z[b], zref[b])
        assert e <= TOL, "tx %d: spectrum relative L2 %.3e" % (b, e)
        assert np.abs(zref[b]).max() > 0
    # transmittance agrees except where a cut-off decision flipped
    close = np.isclose(T, Tref, rtol=1e-3, atol=1e-6)
    assert close.mean() > 0.995
    return z, zref


def test_render_c1_single_query_fp32():
    """1,024 Gaussians, 1 subcarrier, 360x90, hidden 32 (the single-query workload)."""
    _check(1024, 90, 360, 1, 1, 32, seed=0)


@pytest.mark.parametrize("K", [64, 37, 5, 2])
def test_render_subcarrier_strips(K):
    """Strip widths and ragged strip tails (K not a multiple of the strip)."""
    _check(2000, 90, 360, K, 2, 32, seed=1)


def test_render_720x180_multi_tx():
    _check(3000, 180, 720, 3, 3, 64, seed=2)


def test_render_180x45_ragged_rows():
    _check(1500, 45, 180, 16, 2, 16, seed=3, widen=0.3)


def test_render_full_size_sampled_pixels():
    """50,000 Gaussians, 64 subcarriers, 360x90, in the benchmark's launch
    configuration; the oracle evaluates 512 seeded pixels one by one."""
    rng = np.random.default_rng(99)
    pix = np.sort(rng.choice(90 * 360, size=512, replace=False)).astype(np.int32)
    _check(50_000, 90, 360, 64, 1, 32, seed=0, pixels=pix)


@pytest.mark.parametrize("precision,tol", [(G.GSPARC_BF16X2, TOL), (G.GSPARC_BF16, 1e-2)])
def test_render_batched_tensor_core_network_full_size_sampled(precision, tol):
    """The batched inference form at full size: 200,000 Gaussians, 256 subcarriers,
    720x180, hidden 64, BF16-representable weights and latents, the network on the
    tensor cores and FP32 compositing; 4 transmitters in one launch, 256 seeded
    pixels per spectrum evaluated by the oracle.  BF16X2 must meet the 1e-3 bound;
    the single-term BF16 network is reported against a looser 1e-2 bound."""
    n, H, W, K, B = 200_000, 180, 720, 256, 4
    sc = synth.make_scene(n, seed=0, bf16_latent=True)
    mlp = synth.make_mlp(64, seed=3, bf16_weights=True)
    tx = synth.make_tx(B, seed=2)
    _, _, _, _, _, spec, _, _ = gpu_forward(sc, mlp, H, W, K, tx, precision=precision)
    rng = np.random.default_rng(5)
    pix = np.sort(rng.choice(H * W, size=256, replace=False)).astype(np.int32)
    view, band = synth.View(H=H, W=W), synth.Band(K=K)
    g, attrs = oracle_geo_attr(sc, mlp, view, tx)
    zref, _, _ = oracle_render(g, attrs, view, band, pixels=pix)
    z = spectrum_to_complex(spec)[:, pix]
    errs = [rel_l2(z[b], zref[b]) for b in range(B)]
    print("per-spectrum relative L2 (precision %d):" % precision, ["%.2e" % e for e in errs])
    assert max(errs) <= tol


def test_render_empty_and_all_culled():
    sc = synth.make_scene(64, seed=5)
    sc.means[:] = 0.0                          # every Gaussian inside the near distance
    mlp = synth.make_mlp(8)
    _, _, _, _, _, spec, logT, nc = gpu_forward(sc, mlp, 45, 180, 3, synth.make_tx(1))
    assert float(spec.abs().max()) == 0.0 and float(logT.abs().max()) == 0.0
    assert int(nc.max()) == 0
    sc0 = synth.make_scene(0, seed=5)
    _, _, _, _, _, spec0, _, _ = gpu_forward(sc0, mlp, 45, 180, 3, synth.make_tx(1))
    assert float(spec0.abs().max()) == 0.0


def test_render_deterministic():
    sc = synth.make_scene(4000, seed=6)
    mlp = synth.make_mlp(32)
    tx = synth.make_tx(1)
    a = gpu_forward(sc, mlp, 90, 360, 8, tx)[5].cpu()
    b = gpu_forward(sc, mlp, 90, 360, 8, tx)[5].cpu()
    assert torch.equal(a, b)


@pytest.mark.parametrize("n,H,W,K,B,hidden,seed", [(1024, 90, 360, 1, 1, 32, 0), (2000, 90, 360, 64, 2, 32, 1),
                                                   (2000, 90, 360, 37, 2, 32, 1), (1500, 45, 180, 16, 2, 16, 3),
                                                   (3000, 180, 720, 100, 2, 64, 2)])
def test_render_fwd_tensor_cores_matches_oracle_and_fp32_kernel(n, H, W, K, B, hidden, seed):
    """gsparc_render_fwd_tc: same per-pixel decisions as gsparc_render_fwd (bit-identical
    final log2 T, contributor position and count), spectra within 1e-3 of the FP64
    oracle and within 1e-4 of the FP32 kernel."""
    sc = synth.make_scene(n, seed=seed)
    if H == 45:
        sc.log_scales = sc.log_scales + np.float32(0.3)
    mlp = synth.make_mlp(hidden, seed=3)
    tx = synth.make_tx(B, seed=2 + seed)
    r, ds, dm, txd, attr, spec, logT, nc = gpu_forward(sc, mlp, H, W, K, tx)
    nu = torch.empty_like(nc)
    spec_tc, logT_tc, nc_tc = r.render(attr, n_used=nu, tensor_cores=True)
    nu_ref = torch.empty_like(nc)
    r.render(attr, n_used=nu_ref)
    torch.cuda.synchronize()
    assert torch.equal(logT_tc, logT) and torch.equal(nc_tc, nc) and torch.equal(nu, nu_ref)
    a = spectrum_to_complex(spec_tc)
    f = spectrum_to_complex(spec)
    view, band = synth.View(H=H, W=W), synth.Band(K=K)
    g, attrs = oracle_geo_attr(sc, mlp, view, tx)
    zref, _, _ = oracle_render(g, attrs, view, band)
    for b in range(B):
        assert rel_l2(a[b], f[b]) <= 1e-4
        assert rel_l2(a[b], zref[b]) <= TOL


def test_render_fwd_tensor_cores_full_size_sampled():
    """50,000 Gaussians, 64 subcarriers, 360x90 (the benchmark workload), 512 sampled pixels."""
    rng = np.random.default_rng(99)
    pix = np.sort(rng.choice(90 * 360, size=512, replace=False)).astype(np.int32)
    sc = synth.make_scene(50_000, seed=0)
    mlp = synth.make_mlp(32, seed=3)
    tx = synth.make_tx(1, seed=2)
    r, ds, dm, txd, attr, spec, logT, nc = gpu_forward(sc, mlp, 90, 360, 64, tx)
    spec_tc, _, _ = r.render(attr, tensor_cores=True)
    view, band = synth.View(H=90, W=360), synth.Band(K=64)
    g, attrs = oracle_geo_attr(sc, mlp, view, tx)
    zref, _, _ = oracle_render(g, attrs, view, band, pixels=pix)
    z = spectrum_to_complex(spec_tc)[:, pix]
    assert rel_l2(z[0], zref[0]) <= TOL
