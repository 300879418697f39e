"""GPU parity of the per-Gaussian stages against the FP64 oracle:
projection (FP32 vs FP64 within a derived tolerance), binning and sorting
(bit-exact on shared FP32 records), the attribute network."""
import numpy as np
import pytest
import torch

from gpu_util import DEV, oracle_geo_attr
from oracle import binsort as obs
from paper_2511_22793_gb300 import gsparc as G
from paper_2511_22793_gb300 import synth
from paper_2511_22793_gb300.pipeline import DeviceMLP, DeviceScene, Renderer

pytestmark = pytest.mark.gpu


def _wrapdiff(a, b, W):
    d = a - b
    return d - W * np.round(d / W)


@pytest.mark.parametrize("n,H,W,seed", [(1024, 90, 360, 0), (50_000, 90, 360, 0), (3001, 180, 720, 9),
                                        (777, 45, 180, 4)])
def test_project_matches_oracle(n, H, W, seed):
    sc = synth.make_scene(n, seed=seed)
    view = synth.View(H=H, W=W)
    r = Renderer(H, W, 1, n, device=DEV)
    ds = DeviceScene.from_host(sc, DEV)
    G.gsparc_project(r.view, ds.means, ds.log_scales, ds.quats, r.proj)
    p = r.proj.cpu().numpy().astype(np.float64)
    g, _ = oracle_geo_attr(sc, synth.make_mlp(8), view, np.zeros((1, 3)))
    valid = g["valid"]
    assert np.array_equal(p[:, 3] >= 0, valid)
    v = valid
    # FP32 map: a few ulps of W (atan2/asin), i.e. ~1e-4 px at W = 720
    assert np.max(np.abs(_wrapdiff(p[v, 0], g["px"][v], W))) < 2e-4 * W / 360
    assert np.max(np.abs(p[v, 1] - g["py"][v])) < 2e-4 * H / 90
    # Sigma' has relative error ~1e-6 per entry; the conic and extents inherit it,
    # amplified by the condition number of Sigma' (bounded by the 0.3 px^2 dilation)
    for j, k in ((2, "ext_x"), (3, "ext_y"), (7, "r")):
        np.testing.assert_allclose(p[v, j], g[k][v], rtol=2e-5)
    scale = np.sqrt(g["cxx"][v] * g["cyy"][v])
    for j, k in ((4, "cxx"), (5, "cxy"), (6, "cyy")):
        assert np.max(np.abs(p[v, j] - g[k][v]) / scale) < 1e-4


def test_project_edge_cases():
    """Culled (inside near distance), zenith, seam and N = 0."""
    means = np.array([[0.0, 0.05, 0.0], [0.0, 3.0, 0.0], [1e-6, 3.0, 1e-6], [0.0, 1.0, -2.0],
                      [-1e-5, 1.0, -2.0]], dtype=np.float32)
    n = means.shape[0]
    sc = synth.Scene(means=means, log_scales=np.full((n, 3), -1.5, np.float32),
                     quats=np.tile(np.array([[1, 0, 0, 0]], np.float32), (n, 1)),
                     opacity_logit=np.zeros(n, np.float32), latent=np.zeros((n, 16), np.float32))
    r = Renderer(90, 360, 1, n, device=DEV)
    ds = DeviceScene.from_host(sc, DEV)
    G.gsparc_project(r.view, ds.means, ds.log_scales, ds.quats, r.proj)
    p = r.proj.cpu().numpy()
    assert p[0, 2] == -1 and p[0, 3] == -1
    assert np.all(np.isfinite(p[1:]))
    assert abs(p[1, 1] - 90.0) < 1e-3            # zenith row
    assert p[1, 2] >= 180.0                       # azimuth extent covers every column
    assert abs(p[3, 0] - 360.0) < 1e-3 or abs(p[3, 0]) < 1e-3    # on the +-pi seam
    r0 = Renderer(90, 360, 1, 0, device=DEV)
    e = torch.empty((0, 3), device=DEV)
    G.gsparc_project(r0.view, e, e, torch.empty((0, 4), device=DEV), r0.proj)


def _gpu_binsort(rec, H, W, capacity=None):
    n = rec.shape[0]
    cap = capacity if capacity is not None else max(16, 40 * n)
    r = Renderer(H, W, 1, n, pair_capacity=cap, device=DEV)
    r.proj.copy_(torch.tensor(rec, device=DEV))
    keys = torch.empty(max(1, cap), dtype=torch.int64, device=DEV)
    r.status.zero_()
    G.gsparc_bin_sort(r.view, n, r.proj, cap, r.ws, r.sorted_ids, keys, r.tile_ranges, r.n_pairs,
                      r.status)
    st = r.check()
    npairs = int(r.n_pairs.item()) & 0xFFFFFFFF
    m = min(npairs, cap)
    return (st, npairs, keys[:m].cpu().numpy().view(np.uint64), r.sorted_ids[:m].cpu().numpy().view(np.uint32),
            r.tile_ranges.cpu().numpy().view(np.uint32))


@pytest.mark.parametrize("n,H,W,seed", [(1, 90, 360, 1), (17, 90, 360, 2), (1000, 90, 360, 3),
                                        (20_011, 90, 360, 4), (5000, 180, 720, 5), (3000, 45, 180, 6),
                                        (50_000, 90, 360, 7)])
def test_bin_sort_bit_exact(n, H, W, seed):
    rec = synth.make_proj_records(n, H, W, seed=seed)
    st, npairs, keys, ids, ranges = _gpu_binsort(rec, H, W)
    assert st == 0
    ok, ov, orng = obs.bin_sort(rec, H, W)
    assert npairs == len(ov)
    assert np.array_equal(keys, ok)
    assert np.array_equal(ids, ov)
    assert np.array_equal(ranges, orng)


def test_bin_sort_many_passes_and_empty():
    # 720x180: 540 tiles, more than one tile-id byte in the sorted keys
    rec = synth.make_proj_records(4000, 180, 720, seed=11)
    st, npairs, keys, ids, ranges = _gpu_binsort(rec, 180, 720)
    ok, ov, orng = obs.bin_sort(rec, 180, 720)
    assert st == 0 and np.array_equal(ids, ov) and np.array_equal(ranges, orng)
    # every record culled: no pairs, empty ranges
    rec[:, 2:4] = -1
    st, npairs, keys, ids, ranges = _gpu_binsort(rec, 90, 360)
    assert st == 0 and npairs == 0 and not ranges.any()


def test_bin_sort_capacity_overflow_reported():
    rec = synth.make_proj_records(2000, 90, 360, seed=12)
    ok, ov, _ = obs.bin_sort(rec, 90, 360)
    cap = len(ov) // 2
    st, npairs, keys, ids, ranges = _gpu_binsort(rec, 90, 360, capacity=cap)
    assert st == G.GSPARC_ERR_CAPACITY
    assert npairs == len(ov)
    assert len(ids) == cap
    # tiles whose lists end at or below the capacity are complete and sorted, later ones empty
    _, _, orng = obs.bin_sort(rec, 90, 360)
    fits = orng[:, 1] <= cap
    assert fits.any() and not fits.all()
    assert np.array_equal(ranges[fits], orng[fits])
    assert np.all(ranges[~fits, 0] == ranges[~fits, 1])
    last = orng[fits][:, 1].max()
    assert np.array_equal(ids[:last], ov[:last])


@pytest.mark.parametrize("depths", ["spread", "few"])
def test_bin_sort_buckets_above_shared_memory_capacity(depths):
    """Every tile of a 180x45 view holds 26k-39k pairs, more than a thread block
    sorts in shared memory (24576).  Spread depths: those buckets take the
    distribution sort with the keys scattered in the workspace.  Three distinct
    depths: its sub-buckets overflow and the buckets are radix sorted there."""
    rec = synth.make_proj_records(60_000, 45, 180, seed=13, frac_wide=0.6)
    rec[:, 3] = np.where(rec[:, 3] < 0, -1.0, np.maximum(rec[:, 3], 30.0))
    if depths == "few":
        rec[:, 7] = np.random.default_rng(16).choice(np.float32([1.5, 2.0, 7.25]), size=len(rec))
    st, npairs, keys, ids, ranges = _gpu_binsort(rec, 45, 180)
    ok, ov, orng = obs.bin_sort(rec, 45, 180)
    assert (orng[:, 1] - orng[:, 0]).min() > 24576
    assert st == 0 and npairs == len(ov)
    assert np.array_equal(keys, ok)
    assert np.array_equal(ids, ov)
    assert np.array_equal(ranges, orng)


def test_bin_sort_few_distinct_depths():
    """Three distinct depths: each tile's depth sub-buckets hold far more than 64
    keys, so the tiles take the radix path in the workspace; ties go by index."""
    rec = synth.make_proj_records(5000, 90, 360, seed=14)
    rec[:, 7] = np.random.default_rng(15).choice(np.float32([1.5, 2.0, 7.25]), size=len(rec))
    st, npairs, keys, ids, ranges = _gpu_binsort(rec, 90, 360)
    ok, ov, orng = obs.bin_sort(rec, 90, 360)
    assert st == 0 and npairs == len(ov)
    assert np.array_equal(keys, ok)
    assert np.array_equal(ids, ov)
    assert np.array_equal(ranges, orng)


@pytest.mark.parametrize("H,W", [(180, 720), (90, 360), (45, 180)])
def test_bin_sort_serving_scale_sampled_tiles(H, W):
    """The 500k-Gaussian serving scene at its three resolutions (1.7M to 11M pairs; the densest
    tiles above the shared-memory capacity): at 720x180 the tiles outnumber the SMs and such
    buckets are sorted whole, at 360x90 and 180x45 they are cut into slices sorted by blocks of
    their own.  The GPU's own projection records binned and sorted, every tile's pair count
    against the oracle's footprint rule, and the full (r, id) lists of the 8 largest tiles and 8
    random ones bit for bit."""
    sc = synth.make_scene(500_000, seed=0, bf16_latent=True)
    ds = DeviceScene.from_host(sc, DEV)
    r = Renderer(H, W, 1, sc.n, device=DEV)
    r.geometry(ds)
    assert r.check() == 0
    npairs = int(r.n_pairs.item())
    rec = r.proj.cpu().numpy()
    ids = r.sorted_ids[:npairs].cpu().numpy().view(np.uint32)
    rng = r.tile_ranges.cpu().numpy().view(np.uint32).astype(np.int64)
    tiles = obs.footprint_tiles(rec, H, W)
    lens = np.fromiter((len(t) for t in tiles), dtype=np.int64, count=len(tiles))
    flat = np.fromiter((t for ts in tiles for t in ts), dtype=np.int64, count=int(lens.sum()))
    owner = np.repeat(np.arange(len(tiles), dtype=np.int64), lens)
    counts = np.bincount(flat, minlength=r.T)
    assert npairs == len(flat)
    assert np.array_equal(rng[:, 1] - rng[:, 0], counts)
    assert counts.max() > 24576
    pick = np.unique(np.concatenate([np.argsort(counts)[-8:],
                                     np.random.default_rng(17).choice(r.T, 8, replace=False)]))
    rr = rec[:, 7]
    for t in pick:
        mem = owner[flat == t]
        want = mem[np.lexsort((mem, rr[mem].astype(np.float64)))]
        assert np.array_equal(ids[rng[t, 0]:rng[t, 1]], want.astype(np.uint32)), t


def test_bin_sort_properties_full_size_scene():
    """50k-Gaussian scene projected on the GPU: every tile list is ordered by
    (r, id) and holds each Gaussian at most once; pair count = sum of footprints."""
    sc = synth.make_scene(50_000, seed=0)
    r = Renderer(90, 360, 64, sc.n, device=DEV)
    ds = DeviceScene.from_host(sc, DEV)
    r.geometry(ds, keep_keys=True)
    assert r.check() == 0
    npairs = int(r.n_pairs.item())
    keys = r.sorted_keys[:npairs].cpu().numpy().view(np.uint64)
    ids = r.sorted_ids[:npairs].cpu().numpy().view(np.uint32)
    assert np.all(keys[1:] >= keys[:-1])
    rr = r.proj[:, 7].cpu().numpy()
    assert np.array_equal((keys & np.uint64(0xFFFFFFFF)).astype(np.uint32), rr[ids].view(np.uint32))
    tiles = (keys >> np.uint64(32)).astype(np.int64)
    same = (tiles[1:] == tiles[:-1]) & (keys[1:] == keys[:-1])
    assert np.all(ids[1:][same] > ids[:-1][same])
    rng = r.tile_ranges.cpu().numpy()
    assert rng[:, 1].max() == npairs
    counts = np.bincount(tiles, minlength=r.T)
    assert np.array_equal(rng[:, 1] - rng[:, 0], counts)


@pytest.mark.parametrize("hidden,B,n", [(8, 1, 100), (16, 2, 1031), (32, 3, 4099), (64, 2, 2500)])
def test_attr_mlp_matches_oracle(hidden, B, n):
    sc = synth.make_scene(n, seed=hidden)
    mlp = synth.make_mlp(hidden, seed=3)
    tx = synth.make_tx(B, seed=2)
    tx[0] = sc.means[5]          # a transmitter on a Gaussian: exercises the d clamp
    r = Renderer(90, 360, 1, n, device=DEV)
    ds = DeviceScene.from_host(sc, DEV)
    dm = DeviceMLP.from_host(mlp, DEV)
    attr = r.attributes(ds, dm, torch.tensor(tx, device=DEV)).cpu().numpy().astype(np.float64)
    _, ref = oracle_geo_attr(sc, mlp, synth.View(90, 360), tx)
    for b in range(B):
        for j, k in enumerate(("a", "phi0", "sigma", "L")):
            np.testing.assert_allclose(attr[b, :, j], ref[b][k], rtol=2e-5,
                                       atol=2e-6 * max(1.0, np.abs(ref[b][k]).max()))


@pytest.mark.parametrize("hidden,B,n", [(16, 2, 1000), (32, 3, 4099), (64, 2, 2500)])
def test_attr_mlp_tensor_cores(hidden, B, n):
    """The tcgen05 network: BF16X2 (split operands) within 1e-4 of the FP64 oracle,
    BF16 within 3e-2 (one BF16 rounding of inputs and activations), no NaN."""
    sc = synth.make_scene(n, seed=hidden + 1)
    mlp = synth.make_mlp(hidden, seed=3)
    tx = synth.make_tx(B, seed=4)
    r = Renderer(90, 360, 1, n, device=DEV)
    ds = DeviceScene.from_host(sc, DEV)
    dm = DeviceMLP.from_host(mlp, DEV)
    txd = torch.tensor(tx, device=DEV)
    _, ref = oracle_geo_attr(sc, mlp, synth.View(90, 360), tx)
    for prec, tol in ((G.GSPARC_BF16X2, 1e-4), (G.GSPARC_BF16, 3e-2)):
        attr = r.attributes(ds, dm, txd, precision=prec).cpu().numpy().astype(np.float64)
        assert np.all(np.isfinite(attr))
        for b in range(B):
            for j, k in enumerate(("a", "phi0", "sigma", "L")):
                err = np.linalg.norm(attr[b, :, j] - ref[b][k]) / np.linalg.norm(ref[b][k])
                assert err <= tol, (prec, k, err)
