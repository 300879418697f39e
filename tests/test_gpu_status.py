"""Device-side conditions reach the caller's status word (the boundary's convention).

- An expired bounded wait in each tensor-core compositing call: gsparc_set_wait_limit(1) lets
  every pipeline wait poll its mbarrier once, so waits run out without any fault or hang; the
  call must report GSPARC_ERR_TIMEOUT through gsparc_check, return, and leave the context usable
  (the same call with the default limit afterwards gives the FP32 kernel's result).
- Inputs only the device sees: a list id outside the scene (every compositing call skips the
  entry and reports GSPARC_ERR_INPUT), a zero quaternion or a non-finite mean (the projection
  culls the Gaussian and reports GSPARC_ERR_INPUT).
"""
import numpy as np
import pytest
import torch

from gpu_util import DEV
from paper_2511_22793_gb300 import gsparc as G
from paper_2511_22793_gb300 import synth
from paper_2511_22793_gb300.pipeline import DeviceMLP, DeviceScene, Renderer

pytestmark = pytest.mark.gpu


def _setup(n=50_000, H=90, W=360, K=64, B=1):
    sc = synth.make_scene(n, seed=0)
    mlp = synth.make_mlp(32, seed=3)
    r = Renderer(H, W, K, n, device=DEV)
    ds = DeviceScene.from_host(sc, DEV)
    dm = DeviceMLP.from_host(mlp, DEV)
    txd = torch.tensor(synth.make_tx(B, seed=2), device=DEV)
    r.geometry(ds)
    attr = r.attributes(ds, dm, txd)
    torch.cuda.synchronize()
    assert r.check() == 0
    return r, attr


class _Limit:
    def __init__(self, polls):
        self.polls = polls

    def __enter__(self):
        self.prev = G.gsparc_set_wait_limit(self.polls)

    def __exit__(self, *exc):
        G.gsparc_set_wait_limit(self.prev)


def test_set_wait_limit_returns_previous():
    assert G.gsparc_set_wait_limit(7) == 0
    assert G.gsparc_set_wait_limit(0) == 7


def test_expired_waits_report_timeout_and_leave_the_context_usable():
    r, attr = _setup()
    B, n = 1, r.n
    spec, logT, nc = r.alloc_outputs(B)
    ref_spec, ref_logT, ref_nc = r.alloc_outputs(B)
    G.gsparc_render_fwd(r.view, r.band, B, n, r.proj, r.tile_ranges, r.sorted_ids, attr, ref_spec, ref_logT,
                        ref_nc)
    d_spec = torch.randn_like(ref_spec) * 1e-3
    ref_dattr, ref_dproj = torch.zeros_like(attr), torch.zeros_like(r.proj)
    G.gsparc_render_bwd(r.view, r.band, B, n, r.proj, r.tile_ranges, r.sorted_ids, attr, ref_logT, ref_nc, d_spec,
                        ref_dattr, ref_dproj)
    torch.cuda.synchronize()
    status = torch.zeros(1, dtype=torch.int32, device=DEV)
    target = torch.zeros_like(ref_spec)
    loss = torch.zeros(1, device=DEV)
    dz = torch.empty_like(ref_spec)
    csi = torch.empty((B, r.K, 2), device=DEV)
    ws = torch.zeros(G.gsparc_render_bwd_tc_workspace(r.view, r.band, B), dtype=torch.uint8, device=DEV)
    d_attr, d_proj = torch.zeros_like(attr), torch.zeros_like(r.proj)
    calls = {
        "fwd_tc": lambda st: G.gsparc_render_fwd_tc(r.view, r.band, B, n, r.proj, r.tile_ranges, r.sorted_ids, attr,
                                                    spec, logT, nc, d_status=st),
        "fwd_l2_tc": lambda st: G.gsparc_render_fwd_l2_tc(r.view, r.band, B, n, r.proj, r.tile_ranges,
                                                          r.sorted_ids, attr, target, loss, dz, spec, logT, nc,
                                                          d_status=st),
        "csi_tc": lambda st: G.gsparc_render_csi_tc(r.view, r.band, B, n, r.proj, r.tile_ranges, r.sorted_ids,
                                                    attr, csi, d_status=st),
        "bwd_tc": lambda st: G.gsparc_render_bwd_tc(r.view, r.band, B, n, r.proj, r.tile_ranges, r.sorted_ids,
                                                    attr, ref_logT, ref_nc, d_spec, d_attr, d_proj, d_status=st),
        "bwd_tc_balanced": lambda st: G.gsparc_render_bwd_tc_balanced(
            r.view, r.band, B, n, r.proj, r.tile_ranges, r.sorted_ids, attr, ref_spec, None, ref_logT, ref_nc,
            d_spec, ws, d_attr, d_proj, d_status=st),
    }
    for name, call in calls.items():
        status.zero_()
        with _Limit(1):
            call(status)
        assert G.gsparc_check(status) == G.GSPARC_ERR_TIMEOUT, name
        # the context still works, and with the default limit the call is correct again
        status.zero_()
        d_attr.zero_()
        d_proj.zero_()
        call(status)
        assert G.gsparc_check(status) == G.GSPARC_OK, name
        if name in ("fwd_tc", "fwd_l2_tc"):
            e = float((spec - ref_spec).norm() / ref_spec.norm())
            assert e < 1e-4, (name, e)
            assert torch.equal(nc, ref_nc) and torch.equal(logT, ref_logT), name
        elif name.startswith("bwd"):
            e = float((d_attr - ref_dattr).norm() / ref_dattr.norm())
            assert e < 1e-3, (name, e)


def test_list_id_outside_the_scene_reports_input_error():
    r, attr = _setup(n=3000, K=8)
    B, n = 1, r.n
    ids = r.sorted_ids.clone()
    rng = r.tile_ranges.cpu().numpy()
    t = int(np.argmax(rng[:, 1] - rng[:, 0]))
    assert rng[t, 1] > rng[t, 0]
    ids[int(rng[t, 0])] = n + 5          # one entry of the busiest tile points past the scene
    spec, logT, nc = r.alloc_outputs(B)
    d_spec = torch.randn_like(spec) * 1e-3
    status = torch.zeros(1, dtype=torch.int32, device=DEV)
    for tc in (False, True):
        status.zero_()
        fn = G.gsparc_render_fwd_tc if tc else G.gsparc_render_fwd
        fn(r.view, r.band, B, n, r.proj, r.tile_ranges, ids, attr, spec, logT, nc, d_status=status)
        assert G.gsparc_check(status) == G.GSPARC_ERR_INPUT
        assert torch.isfinite(spec).all()
        status.zero_()
        d_attr, d_proj = torch.zeros_like(attr), torch.zeros_like(r.proj)
        fb = G.gsparc_render_bwd_tc if tc else G.gsparc_render_bwd
        fb(r.view, r.band, B, n, r.proj, r.tile_ranges, ids, attr, logT, nc, d_spec, d_attr, d_proj, d_status=status)
        assert G.gsparc_check(status) == G.GSPARC_ERR_INPUT
        assert torch.isfinite(d_attr).all() and torch.isfinite(d_proj).all()
    # the untouched list reports nothing
    status.zero_()
    G.gsparc_render_fwd(r.view, r.band, B, n, r.proj, r.tile_ranges, r.sorted_ids, attr, spec, logT, nc,
                        d_status=status)
    assert G.gsparc_check(status) == G.GSPARC_OK


def test_projection_culls_and_reports_degenerate_gaussians():
    sc = synth.make_scene(1000, seed=0)
    ds = DeviceScene.from_host(sc, DEV)
    r = Renderer(90, 360, 1, sc.n, device=DEV)
    status = torch.zeros(1, dtype=torch.int32, device=DEV)
    G.gsparc_project(r.view, ds.means, ds.log_scales, ds.quats, r.proj, d_status=status)
    assert G.gsparc_check(status) == G.GSPARC_OK
    good = r.proj.clone()
    ds.quats[3].zero_()
    ds.means[7, 1] = float("nan")
    ds.log_scales[11, 0] = float("inf")
    G.gsparc_project(r.view, ds.means, ds.log_scales, ds.quats, r.proj, d_status=status)
    assert G.gsparc_check(status) == G.GSPARC_ERR_INPUT
    p = r.proj.cpu()
    for i in (3, 7, 11):
        assert p[i, 2] == -1 and p[i, 3] == -1, i          # culled
    assert torch.isfinite(p).all()
    keep = torch.ones(sc.n, dtype=torch.bool)
    keep[[3, 7, 11]] = False
    assert torch.equal(p[keep], good.cpu()[keep])
    # no gradient for them, and none of it NaN
    d_proj = torch.ones_like(r.proj)
    gm, gl, gq = torch.zeros_like(ds.means), torch.zeros_like(ds.log_scales), torch.zeros_like(ds.quats)
    G.gsparc_project_bwd(r.view, ds.means, ds.log_scales, ds.quats, d_proj, gm, gl, gq)
    torch.cuda.synchronize()
    for t in (gm, gl, gq):
        assert torch.isfinite(t).all()
    assert float(gq[3].abs().sum()) == 0 and float(gl[11].abs().sum()) == 0
