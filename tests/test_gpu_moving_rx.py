"""Moving receiver (Sec. 4.2 "Directional Projection and Splatting": a receiver pose per
sample): one Renderer moved between poses against the oracle at each pose, and the query
server mixing fixed-receiver and moving-receiver requests."""
import math

import numpy as np
import pytest
import torch

from gpu_util import DEV, oracle_geo_attr, oracle_render, rel_l2, spectrum_to_complex
from paper_2511_22793_gb300 import gsparc as G
from paper_2511_22793_gb300 import synth
from paper_2511_22793_gb300.pipeline import DeviceMLP, DeviceScene, Renderer
from paper_2511_22793_gb300.serve import Request, Server

pytestmark = pytest.mark.gpu
TOL = 1e-3   # spectrum relative L2 against the FP64 oracle, as the fixed-receiver render tests


def _rot(yaw, pitch):
    """World-to-receiver rotation: yaw about +y, then pitch about +x (row-major 3x3)."""
    cy, sy, cp, sp = math.cos(yaw), math.sin(yaw), math.cos(pitch), math.sin(pitch)
    Ry = np.array([[cy, 0, sy], [0, 1, 0], [-sy, 0, cy]])
    Rx = np.array([[1, 0, 0], [0, cp, -sp], [0, sp, cp]])
    return tuple((Rx @ Ry).reshape(-1))


POSES = [((0.0, 0.0, 0.0), None),
         ((1.5, 0.8, -2.0), None),
         ((-0.7, 1.2, 0.4), _rot(0.5, 0.2)),
         ((2.5, -0.5, 3.0), _rot(-1.1, -0.15))]


def test_receiver_moved_between_poses_matches_oracle():
    n, H, W, K, B = 3000, 90, 360, 16, 2
    sc = synth.make_scene(n, seed=81)
    mlp = synth.make_mlp(32, seed=82)
    tx = synth.make_tx(B, seed=83)
    r = Renderer(H, W, K, n, device=DEV)
    ds = DeviceScene.from_host(sc, DEV)
    dm = DeviceMLP.from_host(mlp, DEV)
    txd = torch.tensor(tx, device=DEV)
    for rx, V in POSES:
        r.set_receiver(rx, V if V is not None else (1, 0, 0, 0, 1, 0, 0, 0, 1))
        r.geometry(ds)
        attr = r.attributes(ds, dm, txd)
        spec, _, _ = r.render(attr)
        spec_tc, _, _ = r.render(attr, tensor_cores=True)
        torch.cuda.synchronize()
        assert r.check() == 0
        view = synth.View(H=H, W=W, rx=rx, V=V if V is not None else synth.View(H=H, W=W).V)
        g, attrs = oracle_geo_attr(sc, mlp, view, tx)
        zref, _, _ = oracle_render(g, attrs, view, synth.Band(K=K))
        z = spectrum_to_complex(spec)
        z_tc = spectrum_to_complex(spec_tc)
        for b in range(B):
            assert rel_l2(z[b], zref[b]) <= TOL, (rx, b)
            assert rel_l2(z_tc[b], zref[b]) <= TOL, (rx, b)


def test_server_mixes_fixed_and_moving_receivers():
    """Moving-receiver requests run on their own geometry; every served spectrum equals the
    same request rendered directly for its pose (same kernels, same precision), and the
    fixed-receiver requests in the mix are unaffected."""
    sc = synth.make_scene(8000, seed=84, bf16_latent=True)
    mlp = synth.make_mlp(32, seed=85, bf16_weights=True)
    ds, dm = DeviceScene.from_host(sc, DEV), DeviceMLP.from_host(mlp, DEV)
    res = [(45, 180), (90, 360)]
    tx = synth.make_tx(12, seed=86)
    reqs = []
    for i in range(12):
        rx, V = POSES[i % len(POSES)] if i % 3 else (None, None)
        reqs.append(Request(i, tuple(float(v) for v in tx[i]), res[i % 2], (1, 8, 16)[i % 3], rx=rx, V=V))
    srv = Server(ds, dm, res, mem_budget_bytes=2 << 30, max_batch=4, n_streams=3)
    srv.run(reqs, np.zeros(len(reqs)))
    torch.cuda.synchronize()
    assert all(not q.rejected for q in reqs)
    for q in reqs:
        H, W = q.res
        r = Renderer(H, W, q.K, ds.n, device=DEV)
        if q.rx is not None:
            r.set_receiver(q.rx, q.V if q.V is not None else (1, 0, 0, 0, 1, 0, 0, 0, 1))
        r.geometry(ds)
        attr = r.attributes(ds, dm, torch.tensor([q.tx], dtype=torch.float32, device=DEV), G.GSPARC_BF16X2)
        spec, _, _ = r.render(attr, tensor_cores=True)
        torch.cuda.synchronize()
        ref = spec[0]
        assert float((q.spectrum - ref).norm() / ref.norm().clamp_min(1e-30)) <= 1e-6, q.rid
