"""Launch overlap (programmatic dependent launch of the library's follow-on kernels: tile emit and
sort, the compositing forward, the backward's schedule and walks, the network backward) changes no
result.  The 50,000-Gaussian, 64-subcarrier, 360x90 training step, in both arithmetic forms, run
eagerly and as the CUDA graph the benchmark replays, gives with the overlap off and on the same
tile ranges, sorted ids and upstream gradient dL/dz bit for bit, and the same loss and parameter
gradients (summed by atomics in an order that varies from run to run, so compared at 1e-5
relative L2).
"""
import pytest
import torch

from gpu_util import DEV
from paper_2511_22793_gb300 import gsparc as G
from paper_2511_22793_gb300 import synth
from paper_2511_22793_gb300.pipeline import DeviceMLP, DeviceScene, Renderer
from paper_2511_22793_gb300.step import TrainStep

pytestmark = pytest.mark.gpu

H, W, K, N, HIDDEN = 90, 360, 64, 50_000, 32


def _step(form, overlap, graph):
    prev = G.gsparc_set_launch_overlap(overlap)
    try:
        sc = synth.make_scene(N, seed=0)
        mlp = synth.make_mlp(HIDDEN, seed=3)
        r = Renderer(H, W, K, N, device=DEV)
        ds = DeviceScene.from_host(sc, DEV)
        dm = DeviceMLP.from_host(mlp, DEV)
        txd = torch.tensor(synth.make_tx(1, seed=2), device=DEV)
        # a seeded random target (a nonzero, uneven dL/dz)
        target = 0.5 * torch.randn((1, K, H, W, 2), generator=torch.Generator(DEV).manual_seed(7),
                                   device=DEV) * 1e-3
        st = TrainStep(r, ds, dm, txd, target, form=form)
        if graph:
            st.enqueue()
            g = st.capture()
            for _ in range(3):
                g.replay()
        else:
            for _ in range(2):
                st.enqueue()
        torch.cuda.synchronize()
        assert r.check() == 0
        n_pairs = int(r.n_pairs.item())
        return {"ranges": r.tile_ranges.clone(), "ids": r.sorted_ids[:n_pairs].clone(),
                "dz": st.d_spec.clone(), "loss": float(st.loss.item()), "grads": [t.clone() for t in st.grads],
                "d_attr": st.d_attr.clone()}
    finally:
        G.gsparc_set_launch_overlap(prev)


@pytest.mark.parametrize("form", ["fp32", "tc"])
@pytest.mark.parametrize("graph", [False, True])
def test_launch_overlap_changes_no_result(form, graph):
    assert G.gsparc_set_launch_overlap(True) == G.GSPARC_OVERLAP_ALL      # every group by default
    off = _step(form, False, graph)
    on = _step(form, True, graph)
    assert torch.equal(on["ranges"], off["ranges"])
    assert torch.equal(on["ids"], off["ids"])
    assert torch.equal(on["dz"], off["dz"])
    assert abs(on["loss"] - off["loss"]) <= 1e-5 * abs(off["loss"])
    for a, b in zip(on["grads"] + [on["d_attr"]], off["grads"] + [off["d_attr"]]):
        den = float(b.double().norm())
        assert den > 0
        assert float((a.double() - b.double()).norm()) <= 1e-5 * den


def test_set_launch_overlap_returns_previous():
    prev = G.gsparc_set_launch_overlap(False)
    try:
        assert G.gsparc_set_launch_overlap(G.GSPARC_OVERLAP_FORWARD | 64) == 0
        assert G.gsparc_set_launch_overlap(0) == G.GSPARC_OVERLAP_FORWARD    # unknown bits dropped
    finally:
        G.gsparc_set_launch_overlap(prev)
