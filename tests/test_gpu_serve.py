"""Continuous-batching server: every result is the same alone and in the mix,
admission respects the memory budget, and the served spectra match the plain FP32
path within the 1e-3 bound."""
import numpy as np
import pytest
import torch

from paper_2511_22793_gb300 import gsparc as G
from paper_2511_22793_gb300 import synth
from paper_2511_22793_gb300.pipeline import DeviceMLP, DeviceScene
from paper_2511_22793_gb300.serve import Request, Server, serve_plain

pytestmark = pytest.mark.gpu
RES = [(45, 180), (90, 360), (180, 720)]


def _scene():
    sc = synth.make_scene(20_000, seed=41, bf16_latent=True)
    mlp = synth.make_mlp(32, seed=42, bf16_weights=True)
    return DeviceScene.from_host(sc), DeviceMLP.from_host(mlp)


def _requests(n, seed):
    rng = np.random.default_rng(seed)
    tx = synth.make_tx(n, seed=seed)
    Ks = [1, 8, 64]
    return [Request(i, tuple(float(v) for v in tx[i]), RES[rng.integers(3)], Ks[rng.integers(3)])
            for i in range(n)]


def _rel(a, b):
    return float((a - b).norm() / b.norm().clamp_min(1e-30))


def test_results_same_alone_and_in_the_mix():
    ds, dm = _scene()
    reqs = _requests(30, 43)
    srv = Server(ds, dm, RES, mem_budget_bytes=4 << 30, max_batch=8, n_streams=3)
    srv.run(reqs, np.zeros(len(reqs)))             # one burst: batched and overlapped
    torch.cuda.synchronize()
    assert all(q.t_done >= q.t_arrival and not q.rejected for q in reqs)
    mixed = {q.rid: q.spectrum.clone() for q in reqs}
    batched = sum(1 for q in reqs) > len(set((q.res, q.K) for q in reqs))
    assert batched
    for q in reqs:
        srv.release(q)
    assert srv.used == 0                           # every block back in the arena
    alone = Server(ds, dm, RES, mem_budget_bytes=1 << 30, max_batch=1, n_streams=1)
    for q in reqs:                                 # each alone, same arithmetic
        solo = Request(q.rid, q.tx, q.res, q.K)
        alone.run([solo], np.zeros(1))
        torch.cuda.synchronize()
        assert _rel(mixed[q.rid], solo.spectrum) <= 1e-6
        alone.release(solo)
    plain = _requests(30, 43)
    serve_plain(ds, dm, plain, np.zeros(len(plain)), RES)
    for q, p in zip(reqs, plain):
        assert _rel(mixed[q.rid], p.spectrum) <= 1e-3


def test_memory_admission_and_rejection():
    ds, dm = _scene()
    big = Request(0, (1.0, 2.0, 0.5), (180, 720), 64)
    srv = Server(ds, dm, RES, mem_budget_bytes=1, max_batch=4, n_streams=2)
    srv.run([big], np.zeros(1))
    assert big.rejected
    one = srv.request_bytes(180, 720, 64)
    reqs = [Request(i, (0.5 * i, 1.0, -1.0), (180, 720), 64) for i in range(6)]
    srv = Server(ds, dm, RES, mem_budget_bytes=one + one // 2, max_batch=4, n_streams=2, keep_results=False)
    srv.run(reqs, np.zeros(len(reqs)))
    assert all(not q.rejected and q.t_done >= q.t_arrival for q in reqs)
    assert srv.used == 0
    # kept results hold their memory until released: with room for one, a second request waits
    # for the first one's release, and the server says so instead of waiting forever
    srv = Server(ds, dm, RES, mem_budget_bytes=one + one // 2, max_batch=4, n_streams=2)
    a, b = Request(10, (1.0, 1.0, 1.0), (180, 720), 64), Request(11, (2.0, 1.0, 1.0), (180, 720), 64)
    srv.run([a], np.zeros(1))
    assert a.spectrum is not None and srv.used > 0
    with pytest.raises(RuntimeError):
        srv.run([b], np.zeros(1))
    srv.release(a)
    assert srv.used == 0
    srv.waiting.clear()
    srv.run([Request(12, (2.0, 1.0, 1.0), (180, 720), 64)], np.zeros(1))
    assert srv.used > 0
