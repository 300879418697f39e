"""Training extras on the GPU against the FP64 oracle: the confidence-weighted objective of Eq. 5
(gsparc_confidence) -- objective, confidence, dObj/dL_task and the weight gradients, their
accumulation, optional outputs, the empty batch and run-to-run equality -- and the adaptive
density control of Algorithm 1 (gsparc_densify_accumulate, gsparc_densify,
gsparc_opacity_reset)."""
import numpy as np
import pytest
import torch

from extras_cases import (accumulate_check, conf_case, conf_oracle, dens_case, dens_check, dens_oracle,
                          reset_check)
from gpu_util import DEV
from paper_2511_22793_gb300 import gsparc as G

pytestmark = pytest.mark.gpu


def _d(a):
    return torch.tensor(np.ascontiguousarray(a), device=DEV)


@pytest.mark.parametrize("B,hidden", [(1, 32), (4, 32), (37, 32), (1000, 32), (300, 8), (9, 1)])
def test_confidence_matches_oracle(B, hidden):
    pos, L, w = conf_case(B, hidden, 100 + B + hidden)
    o_obj, o_C, o_dL, o_dw, kink = conf_oracle(pos, L, w, hidden)
    assert kink > 1e-5            # no ReLU decision within FP32 rounding of the kink
    obj = torch.full((1,), 5.0, device=DEV)
    C = torch.empty(B, device=DEV)
    dL = torch.empty(B, device=DEV)
    dw = torch.zeros(5 * hidden + 1, device=DEV)
    G.gsparc_confidence(_d(pos), _d(L), _d(w), hidden, obj, C, dL, dw)
    torch.cuda.synchronize()
    assert abs(float(obj) - o_obj) <= 1e-5 * abs(o_obj)
    assert np.allclose(C.cpu().numpy(), o_C, rtol=2e-6, atol=0)
    assert np.allclose(dL.cpu().numpy(), o_dL, rtol=2e-6, atol=0)
    g = dw.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(g - o_dw) <= 1e-5 * np.linalg.norm(o_dw)


def test_confidence_accumulates_and_repeats():
    B, hidden = 64, 32
    pos, L, w = conf_case(B, hidden, 7)
    args = (_d(pos), _d(L), _d(w), hidden)
    obj1, obj2 = torch.empty(1, device=DEV), torch.empty(1, device=DEV)
    C1, C2 = torch.empty(B, device=DEV), torch.empty(B, device=DEV)
    dw = torch.zeros(5 * hidden + 1, device=DEV)
    G.gsparc_confidence(*args, obj1, C1, None, dw)
    once = dw.clone()
    G.gsparc_confidence(*args, obj2, C2, None, dw)
    torch.cuda.synchronize()
    assert torch.equal(obj1, obj2) and torch.equal(C1, C2)
    assert torch.equal(dw, 2.0 * once)
    # optional outputs left out: the same objective
    obj3 = torch.empty(1, device=DEV)
    G.gsparc_confidence(*args, obj3)
    torch.cuda.synchronize()
    assert torch.equal(obj3, obj1)


def test_confidence_empty_batch():
    obj = torch.full((1,), 5.0, device=DEV)
    w = _d(conf_case(1, 32, 3)[2])
    empty = torch.empty((0,), device=DEV)
    G.gsparc_confidence(torch.empty((0, 3), device=DEV), empty, w, 32, obj)
    torch.cuda.synchronize()
    assert float(obj) == 0.0


def _dens_gpu(c, th, cap):
    N, P = c["payload"].shape
    f = lambda *shape: torch.full(shape, float("nan"), device=DEV)
    out = {"means": f(cap, 3), "log_scales": f(cap, 3), "quats": f(cap, 4), "opacity_logit": f(cap),
           "payload": f(cap, P) if P > 0 else None,
           "parent": torch.full((cap,), -1, dtype=torch.int32, device=DEV)}
    n_out = torch.full((1,), -1, dtype=torch.int32, device=DEV)
    status = torch.zeros(1, dtype=torch.int32, device=DEV)
    ws = torch.empty(max(G.gsparc_densify_workspace(N), 1), dtype=torch.uint8, device=DEV)
    params = G.densify_params(tau_grad=th.tau_grad, clone_scale=th.eps * th.r_scene, sigma_min=th.sigma_min,
                              r_max=th.r_max, n_split=th.n_split)
    count = _d(c["count"].view(np.int32))
    G.gsparc_densify(_d(c["means"]), _d(c["log_scales"]), _d(c["quats"]), _d(c["opacity_logit"]),
                     _d(c["payload"]) if P > 0 else None, _d(c["proj"]), _d(c["norm_sum"]), count, _d(c["xi"]),
                     params, ws, out, n_out, status)
    torch.cuda.synchronize()
    res = {k: out[k].cpu().numpy() for k in ("means", "log_scales", "quats", "opacity_logit")}
    res["payload"] = out["payload"].cpu().numpy() if P > 0 else np.zeros((cap, 0), np.float32)
    res["parent"] = out["parent"].cpu().numpy().view(np.uint32)
    res["n_out"] = int(n_out.cpu().numpy().view(np.uint32)[0])
    res["status"] = int(status.item())
    return res


@pytest.mark.parametrize("N,P,n_split,cap_frac,seed", [(3000, 5, 2, 2.0, 0), (3000, 0, 3, 2.0, 1),
                                                        (257, 16, 2, 0.5, 2), (1, 3, 4, 4.0, 3),
                                                        (700, 2, 8, 0.0, 4), (300_000, 16, 2, 1.5, 6)])
def test_densify_matches_oracle(N, P, n_split, cap_frac, seed):
    """gsparc_densify against the oracle: row count and parents bit-exact, copies exact, children
    within FP32 rounding; ragged blocks, no payload, capacity below the row count (and zero),
    n_split 2 to 8, and 300k Gaussians (more blocks than the one-block scan has threads)."""
    c, th = dens_case(N, P, n_split, seed)
    o = dens_oracle(c, th)
    cap = int(cap_frac * N)
    res = _dens_gpu(c, th, cap)
    dens_check(res, o, c, cap)
    again = _dens_gpu(c, th, cap)
    for k in res:
        assert np.array_equal(np.asarray(res[k]), np.asarray(again[k]), equal_nan=True), k


def test_densify_accumulate_and_opacity_reset():
    c, th = dens_case(5000, 0, 2, 9)
    o = dens_oracle(c, th)
    norm = _d(c["norm_sum"]).clone()
    cnt = _d(c["count"].view(np.int32)).clone()
    G.gsparc_densify_accumulate(_d(c["proj"]), _d(c["d_means"]), norm, cnt)
    logit = _d(c["opacity_logit"]).clone()
    G.gsparc_opacity_reset(logit, 0.01)
    torch.cuda.synchronize()
    accumulate_check(norm.cpu().numpy(), cnt.cpu().numpy().view(np.uint32), o)
    reset_check(logit.cpu().numpy(), o)


def test_densify_empty_set():
    n_out = torch.full((1,), 7, dtype=torch.int32, device=DEV)
    e = lambda *s: torch.empty(s, device=DEV)
    out = {"means": e(0, 3), "log_scales": e(0, 3), "quats": e(0, 4), "opacity_logit": e(0),
           "parent": torch.empty((0,), dtype=torch.int32, device=DEV)}
    ws = torch.empty(256, dtype=torch.uint8, device=DEV)
    G.gsparc_densify(e(0, 3), e(0, 3), e(0, 4), e(0), None, e(0, 8), e(0), torch.empty((0,), dtype=torch.int32,
                     device=DEV), e(0, 2, 3), G.densify_params(), ws, out, n_out)
    torch.cuda.synchronize()
    assert int(n_out.item()) == 0
