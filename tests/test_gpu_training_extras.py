"""Training extras on the GPU against the FP64 oracle: the confidence-weighted objective of Eq. 5
(gsparc_confidence) -- objective, confidence, dObj/dL_task and the weight gradients, their
accumulation, optional outputs, the empty batch and run-to-run equality."""
import numpy as np
import pytest
import torch

from extras_cases import conf_case, conf_oracle
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
