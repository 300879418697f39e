"""The library's training constants against the values the paper's table of hyperparameters
prints (tests/golden/hyperparameters.txt), and the position-rate anneal of the training loop
against the oracle's (host logic only)."""
import math
import os
import types

import pytest

from oracle import adam as OA
from oracle import confidence as CF
from oracle import spectrum_loss as S
from paper_2511_22793_gb300 import train

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "hyperparameters.txt")


def _table():
    out = {}
    for line in open(GOLDEN):
        line = line.strip()
        if line and not line.startswith("#"):
            k, v = line.split()
            out[k] = float(v)
    return out


def test_training_rates_match_the_table():
    t = _table()
    assert train.POS_LR_INIT == t["position_lr_init"] and train.POS_LR_FINAL == t["position_lr_final"]
    assert train.LR["opacity_logit"] == t["opacity_lr"]
    assert train.LR["log_scales"] == t["scaling_lr"]
    assert train.LR["quats"] == t["rotation_lr"]
    for k in ("W1", "b1", "W2", "b2", "W3", "b3"):
        assert train.LR[k] == t["emission_mlp_lr"], k


def test_loss_weights_match_the_table():
    """The oracle's weights and the binding's defaults of Eq. 4 and Eq. 5."""
    import inspect

    from paper_2511_22793_gb300 import gsparc as G

    t = _table()
    assert CF.ALPHA == t["alpha"]
    assert S.LAMBDA == t["lambda_1"]
    assert inspect.signature(G.gsparc_spectrum_loss).parameters["lam"].default == t["lambda_1"]
    assert inspect.signature(G.gsparc_confidence).parameters["alpha"].default == t["alpha"]


@pytest.mark.parametrize("total", [2, 100, 1000])
def test_position_rate_anneal_matches_the_oracle(total):
    for step in (0, 1, total // 3, total // 2, total - 1, total + 5):
        fake = types.SimpleNamespace(step_count=step, total_steps=total)
        got = train.Trainer.pos_lr(fake)
        assert math.isclose(got, OA.position_lr(min(step, total - 1), total), rel_tol=1e-12)
