"""The on-device training loop: it fits a ground-truth scene (loss and held-out error
fall), and checkpoint/resume reproduces the loss trajectory."""
import numpy as np
import pytest
import torch

from paper_2511_22793_gb300 import synth
from paper_2511_22793_gb300.train import Trainer

pytestmark = pytest.mark.gpu


def _trainer(steps=200):
    gt = synth.make_scene(600, seed=31)
    gt.log_scales = gt.log_scales + np.float32(0.5)
    gt_mlp = synth.make_mlp(16, seed=32)
    train_tx = synth.make_tx(64, seed=33)
    return Trainer(3000, gt, gt_mlp, train_tx, H=45, W=180, K=8, hidden=16, batch=4,
                   total_steps=steps, seed=34)


def test_training_from_scratch_reduces_loss():
    tr = _trainer()
    losses = [float(tr.step()) for _ in range(200)]
    assert np.isfinite(losses).all()
    assert np.mean(losses[-20:]) < 0.8 * np.mean(losses[:20]), (losses[:5], losses[-5:])


def test_training_recovers_perturbed_scene_on_heldout_transmitters():
    """Start from the ground truth with shifted opacities and a perturbed network: the
    fit must bring the error on unseen transmitters down."""
    gt = synth.make_scene(600, seed=31)
    gt.log_scales = gt.log_scales + np.float32(0.5)
    gt_mlp = synth.make_mlp(16, seed=32)
    start = synth.Scene(gt.means.copy(), gt.log_scales.copy(), gt.quats.copy(),
                        gt.opacity_logit - np.float32(1.0), gt.latent.copy())
    noise = synth.make_mlp(16, seed=36)
    mlp0 = synth.MLPWeights(16, *[a + 0.3 * b for a, b in zip(gt_mlp.arrays(), noise.arrays())])
    tr = Trainer(600, gt, gt_mlp, synth.make_tx(64, seed=33), H=45, W=180, K=8, hidden=16, batch=4,
                 total_steps=300, seed=34, init=(start, mlp0))
    held = synth.make_tx(16, seed=35)
    e0 = tr.evaluate(held)
    for _ in range(300):
        tr.step()
    e1 = tr.evaluate(held)
    assert e1 < 0.7 * e0, (e0, e1)


def test_checkpoint_resume_reproduces_trajectory():
    tr = _trainer()
    for _ in range(20):
        tr.step()
    st = tr.state_dict()
    a = [float(tr.step()) for _ in range(10)]
    tr.load_state_dict(st)
    b = [float(tr.step()) for _ in range(10)]
    # gradient sums use float atomics, so the last bits may differ between runs
    np.testing.assert_allclose(a, b, rtol=1e-4)
