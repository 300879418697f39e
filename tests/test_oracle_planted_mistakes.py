"""Planted mistakes: a copy of the oracle with one deliberate error must fail the pin that guards
that part, so that the pins are not vacuous.  Every mistake is planted in the oracle, on the
CPU: a patched copy of the C renderer compiled into a temporary library, or a monkeypatched
Python function; the real oracle is restored afterwards."""
import numpy as np
import pytest
import torch

import test_oracle_adam as TAD
import test_oracle_attributes as TA
import test_oracle_binsort as TB
import test_oracle_confidence as TCF
import test_oracle_csi as TC
import test_oracle_densify as TD
import test_oracle_emission as TE
import test_oracle_grad as TG
import test_oracle_projection as TP
import test_oracle_render as TR
import test_oracle_spectrum_loss as TS
from oracle import adam as AD
from oracle import attributes as A
from oracle import binsort as B
from oracle import confidence as CF
from oracle import csi as CS
from oracle import densify as DN
from oracle import emission as E
from oracle import projection as P
from oracle import render as R
from oracle import spectrum_loss as S


def _plant_in_renderer(tmp_path, monkeypatch, old, new):
    src = open(R._SRC).read()
    assert src.count(old) >= 1, "the line to plant the mistake in is gone"
    planted = tmp_path / "render_oracle_planted.c"
    planted.write_text(src.replace(old, new))
    monkeypatch.setattr(R, "_SRC", str(planted))
    monkeypatch.setattr(R, "_LIB", str(tmp_path / "liboracle_planted.so"))
    monkeypatch.setattr(R, "_lib", None)


@pytest.mark.parametrize("old,new,pin", [
    # the delay phase with the wrong sign (forward and backward alike)
    ("double psi = phi0[i] - 2.0 * ORC_PI", "double psi = phi0[i] + 2.0 * ORC_PI",
     lambda: TR.test_subcarrier_ratio_single_gaussian(R)),
    # no azimuth wrap: footprints stop at the seam
    ("return d - (double)W * floor(d / (double)W + 0.5);", "return d;",
     lambda: TR.test_zenith_rotation_shifts_columns(R)),
    # the backward without the suffix term of d/d alpha
    ("- suffix / (1.0 - h->alpha)", "",
     lambda: TG.test_render_gradient_vs_central_differences(R, False)),
])
def test_planted_renderer_mistake_fails_its_pin(tmp_path, monkeypatch, old, new, pin):
    _plant_in_renderer(tmp_path, monkeypatch, old, new)
    with pytest.raises(AssertionError):
        pin()


def test_planted_dilation_mistake_fails_its_pin(monkeypatch):
    monkeypatch.setattr(P, "DILATION", 0.0)
    with pytest.raises(AssertionError):
        TP.test_isotropic_closed_form_random_directions(90, 360)


def test_planted_network_input_mistake_fails_its_pin(monkeypatch):
    orig = A.mlp_outputs
    monkeypatch.setattr(A, "mlp_outputs",
                        lambda tx, latent, logd, *w: orig(tx, latent, torch.zeros_like(logd), *w))
    with pytest.raises(AssertionError):
        TA.test_log_distance_feature_wiring()


def test_planted_emission_mistake_fails_its_pin(monkeypatch):
    orig = E.network
    monkeypatch.setattr(E, "network", lambda flat, hidden, tx: orig(flat, hidden, tx) - E.unpack(flat, hidden)[3])
    with pytest.raises(AssertionError):
        TE.test_zero_output_weights_closed_form()


def test_planted_ssim_padding_mistake_fails_its_pin(monkeypatch):
    def replicate(img):
        w = torch.tensor(S.window_2d(), dtype=torch.float64).reshape(1, 1, S.WINDOW, S.WINDOW)
        r = S.WINDOW // 2
        x = torch.nn.functional.pad(img.unsqueeze(1), (r, r, r, r), mode="replicate")
        return torch.nn.functional.conv2d(x, w).squeeze(1)

    monkeypatch.setattr(S, "_filter", replicate)
    with pytest.raises(AssertionError):
        TS.test_ssim_map_against_brute_force()


def test_planted_adam_bias_correction_mistake_fails_its_pin(monkeypatch):
    orig = AD.adam_step
    # no bias correction: 1 - b^t taken as 1
    monkeypatch.setattr(AD, "adam_step", lambda p, g, m, v, t, lr, **k: orig(p, g, m, v, 10 ** 9, lr, **k))
    with pytest.raises(AssertionError):
        TAD.test_adam_matches_torch_fp64()


def test_planted_pixel_centre_mistake_fails_its_pin(monkeypatch):
    orig = B.footprint_tiles

    def integer_centres(rec, H, W):
        shifted = np.array(rec, dtype=np.float32, copy=True)
        shifted[:, :2] += np.float32(0.5)     # pixel centres at (x, y) instead of (x + 0.5, y + 0.5)
        return orig(shifted, H, W)

    monkeypatch.setattr(B, "footprint_tiles", integer_centres)
    with pytest.raises(AssertionError):
        TB.test_footprint_matches_pixel_bruteforce()


def test_planted_csi_mean_mistake_fails_its_pin(monkeypatch):
    orig = CS.csi_head
    # the spatial sum instead of the mean of Eq. 2
    monkeypatch.setattr(CS, "csi_head", lambda z, H, W: orig(z, H, W) * (H * W))
    with pytest.raises(AssertionError):
        TC.test_csi_head_closed_forms()


def test_planted_confidence_offset_mistake_fails_its_pin(monkeypatch):
    # C = exp(g) without the offset that keeps it above 1
    monkeypatch.setattr(CF, "confidence", lambda pos, w: torch.exp(CF.network(pos, *w)))
    with pytest.raises(AssertionError):
        TCF.test_confidence_exceeds_one()


def _patched_module(monkeypatch, mod, old, new):
    """A copy of an oracle module with one line changed, loaded as a sibling in the package."""
    import sys
    import types

    src = open(mod.__file__).read()
    assert src.count(old) == 1, "the line to plant the mistake in is gone"
    planted = types.ModuleType(mod.__name__ + "_planted")
    planted.__package__ = "oracle"
    planted.__file__ = mod.__file__
    monkeypatch.setitem(sys.modules, planted.__name__, planted)
    exec(compile(src.replace(old, new), mod.__file__, "exec"), planted.__dict__)
    return planted


@pytest.mark.parametrize("old,new,pin", [
    # children scaled by 1/N instead of 1/(0.8 N)
    ("math.log(0.8 * th.n_split)", "math.log(th.n_split)", lambda: TD.test_split_scale_rule(2)),
    # children offset by diag(s) R xi instead of R diag(s) xi
    ("R[i] @ (scale[i] * xi[i, c])", "scale[i] * (R[i] @ xi[i, c])",
     TD.test_split_children_at_mahalanobis_distance_xi),
])
def test_planted_densify_mistake_fails_its_pin(monkeypatch, old, new, pin):
    monkeypatch.setattr(TD, "D", _patched_module(monkeypatch, DN, old, new))
    with pytest.raises(AssertionError):
        pin()


@pytest.mark.parametrize("old,new,pin", [
    # the azimuth and elevation scales of the Jacobian swapped (equal on the W = 4H grids)
    ("    sx = W / (2.0 * math.pi)\n    sy = 2.0 * H / math.pi\n", "    sy = W / (2.0 * math.pi)\n    sx = 2.0 * H / math.pi\n",
     lambda: TP.test_jacobian_matches_central_differences(60, 100)),
])
def test_planted_projection_scale_mistake_fails_its_pin(monkeypatch, old, new, pin):
    monkeypatch.setattr(TP, "P", _patched_module(monkeypatch, P, old, new))
    with pytest.raises(AssertionError):
        pin()


def test_planted_spectrum_loss_weight_mistake_fails_its_pin(monkeypatch):
    # the weights of L1 and SSIM in Eq. 4 exchanged
    monkeypatch.setattr(TS, "S", _patched_module(monkeypatch, S, "    return (1.0 - lam) * l1 + lam * (1.0 - ssim)",
                                                 "    return lam * l1 + (1.0 - lam) * (1.0 - ssim)"))
    with pytest.raises(AssertionError):
        TS.test_l1_part_by_hand()


def test_planted_attribute_output_order_mistake_fails_its_pin(monkeypatch):
    # phase and opacity read from each other's network output
    monkeypatch.setattr(TA, "A", _patched_module(
        monkeypatch, A, "    phi0 = o[:, 1]\n    sigma = torch.sigmoid(opacity_logit + o[:, 2])",
        "    phi0 = o[:, 2]\n    sigma = torch.sigmoid(opacity_logit + o[:, 1])"))
    with pytest.raises(AssertionError):
        TA.test_constant_network_closed_form()


def test_planted_channel_loss_gradient_mistake_fails_its_pin(monkeypatch):
    # the derivative of the squared error without its factor 2
    monkeypatch.setattr(TC, "C", _patched_module(monkeypatch, CS, "    return loss, 2.0 * d / m",
                                                 "    return loss, d / m"))
    with pytest.raises(AssertionError):
        TC.test_channel_loss_closed_forms_and_gradient()


def test_planted_tie_order_mistake_fails_its_pin(monkeypatch):
    # equal distances ordered by descending Gaussian index
    monkeypatch.setattr(TB, "B", _patched_module(
        monkeypatch, B, '    order = np.argsort(keys, kind="stable")',
        '    keys, vals = keys[::-1], vals[::-1]\n    order = np.argsort(keys, kind="stable")'))
    with pytest.raises(AssertionError):
        TB.test_ties_keep_index_order()
