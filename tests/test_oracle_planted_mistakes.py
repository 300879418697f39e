"""Planted mistakes: a copy of the oracle with one deliberate error must fail the pin that guards
that part, so that the pins are not vacuous.  Every mistake is planted in the oracle, on the
CPU: a patched copy of the C renderer compiled into a temporary library, or a monkeypatched
Python function; the real oracle is restored afterwards."""
import pytest
import torch

import test_oracle_attributes as TA
import test_oracle_emission as TE
import test_oracle_grad as TG
import test_oracle_projection as TP
import test_oracle_render as TR
import test_oracle_spectrum_loss as TS
from oracle import attributes as A
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
        TP.test_isotropic_closed_form_random_directions()


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
