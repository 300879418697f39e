"""Pins for the oracle's projection (Sec. 4.2 map and Sigma' = J V Sigma V^T J^T)."""
import math
import os

import numpy as np
import pytest
import torch

from oracle import projection as P
from paper_2511_22793_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    rows = []
    for line in open(os.path.join(GOLD, name)):
        line = line.split("#")[0].strip()
        if line:
            rows.append([float(v) for v in line.split()])
    return np.array(rows)


def _view(H=90, W=360, rx=(0.0, 0.0, 0.0), V=None):
    v = synth.View(H=H, W=W, rx=rx)
    if V is not None:
        v.V = tuple(np.asarray(V, dtype=np.float64).reshape(-1).tolist())
    return v


def test_map_cardinal_directions_golden():
    g = _load("equirect_cardinal.txt")
    xp = torch.tensor(g[:, 0:3], dtype=torch.float64)
    px, py, r = P.equirect_map(xp, 90, 360)
    np.testing.assert_allclose(px.numpy(), g[:, 3], rtol=0, atol=1e-12)
    np.testing.assert_allclose(py.numpy(), g[:, 4], rtol=0, atol=1e-12)


def test_isotropic_footprint_golden():
    g = _load("isotropic_footprint.txt")
    means = torch.tensor(g[:, 0:3], dtype=torch.float64)
    ls = torch.log(torch.tensor(g[:, 3:4], dtype=torch.float64)).expand(-1, 3).contiguous()
    q = torch.tensor([[1.0, 0.0, 0.0, 0.0]] * len(g), dtype=torch.float64)
    out = P.project(means, ls, q, _view())
    np.testing.assert_allclose(out["sxx"].numpy(), g[:, 4], rtol=1e-13)
    np.testing.assert_allclose(out["sxy"].numpy(), g[:, 5], atol=1e-12)
    np.testing.assert_allclose(out["syy"].numpy(), g[:, 6], rtol=1e-13)


@pytest.mark.parametrize("H,W", [(90, 360), (60, 100)])
def test_isotropic_closed_form_random_directions(H, W):
    """Sigma' = diag(s^2 s_x^2/rho^2, s^2 s_y^2/r^2) + 0.3 I for any direction
    and any rotation quaternion (an isotropic Sigma ignores the rotation).  With W = 4H (the
    1-degree grids) s_x = s_y; the 60 x 100 grid tells the two scales apart."""
    rng = np.random.default_rng(11)
    n = 200
    means = rng.uniform(-5, 5, (n, 3))
    means[:, 1] = rng.uniform(0.2, 5, n)
    s = np.exp(rng.normal(-1.5, 0.5, n))
    ls = np.log(s)[:, None].repeat(3, 1)
    q = rng.normal(size=(n, 4))
    out = P.project(torch.tensor(means), torch.tensor(ls), torch.tensor(q), _view(H, W))
    x, y, z = means.T
    rho2 = x * x + z * z
    r2 = rho2 + y * y
    sx, sy = W / (2 * math.pi), 2 * H / math.pi
    np.testing.assert_allclose(out["sxx"].numpy(), s * s * sx * sx / rho2 + 0.3, rtol=1e-11)
    np.testing.assert_allclose(out["syy"].numpy(), s * s * sy * sy / r2 + 0.3, rtol=1e-11)
    np.testing.assert_allclose(out["sxy"].numpy(), 0.0, atol=1e-9 * (s * s * sx * sy).max())


@pytest.mark.parametrize("H,W", [(90, 360), (60, 100)])
def test_jacobian_matches_central_differences(H, W):
    rng = np.random.default_rng(12)
    xp = rng.uniform(-5, 5, (64, 3))
    xp[:, 1] = rng.uniform(0.1, 5, 64)
    J = P.map_jacobian(torch.tensor(xp), H, W).numpy()
    h = 1e-6
    for c in range(3):
        e = np.zeros(3)
        e[c] = h
        pp = P.equirect_map(torch.tensor(xp + e), H, W)
        pm = P.equirect_map(torch.tensor(xp - e), H, W)
        dpx = (pp[0] - pm[0]).numpy() / (2 * h)
        dpy = (pp[1] - pm[1]).numpy() / (2 * h)
        np.testing.assert_allclose(J[:, 0, c], dpx, rtol=1e-6, atol=1e-6)
        np.testing.assert_allclose(J[:, 1, c], dpy, rtol=1e-6, atol=1e-6)


def test_rotation_matches_scipy():
    Rot = pytest.importorskip("scipy.spatial.transform").Rotation
    rng = np.random.default_rng(13)
    q = rng.normal(size=(100, 4))
    R = P.quat_to_rotmat(torch.tensor(q)).numpy()
    ref = Rot.from_quat(q[:, [1, 2, 3, 0]]).as_matrix()   # scipy takes (x, y, z, w)
    np.testing.assert_allclose(R, ref, atol=1e-13)


def test_covariance_spectrum_is_scales_squared():
    rng = np.random.default_rng(14)
    ls = rng.normal(-1.5, 0.5, (50, 3))
    q = rng.normal(size=(50, 4))
    S = P.covariance3d(torch.tensor(ls), torch.tensor(q)).numpy()
    ev = np.sort(np.linalg.eigvalsh(S), axis=1)
    np.testing.assert_allclose(ev, np.sort(np.exp(2 * ls), axis=1), rtol=1e-10)


def test_view_rotation_consistency():
    """Rotating the world and the view matrix together leaves every output unchanged;
    a receiver offset is the same as shifting the scene."""
    sc = synth.make_scene(128, seed=21)
    Rot = pytest.importorskip("scipy.spatial.transform").Rotation
    Q = Rot.from_euler("xyz", [0.3, -1.1, 0.7]).as_matrix()
    rx = np.array([0.4, -0.2, 0.9])
    base = P.project(torch.tensor(sc.means, dtype=torch.float64) - torch.tensor(rx),
                     torch.tensor(sc.log_scales, dtype=torch.float64),
                     torch.tensor(sc.quats, dtype=torch.float64), _view())
    # world' = Q world; quaternion of Q composed with each Gaussian's rotation
    qQ = Rot.from_matrix(Q).as_quat()   # x, y, z, w
    qg = Rot.from_quat(sc.quats.astype(np.float64)[:, [1, 2, 3, 0]])
    qnew = (Rot.from_quat(qQ) * qg).as_quat()[:, [3, 0, 1, 2]]
    means2 = sc.means.astype(np.float64) @ Q.T
    rx2 = Q @ rx
    out = P.project(torch.tensor(means2), torch.tensor(sc.log_scales, dtype=torch.float64),
                    torch.tensor(qnew), _view(rx=tuple(rx2), V=Q.T))
    for k in ("px", "py", "sxx", "sxy", "syy", "r"):
        np.testing.assert_allclose(out[k].numpy(), base[k].numpy(), rtol=1e-9, atol=1e-9)


def test_zenith_quarter_turn_shifts_azimuth():
    """Rotating the scene by +90 degrees about the vertical axis adds W/4 to p_x (mod W)
    and leaves p_y and the footprint's size unchanged."""
    sc = synth.make_scene(256, seed=22)
    m = sc.means.astype(np.float64)
    # atan2(x, z) + pi/2 = atan2(z, -x): new point (x, y, z) -> (z, y, -x)
    m2 = np.stack([m[:, 2], m[:, 1], -m[:, 0]], 1)
    Rot = pytest.importorskip("scipy.spatial.transform").Rotation
    R90 = Rot.from_euler("y", 90, degrees=True)
    assert np.allclose(R90.apply(m), m2, atol=1e-12)
    q2 = (R90 * Rot.from_quat(sc.quats.astype(np.float64)[:, [1, 2, 3, 0]])).as_quat()[:, [3, 0, 1, 2]]
    ls = torch.tensor(sc.log_scales, dtype=torch.float64)
    a = P.project(torch.tensor(m), ls, torch.tensor(sc.quats, dtype=torch.float64), _view())
    b = P.project(torch.tensor(m2), ls, torch.tensor(q2), _view())
    d = (b["px"] - a["px"]).numpy() - 90.0
    d = d - 360.0 * np.round(d / 360.0)
    np.testing.assert_allclose(d, 0.0, atol=1e-9)
    for k in ("py", "sxx", "sxy", "syy", "r"):
        np.testing.assert_allclose(b[k].numpy(), a[k].numpy(), rtol=1e-9, atol=1e-9)


def test_cull_and_extents():
    means = torch.tensor([[0.0, 0.05, 0.05], [0.0, 0.0, 3.0]], dtype=torch.float64)
    ls = torch.full((2, 3), math.log(0.1), dtype=torch.float64)
    q = torch.tensor([[1.0, 0, 0, 0]] * 2, dtype=torch.float64)
    out = P.project(means, ls, q, _view())
    assert not bool(out["valid"][0]) and bool(out["valid"][1])
    np.testing.assert_allclose(out["ext_x"][1].item(), math.sqrt(P.Q_MAX * out["sxx"][1].item()))
    # at the bounding box's x extent the kernel equals 1/255 along the principal axis
    qv = out["ext_x"][1] ** 2 * out["cxx"][1]
    np.testing.assert_allclose(math.exp(-0.5 * qv.item()), 1 / 255.0, rtol=1e-12)


def test_zenith_footprint_closed_form():
    """Exactly at the zenith (x' = z' = 0) the azimuth row of J is (s_x / (1e-3 r), 0, 0)
    and the elevation row (0, 0, -s_y / r), so for an isotropic Gaussian
    Sigma' = diag(s^2 s_x^2 / (1e-3 r)^2, s^2 s_y^2 / r^2) + 0.3 I: the footprint spans
    every azimuth column."""
    r, s = 3.0, 0.2
    out = P.project(torch.tensor([[0.0, r, 0.0]], dtype=torch.float64),
                    torch.full((1, 3), math.log(s), dtype=torch.float64),
                    torch.tensor([[1.0, 0, 0, 0]], dtype=torch.float64), _view())
    sx = sy = 180.0 / math.pi
    np.testing.assert_allclose(out["sxx"].item(), s * s * sx * sx / (1e-3 * r) ** 2 + 0.3, rtol=1e-12)
    np.testing.assert_allclose(out["syy"].item(), s * s * sy * sy / r ** 2 + 0.3, rtol=1e-12)
    assert abs(out["sxy"].item()) < 1e-9
    assert out["ext_x"].item() > 180.0
    np.testing.assert_allclose(out["py"].item(), 90.0, rtol=1e-14)


def test_jacobian_cap_continuous_at_threshold():
    """Just outside the cap the azimuth row is the exact 1/rho; inside it is capped
    at 1/(1e-3 r) with the same direction: the row's norm is continuous at rho = 1e-3 r."""
    r = 2.0
    rhos = np.array([0.5e-3, 0.999e-3, 1.0e-3, 1.001e-3, 2e-3]) * r
    ang = 0.7
    xp = np.stack([rhos * math.sin(ang), np.sqrt(r * r - rhos ** 2), rhos * math.cos(ang)], 1)
    J = P.map_jacobian(torch.tensor(xp), 90, 360).numpy()
    sx = 180.0 / math.pi
    expect = sx / np.maximum(rhos, 1e-3 * r)
    np.testing.assert_allclose(np.linalg.norm(J[:, 0, :], axis=1), expect, rtol=1e-12)
    np.testing.assert_allclose(J[:, 0, 0] / np.linalg.norm(J[:, 0, :], axis=1), math.cos(ang), rtol=1e-12)
