"""Pins of the oracle's adaptive density control (Algorithm 1, densification branch): the
schedule and statistics worked by hand, identity when nothing qualifies, clones worked by hand,
split children placed by an independent rotation (scipy) and at Mahalanobis distance |xi| from
the parent, the 0.8 N scale rule, the pruning boundaries, the opacity reset and the output count
on a random scene."""
import math

import numpy as np
import pytest
import torch

from oracle import densify as D
from oracle import projection as PR


def _set(n, seed, log_scale=-1.5):
    rng = np.random.default_rng(seed)
    q = rng.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return {"means": rng.uniform(-5, 5, size=(n, 3)), "log_scales": log_scale + 0.5 * rng.normal(size=(n, 3)),
            "quats": q, "opacity_logit": rng.normal(size=n), "payload": rng.normal(size=(n, 5))}


def test_schedule_by_hand():
    th = D.Thresholds(densify_every=100, reset_every=300, densify_until=1000)
    assert D.schedule(1, th) == (True, False, False)
    assert D.schedule(100, th) == (True, True, False)
    assert D.schedule(300, th) == (True, True, True)
    assert D.schedule(999, th) == (True, False, False)
    assert D.schedule(1000, th) == (False, False, False)


def test_statistics_and_decision_by_hand():
    t = 2.0 ** -12       # tau_grad; the gradients below are exact in binary
    s, c = np.zeros(4), np.zeros(4, dtype=np.int64)
    s, c = D.accumulate(s, c, [[3, 4, 0], [0, 0, t / 2], [1, 0, 0], [5, 5, 5]], [True, True, True, False])
    s, c = D.accumulate(s, c, [[0, 0, 0], [0, 1.5 * t, 0], [1, 0, 0], [5, 5, 5]], [True, True, False, False])
    assert list(s) == [5.0, 2 * t, 1.0, 0.0] and list(c) == [2, 2, 1, 0]
    th = D.Thresholds(tau_grad=t, eps=0.01, r_scene=10.0)
    ls = np.log(np.array([[0.05, 0.099, 0.09], [0.2, 0.05, 0.05], [0.1, 0.1, 0.101], [0.01, 0.01, 0.01]]))
    # means 2.5, exactly tau (a candidate), 1.0, never visible; the small/large cut is eps r_scene = 0.1
    assert list(D.decide(s, c, ls, th)) == [1, 2, 2, 0]


def test_nothing_qualifies_is_the_identity():
    g = _set(50, 1)
    th = D.Thresholds(sigma_min=0.0, r_max=math.inf)
    out, parent = D.densify_and_prune(g, np.full(50, 7.0), np.zeros(50, dtype=int), np.zeros((50, 2, 3)), th)
    assert list(parent) == list(range(50))
    for k in g:
        assert np.array_equal(out[k], g[k]), k


def test_clone_by_hand():
    g = _set(3, 2)
    g["opacity_logit"][:] = 0.0
    out, parent = D.densify_and_prune(g, np.zeros(3), np.array([0, 1, 0]), np.zeros((3, 2, 3)), D.Thresholds())
    assert list(parent) == [0, 1, 1, 2]
    for k in g:
        assert np.array_equal(out[k][[0, 1, 3]], g[k]) and np.array_equal(out[k][2], g[k][1]), k


def test_split_children_against_an_independent_rotation():
    """Child = mu + R diag(s) xi with R from scipy's rotation of the same quaternion."""
    Rot = pytest.importorskip("scipy.spatial.transform").Rotation
    g = _set(6, 3, log_scale=0.0)
    g["opacity_logit"][:] = 1.0
    act = np.array([2, 0, 2, 2, 0, 2])
    th = D.Thresholds(n_split=3)
    xi = np.random.default_rng(4).normal(size=(6, 3, 3))
    out, parent = D.densify_and_prune(g, np.zeros(6), act, xi, th)
    assert list(parent) == [0, 0, 0, 1, 2, 2, 2, 3, 3, 3, 4, 5, 5, 5]
    for i in np.flatnonzero(act == 2):
        w, x, y, z = g["quats"][i]
        R = Rot.from_quat([x, y, z, w]).as_matrix()
        rows = np.flatnonzero(parent == i)
        for c, j in enumerate(rows):
            expect = g["means"][i] + R @ (np.exp(g["log_scales"][i]) * xi[i, c])
            assert np.allclose(out["means"][j], expect, rtol=0, atol=1e-12)
            for key in ("quats", "opacity_logit", "payload"):
                assert np.array_equal(out[key][j], g[key][i])


def test_split_children_at_mahalanobis_distance_xi():
    """(c - mu)^T Sigma^-1 (c - mu) = |xi|^2 with Sigma = R S^2 R^T of the parent."""
    g = _set(20, 5, log_scale=-0.5)
    act = np.full(20, 2)
    xi = np.random.default_rng(6).normal(size=(20, 2, 3))
    th = D.Thresholds(sigma_min=0.0)
    out, parent = D.densify_and_prune(g, np.zeros(20), act, xi, th)
    Sig = PR.covariance3d(torch.tensor(g["log_scales"]), torch.tensor(g["quats"])).numpy()
    for j in range(out["means"].shape[0]):
        i = parent[j]
        d = out["means"][j] - g["means"][i]
        m2 = d @ np.linalg.solve(Sig[i], d)
        assert abs(m2 - float(xi[i, j - 2 * i] @ xi[i, j - 2 * i])) <= 1e-9 * max(1.0, m2)


@pytest.mark.parametrize("n_split", [2, 3, 4])
def test_split_scale_rule(n_split):
    """Children's per-axis scales are the parent's divided by 0.8 N; with xi = 0 they sit on the
    parent's mean."""
    g = _set(4, 7)
    g["opacity_logit"][:] = 0.0
    out, parent = D.densify_and_prune(g, np.zeros(4), np.array([0, 2, 0, 0]), np.zeros((4, n_split, 3)),
                                      D.Thresholds(n_split=n_split))
    rows = np.flatnonzero(parent == 1)
    assert len(rows) == n_split and out["means"].shape[0] == 3 + n_split
    for j in rows:
        assert np.allclose(np.exp(out["log_scales"][j]) * 0.8 * n_split, np.exp(g["log_scales"][1]),
                           rtol=1e-14, atol=0)
        assert np.array_equal(out["means"][j], g["means"][1])


def test_pruning_boundaries():
    """Opacity strictly below sigma_min and radius strictly above r_max go; clones and children
    of a too-wide parent stay (they have no footprint yet), the parent itself goes."""
    g = _set(6, 8)
    smin = 0.005
    lg = math.log(smin / (1 - smin))
    g["opacity_logit"][:] = [lg - 1e-6, lg + 1e-6, 2.0, 2.0, 2.0, lg - 1.0]
    radius = np.array([0.0, 0.0, 20.0, 20.0 + 1e-9, 25.0, 0.0])
    act = np.array([0, 0, 0, 0, 1, 1])
    out, parent = D.densify_and_prune(g, radius, act, np.zeros((6, 2, 3)), D.Thresholds(sigma_min=smin, r_max=20.0))
    # 0 faint; 1 kept; 2 at r_max kept; 3 wide; 4 wide but its clone stays; 5 and its clone faint
    assert list(parent) == [1, 2, 4]
    assert np.array_equal(out["means"][2], g["means"][4])


def test_opacity_reset():
    lg = np.linspace(-9.0, 9.0, 37)
    sig = 1.0 / (1.0 + np.exp(-lg))
    new = 1.0 / (1.0 + np.exp(-D.reset_opacity(lg)))
    assert np.allclose(new, np.minimum(sig, 0.01), rtol=1e-14, atol=0)
    assert np.array_equal(D.reset_opacity(lg)[lg < -5.0], lg[lg < -5.0])


def test_output_count_on_a_random_scene():
    n = 400
    g = _set(n, 9)
    rng = np.random.default_rng(10)
    s, c = D.accumulate(np.zeros(n), np.zeros(n, dtype=np.int64), rng.normal(scale=3e-4, size=(n, 3)),
                        rng.uniform(size=n) < 0.9)
    th = D.Thresholds(r_scene=22.0, r_max=15.0)
    act = D.decide(s, c, g["log_scales"], th)
    assert (act == 1).any() and (act == 2).any() and (act == 0).any()
    radius = rng.uniform(0.0, 20.0, size=n)
    xi = rng.normal(size=(n, th.n_split, 3))
    out, parent = D.densify_and_prune(g, radius, act, xi, th)
    sig = 1.0 / (1.0 + np.exp(-g["opacity_logit"]))
    faint = sig < th.sigma_min
    wide = radius > th.r_max
    expect = int(((act == 0) & ~faint & ~wide).sum() + ((act == 1) & ~faint & ~wide).sum()
                 + ((act == 1) & ~faint).sum() + th.n_split * ((act == 2) & ~faint).sum())
    assert out["means"].shape[0] == expect == parent.shape[0]
    assert np.all(np.diff(parent) >= 0)
