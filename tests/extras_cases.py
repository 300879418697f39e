"""Seeded cases and FP64 oracle results shared by the host-shim and GPU tests of the training
extras (the confidence objective of Eq. 5, adaptive density control)."""
import math

import numpy as np
import torch

from oracle import confidence as CF


def conf_case(B, hidden, seed):
    rng = np.random.default_rng(seed)
    pos = rng.uniform(-5, 5, size=(B, 3)).astype(np.float32)
    L = rng.uniform(0.01, 0.6, size=B).astype(np.float32)
    w = np.concatenate([rng.normal(size=3 * hidden) / math.sqrt(3) * 0.5, 0.3 * rng.normal(size=hidden),
                        rng.normal(size=hidden) / math.sqrt(hidden), [0.1]]).astype(np.float32)
    return pos, L, w


def conf_oracle(pos, L, w, hidden, alpha=0.3):
    h = hidden
    t = [torch.tensor(w[0:3 * h].reshape(3, h).astype(np.float64), requires_grad=True),
         torch.tensor(w[3 * h:4 * h].astype(np.float64), requires_grad=True),
         torch.tensor(w[4 * h:5 * h].reshape(h, 1).astype(np.float64), requires_grad=True),
         torch.tensor(w[5 * h:5 * h + 1].astype(np.float64), requires_grad=True)]
    P = torch.tensor(pos.astype(np.float64))
    Lt = torch.tensor(L.astype(np.float64), requires_grad=True)
    obj = CF.objective(P, t, Lt, alpha=alpha)
    grads = torch.autograd.grad(obj, t + [Lt])
    C = CF.confidence(P, [x.detach() for x in t])
    dw = np.concatenate([g.reshape(-1).numpy() for g in grads[:4]])
    pre = (P @ t[0] + t[1]).detach().numpy()
    return float(obj.detach()), C.numpy(), grads[4].numpy(), dw, np.abs(pre).min()


TAU = 2.0 ** -12            # exact in FP32 and FP64
EPS, R_SCENE = 0.01, 20.0   # clone_scale 0.2 m
SIGMA_MIN, R_MAX = 0.005, 20.0


def dens_case(N, P, n_split, seed, margin=1e-4):
    """Seeded Gaussians with a mix of keep / clone / split / faint / wide / culled / never-visible
    entries; every FP32 decision at least `margin` (relative) away from its threshold, so that FP32
    and FP64 take the same decisions."""
    from oracle import densify as D

    rng = np.random.default_rng(seed)
    c = {}
    c["means"] = rng.uniform(-5, 5, size=(N, 3)).astype(np.float32)
    c["log_scales"] = rng.normal(-1.6, 0.5, size=(N, 3)).astype(np.float32)
    c["quats"] = rng.normal(size=(N, 4)).astype(np.float32)
    c["opacity_logit"] = rng.normal(-1.0, 2.5, size=N).astype(np.float32)
    c["payload"] = rng.normal(size=(N, P)).astype(np.float32)
    proj = rng.normal(size=(N, 8)).astype(np.float32)
    proj[:, 2:4] = rng.uniform(0.5, 30.0, size=(N, 2))
    culled = rng.uniform(size=N) < 0.05
    proj[culled, 2:4] = -1.0
    c["proj"] = proj
    count = rng.integers(0, 5, size=N).astype(np.uint32)
    avg = TAU * np.exp(rng.normal(0.0, 0.7, size=N))
    c["norm_sum"] = (avg * count).astype(np.float32)
    c["count"] = count
    c["xi"] = rng.normal(size=(N, n_split, 3)).astype(np.float32)
    c["d_means"] = (1e-3 * rng.normal(size=(N, 3))).astype(np.float32)
    # move the few entries that fall within `margin` of a threshold away from it, then check
    for _ in range(2):
        ns, cnt = c["norm_sum"].astype(np.float64), count.astype(np.float64)
        a = np.where(count > 0, ns / np.maximum(cnt, 1), 10.0)
        smax = np.exp(c["log_scales"].astype(np.float64).max(axis=1))
        sig = 1.0 / (1.0 + np.exp(-c["opacity_logit"].astype(np.float64)))
        rad = proj[:, 2:4].astype(np.float64).max(axis=1)
        near = [np.abs(a / TAU - 1) <= margin, np.abs(smax / (EPS * R_SCENE) - 1) <= margin,
                np.abs(sig / SIGMA_MIN - 1) <= margin, np.abs(rad - R_MAX) <= margin]
        c["norm_sum"][near[0]] *= np.float32(1.01)
        c["log_scales"][near[1]] += np.float32(0.01)
        c["opacity_logit"][near[2]] += np.float32(0.05)
        proj[near[3], 2:4] += np.float32(0.5)
    assert not any(m.any() for m in near), "seed %d: a decision within %g of its threshold" % (seed, margin)
    th = D.Thresholds(tau_grad=TAU, eps=EPS, r_scene=R_SCENE, n_split=n_split, sigma_min=SIGMA_MIN, r_max=R_MAX)
    return c, th


def dens_oracle(c, th):
    """The oracle's accumulate, decide, densify-and-prune and reset on the case's FP32 values."""
    from oracle import densify as D

    f64 = {k: np.asarray(v, dtype=np.float64) for k, v in c.items() if k != "count"}
    radius = f64["proj"][:, 2:4].max(axis=1)
    acc_norm, acc_count = D.accumulate(f64["norm_sum"], c["count"].astype(np.int64), f64["d_means"], radius > 0)
    action = D.decide(f64["norm_sum"], c["count"].astype(np.int64), f64["log_scales"], th)
    g = {k: f64[k] for k in ("means", "log_scales", "quats", "opacity_logit", "payload")}
    out, parent = D.densify_and_prune(g, radius, action, f64["xi"], th)
    reset = D.reset_opacity(f64["opacity_logit"])
    return dict(out=out, parent=parent, action=action, acc_norm=acc_norm, acc_count=acc_count, reset=reset)


def dens_check(res, o, c, cap):
    """GPU (or host-shim) densification result against the oracle: the row count and parents
    bit-exact, kept and cloned rows exact copies, children's means within 2e-5 m and log-scales
    within 1e-6 of the oracle, rows past the capacity left alone, and the capacity status."""
    total = len(o["parent"])
    assert res["n_out"] == total
    assert res["status"] == (-5 if total > cap else 0)
    k = min(total, cap)
    par = o["parent"][:k]
    assert np.array_equal(res["parent"][:k], par)
    child = o["action"][par] == 2
    for key in ("quats", "opacity_logit", "payload"):
        assert np.array_equal(res[key][:k], c[key][par]), key
    assert np.array_equal(res["means"][:k][~child], c["means"][par[~child]])
    assert np.array_equal(res["log_scales"][:k][~child], c["log_scales"][par[~child]])
    assert np.allclose(res["means"][:k][child], o["out"]["means"][:k][child], rtol=0, atol=2e-5)
    assert np.allclose(res["log_scales"][:k][child], o["out"]["log_scales"][:k][child], rtol=0, atol=1e-6)
    if cap > k:
        assert np.all(res["parent"][k:] == 0xFFFFFFFF)


def accumulate_check(acc_norm, acc_count, o):
    assert np.array_equal(acc_count.astype(np.int64), o["acc_count"])
    assert np.allclose(acc_norm, o["acc_norm"], rtol=1e-6, atol=1e-12)


def reset_check(reset, o):
    assert np.allclose(reset, o["reset"], rtol=0, atol=1e-6)
    below = o["reset"] < np.log(0.01 / 0.99) - 1e-6
    assert np.array_equal(reset[below].astype(np.float64), o["reset"][below])
