"""Parity at the benchmarked sizes, against the FP64 oracle.

- The 50,000-Gaussian, 64-subcarrier, 360x90 training step, in both arithmetic forms of
  `step.TrainStep` (the object and the CUDA graph the benchmark times): its loss and the
  gradients of all eleven parameter tensors against the oracle's analytic FP64 gradient
  (Algorithm 1 Backprop), with an upstream gradient that is nonzero only on 512 seeded pixels
  so that the per-pixel oracle evaluates exactly those pixels.  The target equals the step's
  own spectrum everywhere else, so dL/dz is exactly zero there (asserted); the oracle takes the
  GPU's dL/dz on the sample as its seed.  Bound: 1e-3 relative L2 per tensor.
- Central finite differences of the same FP32 loss (evaluated in FP64 from the GPU's spectrum
  at the sampled pixels) on 32 sampled parameters against the GPU's analytic gradient.
- Served spectra (tensor-core server, split-BF16 network) for 256 and 1,024 subcarriers at
  720x180 over a 500,000-Gaussian resident scene, and a moving-receiver request, against the
  oracle on 256 sampled pixels each (the 1e-3 bound).
- One `train.Trainer.step` in both forms: its gradient buffers against `oracle.pipeline`
  and its Adam update against `oracle.adam` applied to the same gradient, over two steps.
"""
import math

import numpy as np
import pytest
import torch

from gpu_util import DEV, rel_l2, spectrum_to_complex
from oracle import adam as oadam
from oracle import pipeline as opl
from paper_2511_22793_gb300 import gsparc as G
from paper_2511_22793_gb300 import synth
from paper_2511_22793_gb300.pipeline import DeviceMLP, DeviceScene, Renderer
from paper_2511_22793_gb300.step import PARAM_NAMES, TrainStep

pytestmark = pytest.mark.gpu

H, W, K, N, HIDDEN = 90, 360, 64, 50_000, 32
NPIX = 512


def _c2(form):
    sc = synth.make_scene(N, seed=0)
    mlp = synth.make_mlp(HIDDEN, seed=3)
    tx = synth.make_tx(1, seed=2)
    r = Renderer(H, W, K, N, device=DEV)
    ds = DeviceScene.from_host(sc, DEV)
    dm = DeviceMLP.from_host(mlp, DEV)
    txd = torch.tensor(tx, device=DEV)
    target = torch.zeros((1, K, H, W, 2), device=DEV)
    st = TrainStep(r, ds, dm, txd, target, form=form)
    st.enqueue()                      # geometry and attributes of this form
    torch.cuda.synchronize()
    assert r.check() == 0
    # the step's own spectrum: the same forward kernel, spectrum stored
    z = st.spectrum(torch.empty_like(st.spec))
    torch.cuda.synchronize()
    zc = spectrum_to_complex(z)[0]                                 # [HW, K]
    rng = np.random.default_rng(512)
    lit = np.flatnonzero(np.abs(zc).sum(1) > 0)
    pix = np.sort(rng.choice(lit, NPIX, replace=False))
    scale = np.sqrt(np.mean(np.abs(zc[pix]) ** 2))
    delta = 0.3 * scale * (rng.normal(size=(NPIX, K)) + 1j * rng.normal(size=(NPIX, K)))
    tgt = zc.copy()
    tgt[pix] -= delta
    dev_t = np.stack([tgt.real, tgt.imag], -1).reshape(H, W, K, 2).transpose(2, 0, 1, 3)[None]
    target.copy_(torch.tensor(np.ascontiguousarray(dev_t), dtype=torch.float32))
    # the exact FP32 target the GPU sees, back in the oracle's layout
    t32 = spectrum_to_complex(target)[0]
    return dict(sc=sc, mlp=mlp, tx=tx, r=r, ds=ds, dm=dm, st=st, z=zc, pix=pix, t32=t32,
                view=synth.View(H=H, W=W), band=synth.Band(K=K))


def _oracle_grads(c, gz):
    """Oracle vector-Jacobian product of the whole chain (projection, network, compositing) with
    the GPU step's own upstream gradient gz = dL/dz [NPIX, K] on the sampled pixels: the oracle's
    loss_and_grad takes the mean squared error over its pixel subset, so the target is placed so
    that its upstream gradient is exactly gz.  (The oracle's own 2 (z - t) / M would differ from
    the GPU's wherever |z| is far above the sample's rms: Gaussians next to the transmitter have
    amplitudes ~1/d, and there the ~1e-5 spectrum difference is a percent of the seed.)  Returns
    the oracle's loss L = sum |z - t|^2 / (K H W) on the sample, its spectrum and gradient."""
    pix = c["pix"]
    fwd = opl.forward(c["sc"], c["mlp"], c["view"], c["band"], c["tx"], pixels=pix)
    z_or = fwd["z"][0]
    M, Msub = K * H * W, NPIX * K
    t_sub = z_or - gz * Msub / 2.0
    loss_sub, g = opl.loss_and_grad(c["sc"], c["mlp"], c["view"], c["band"], c["tx"], t_sub[None], pixels=pix)
    loss = float(np.sum(np.abs(z_or - c["t32"][pix]) ** 2) / M)
    return loss, z_or, g


@pytest.mark.parametrize("form", ["fp32", "tc"])
def test_c2_training_step_matches_oracle_on_sampled_pixels(form):
    c = _c2(form)
    st, r = c["st"], c["r"]
    graph = st.capture()
    for _ in range(2):
        graph.replay()
    torch.cuda.synchronize()
    assert r.check() == 0
    d = spectrum_to_complex(st.d_spec)[0]
    off = np.ones(H * W, bool)
    off[c["pix"]] = False
    assert np.all(d[off] == 0), "dL/dz nonzero outside the sampled pixels"
    assert np.count_nonzero(d[c["pix"]]) > 0.99 * NPIX * K
    loss_gpu = float(st.loss)
    loss_or, z_or, g_or = _oracle_grads(c, d[c["pix"]])
    assert rel_l2(c["z"][c["pix"]], z_or) <= 1e-3
    assert abs(loss_gpu - loss_or) <= 1e-3 * loss_or, (loss_gpu, loss_or)
    got = st.gradients()
    errs = {}
    for k in PARAM_NAMES:
        gk = got[k].detach().cpu().numpy().astype(np.float64)
        assert np.all(np.isfinite(gk)), k
        errs[k] = rel_l2(gk, g_or[k])
    print(form, {k: "%.2e" % v for k, v in errs.items()})
    for k, e in errs.items():
        assert e <= 1e-3, "%s: relative L2 %.3e (%s)" % (k, e, form)


def test_c2_finite_differences_through_gpu_loss():
    """FP32 form: the loss over the sampled pixels, formed in FP64 from the GPU's spectrum, is
    differenced at theta +- h for 32 parameters (h = 1e-3 max(1, |theta|), reduced to 1e-4 and
    1e-5 times that while the perturbation changes any composited set at the sampled pixels, as
    n_used and n_contrib show; a parameter for which even the smallest h does is resampled).  Each difference quotient is within 2e-2 of the analytic GPU gradient (relative),
    and their relative L2 over the 32 is within 5e-3.

    The 32 are drawn from the per-Gaussian tensors (means, log-scales, quaternions, opacity
    logits, latents; the latents reach the loss through the network).  A shared network weight
    moves every Gaussian's alpha at once, so at any h that rises above FP32 rounding some of the
    ~5e5 (pixel, Gaussian) pairs at the sampled pixels cross a cut-off and the loss jumps; the
    weights' gradients are compared with the oracle's analytic gradient (itself checked by
    finite differences on the CPU) in the test above."""
    c = _c2("fp32")
    st, r, pix = c["st"], c["r"], c["pix"]
    graph = st.capture()
    graph.replay()
    torch.cuda.synchronize()
    an = {k: v.detach().cpu().numpy().astype(np.float64) for k, v in st.gradients().items()}
    params = dict(zip(PARAM_NAMES, list(c["ds"].tensors()) + list(c["dm"].tensors())))
    t_pix = c["t32"][pix]
    M = K * H * W

    def loss_at():
        graph.replay()
        st.spectrum()
        torch.cuda.synchronize()
        zz = spectrum_to_complex(st.spec)[0][pix]
        nu = st.n_used.view(-1)[torch.as_tensor(pix, device=DEV)].cpu().numpy()
        ncn = st.nc.view(-1)[torch.as_tensor(pix, device=DEV)].cpu().numpy()
        return float(np.sum(np.abs(zz - t_pix) ** 2) / M), nu, ncn

    _, nu0, nc0 = loss_at()
    quota = {"means": 8, "log_scales": 6, "quats": 6, "opacity_logit": 6, "latent": 6}
    rng = np.random.default_rng(77)
    fd_all, an_all = [], []
    for k, q in quota.items():
        g = an[k].reshape(-1)
        cand = np.flatnonzero(np.abs(g) >= 0.1 * np.abs(g).max())
        rng.shuffle(cand)
        taken = 0
        for idx in cand:
            if taken == q:
                break
            flat = params[k].view(-1)
            x0 = float(flat[idx])
            fd = None
            for rel_h in (1e-3, 1e-4, 1e-5):
                h = rel_h * max(1.0, abs(x0))
                flat[idx] = x0 + h
                lp, nup, ncp = loss_at()
                flat[idx] = x0 - h
                lm, num, ncm = loss_at()
                flat[idx] = x0
                if (np.array_equal(nup, nu0) and np.array_equal(num, nu0) and np.array_equal(ncp, nc0)
                        and np.array_equal(ncm, nc0)):
                    # the perturbed values as stored in FP32
                    hp = float(np.float32(x0 + h)) - x0
                    hm = x0 - float(np.float32(x0 - h))
                    fd = (lp - lm) / (hp + hm)
                    break
            if fd is None:
                continue          # a cut-off or termination decision moves even at the smallest h
            fd_all.append(fd)
            an_all.append(g[idx])
            assert abs(fd - g[idx]) <= 2e-2 * abs(g[idx]), (k, int(idx), fd, g[idx])
            taken += 1
        assert taken == q, "%s: only %d smooth parameters" % (k, taken)
    loss_at()
    assert len(fd_all) == 32
    e = rel_l2(np.array(an_all), np.array(fd_all))
    print("FD relative L2 over 32 parameters: %.3e" % e)
    assert e <= 5e-3


def test_served_spectra_match_oracle_large_subcarrier_counts():
    """The tensor-core server at 720x180 with 256 and 1,024 subcarriers over a 500,000-Gaussian
    resident scene, and a moving-receiver request (rotated and displaced receiver, 256
    subcarriers): each served spectrum against the oracle on 256 seeded pixels <= 1e-3."""
    from oracle import attributes as oattr
    from oracle import projection as oproj
    from oracle import render as orender
    from paper_2511_22793_gb300.serve import Request, Server

    n = 500_000
    sc = synth.make_scene(n, seed=4)
    mlp = synth.make_mlp(32, seed=3)
    ds, dm = DeviceScene.from_host(sc, DEV), DeviceMLP.from_host(mlp, DEV)
    res = (180, 720)
    c, s = math.cos(0.7), math.sin(0.7)
    V = (c, 0.0, -s, 0.0, 1.0, 0.0, s, 0.0, c)
    rx_m = (0.6, 0.3, -0.4)
    txs = synth.make_tx(3, seed=44)
    reqs = [Request(0, tuple(map(float, txs[0])), res, 256), Request(1, tuple(map(float, txs[1])), res, 1024),
            Request(2, tuple(map(float, txs[2])), res, 256, rx=rx_m, V=V)]
    srv = Server(ds, dm, [res], mem_budget_bytes=24 << 30, max_batch=4, n_streams=3)
    srv.run(reqs, np.zeros(len(reqs)))
    torch.cuda.synchronize()
    assert all(not q.rejected for q in reqs)
    rng = np.random.default_rng(45)
    f64 = lambda a: torch.tensor(np.asarray(a), dtype=torch.float64)
    weights = [f64(a) for a in mlp.arrays()]
    for q in reqs:
        view = synth.View(H=res[0], W=res[1], rx=q.rx or (0.0, 0.0, 0.0),
                          V=q.V or (1.0, 0.0, 0.0, 0.0, 1.0, 0.0, 0.0, 0.0, 1.0))
        band = synth.Band(K=q.K)
        geo = oproj.project(f64(sc.means), f64(sc.log_scales), f64(sc.quats), view)
        g = {k: geo[k].numpy() for k in ("px", "py", "cxx", "cxy", "cyy", "r", "valid")}
        at = oattr.attributes(f64(sc.means), f64(sc.opacity_logit), f64(sc.latent), weights, f64(q.tx), view.rx)
        at = {k: at[k].numpy() for k in ("sigma", "a", "phi0", "L")}
        pix = np.sort(rng.choice(res[0] * res[1], 256, replace=False))
        z_or, _, n_or = orender.render_fwd(g, at, view.H, view.W, band.K, band.f_c, band.df, pixels=pix)
        z = spectrum_to_complex(q.spectrum[None])[0][pix]
        e = rel_l2(z, z_or)
        print("request %d (K=%d%s): relative L2 %.2e, composited per pixel %.0f" %
              (q.rid, q.K, ", moving" if q.rx else "", e, n_or.mean()))
        assert n_or.mean() > 10
        assert e <= 1e-3, (q.rid, e)


@pytest.mark.parametrize("tensor_cores", [False, True])
def test_trainer_step_matches_oracle_pipeline_and_adam(tensor_cores):
    from paper_2511_22793_gb300.train import LR, MLP_KEYS, SCENE_KEYS, Trainer

    Hh, Ww, Kk, n = 45, 180, 16, 3000
    gt = synth.make_scene(2000, seed=61)
    gt_mlp = synth.make_mlp(32, seed=62)
    train_tx = synth.make_tx(16, seed=63)
    tr = Trainer(n, gt, gt_mlp, train_tx, H=Hh, W=Ww, K=Kk, hidden=32, batch=2, total_steps=100,
                 device=DEV, seed=64, tensor_cores=tensor_cores)
    # start from a seeded scene with spread opacities rather than the flat initialisation, so
    # that the gradient reaches every kind of parameter
    init, init_mlp = synth.make_scene(n, seed=65), synth.make_mlp(32, seed=66)
    for k, a in zip(SCENE_KEYS, init.arrays()):
        tr.params[k].copy_(torch.tensor(a, device=DEV))
    for k, a in zip(MLP_KEYS, init_mlp.arrays()):
        tr.params[k].copy_(torch.tensor(a, device=DEV))
    view, band = synth.View(H=Hh, W=Ww), synth.Band(K=Kk)
    m = {k: np.zeros(p.shape) for k, p in tr.params.items()}
    v = {k: np.zeros(p.shape) for k, p in tr.params.items()}
    for step in (1, 2):
        theta0 = {k: p.detach().cpu().numpy().astype(np.float64) for k, p in tr.params.items()}
        tr.step()
        pos_lr = tr.pos_lr()          # the rate of this step (annealed with the step count)
        torch.cuda.synchronize()
        assert tr.r.check() == 0
        tx = tr.tx.cpu().numpy().astype(np.float64)
        tgt = spectrum_to_complex(tr.batch_target)
        sc0 = synth.Scene(*[theta0[k].astype(np.float32) for k in SCENE_KEYS])
        mlp0 = synth.MLPWeights(32, *[theta0[k].astype(np.float32) for k in MLP_KEYS])
        _, g_or = opl.loss_and_grad(sc0, mlp0, view, band, tx, tgt)
        g_gpu = {k: tr.grads[k].detach().cpu().numpy().astype(np.float64) for k in tr.params}
        for k in tr.params:
            e = rel_l2(g_gpu[k], g_or[k])
            assert e <= 5e-3, "step %d %s: gradient relative L2 %.3e" % (step, k, e)
        for k, p in tr.params.items():
            lr = pos_lr if k == "means" else LR[k]
            want, m[k], v[k] = oadam.adam_step(theta0[k], g_gpu[k], m[k], v[k], step, lr)
            got = p.detach().cpu().numpy().astype(np.float64)
            # the update is ~lr per element: FP32 rounding of theta and of the update; a gradient
            # whose square underflows FP32 (|g| < 1e-18) may take any update up to lr
            tiny = np.abs(g_gpu[k]) < 1e-18
            tol = 1e-6 * np.abs(theta0[k]) + np.where(tiny, 1.01 * lr, 1e-4 * lr)
            assert np.all(np.abs(got - want) <= tol), "step %d %s: Adam update" % (step, k)
            # (FP32 1 - b1 and 1 - b2 are 2.4e-7 and 1.3e-5 off their FP64 values, relative)
            assert np.allclose(tr.m[k].cpu().numpy(), m[k], rtol=1e-5, atol=1e-12), k
            assert np.allclose(tr.v[k].cpu().numpy(), v[k], rtol=5e-5, atol=1e-20), k
