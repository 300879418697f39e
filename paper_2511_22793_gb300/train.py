"""On-device training loop (Algorithm 1: render, loss, Backprop, Adam, densification) over the C ABI.

Every step takes the next batch of training transmitters, renders their spectra (projection,
bin/sort, attribute network, compositing), takes the loss against the targets, runs the
hand-written backward (per-pixel state recomputed from the stored final log-transmittance,
network activations recomputed) and updates every parameter group with Adam at the learning
rates of the paper's hyperparameter table (position rate annealed exponentially from 1.6e-4 to
1.6e-7 over the run), in one launch over the flat parameter buffer.

Arithmetic: tensor_cores=True runs the network and the compositing contractions on the tensor
cores (split-BF16 operands, FP32 accumulation and FP32 master weights); False runs everything in
FP32 on the CUDA cores.

Losses (`loss`):
  "l2"     complex L2 (mean |z - z*|^2), fused into the forward's epilogue;
  "l1ssim" Eq. 4 on magnitude spectra, (1 - lambda_1) L1(|z|, |z*|) + lambda_1 (1 - SSIM), the
           paper's loss for spectrum targets.
With confidence=True the objective is Eq. 5 over the batch, mean_b (C_b L_b - alpha ln C_b) with
C_b = 1 + exp(g(tx_b)) from a 3 -> 32 -> 1 network trained alongside (its rate in the table):
each sample's dL_b/dz is scaled by dObj/dL_b = C_b / B.

Densification (densify_every > 0, Algorithm 1's branch; the paper gives no thresholds, the
proposed ones are gsparc.densify_params()): after every backward the positional gradient norm of
every visible Gaussian is accumulated; every densify_every steps until densify_until, Gaussians
are cloned, split and pruned (gsparc_densify), their Adam moments and latents carried along as
the kernel's per-Gaussian payload (new clones and children inherit their parent's moments), and
every opacity_reset_every steps the opacities are capped at 0.01 (gsparc_opacity_reset).

Targets: spectra of a ground-truth scene rendered by the FP32 path (whose parity with the FP64
oracle the tests establish).  With resident_targets (the default when they fit the budget) all
training targets are rendered once at set-up and kept in HBM in a seeded shuffled order, so that
every batch is a contiguous view of the stored dataset; otherwise each batch's targets are
rendered when it is drawn.

Checkpoint/resume: `state_dict()` holds parameters, Adam moments, the step counter and the batch
cursor; `load_state_dict()` restores them (the Gaussian count must match).
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import gsparc as G
from . import synth
from .pipeline import DeviceMLP, DeviceScene, Renderer

SCENE_KEYS = ("means", "log_scales", "quats", "opacity_logit", "latent")
MLP_KEYS = ("W1", "b1", "W2", "b2", "W3", "b3")
# learning rates (Table of hyperparameters); the latent codes share the emission network's rate
LR = {"log_scales": 0.005, "quats": 0.001, "opacity_logit": 0.0055, "latent": 0.005,
      "W1": 0.005, "b1": 0.005, "W2": 0.005, "b2": 0.005, "W3": 0.005, "b3": 0.005}
POS_LR_INIT, POS_LR_FINAL = 1.6e-4, 1.6e-7
CONFIDENCE_LR = 0.005
CONFIDENCE_HIDDEN = 32
LAMBDA_1 = 0.2


def init_scene(n, seed=10, init_scale=0.2, init_opacity=0.1):
    """Geometry-agnostic initialisation (Sec. 4.1): uniform centres, isotropic scales,
    identity rotations, small constant opacity, N(0,1) latents."""
    rng = np.random.default_rng(seed)
    means = rng.uniform(-synth.CUBE_HALF, synth.CUBE_HALF, size=(n, 3))
    means[:, 1] = rng.uniform(0.0, synth.CUBE_HALF, size=n)
    log_scales = np.full((n, 3), math.log(init_scale))
    quats = np.tile([1.0, 0.0, 0.0, 0.0], (n, 1))
    ologit = np.full(n, math.log(init_opacity / (1.0 - init_opacity)))
    latent = rng.normal(0.0, 1.0, size=(n, synth.LATENT_DIM))
    f = lambda a: np.ascontiguousarray(a, dtype=np.float32)
    return synth.Scene(f(means), f(log_scales), f(quats), f(ologit), f(latent))


def _confidence_init(hidden, seed):
    """W1 [3, h] N(0,1)/sqrt(3), b1 0, W2 [h] N(0,1)/sqrt(h) * 0.1, b2 0: C starts near 2."""
    rng = np.random.default_rng(seed)
    w1 = rng.normal(0.0, 1.0, size=(3, hidden)) / math.sqrt(3.0)
    w2 = 0.1 * rng.normal(0.0, 1.0, size=hidden) / math.sqrt(hidden)
    return np.concatenate([w1.reshape(-1), np.zeros(hidden), w2, np.zeros(1)]).astype(np.float32)


class Trainer:
    def __init__(self, n, gt_scene, gt_mlp, train_tx, H=90, W=360, K=128, hidden=32, batch=4,
                 total_steps=1000, device="cuda", seed=10, tensor_cores=True, init=None, loss="l2",
                 confidence=False, densify_every=0, densify_until=15000, opacity_reset_every=3000,
                 densify_params=None, resident_targets=None, target_budget_bytes=120 << 30):
        """init: optional (Scene, MLPWeights) to start from instead of the paper's
        geometry-agnostic initialisation."""
        if loss not in ("l2", "l1ssim"):
            raise ValueError("loss must be 'l2' or 'l1ssim'")
        self.dev = torch.device(device)
        self.H, self.W, self.K, self.batch = H, W, K, batch
        self.total_steps = total_steps
        self.tensor_cores = tensor_cores
        self.loss_kind, self.confidence = loss, confidence
        self.densify_every, self.densify_until = int(densify_every), int(densify_until)
        self.opacity_reset_every = int(opacity_reset_every)
        self.dparams = densify_params if densify_params is not None else G.densify_params()
        self.seed = seed
        if init is None:
            sc = init_scene(n, seed=seed)
            mlp = synth.make_mlp(hidden, seed=seed + 1)
        else:
            sc, mlp = init
        self.hidden = mlp.hidden
        self.mlp_arrays = list(mlp.arrays())
        self.conf_w0 = _confidence_init(CONFIDENCE_HIDDEN, seed + 3) if confidence else None
        self.step_count = 0
        self.cursor = 0
        self.rng = np.random.default_rng(seed + 2)
        self._build(sc.arrays(), None)
        self.loss = torch.zeros(1, device=self.dev)
        self.loss_b = torch.zeros(batch, device=self.dev)
        self.conf_c = torch.zeros(batch, device=self.dev)
        self.conf_d = torch.zeros(batch, device=self.dev)
        self.objective = torch.zeros(1, device=self.dev)
        # ground truth: its own renderer with cached geometry (receiver fixed)
        self.gt = DeviceScene.from_host(gt_scene, self.dev)
        self.gt_mlp = DeviceMLP.from_host(gt_mlp, self.dev)
        self.rg = Renderer(H, W, K, gt_scene.n, device=self.dev)
        self.rg.geometry(self.gt)
        self.gt_attr = torch.empty((batch, gt_scene.n, 4), device=self.dev)
        self.target = self.rg.alloc_outputs(batch)
        self.mag_target = torch.empty((batch, K, H, W), device=self.dev) if loss == "l1ssim" else None
        self.ssim_ws = None
        if loss == "l1ssim":
            self.ssim_ws = torch.empty(G.gsparc_spectrum_loss_workspace(batch, K, H, W), dtype=torch.uint8,
                                       device=self.dev)
            self.ssim_ws1 = torch.empty(G.gsparc_spectrum_loss_workspace(1, K, H, W), dtype=torch.uint8,
                                        device=self.dev)
        # the dataset, in a seeded shuffled order (every batch a contiguous slice of it)
        order = np.random.default_rng(seed + 4).permutation(len(train_tx))
        self.n_train = len(train_tx) - len(train_tx) % batch
        self.train_tx = torch.tensor(np.asarray(train_tx, dtype=np.float32)[order[:self.n_train]], device=self.dev)
        per = K * H * W * (4 if loss == "l1ssim" else 8)
        self.resident = resident_targets if resident_targets is not None else \
            self.n_train * per <= target_budget_bytes
        self.dataset = None
        if self.resident:
            shape = (self.n_train, K, H, W) if loss == "l1ssim" else (self.n_train, K, H, W, 2)
            self.dataset = torch.empty(shape, device=self.dev)
            for s in range(0, self.n_train, batch):
                z = self.render_targets(self.train_tx[s:s + batch])
                if loss == "l1ssim":
                    torch.linalg.vector_norm(z, dim=-1, out=self.dataset[s:s + batch])
                else:
                    self.dataset[s:s + batch].copy_(z)
            torch.cuda.synchronize(self.dev)

    # -- buffers of the current Gaussian set -------------------------------------------------
    def _build(self, scene_arrays, carry):
        """(Re)allocate parameters, gradients, moments, the renderer and the per-step buffers for
        the Gaussians in scene_arrays; carry: optional (m, v) dicts of moments to install."""
        n = int(np.shape(scene_arrays[0])[0]) if not isinstance(scene_arrays[0], torch.Tensor) else \
            int(scene_arrays[0].shape[0])
        self.n = n
        keys = list(SCENE_KEYS) + list(MLP_KEYS) + (["conf"] if self.confidence else [])
        arrays = list(scene_arrays) + list(self.mlp_arrays) + ([self.conf_w0] if self.confidence else [])
        shapes = {k: tuple(a.shape) for k, a in zip(keys, arrays)}
        self.params, self._pbuf = self._flat(shapes)
        for k, a in zip(keys, arrays):
            src = a if isinstance(a, torch.Tensor) else torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32))
            self.params[k].copy_(src)
        self.scene = DeviceScene(*[self.params[k] for k in SCENE_KEYS])
        self.mlp = DeviceMLP(self.hidden, *[self.params[k] for k in MLP_KEYS])
        self.grads, self._gbuf = self._flat(shapes)
        self.m, self._mbuf = self._flat(shapes)
        self.v, self._vbuf = self._flat(shapes)
        if carry is not None:
            for k in keys:
                if k in carry[0]:
                    self.m[k].copy_(carry[0][k])
                    self.v[k].copy_(carry[1][k])
        self.r = Renderer(self.H, self.W, self.K, n, device=self.dev)
        B = self.batch
        self.attr = torch.empty((B, n, 4), device=self.dev)
        self.out = self.r.alloc_outputs(B)
        self.d_spec = torch.empty_like(self.out[0])
        self.d_attr = torch.empty_like(self.attr)
        self.d_proj = torch.empty_like(self.r.proj)
        tc = self.tensor_cores
        strips = G.s_tot_strips(self.K) if tc else G.fp32_strips(self.K)
        self.s_tot = torch.empty((B, strips, self.H, self.W), device=self.dev)
        self.walks = self.r.walk_buffer(B)
        ws = G.gsparc_render_bwd_tc_workspace(self.r.view, self.r.band, B) if tc else \
            G.gsparc_render_bwd_workspace(self.r.view, self.r.band, B)
        self.bwd_ws = torch.zeros(ws, dtype=torch.uint8, device=self.dev)
        if self.densify_every > 0:
            self.norm_sum = torch.zeros(n, device=self.dev)
            self.count = torch.zeros(n, dtype=torch.int32, device=self.dev)
            self.dens_ws = torch.empty(G.gsparc_densify_workspace(n), dtype=torch.uint8, device=self.dev)

    def _flat(self, shapes):
        sizes = [int(np.prod(sh)) for sh in shapes.values()]
        offs = np.cumsum([0] + [(z + 63) // 64 * 64 for z in sizes])
        buf = torch.zeros(int(offs[-1]), device=self.dev)
        views = {k: buf[int(o):int(o) + z].view(sh) for (k, sh), o, z in zip(shapes.items(), offs[:-1], sizes)}
        # the groups' ends in the flat buffer (the padding after a group belongs to it)
        self._seg_end = [int(o) for o in offs[1:]]
        return views, buf

    def pos_lr(self):
        t = min(max(self.step_count / max(self.total_steps - 1, 1), 0.0), 1.0)
        return math.exp(math.log(POS_LR_INIT) * (1 - t) + math.log(POS_LR_FINAL) * t)

    def render_targets(self, tx):
        self.rg.attributes(self.gt, self.gt_mlp, tx, G.GSPARC_FP32, out=self.gt_attr[:tx.shape[0]])
        return self.rg.render(self.gt_attr[:tx.shape[0]], out=tuple(t[:tx.shape[0]] for t in self.target))[0]

    def forward(self, tx, out=None):
        """Spectra of the current model for transmitters tx [b, 3] (b <= batch)."""
        b = int(tx.shape[0])
        prec = G.GSPARC_BF16X2 if self.tensor_cores else G.GSPARC_FP32
        self.r.geometry(self.scene)
        attr = self.r.attributes(self.scene, self.mlp, tx, prec, out=self.attr[:b])
        outs = out if out is not None else tuple(t[:b] for t in self.out)
        return self.r.render(attr, out=outs, tensor_cores=self.tensor_cores), attr

    def _batch(self):
        """The next batch's transmitters and targets (contiguous views when resident)."""
        if self.cursor + self.batch > self.n_train:
            self.cursor = 0
        c = self.cursor
        self.cursor += self.batch
        tx = self.train_tx[c:c + self.batch]
        if self.resident:
            return tx, self.dataset[c:c + self.batch]
        z = self.render_targets(tx)
        if self.loss_kind == "l1ssim":
            torch.linalg.vector_norm(z, dim=-1, out=self.mag_target)
            return tx, self.mag_target
        return tx, z

    def step(self):
        tx, target = self._batch()
        self.tx, self.batch_target = tx, target      # the batch this step trained on
        r, B, tc = self.r, self.batch, self.tensor_cores
        self._gbuf.zero_()
        self.d_attr.zero_()
        self.d_proj.zero_()
        prec = G.GSPARC_BF16X2 if tc else G.GSPARC_FP32
        r.geometry(self.scene)
        attr = r.attributes(self.scene, self.mlp, tx, prec, out=self.attr)
        spec, logT, nc = self.out
        fused = self.loss_kind == "l2" and not self.confidence
        if fused:
            # the loss fused into the forward's epilogue: dL/dz and the loss, no spectrum
            fn = G.gsparc_render_fwd_l2_tc if tc else G.gsparc_render_fwd_l2
            fn(r.view, r.band, B, self.n, r.proj, r.tile_ranges, r.sorted_ids, attr, target, self.loss, self.d_spec,
               None, logT, nc, s_tot=self.s_tot, tile_walk=self.walks, d_status=r.status)
        else:
            r.render(attr, out=self.out, tensor_cores=tc)
            if self.loss_kind == "l2":
                for b in range(B):
                    G.gsparc_l2_loss(spec[b], target[b], self.loss_b[b:b + 1], self.d_spec[b])
            elif self.confidence:
                for b in range(B):
                    G.gsparc_spectrum_loss(spec[b:b + 1], target[b:b + 1], self.ssim_ws1, self.loss_b[b:b + 1],
                                           self.d_spec[b:b + 1], lam=LAMBDA_1)
            else:
                G.gsparc_spectrum_loss(spec, target, self.ssim_ws, self.loss, self.d_spec, lam=LAMBDA_1)
            if self.confidence:
                # Eq. 5: objective, C and dObj/dL_b = C_b / B; each sample's gradient scaled by it
                G.gsparc_confidence(tx, self.loss_b, self.params["conf"], CONFIDENCE_HIDDEN, self.objective,
                                    self.conf_c, self.conf_d, self.grads["conf"])
                G.gsparc_scale_rows(self.d_spec, self.conf_d)
                self.loss = self.objective
        if fused:
            r.render_backward(attr, logT, nc, self.d_spec, self.d_attr, self.d_proj, tensor_cores=tc,
                              s_tot=self.s_tot, tile_walk=self.walks, ws=self.bwd_ws)
        else:
            r.render_backward(attr, logT, nc, self.d_spec, self.d_attr, self.d_proj, tensor_cores=tc, spectrum=spec,
                              ws=self.bwd_ws)
        g = self.grads
        r.attributes_backward(self.scene, self.mlp, tx, self.d_attr, g["means"], g["opacity_logit"], g["latent"],
                              [g[k] for k in MLP_KEYS], tensor_cores=tc and self.hidden in (16, 32))
        r.project_backward(self.scene, self.d_proj, g["means"], g["log_scales"], g["quats"])
        self.step_count += 1
        if self.densify_every > 0:
            G.gsparc_densify_accumulate(r.proj, g["means"], self.norm_sum, self.count)
        # one Adam launch over every group, each at its learning rate
        lrs = [self.pos_lr() if k == "means" else (CONFIDENCE_LR if k == "conf" else LR[k]) for k in self.params]
        G.gsparc_adam_segments(self._pbuf, self._gbuf, self._mbuf, self._vbuf, self._seg_end, lrs, self.step_count)
        if self.densify_every > 0 and self.step_count < self.densify_until:
            if self.step_count % self.densify_every == 0:
                self.densify()
            if self.opacity_reset_every > 0 and self.step_count % self.opacity_reset_every == 0:
                G.gsparc_opacity_reset(self.params["opacity_logit"], 0.01)
        return self.loss

    def densify(self):
        """Clone / split / prune (gsparc_densify) with the statistic accumulated since the last
        call; latents and the per-Gaussian Adam moments travel as the kernel's payload."""
        n, ns = self.n, int(self.dparams.n_split)
        per_g = [k for k in SCENE_KEYS]
        cols = [self.params["latent"]] + [self.m[k].reshape(n, -1) for k in per_g] + \
            [self.v[k].reshape(n, -1) for k in per_g]
        payload = torch.cat(cols, dim=1).contiguous()
        widths = [c.shape[1] for c in cols]
        xi = torch.tensor(self.rng.standard_normal((n, ns, 3)), dtype=torch.float32, device=self.dev)
        cap = n * max(ns, 2)
        out = {"means": torch.empty((cap, 3), device=self.dev), "log_scales": torch.empty((cap, 3), device=self.dev),
               "quats": torch.empty((cap, 4), device=self.dev), "opacity_logit": torch.empty(cap, device=self.dev),
               "payload": torch.empty((cap, payload.shape[1]), device=self.dev),
               "parent": torch.empty(cap, dtype=torch.int32, device=self.dev)}
        n_out = torch.zeros(1, dtype=torch.int32, device=self.dev)
        status = torch.zeros(1, dtype=torch.int32, device=self.dev)
        s = self.scene
        G.gsparc_densify(s.means, s.log_scales, s.quats, s.opacity_logit, payload, self.r.proj, self.norm_sum,
                         self.count, xi, self.dparams, self.dens_ws, out, n_out, d_status=status)
        if G.gsparc_check(status) != 0:
            raise RuntimeError("densification status %d" % G.gsparc_check(status))
        m = int(n_out.item())
        if m == 0:
            raise RuntimeError("densification removed every Gaussian")
        self.last_parent = out["parent"][:m].clone()   # input row of every output row
        pl = out["payload"][:m]
        parts = torch.split(pl, widths, dim=1)
        latent = parts[0]
        shapes = {"means": (m, 3), "log_scales": (m, 3), "quats": (m, 4), "opacity_logit": (m,), "latent": (m, 16)}
        carry_m = {k: parts[1 + i].reshape(shapes[k]) for i, k in enumerate(per_g)}
        carry_v = {k: parts[1 + len(per_g) + i].reshape(shapes[k]) for i, k in enumerate(per_g)}
        for k in list(MLP_KEYS) + (["conf"] if self.confidence else []):
            carry_m[k] = self.m[k].clone()
            carry_v[k] = self.v[k].clone()
        self.mlp_arrays = [self.params[k].clone() for k in MLP_KEYS]
        if self.confidence:
            self.conf_w0 = self.params["conf"].clone()
        scene = [out["means"][:m].clone(), out["log_scales"][:m].clone(), out["quats"][:m].clone(),
                 out["opacity_logit"][:m].clone(), latent.clone()]
        self._build(scene, (carry_m, carry_v))

    def evaluate(self, tx_all, chunk=None, magnitude=False):
        """Relative L2 error ||z - z*|| / ||z*|| over all spectra of tx_all (of |z| with
        magnitude=True)."""
        chunk = chunk or self.batch
        num = 0.0
        den = 0.0
        txs = torch.tensor(np.asarray(tx_all, dtype=np.float32), device=self.dev)
        for s in range(0, txs.shape[0], chunk):
            t = txs[s:s + chunk]
            target = self.render_targets(t)
            (spec, _, _), _ = self.forward(t)
            if magnitude:
                a, b_ = torch.linalg.vector_norm(spec, dim=-1), torch.linalg.vector_norm(target, dim=-1)
                num += float(((a - b_) ** 2).sum())
                den += float((b_ ** 2).sum())
            else:
                num += float(((spec - target) ** 2).sum())
                den += float((target ** 2).sum())
        return math.sqrt(num / den) if den > 0 else float("nan")

    def state_dict(self):
        return {"params": {k: p.detach().clone() for k, p in self.params.items()},
                "m": self._mbuf.clone(), "v": self._vbuf.clone(), "step": self.step_count, "cursor": self.cursor,
                "rng": self.rng.bit_generator.state}

    def load_state_dict(self, st):
        for k, p in self.params.items():
            p.copy_(st["params"][k])
        self._mbuf.copy_(st["m"])
        self._vbuf.copy_(st["v"])
        self.step_count = int(st["step"])
        self.cursor = int(st["cursor"])
        self.rng.bit_generator.state = st["rng"]
