"""On-device training loop (Algorithm 1: render, loss, Backprop, Adam) over the C ABI.

Every step samples a batch of training transmitters, renders their spectra
(projection, bin/sort, attribute network on the tensor cores in split-BF16
with FP32 master weights, compositing), takes the complex L2 loss against the
targets, runs the hand-written backward (per-pixel state recomputed from the
stored final log-transmittance, network activations recomputed) and updates
every parameter group with Adam at the learning rates of the paper's
hyperparameter table (position rate annealed exponentially from 1.6e-4 to
1.6e-7 over the run), in one launch over the flat parameter buffer.  Densification, pruning and the confidence network are
not part of this loop.

Targets are spectra of a ground-truth scene rendered by the same FP32 path
(whose parity with the FP64 oracle the tests establish), recomputed for the
sampled transmitters each step instead of being stored.

Checkpoint/resume: `state_dict()` holds parameters, Adam moments, the step
counter and the sampling RNG state; `load_state_dict()` restores them.
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


class Trainer:
    def __init__(self, n, gt_scene, gt_mlp, train_tx, H=90, W=360, K=128, hidden=32, batch=4,
                 total_steps=1000, device="cuda", seed=10, tensor_cores=True, init=None):
        """init: optional (Scene, MLPWeights) to start from instead of the paper's
        geometry-agnostic initialisation."""
        self.dev = torch.device(device)
        self.H, self.W, self.K, self.n, self.batch = H, W, K, n, batch
        self.total_steps = total_steps
        self.tensor_cores = tensor_cores
        self.s_tot = None   # fused forward's s_tot and tile walks for the scheduled backward
        self.walks = None
        if init is None:
            sc = init_scene(n, seed=seed)
            mlp = synth.make_mlp(hidden, seed=seed + 1)
        else:
            sc, mlp = init
            n = sc.n
            self.n = n
        # parameters, gradients and Adam moments: one flat allocation each, with the same layout
        # (every group at a 64-float boundary), so that one launch updates every group
        shapes = {k: np.shape(a) for k, a in zip(SCENE_KEYS + MLP_KEYS, list(sc.arrays()) + list(mlp.arrays()))}
        self.params, self._pbuf = self._flat(shapes)
        for k, a in zip(SCENE_KEYS + MLP_KEYS, list(sc.arrays()) + list(mlp.arrays())):
            self.params[k].copy_(torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32)))
        self.scene = DeviceScene(*[self.params[k] for k in SCENE_KEYS])
        self.mlp = DeviceMLP(mlp.hidden, *[self.params[k] for k in MLP_KEYS])
        self.grads, self._gbuf = self._flat(shapes)
        self.m, self._mbuf = self._flat(shapes)
        self.v, self._vbuf = self._flat(shapes)
        self.step_count = 0
        self.rng = np.random.default_rng(seed + 2)
        self.r = Renderer(H, W, K, n, device=self.dev)
        self.attr = torch.empty((batch, n, 4), device=self.dev)
        self.out = self.r.alloc_outputs(batch)
        self.d_spec = torch.empty_like(self.out[0])
        self.d_attr = torch.empty_like(self.attr)
        self.d_proj = torch.empty_like(self.r.proj)
        self.loss = torch.zeros(1, device=self.dev)
        # ground truth: its own renderer with cached geometry (receiver fixed)
        self.gt = DeviceScene.from_host(gt_scene, self.dev)
        self.gt_mlp = DeviceMLP.from_host(gt_mlp, self.dev)
        self.rg = Renderer(H, W, K, gt_scene.n, device=self.dev)
        self.rg.geometry(self.gt)
        self.gt_attr = torch.empty((batch, gt_scene.n, 4), device=self.dev)
        self.target = self.rg.alloc_outputs(batch)
        self.train_tx = torch.tensor(np.asarray(train_tx, dtype=np.float32), device=self.dev)
        self.tx = torch.empty((batch, 3), device=self.dev)

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

    def step(self):
        idx = self.rng.integers(0, self.train_tx.shape[0], size=self.batch)
        self.tx.copy_(self.train_tx[torch.as_tensor(idx, device=self.dev)])
        target = self.render_targets(self.tx)
        self._gbuf.zero_()
        self.d_attr.zero_()
        self.d_proj.zero_()
        if self.tensor_cores:
            # the loss fused into the tensor-core forward: dL/dz and the loss, no spectrum
            prec = G.GSPARC_BF16X2
            self.r.geometry(self.scene)
            attr = self.r.attributes(self.scene, self.mlp, self.tx, prec, out=self.attr)
            _, logT, nc = self.out
            if self.s_tot is None:
                self.s_tot = self.r.s_tot_buffer(self.batch)
                self.walks = self.r.walk_buffer(self.batch)
            G.gsparc_render_fwd_l2_tc(self.r.view, self.r.band, self.batch, self.n, self.r.proj, self.r.tile_ranges,
                                      self.r.sorted_ids, attr, target, self.loss, self.d_spec, None, logT, nc,
                                      s_tot=self.s_tot, tile_walk=self.walks)
        else:
            (spec, logT, nc), attr = self.forward(self.tx)
            G.gsparc_l2_loss(spec, target, self.loss, self.d_spec)
        self.r.render_backward(attr, logT, nc, self.d_spec, self.d_attr, self.d_proj,
                               tensor_cores=self.tensor_cores, s_tot=self.s_tot,
                               tile_walk=self.walks if self.tensor_cores else None)
        g = self.grads
        self.r.attributes_backward(self.scene, self.mlp, self.tx, self.d_attr, g["means"],
                                   g["opacity_logit"], g["latent"], [g[k] for k in MLP_KEYS],
                                   tensor_cores=self.tensor_cores and self.mlp.hidden in (16, 32))
        self.r.project_backward(self.scene, self.d_proj, g["means"], g["log_scales"], g["quats"])
        self.step_count += 1
        # one Adam launch over every group, each at its learning rate
        lrs = [self.pos_lr() if k == "means" else LR[k] for k in self.params]
        G.gsparc_adam_segments(self._pbuf, self._gbuf, self._mbuf, self._vbuf, self._seg_end, lrs, self.step_count)
        return self.loss

    def evaluate(self, tx_all, chunk=None):
        """Relative L2 error ||z - z*|| / ||z*|| over all spectra of tx_all."""
        chunk = chunk or self.batch
        num = 0.0
        den = 0.0
        txs = torch.tensor(np.asarray(tx_all, dtype=np.float32), device=self.dev)
        for s in range(0, txs.shape[0], chunk):
            t = txs[s:s + chunk]
            target = self.render_targets(t)
            (spec, _, _), _ = self.forward(t)
            num += float(((spec - target) ** 2).sum())
            den += float((target ** 2).sum())
        return math.sqrt(num / den) if den > 0 else float("nan")

    def state_dict(self):
        return {"params": {k: p.detach().clone() for k, p in self.params.items()},
                "m": self._mbuf.clone(), "v": self._vbuf.clone(), "step": self.step_count,
                "rng": self.rng.bit_generator.state}

    def load_state_dict(self, st):
        for k, p in self.params.items():
            p.copy_(st["params"][k])
        self._mbuf.copy_(st["m"])
        self._vbuf.copy_(st["v"])
        self.step_count = int(st["step"])
        self.rng.bit_generator.state = st["rng"]
