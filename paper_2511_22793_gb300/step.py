"""One training step of the splatting path (Algorithm 1: render, loss, Backprop) on the device.

`TrainStep` owns the buffers of one configuration and enqueues the step's library calls:
projection -> bin/sort -> attribute network -> compositing forward -> complex L2 loss ->
compositing backward -> network backward -> projection backward.  Two arithmetic forms:

  form="fp32": every stage on the CUDA cores in FP32 (gsparc_attr_mlp FP32, the loss fused into
               gsparc_render_fwd_l2, the scheduled gsparc_render_bwd_balanced fed by its s_tot
               and tile walks, gsparc_attr_mlp_bwd);
  form="tc":   the subcarrier contractions and the network's products on the tensor cores with
               split-BF16 operands and FP32 accumulation (gsparc_attr_mlp BF16X2, the loss fused
               into gsparc_render_fwd_l2_tc, the scheduled gsparc_render_bwd_tc_balanced fed by
               its s_tot and tile walks, gsparc_attr_mlp_bwd_tc); transmittance, alpha and the
               per-pixel recursions stay FP32.

`enqueue(concurrent=True)` puts the gradient zeroing and the network forward beside projection
and bin/sort, and the projection backward beside the network backward, on a second stream (the
form captured as one CUDA graph by `capture()`); `concurrent=False` keeps one stream, with an
optional per-stage event hook for timing.  Every gradient is a view of one flat buffer (one
memset per step).
"""
from __future__ import annotations

import numpy as np
import torch

from . import gsparc as G
from .pipeline import DeviceMLP, DeviceScene, Renderer

PARAM_NAMES = ("means", "log_scales", "quats", "opacity_logit", "latent", "W1", "b1", "W2", "b2", "W3", "b3")
STAGES = ("project", "bin_sort", "attr_mlp", "render_fwd", "render_bwd", "attr_mlp_bwd", "project_bwd")


class TrainStep:
    def __init__(self, r: Renderer, scene: DeviceScene, mlp: DeviceMLP, tx: torch.Tensor, target: torch.Tensor,
                 form="fp32"):
        if form not in ("fp32", "tc"):
            raise ValueError("form must be 'fp32' or 'tc'")
        self.r, self.scene, self.mlp, self.tx, self.target = r, scene, mlp, tx, target
        self.form = form
        dev = r.device
        self.B = int(tx.shape[0])
        B, n = self.B, r.n
        self.attr = torch.empty((B, n, 4), device=dev)
        self.spec, self.logT, self.nc = r.alloc_outputs(B)
        self.n_used = torch.zeros((B, r.H, r.W), dtype=torch.int32, device=dev)
        self.loss = torch.zeros(1, device=dev)
        self.d_spec = torch.empty_like(self.spec)
        shapes = [self.attr.shape, r.proj.shape] + [t.shape for t in scene.tensors()] + \
                 [t.shape for t in mlp.tensors()]
        sizes = [int(np.prod(sh)) for sh in shapes]
        offs = np.cumsum([0] + [(z + 63) // 64 * 64 for z in sizes])
        self.gbuf = torch.zeros(int(offs[-1]), device=dev)
        views = [self.gbuf[int(o):int(o) + z].view(sh) for o, z, sh in zip(offs[:-1], sizes, shapes)]
        self.d_attr, self.d_proj, self.grads = views[0], views[1], views[2:]
        self.mlp_s = mlp.struct()
        self.grad_s = G.make_mlp_grad(*self.grads[5:])
        tc = form == "tc"
        self.mlp_tc = tc and mlp.hidden in (16, 32)
        self.mlp_prec = G.GSPARC_BF16X2 if tc else G.GSPARC_FP32
        # The FP32 network backward recomputes the forward's activations: storing them in the forward
        # (gsparc_attr_mlp's `hidden`) makes the backward 33 -> 29 us, but the forward's 12.8 MB of
        # extra stores, on the second stream beside projection and bin/sort, cost the step more.
        self.hidden = None
        strips = G.s_tot_strips(r.K) if tc else G.fp32_strips(r.K)
        self.s_tot = torch.empty((B, strips, r.H, r.W), dtype=torch.float32, device=dev)
        self.walks = r.walk_buffer(B)
        ws = G.gsparc_render_bwd_tc_workspace(r.view, r.band, B) if tc else \
            G.gsparc_render_bwd_workspace(r.view, r.band, B)
        self.bwd_ws = torch.zeros(ws, dtype=torch.uint8, device=dev)
        self.side = torch.cuda.Stream(dev)
        # the host-input step's third stream and the pinned word its loss is copied to (made here:
        # neither can be created while a graph is being captured)
        self.copy_s = torch.cuda.Stream(dev)
        self.host_loss = torch.empty(1, dtype=torch.float32).pin_memory()
        self.stages = STAGES
        # kernels of the library launched by one step: project 1, bin/sort 3, network 1, forward
        # with the loss fused 1, backward 2 (its schedule and the scheduled walks), network
        # backward 1, projection backward 1
        self.launches = 1 + 3 + 1 + 1 + 2 + 1 + 1

    def spectrum(self, out=None):
        """The step's spectrum [B,K,H,W,2] (the step itself stores only dL/dz): the same forward
        kernel once more with the spectrum stored, on the current stream."""
        r, B = self.r, self.B
        z = out if out is not None else self.spec
        fn = G.gsparc_render_fwd_l2_tc if self.form == "tc" else G.gsparc_render_fwd_l2
        fn(r.view, r.band, B, r.n, r.proj, r.tile_ranges, r.sorted_ids, self.attr, self.target, self.loss,
           self.d_spec, z, self.logT, self.nc, d_status=r.status)
        return z

    def gradients(self):
        """Name -> gradient view (the flat buffer's views, valid after a step)."""
        return dict(zip(PARAM_NAMES, self.grads))

    def _mlp_fwd(self, stream=None):
        s = self.scene
        G.gsparc_attr_mlp(self.tx, self.r.rx, s.means, s.opacity_logit, s.latent, self.mlp_s, self.mlp_prec,
                          self.attr, stream, hidden=self.hidden)

    def _mlp_bwd(self, stream=None):
        s, g = self.scene, self.grads
        if self.mlp_tc:
            G.gsparc_attr_mlp_bwd_tc(self.tx, self.r.rx, s.means, s.opacity_logit, s.latent, self.mlp_s,
                                     G.GSPARC_BF16X2, self.d_attr, g[0], g[3], g[4], self.grad_s, stream)
        else:
            G.gsparc_attr_mlp_bwd(self.tx, self.r.rx, s.means, s.opacity_logit, s.latent, self.mlp_s,
                                  self.d_attr, g[0], g[3], g[4], self.grad_s, stream, hidden=self.hidden)

    def _proj_bwd(self, stream=None):
        s, g = self.scene, self.grads
        G.gsparc_project_bwd(self.r.view, s.means, s.log_scales, s.quats, self.d_proj, g[0], g[1], g[2], stream)

    def _render_fwd(self):
        r, B = self.r, self.B
        if self.form == "tc":
            # the loss fused into the forward's epilogue: it writes dL/dz, not the spectrum
            G.gsparc_render_fwd_l2_tc(r.view, r.band, B, r.n, r.proj, r.tile_ranges, r.sorted_ids, self.attr,
                                      self.target, self.loss, self.d_spec, None, self.logT, self.nc, self.n_used,
                                      s_tot=self.s_tot, tile_walk=self.walks, d_status=r.status)
        else:
            # dL/dz and the loss, no spectrum (training needs only the gradient)
            G.gsparc_render_fwd_l2(r.view, r.band, B, r.n, r.proj, r.tile_ranges, r.sorted_ids, self.attr,
                                   self.target, self.loss, self.d_spec, None, self.logT, self.nc, self.n_used,
                                   s_tot=self.s_tot, tile_walk=self.walks, d_status=r.status)

    def _render_bwd(self):
        r, B = self.r, self.B
        if self.form == "tc":
            G.gsparc_render_bwd_tc_balanced(r.view, r.band, B, r.n, r.proj, r.tile_ranges, r.sorted_ids, self.attr,
                                            None, self.s_tot, self.logT, self.nc, self.d_spec, self.bwd_ws,
                                            self.d_attr, self.d_proj, tile_walk=self.walks, d_status=r.status)
        else:
            G.gsparc_render_bwd_balanced(r.view, r.band, B, r.n, r.proj, r.tile_ranges, r.sorted_ids, self.attr,
                                         None, self.s_tot, self.logT, self.nc, self.d_spec, self.bwd_ws,
                                         self.d_attr, self.d_proj, tile_walk=self.walks, d_status=r.status)

    def enqueue(self, concurrent=False, events=None):
        """Enqueue one step on the current stream.  events: optional dict stage -> (start, end)
        CUDA events recorded around each stage (single-stream form only)."""
        r, s = self.r, self.scene
        cur = torch.cuda.current_stream(r.device)

        def stage(name, fn):
            if events is not None and name in events:
                events[name][0].record(cur)
            fn()
            if events is not None and name in events:
                events[name][1].record(cur)

        if concurrent:
            fork = torch.cuda.Event()
            fork.record(cur)
            self.side.wait_event(fork)
            with torch.cuda.stream(self.side):
                self.gbuf.zero_()   # the gradients are first written by the compositing backward
            self._mlp_fwd(self.side)
            joined = torch.cuda.Event()
            joined.record(self.side)
        else:
            self.gbuf.zero_()
        stage("project", lambda: G.gsparc_project(r.view, s.means, s.log_scales, s.quats, r.proj,
                                                  d_status=r.status))
        stage("bin_sort", lambda: G.gsparc_bin_sort(r.view, r.n, r.proj, r.capacity, r.ws, r.sorted_ids, None,
                                                    r.tile_ranges, r.n_pairs, r.status))
        if concurrent:
            cur.wait_event(joined)
        else:
            stage("attr_mlp", self._mlp_fwd)
        stage("render_fwd", self._render_fwd)
        stage("render_bwd", self._render_bwd)
        if concurrent:
            fork2 = torch.cuda.Event()
            fork2.record(cur)
            self.side.wait_event(fork2)
            self._proj_bwd(self.side)
            joined2 = torch.cuda.Event()
            joined2.record(self.side)
            self._mlp_bwd()
            cur.wait_event(joined2)
        else:
            stage("attr_mlp_bwd", self._mlp_bwd)
            stage("project_bwd", self._proj_bwd)

    def enqueue_from_host(self, inp):
        """The step with its inputs in pinned host memory (`inp`: a PackedInputs whose views are
        this step's scene (means, log-scales, quaternions first), network, transmitters and, last,
        the target): the projection's inputs are copied first, then the rest of the scene, the
        network and the transmitters on the second stream ahead of the network forward, and the
        target on a third stream after them, beside projection, binning and the forward, which
        therefore writes the spectrum (the fused loss would wait for the whole target); the loss
        and dL/dz follow once the target is in, and the backward forms s_tot from the spectrum.
        The loss is copied to pinned host memory (`host_loss`) on the third stream while the
        backward runs.  Same loss and gradients as enqueue()."""
        r, s = self.r, self.scene
        cur = torch.cuda.current_stream(r.device)
        inp.upload(0, 3)
        geo_in = torch.cuda.Event()
        geo_in.record(cur)
        self.side.wait_event(geo_in)
        with torch.cuda.stream(self.side):
            inp.upload(3, len(inp.views) - 1)
            rest_in = torch.cuda.Event()
            rest_in.record(self.side)
            self.gbuf.zero_()
        self.copy_s.wait_event(rest_in)
        with torch.cuda.stream(self.copy_s):
            inp.upload(len(inp.views) - 1)
        tgt_in = torch.cuda.Event()
        tgt_in.record(self.copy_s)
        self._mlp_fwd(self.side)
        joined = torch.cuda.Event()
        joined.record(self.side)
        G.gsparc_project(r.view, s.means, s.log_scales, s.quats, r.proj, d_status=r.status)
        G.gsparc_bin_sort(r.view, r.n, r.proj, r.capacity, r.ws, r.sorted_ids, None, r.tile_ranges, r.n_pairs,
                          r.status)
        cur.wait_event(joined)
        B = self.B
        if self.form == "tc":
            G.gsparc_render_fwd_tc(r.view, r.band, B, r.n, r.proj, r.tile_ranges, r.sorted_ids, self.attr, self.spec,
                                   self.logT, self.nc, self.n_used, d_status=r.status)
        else:
            G.gsparc_render_fwd(r.view, r.band, B, r.n, r.proj, r.tile_ranges, r.sorted_ids, self.attr, self.spec,
                                self.logT, self.nc, self.n_used, d_status=r.status)
        cur.wait_event(tgt_in)
        G.gsparc_l2_loss(self.spec, self.target, self.loss, self.d_spec)
        loss_done = torch.cuda.Event()
        loss_done.record(cur)
        self.copy_s.wait_event(loss_done)
        with torch.cuda.stream(self.copy_s):
            self.host_loss.copy_(self.loss, non_blocking=True)
        loss_out = torch.cuda.Event()
        loss_out.record(self.copy_s)
        fn = G.gsparc_render_bwd_tc_balanced if self.form == "tc" else G.gsparc_render_bwd_balanced
        fn(r.view, r.band, B, r.n, r.proj, r.tile_ranges, r.sorted_ids, self.attr, self.spec, None, self.logT,
           self.nc, self.d_spec, self.bwd_ws, self.d_attr, self.d_proj, d_status=r.status)
        fork2 = torch.cuda.Event()
        fork2.record(cur)
        self.side.wait_event(fork2)
        self._proj_bwd(self.side)
        joined2 = torch.cuda.Event()
        joined2.record(self.side)
        self._mlp_bwd()
        cur.wait_event(joined2)
        cur.wait_event(loss_out)

    def capture(self, inp=None):
        """The concurrent step (with inp: its host-input form) captured as one CUDA graph (the
        library only enqueues stream-ordered work, so it captures); replay() runs a step."""
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            if inp is None:
                self.enqueue(concurrent=True)
            else:
                self.enqueue_from_host(inp)
        return g
