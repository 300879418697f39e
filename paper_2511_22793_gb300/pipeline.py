"""Device buffers and call sequence of the splatting path, over the C ABI.

PyTorch provides device memory and streams only; every step runs in
libgsparc.so through the binding in gsparc.py.  A `Renderer` owns the
buffers of one (view, band, scene size) configuration:

  geometry(scene)            gsparc_project + gsparc_bin_sort   (query-independent)
  attributes(scene, mlp, tx) gsparc_attr_mlp                    (per transmitter)
  render(attr)               gsparc_render_fwd
  backward(...)              gsparc_render_bwd, gsparc_attr_mlp_bwd, gsparc_project_bwd

With the receiver fixed, the geometry depends only on the scene, so it is
computed once per scene and reused by every transmitter query.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import torch

from . import gsparc as G


def _dev(a, device):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device=device)


class PackedInputs:
    """Float32 device tensors that share one allocation (each at a 256-byte aligned offset),
    with a pinned host mirror, so that a step's inputs move from host memory in one copy.

    views[i] has shapes[i]; upload() copies the host mirror (or a run of views) to the device
    on the current stream (asynchronously), nbytes is its size."""

    def __init__(self, shapes, device="cuda"):
        offs, o = [], 0
        for sh in shapes:
            offs.append(o)
            o += (int(np.prod(sh)) * 4 + 255) // 256 * 256
        self.offs = offs + [o]
        self.nbytes = max(o, 256)
        self.flat = torch.zeros(self.nbytes, dtype=torch.uint8, device=device)
        self.host = torch.zeros(self.nbytes, dtype=torch.uint8).pin_memory()
        self.views = [self.flat[off:off + int(np.prod(sh)) * 4].view(torch.float32).view(*sh)
                      for off, sh in zip(offs, shapes)]
        self.host_views = [self.host[off:off + int(np.prod(sh)) * 4].view(torch.float32).view(*sh)
                           for off, sh in zip(offs, shapes)]

    def set_host(self, i, a):
        """Write array a into slot i of the host mirror."""
        self.host_views[i].copy_(torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32))
                                 if not isinstance(a, torch.Tensor) else a.detach().to("cpu", torch.float32))

    def upload(self, first=0, last=None):
        """Copy views[first:last] (one contiguous byte range; all by default) from the host
        mirror on the current stream."""
        last = len(self.views) if last is None else last
        lo, hi = self.offs[first], (self.offs[last] if last < len(self.views) else self.nbytes)
        self.flat[lo:hi].copy_(self.host[lo:hi], non_blocking=True)


@dataclass
class DeviceScene:
    means: torch.Tensor          # [N, 3]
    log_scales: torch.Tensor     # [N, 3]
    quats: torch.Tensor          # [N, 4]
    opacity_logit: torch.Tensor  # [N]
    latent: torch.Tensor         # [N, 16]

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    @staticmethod
    def from_host(scene, device="cuda"):
        return DeviceScene(*[_dev(a, device) for a in scene.arrays()])

    def tensors(self):
        return (self.means, self.log_scales, self.quats, self.opacity_logit, self.latent)


@dataclass
class DeviceMLP:
    hidden: int
    W1: torch.Tensor
    b1: torch.Tensor
    W2: torch.Tensor
    b2: torch.Tensor
    W3: torch.Tensor
    b3: torch.Tensor

    @staticmethod
    def from_host(mlp, device="cuda"):
        return DeviceMLP(mlp.hidden, *[_dev(a, device) for a in mlp.arrays()])

    def tensors(self):
        return (self.W1, self.b1, self.W2, self.b2, self.W3, self.b3)

    def struct(self) -> G.MLP:
        return G.make_mlp(self.hidden, *self.tensors())


class Renderer:
    """Buffers and calls for one view / band / scene size."""

    def __init__(self, H, W, K, n, f_c=2.4e9, df=312.5e3, rx=(0.0, 0.0, 0.0),
                 V=(1, 0, 0, 0, 1, 0, 0, 0, 1), near_dist=0.1, pair_capacity=None, device="cuda"):
        self.device = torch.device(device)
        self.V, self.near = tuple(float(v) for v in V), float(near_dist)
        self.view = G.make_view(H, W, rx, V, near_dist)
        self.band = G.make_band(K, f_c, df)
        self.H, self.W, self.K, self.n = int(H), int(W), int(K), int(n)
        self.rx = tuple(float(v) for v in rx)
        self.T = G.gsparc_num_tiles(self.view)
        self.capacity = int(pair_capacity) if pair_capacity is not None else max(4096, 64 * self.n)
        dev = self.device
        self.proj = torch.empty((self.n, G.PROJ_STRIDE), dtype=torch.float32, device=dev)
        self.sorted_ids = torch.empty(max(1, self.capacity), dtype=torch.int32, device=dev)
        self.sorted_keys = None
        self.tile_ranges = torch.empty((self.T, 2), dtype=torch.int32, device=dev)
        self.n_pairs = torch.zeros(1, dtype=torch.int32, device=dev)
        self.status = torch.zeros(1, dtype=torch.int32, device=dev)
        ws = G.gsparc_bin_sort_workspace(self.view, self.n, self.capacity)
        self.ws = torch.empty(max(256, ws), dtype=torch.uint8, device=dev)
        self.bwd_ws = None   # schedule of the tensor-core backward, allocated on first use

    def set_receiver(self, rx, V=None):
        """Move the receiver (position rx, world-to-receiver rotation V, row-major 3x3): the
        next geometry() projects and bins for that pose (Sec. 4.2 "Directional Projection
        and Splatting", receiver pose x_rx,i per sample)."""
        if V is not None:
            self.V = tuple(float(v) for v in V)
        self.rx = tuple(float(v) for v in rx)
        self.view = G.make_view(self.H, self.W, self.rx, self.V, self.near)

    # -- receiver-dependent geometry (query-independent while the receiver stays) ----
    def geometry(self, scene: DeviceScene, keep_keys=False, stream=None):
        if keep_keys and self.sorted_keys is None:
            self.sorted_keys = torch.empty(max(1, self.capacity), dtype=torch.int64, device=self.device)
        G.gsparc_project(self.view, scene.means, scene.log_scales, scene.quats, self.proj, stream,
                         d_status=self.status)
        G.gsparc_bin_sort(self.view, self.n, self.proj, self.capacity, self.ws, self.sorted_ids,
                          self.sorted_keys if keep_keys else None, self.tile_ranges, self.n_pairs,
                          self.status, stream)

    def check(self, stream=None) -> int:
        """Synchronise and return the device status (0 when every wait, capacity and device-side
        input check held; the first condition raised by any of this renderer's calls otherwise)."""
        return G.gsparc_check(self.status, stream)

    # -- per-query attributes and compositing ---------------------------------------
    def attributes(self, scene: DeviceScene, mlp: DeviceMLP, tx: torch.Tensor, precision=G.GSPARC_FP32,
                   out=None, stream=None, hidden=None):
        """hidden (FP32): a buffer of 2 * mlp.hidden * hidden_ld(B * n) floats that receives the
        network's activations for attributes_backward."""
        B = int(tx.shape[0])
        attr = out if out is not None else torch.empty((B, self.n, 4), dtype=torch.float32,
                                                       device=self.device)
        G.gsparc_attr_mlp(tx, self.rx, scene.means, scene.opacity_logit, scene.latent, mlp.struct(),
                          precision, attr, stream, hidden=hidden)
        return attr

    def alloc_outputs(self, B):
        dev = self.device
        spec = torch.empty((B, self.K, self.H, self.W, 2), dtype=torch.float32, device=dev)
        logT = torch.empty((B, self.H, self.W), dtype=torch.float32, device=dev)
        nc = torch.empty((B, self.H, self.W), dtype=torch.int32, device=dev)
        return spec, logT, nc

    def render(self, attr, out=None, n_used=None, tensor_cores=False, stream=None):
        """Forward compositing; tensor_cores selects gsparc_render_fwd_tc (same outputs)."""
        B = int(attr.shape[0])
        spec, logT, nc = out if out is not None else self.alloc_outputs(B)
        fn = G.gsparc_render_fwd_tc if tensor_cores else G.gsparc_render_fwd
        fn(self.view, self.band, B, self.n, self.proj, self.tile_ranges, self.sorted_ids, attr, spec,
           logT, nc, n_used, stream, d_status=self.status)
        return spec, logT, nc

    def render_csi(self, attr, csi=None, out=None, n_used=None, stream=None):
        """Spatial-mean channel estimate (Eq. 2) fused into the tensor-core forward.

        csi [B, K, 2] out (allocated when None).  out: optional (spectrum, final_logT,
        n_contrib) as render(); with out=None no spectrum is written at all (the state
        buffers are skipped too).  Returns csi."""
        B = int(attr.shape[0])
        if csi is None:
            csi = torch.empty((B, self.K, 2), dtype=torch.float32, device=self.device)
        spec, logT, nc = out if out is not None else (None, None, None)
        G.gsparc_render_csi_tc(self.view, self.band, B, self.n, self.proj, self.tile_ranges,
                               self.sorted_ids, attr, csi, spec, logT, nc, n_used, stream, d_status=self.status)
        return csi

    def s_tot_buffer(self, B):
        """[B, strips, H, W] buffer for the fused L2 forward's s_tot output."""
        return torch.empty((B, G.s_tot_strips(self.K), self.H, self.W), dtype=torch.float32,
                           device=self.device)

    def walk_buffer(self, B):
        """[B, T] buffer for the fused L2 forward's per-tile walk output."""
        return torch.empty((B, self.T), dtype=torch.int32, device=self.device)

    def render_backward(self, attr, logT, nc, d_spec, d_attr, d_proj, tensor_cores=False, stream=None,
                        spectrum=None, s_tot=None, split_min=0, tile_walk=None, ws=None):
        """Compositing gradient scheduled over the SMs: gsparc_render_bwd_tc_balanced
        (tensor_cores) or gsparc_render_bwd_balanced (FP32); long walks are split when the
        spectrum or the fused forward's s_tot is given.  ws: the schedule's workspace (zeroed
        before first use), allocated here when None."""
        B = int(attr.shape[0])
        if tensor_cores:
            need = G.gsparc_render_bwd_tc_workspace(self.view, self.band, B)
            fn = G.gsparc_render_bwd_tc_balanced
        else:
            need = G.gsparc_render_bwd_workspace(self.view, self.band, B)
            fn = G.gsparc_render_bwd_balanced
        if ws is None:
            if self.bwd_ws is None or self.bwd_ws.numel() < need:
                self.bwd_ws = torch.zeros(need, dtype=torch.uint8, device=self.device)
            ws = self.bwd_ws
        fn(self.view, self.band, B, self.n, self.proj, self.tile_ranges, self.sorted_ids, attr, spectrum, s_tot,
           logT, nc, d_spec, ws, d_attr, d_proj, split_min=split_min, tile_walk=tile_walk, stream=stream,
           d_status=self.status)

    def attributes_backward(self, scene, mlp, tx, d_attr, d_means, d_ologit, d_latent, d_weights,
                            stream=None, tensor_cores=False, hidden=None):
        """tensor_cores: the tcgen05 form (split-BF16 products, hidden 16 or 32); hidden: the FP32
        form reads the activations attributes(hidden=...) stored instead of recomputing them."""
        if tensor_cores:
            G.gsparc_attr_mlp_bwd_tc(tx, self.rx, scene.means, scene.opacity_logit, scene.latent,
                                     mlp.struct(), G.GSPARC_BF16X2, d_attr, d_means, d_ologit, d_latent,
                                     G.make_mlp_grad(*d_weights), stream)
        else:
            G.gsparc_attr_mlp_bwd(tx, self.rx, scene.means, scene.opacity_logit, scene.latent,
                                  mlp.struct(), d_attr, d_means, d_ologit, d_latent,
                                  G.make_mlp_grad(*d_weights), stream, hidden=hidden)

    def project_backward(self, scene, d_proj, d_means, d_log_scales, d_quats, stream=None):
        G.gsparc_project_bwd(self.view, scene.means, scene.log_scales, scene.quats, d_proj, d_means,
                             d_log_scales, d_quats, stream)
