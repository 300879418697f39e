"""Continuous-batching CSI query server over one resident scene.

A request asks for the spectrum seen at a receiver for one transmitter
position, at one of several hemisphere resolutions and subcarrier counts.  The
scene stays resident on the device.  For the fixed receiver its projection and
bin/sort are computed once per resolution (the geometry does not depend on the
query) and per request the work is the attribute network and the compositing.
A request may instead carry its own receiver pose (rx, and optionally the
rotation V): the paper's moving-receiver setting, one pose per sample.  Its
geometry is then computed for it, on its stream, into geometry buffers owned
by that stream slot, and it runs alone (no other request shares its tile
lists).

Scheduling (`Server.poll`, admission in `admit`):
  * finished batches are detected with CUDA events (no host synchronisation)
    and release their stream slot and their memory reservation;
  * waiting requests are admitted oldest first while a stream slot is free and
    the memory budget (attribute buffer + spectrum + per-pixel state of every
    admitted request) allows; an admitted request joins a batch with the other
    waiting requests of the same (resolution, subcarrier count), up to
    `max_batch`, so one launch serves several transmitters;
  * batches run on separate CUDA streams, so work admitted while others are on
    the GPU overlaps with them.
A request that alone exceeds the budget is rejected; a waiting request can be withdrawn
(`Server.cancel`).  Latency is measured from
the request's arrival time to the host observing its batch's completion event.

`serve_plain` is the baseline: one request at a time on one stream with the
FP32 network and FP32 compositing (and, for a moving-receiver request, its
geometry computed first).
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import gsparc as G
from .pipeline import DeviceMLP, DeviceScene, Renderer


@dataclass
class Request:
    rid: int
    tx: tuple
    res: tuple          # (H, W)
    K: int
    t_arrival: float = 0.0
    t_done: float = -1.0
    spectrum: torch.Tensor | None = None   # [K, H, W, 2] on the device
    rejected: bool = False
    cancelled: bool = False
    rx: tuple | None = None                # receiver position of a moving-receiver request
    V: tuple | None = None                 # its rotation (row-major 3x3), identity when None


@dataclass
class _Batch:
    reqs: list
    stream: torch.cuda.Stream
    event: torch.cuda.Event
    nbytes: int
    bufs: tuple = field(default_factory=tuple)


def admit(waiting, used, budget, max_batch, request_bytes):
    """Admission of the oldest waiting request and the batch it leads (host logic only).

    The head is admitted if its bytes fit beside `used` within `budget`; a moving-receiver head
    (its own geometry) runs alone; otherwise every later waiting request of the same
    (resolution, subcarrier count) with the fixed receiver joins, oldest first, while the batch
    has fewer than `max_batch` requests and its bytes still fit.  Returns (batch, the requests
    left waiting in their order), or None when the head does not fit (nothing is taken)."""
    head = waiting[0]
    H, W = head.res
    one = request_bytes(H, W, head.K)
    if used + one > budget:
        return None
    rest = collections.deque(waiting)
    if head.rx is not None:
        return [rest.popleft()], rest
    group = []
    left = collections.deque()
    while rest:
        q = rest.popleft()
        if (len(group) < max_batch and q.res == head.res and q.K == head.K and q.rx is None
                and used + one * (len(group) + 1) <= budget):
            group.append(q)
        else:
            left.append(q)
    return group, left


class Server:
    def __init__(self, scene: DeviceScene, mlp: DeviceMLP, resolutions, mem_budget_bytes=16 << 30,
                 max_batch=8, n_streams=4, precision=G.GSPARC_BF16X2, tensor_cores=True,
                 f_c=2.4e9, df=312.5e3, device="cuda", keep_results=True):
        """keep_results=False: a finished request drops its spectrum (the client has taken
        it), so the device memory of retired batches is released as the budget assumes."""
        self.dev = torch.device(device)
        self.keep_results = keep_results
        self.scene, self.mlp = scene, mlp
        self.precision, self.tensor_cores = precision, tensor_cores
        self.f_c, self.df = f_c, df
        self.budget = int(mem_budget_bytes)
        self.used = 0
        self.max_batch = max_batch
        self.streams = [torch.cuda.Stream(self.dev) for _ in range(n_streams)]
        self.free_streams = list(range(n_streams))
        self.waiting = collections.deque()
        self.inflight: list[_Batch] = []
        self.done: list[Request] = []
        self.geom = {}
        for (H, W) in resolutions:
            r = Renderer(H, W, 1, scene.n, f_c=f_c, df=df, device=self.dev)
            r.geometry(scene)
            if r.check() != 0:
                raise RuntimeError("geometry of %dx%d failed" % (W, H))
            self.geom[(H, W)] = r
        self.bands = {}
        self.mlp_s = mlp.struct()
        self.slot_geom = {}   # (slot, H, W) -> Renderer for moving-receiver requests

    def _slot_renderer(self, slot, H, W):
        key = (slot, H, W)
        if key not in self.slot_geom:
            self.slot_geom[key] = Renderer(H, W, 1, self.scene.n, f_c=self.f_c, df=self.df, device=self.dev)
        return self.slot_geom[key]

    def request_bytes(self, H, W, K):
        return self.scene.n * 16 + K * H * W * 8 + H * W * 8

    def submit(self, req: Request):
        H, W = req.res
        if self.request_bytes(H, W, req.K) > self.budget:
            req.rejected = True
            req.t_done = time.perf_counter()
            self.done.append(req)
            return
        self.waiting.append(req)

    def cancel(self, rid) -> bool:
        """Withdraw request `rid` if it is still waiting (one already on the GPU runs to
        completion); it is marked cancelled and counted as done.  Returns whether it was waiting."""
        for q in self.waiting:
            if q.rid == rid:
                self.waiting.remove(q)
                q.cancelled = True
                q.t_done = time.perf_counter()
                self.done.append(q)
                return True
        return False

    def _band(self, K):
        if K not in self.bands:
            self.bands[K] = G.make_band(K, self.f_c, self.df)
        return self.bands[K]

    def _launch(self, reqs, slot):
        H, W = reqs[0].res
        K = reqs[0].K
        B = len(reqs)
        stream = self.streams[slot]
        moving = reqs[0].rx is not None
        if moving:
            r = self._slot_renderer(slot, H, W)
            r.set_receiver(reqs[0].rx, reqs[0].V if reqs[0].V is not None else (1, 0, 0, 0, 1, 0, 0, 0, 1))
        else:
            r = self.geom[(H, W)]
        nbytes = sum(self.request_bytes(H, W, K) for _ in reqs)
        with torch.cuda.stream(stream):
            if moving:
                r.geometry(self.scene, stream=stream)
            tx = torch.tensor([q.tx for q in reqs], dtype=torch.float32).pin_memory().to(self.dev,
                                                                                        non_blocking=True)
            attr = torch.empty((B, self.scene.n, 4), device=self.dev)
            spec = torch.empty((B, K, H, W, 2), device=self.dev)
            logT = torch.empty((B, H, W), device=self.dev)
            nc = torch.empty((B, H, W), dtype=torch.int32, device=self.dev)
            s = stream
            G.gsparc_attr_mlp(tx, r.rx, self.scene.means, self.scene.opacity_logit, self.scene.latent,
                              self.mlp_s, self.precision, attr, s)
            fn = G.gsparc_render_fwd_tc if self.tensor_cores else G.gsparc_render_fwd
            fn(r.view, self._band(K), B, self.scene.n, r.proj, r.tile_ranges, r.sorted_ids, attr, spec,
               logT, nc, None, s)
            ev = torch.cuda.Event()
            ev.record(stream)
        for b, q in enumerate(reqs):
            q.spectrum = spec[b]
        self.used += nbytes
        self.inflight.append(_Batch(reqs, stream, ev, nbytes, (tx, attr, spec, logT, nc)))

    def poll(self):
        """Retire finished batches, then admit and launch what fits.  Returns True when idle."""
        still = []
        for bt in self.inflight:
            if bt.event.query():
                now = time.perf_counter()
                for q in bt.reqs:
                    q.t_done = now
                    if not self.keep_results:
                        q.spectrum = None
                    self.done.append(q)
                self.used -= bt.nbytes
                self.free_streams.append(self.streams.index(bt.stream))
            else:
                still.append(bt)
        self.inflight = still
        while self.waiting and self.free_streams:
            picked = admit(self.waiting, self.used, self.budget, self.max_batch, self.request_bytes)
            if picked is None:
                break                                    # wait for memory to free up
            group, self.waiting = picked
            self._launch(group, self.free_streams.pop())
        return not self.inflight and not self.waiting

    def run(self, requests, arrivals):
        """Serve requests arriving at host times `arrivals` (seconds from now)."""
        t0 = time.perf_counter()
        order = np.argsort(arrivals)
        i = 0
        n = len(requests)
        while len(self.done) < n:
            now = time.perf_counter() - t0
            while i < n and arrivals[order[i]] <= now:
                q = requests[order[i]]
                q.t_arrival = t0 + arrivals[order[i]]
                self.submit(q)
                i += 1
            idle = self.poll()
            if idle and i < n:
                wait = arrivals[order[i]] - (time.perf_counter() - t0)
                if wait > 0:
                    time.sleep(min(wait, 0.001))
        return self.done


def serve_plain(scene: DeviceScene, mlp: DeviceMLP, requests, arrivals, resolutions, f_c=2.4e9,
                df=312.5e3, device="cuda", keep_results=True):
    """Baseline: one request at a time, FP32 network and FP32 compositing, one stream.
    keep_results=False: each request's spectrum is dropped once it is done."""
    dev = torch.device(device)
    geom = {}
    for (H, W) in resolutions:
        r = Renderer(H, W, 1, scene.n, f_c=f_c, df=df, device=dev)
        r.geometry(scene)
        geom[(H, W)] = r
    torch.cuda.synchronize(dev)
    mlp_s = mlp.struct()
    bands = {}
    moving = {}
    t0 = time.perf_counter()
    order = np.argsort(arrivals)
    for idx in order:
        q = requests[idx]
        q.t_arrival = t0 + arrivals[idx]
        now = time.perf_counter()
        if now < q.t_arrival:
            time.sleep(q.t_arrival - now)
        H, W = q.res
        if q.rx is not None:                       # moving receiver: its own geometry first
            if (H, W) not in moving:
                moving[(H, W)] = Renderer(H, W, 1, scene.n, f_c=f_c, df=df, device=dev)
            r = moving[(H, W)]
            r.set_receiver(q.rx, q.V if q.V is not None else (1, 0, 0, 0, 1, 0, 0, 0, 1))
            r.geometry(scene)
        else:
            r = geom[(H, W)]
        if q.K not in bands:
            bands[q.K] = G.make_band(q.K, f_c, df)
        tx = torch.tensor([q.tx], dtype=torch.float32, device=dev)
        attr = torch.empty((1, scene.n, 4), device=dev)
        spec = torch.empty((1, q.K, H, W, 2), device=dev)
        logT = torch.empty((1, H, W), device=dev)
        nc = torch.empty((1, H, W), dtype=torch.int32, device=dev)
        G.gsparc_attr_mlp(tx, r.rx, scene.means, scene.opacity_logit, scene.latent, mlp_s, G.GSPARC_FP32, attr)
        G.gsparc_render_fwd(r.view, bands[q.K], 1, scene.n, r.proj, r.tile_ranges, r.sorted_ids, attr, spec,
                            logT, nc)
        torch.cuda.current_stream(dev).synchronize()
        q.t_done = time.perf_counter()
        q.spectrum = spec[0] if keep_results else None
    return requests


def latency_stats(reqs):
    lat = np.array([(q.t_done - q.t_arrival) * 1e3 for q in reqs if not q.rejected and not q.cancelled])
    if lat.size == 0:
        return {}
    span = max(q.t_done for q in reqs) - min(q.t_arrival for q in reqs)
    return {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean()), "spectra_per_s": len(lat) / span, "served": int(lat.size),
            "rejected": int(sum(q.rejected for q in reqs)), "cancelled": int(sum(q.cancelled for q in reqs))}
