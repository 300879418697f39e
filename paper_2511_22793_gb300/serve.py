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

Memory: the server allocates its whole budget once, as one device arena, and every admitted
batch's buffers (attributes, spectrum, per-pixel state) are carved from it (`Arena`, first fit);
each stream slot owns a pinned host buffer and a device buffer for its batch's transmitters.  No
request allocates device or pinned memory on its way through the server.

Scheduling (`Server.poll`, admission in `admit`):
  * finished batches are detected with CUDA events (no host synchronisation)
    and release their stream slot, and their block of the arena unless their
    results are kept (then `Server.release` returns it);
  * waiting requests are admitted oldest first while a stream slot is free and
    the arena has a block for the batch (attribute buffer + spectrum + per-pixel
    state of every request in it); an admitted request joins a batch with the other
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


class Arena:
    """Offsets in one device allocation of `size` bytes (host bookkeeping only): first fit over a
    sorted free list, every block aligned to `align` bytes, neighbours merged on free.  The
    server carves each admitted batch's buffers from it, so that admission by memory is
    admission into memory that is already there (no allocation on a request's path)."""

    def __init__(self, size, align=256):
        self.size, self.align = int(size), int(align)
        self.free_list = [(0, self.size)]          # (offset, length), sorted by offset
        self.taken = {}                            # offset -> length
        self.used = 0

    def _round(self, n):
        return (int(n) + self.align - 1) // self.align * self.align

    def fits(self, n):
        n = self._round(n)
        return any(ln >= n for _, ln in self.free_list)

    def alloc(self, n):
        """Offset of a block of at least n bytes, or None when no free block is large enough."""
        n = self._round(max(int(n), 1))
        for i, (off, ln) in enumerate(self.free_list):
            if ln >= n:
                if ln == n:
                    del self.free_list[i]
                else:
                    self.free_list[i] = (off + n, ln - n)
                self.taken[off] = n
                self.used += n
                return off
        return None

    def free(self, off):
        n = self.taken.pop(off)
        self.used -= n
        fl = self.free_list
        i = 0
        while i < len(fl) and fl[i][0] < off:
            i += 1
        fl.insert(i, (off, n))
        # merge with the next block, then with the previous one
        if i + 1 < len(fl) and fl[i][0] + fl[i][1] == fl[i + 1][0]:
            fl[i] = (fl[i][0], fl[i][1] + fl[i + 1][1])
            del fl[i + 1]
        if i > 0 and fl[i - 1][0] + fl[i - 1][1] == fl[i][0]:
            fl[i - 1] = (fl[i - 1][0], fl[i - 1][1] + fl[i][1])
            del fl[i]


@dataclass
class _Batch:
    reqs: list
    slot: int
    event: torch.cuda.Event
    offset: int                 # the batch's block in the arena
    nbytes: int
    live: int = 0               # requests whose result still holds the block


def admit(waiting, used, budget, max_batch, request_bytes, fits=None):
    """Admission of the oldest waiting request and the batch it leads (host logic only).

    The head is admitted if its bytes fit beside `used` within `budget`; a moving-receiver head
    (its own geometry) runs alone; otherwise every later waiting request of the same
    (resolution, subcarrier count) with the fixed receiver joins, oldest first, while the batch
    has fewer than `max_batch` requests and its bytes still fit.  fits(bytes), when given, says
    whether a batch of that size has a contiguous block left (the arena may be fragmented): the
    newest members are dropped until it does.  Returns (batch, the requests left waiting in
    their order), or None when the head does not fit (nothing is taken)."""
    head = waiting[0]
    H, W = head.res
    one = request_bytes(H, W, head.K)
    if used + one > budget or (fits is not None and not fits(one)):
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
    if fits is not None:
        while len(group) > 1 and not fits(one * len(group)):
            q = group.pop()
            # back into the queue at its place (the queue is in arrival order)
            left = collections.deque(sorted(list(left) + [q], key=lambda r: _order(waiting, r)))
    return group, left


def _order(waiting, r):
    for i, q in enumerate(waiting):
        if q is r:
            return i
    return len(waiting)


class Server:
    def __init__(self, scene: DeviceScene, mlp: DeviceMLP, resolutions, mem_budget_bytes=16 << 30,
                 max_batch=8, n_streams=4, precision=G.GSPARC_BF16X2, tensor_cores=True,
                 f_c=2.4e9, df=312.5e3, device="cuda", keep_results=True, moving_receiver=True):
        """mem_budget_bytes: the device arena every admitted batch's buffers (attributes,
        spectrum, per-pixel state) are carved from, allocated once here.  keep_results=False: a
        finished request's spectrum is dropped as it completes and its memory returns to the
        arena; True: Request.spectrum stays a view into the arena until release(request)."""
        self.dev = torch.device(device)
        self.keep_results = keep_results
        self.scene, self.mlp = scene, mlp
        self.precision, self.tensor_cores = precision, tensor_cores
        self.f_c, self.df = f_c, df
        self.budget = int(mem_budget_bytes)
        self.arena = Arena(self.budget)
        self.arena_buf = torch.empty(self.budget, dtype=torch.uint8, device=self.dev)
        self.max_batch = max_batch
        self.streams = [torch.cuda.Stream(self.dev) for _ in range(n_streams)]
        # per stream slot: the batch's transmitters in pinned host memory and on the device
        self.tx_host = [torch.zeros((max_batch, 3), dtype=torch.float32).pin_memory() for _ in range(n_streams)]
        self.tx_dev = [torch.zeros((max_batch, 3), dtype=torch.float32, device=self.dev) for _ in range(n_streams)]
        self.free_streams = list(range(n_streams))
        self.waiting = collections.deque()
        self.inflight: list[_Batch] = []
        self.held = {}          # rid -> the batch whose block its result lives in
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
        # per (slot, resolution): the geometry buffers of a moving-receiver request, allocated here
        # (moving_receiver=False leaves them out; such requests are then rejected)
        self.slot_geom = {}
        if moving_receiver:
            for slot in range(n_streams):
                for (H, W) in resolutions:
                    self.slot_geom[(slot, H, W)] = Renderer(H, W, 1, scene.n, f_c=f_c, df=df, device=self.dev)

    @property
    def used(self):
        return self.arena.used

    @staticmethod
    def _layout(n, B, H, W, K):
        """Byte offsets of one batch's buffers inside its block: attributes [B,N,4], spectrum
        [B,K,H,W,2], final log T [B,H,W], contributor positions [B,H,W]; each 256-aligned."""
        al = lambda x: (x + 255) // 256 * 256
        o_attr = 0
        o_spec = o_attr + al(B * n * 16)
        o_logT = o_spec + al(B * K * H * W * 8)
        o_nc = o_logT + al(B * H * W * 4)
        return o_attr, o_spec, o_logT, o_nc, o_nc + al(B * H * W * 4)

    def request_bytes(self, H, W, K):
        return self._layout(self.scene.n, 1, H, W, K)[-1]

    def submit(self, req: Request):
        H, W = req.res
        if self.request_bytes(H, W, req.K) > self.budget or (req.rx is not None and not self.slot_geom) or \
                (H, W) not in self.geom:
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

    def release(self, req: Request):
        """The client is done with req.spectrum (a view into the arena): its memory may be reused."""
        bt = self.held.pop(req.rid, None)
        req.spectrum = None
        if bt is not None:
            bt.live -= 1
            if bt.live == 0:
                self.arena.free(bt.offset)

    def _band(self, K):
        if K not in self.bands:
            self.bands[K] = G.make_band(K, self.f_c, self.df)
        return self.bands[K]

    def _view(self, off, nbytes, dtype, shape):
        return self.arena_buf[off:off + nbytes].view(dtype).view(*shape)

    def _launch(self, reqs, slot, offset):
        H, W = reqs[0].res
        K = reqs[0].K
        B = len(reqs)
        n = self.scene.n
        stream = self.streams[slot]
        moving = reqs[0].rx is not None
        if moving:
            r = self.slot_geom[(slot, H, W)]
            r.set_receiver(reqs[0].rx, reqs[0].V if reqs[0].V is not None else (1, 0, 0, 0, 1, 0, 0, 0, 1))
        else:
            r = self.geom[(H, W)]
        o_attr, o_spec, o_logT, o_nc, total = self._layout(n, B, H, W, K)
        attr = self._view(offset + o_attr, B * n * 16, torch.float32, (B, n, 4))
        spec = self._view(offset + o_spec, B * K * H * W * 8, torch.float32, (B, K, H, W, 2))
        logT = self._view(offset + o_logT, B * H * W * 4, torch.float32, (B, H, W))
        nc = self._view(offset + o_nc, B * H * W * 4, torch.int32, (B, H, W))
        th = self.tx_host[slot].numpy()
        for b, q in enumerate(reqs):
            th[b] = q.tx
        tx = self.tx_dev[slot][:B]
        with torch.cuda.stream(stream):
            if moving:
                r.geometry(self.scene, stream=stream)
            tx.copy_(self.tx_host[slot][:B], non_blocking=True)
            G.gsparc_attr_mlp(tx, r.rx, self.scene.means, self.scene.opacity_logit, self.scene.latent,
                              self.mlp_s, self.precision, attr, stream)
            fn = G.gsparc_render_fwd_tc if self.tensor_cores else G.gsparc_render_fwd
            fn(r.view, self._band(K), B, n, r.proj, r.tile_ranges, r.sorted_ids, attr, spec,
               logT, nc, None, stream, d_status=r.status)
            ev = torch.cuda.Event()
            ev.record(stream)
        for b, q in enumerate(reqs):
            q.spectrum = spec[b]
        self.inflight.append(_Batch(reqs, slot, ev, offset, total, live=B))

    def poll(self):
        """Retire finished batches, then admit and launch what fits.  Returns True when idle."""
        still = []
        for bt in self.inflight:
            if bt.event.query():
                now = time.perf_counter()
                for q in bt.reqs:
                    q.t_done = now
                    self.done.append(q)
                    if self.keep_results:
                        self.held[q.rid] = bt
                    else:
                        q.spectrum = None
                if not self.keep_results:
                    self.arena.free(bt.offset)
                self.free_streams.append(bt.slot)
            else:
                still.append(bt)
        self.inflight = still
        while self.waiting and self.free_streams:
            picked = admit(self.waiting, self.arena.used, self.budget, self.max_batch, self.request_bytes,
                           fits=self.arena.fits)
            if picked is None:
                if not self.inflight:
                    raise RuntimeError("the arena is full of results not yet released (Server.release)")
                break                                    # wait for memory to free up
            group, self.waiting = picked
            H, W = group[0].res
            off = self.arena.alloc(self._layout(self.scene.n, len(group), H, W, group[0].K)[-1])
            self._launch(group, self.free_streams.pop(), off)
        return not self.inflight and not self.waiting

    def run(self, requests, arrivals):
        """Serve requests arriving at host times `arrivals` (seconds from now)."""
        t0 = time.perf_counter()
        order = np.argsort(arrivals)
        i = 0
        n = len(requests)
        start = len(self.done)
        while len(self.done) - start < n:
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
    """Baseline: one request at a time, FP32 network and FP32 compositing, one stream.  Buffers
    are allocated once per (resolution, subcarrier count) and the transmitter goes through a
    pinned buffer.  keep_results=True: each request gets a copy of its spectrum; False: it is
    dropped once the request is done."""
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
    bufs = {}
    tx_host = torch.zeros((1, 3), dtype=torch.float32).pin_memory()
    tx = torch.zeros((1, 3), dtype=torch.float32, device=dev)
    attr = torch.empty((1, scene.n, 4), device=dev)
    stream = torch.cuda.current_stream(dev)
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
        if (H, W, q.K) not in bufs:
            bufs[(H, W, q.K)] = (torch.empty((1, q.K, H, W, 2), device=dev), torch.empty((1, H, W), device=dev),
                                 torch.empty((1, H, W), dtype=torch.int32, device=dev))
        spec, logT, nc = bufs[(H, W, q.K)]
        tx_host.numpy()[0] = q.tx
        tx.copy_(tx_host, non_blocking=True)
        G.gsparc_attr_mlp(tx, r.rx, scene.means, scene.opacity_logit, scene.latent, mlp_s, G.GSPARC_FP32, attr)
        G.gsparc_render_fwd(r.view, bands[q.K], 1, scene.n, r.proj, r.tile_ranges, r.sorted_ids, attr, spec,
                            logT, nc, d_status=r.status)
        stream.synchronize()
        q.t_done = time.perf_counter()
        q.spectrum = spec[0].clone() if keep_results else None
    for r in list(geom.values()) + list(moving.values()):
        if r.check() != 0:
            raise RuntimeError("plain path status %d" % r.check())
    return requests


def latency_stats(reqs):
    lat = np.array([(q.t_done - q.t_arrival) * 1e3 for q in reqs if not q.rejected and not q.cancelled])
    if lat.size == 0:
        return {}
    span = max(q.t_done for q in reqs) - min(q.t_arrival for q in reqs)
    return {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean()), "spectra_per_s": len(lat) / span, "served": int(lat.size),
            "rejected": int(sum(q.rejected for q in reqs)), "cancelled": int(sum(q.cancelled for q in reqs))}
