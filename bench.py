"""Benchmark of the splatting hot path on one GB300 (or N independent replicas).

Workload (one step = one pass of the whole path over one query):
  50,000 Gaussians (seeded synthetic scene: means uniform in a 10 m cube
  around the receiver, upper hemisphere; log-scales N(-1.5, 0.5); random unit
  quaternions; opacity logits N(0,1); 16-dim latents N(0,1)), one transmitter,
  64 subcarriers 312.5 kHz apart about 2.4 GHz, 360x90 hemisphere (1-degree
  bins, 16x16 tiles), attribute network 20 -> 32 -> 32 -> 3 (split-BF16 on
  the tensor cores in the default configuration, FP32 with --render fp32).
  Step = project -> bin/sort -> attribute network -> render forward ->
  complex L2 loss against a target spectrum (rendered by the same path from a
  second seeded scene, once, outside the timed region) -> render backward ->
  network backward -> projection backward.

Metric: Gaussian-pixel-subcarrier units per second, where a unit is one
Gaussian composited at one pixel (counted up to termination by the forward
kernel's per-pixel counter) for one subcarrier; fwd+bwd per step.

`value` times the step on the device with inputs resident in HBM (CUDA
events on the launching stream, L2 flushed by a 256 MiB write between timed
steps; the loss fused into the forward).  `e2e` times the step through the C
ABI with the scene, network, transmitters and target copied from pinned host
memory and the loss read back, inside the timed region; its graph overlaps
the target's copy with projection, binning and the forward (which then writes
the spectrum, and the loss follows once the target is in), and it is checked
against the device-resident step's loss and gradients before timing.  `roofline` reports the dominant kernel against the FP32 ALU
peak; `cpu_baseline` times the FP64 oracle on a bounded pixel sample.

Multi-GPU: queries are independent, so N ranks run N replicas on their own
transmitters (weak scaling) with no data-path collective; timing is the max
over ranks.  `--impl reference` times the FP64 CPU oracle as the reference arm.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Gaussian·pixel·subcarrier/s fwd+bwd and p50/p99 spectrum latency vs plain GPU path"
UNIT = "Gaussian·pixel·subcarrier/s"
WORKLOAD = dict(name="fwd+bwd, 50k Gaussians, 64 subcarriers, 360x90, hidden 32, 1 transmitter",
                n=50_000, K=64, H=90, W=360, hidden=32, B=1, f_c=2.4e9, df=312.5e3)
FLOP_FWD_UNIT = 4     # z += w * e^{j psi}: two FMAs per (pixel, Gaussian, subcarrier)
FLOP_BWD_UNIT = 12    # Re, Im and frequency-weighted Im of conj(g) e^{j psi}: six FMAs
FP32_LANES_PER_SM = 128


def _env_int(k, d):
    try:
        return int(os.environ.get(k, d))
    except ValueError:
        return d


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "25"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def wait_first(self, timeout=3.0):
        """Block until the first sample arrived (nvidia-smi takes a moment to start)."""
        t0 = time.perf_counter()
        while self.proc is not None and not self.lines and time.perf_counter() - t0 < timeout:
            time.sleep(0.01)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f)
    return {}


# --------------------------------------------------------------------------------------------
# our arm
# --------------------------------------------------------------------------------------------

def run_ours(args, rank, world, local_rank):
    import torch

    from paper_2511_22793_gb300 import gsparc as G
    from paper_2511_22793_gb300 import synth
    from paper_2511_22793_gb300.pipeline import DeviceMLP, DeviceScene, PackedInputs, Renderer
    from paper_2511_22793_gb300.replicas import job_totals, rank_queries, throughput

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    wl = WORKLOAD
    n, K, H, W, hidden, B = wl["n"], wl["K"], wl["H"], wl["W"], wl["hidden"], wl["B"]
    sc = synth.make_scene(n, seed=0)
    mlp = synth.make_mlp(hidden, seed=3)
    tx = rank_queries(synth.make_tx(B * world, seed=2), B, rank, world)
    r = Renderer(H, W, K, n, f_c=wl["f_c"], df=wl["df"], device=dev)
    stream = torch.cuda.current_stream(dev)

    # target spectrum: the same path on a second seeded scene (not timed)
    sc_t = synth.make_scene(n, seed=1)
    rt = Renderer(H, W, K, n, f_c=wl["f_c"], df=wl["df"], device=dev)
    dst = DeviceScene.from_host(sc_t, dev)
    dm = DeviceMLP.from_host(mlp, dev)
    txd = torch.tensor(tx, device=dev)
    rt.geometry(dst)
    target = rt.render(rt.attributes(dst, dm, txd))[0].clone()
    del rt, dst

    # the step's inputs (scene, network, transmitters, target spectrum) share one device
    # allocation: the end-to-end step moves them from pinned host memory in one copy
    arrays = list(sc.arrays()) + list(mlp.arrays()) + [txd, target]
    inp = PackedInputs([tuple(np.shape(a)) if not isinstance(a, torch.Tensor) else tuple(a.shape)
                        for a in arrays], dev)
    for i, a in enumerate(arrays):
        inp.set_host(i, a)
    inp.upload()
    torch.cuda.synchronize(dev)
    ds = DeviceScene(*inp.views[0:5])
    dm = DeviceMLP(hidden, *inp.views[5:11])
    txd, target = inp.views[11], inp.views[12]
    attr = torch.empty((B, n, 4), device=dev)
    spec, logT, nc = r.alloc_outputs(B)
    n_used = torch.zeros((B, H, W), dtype=torch.int32, device=dev)
    loss = torch.zeros(1, device=dev)
    d_spec = torch.empty_like(spec)
    # every gradient buffer is a view of one flat allocation, zeroed by one memset per step
    shapes = [attr.shape, r.proj.shape] + [t.shape for t in ds.tensors()] + [t.shape for t in dm.tensors()]
    sizes = [int(np.prod(sh)) for sh in shapes]
    offs = np.cumsum([0] + [(z + 63) // 64 * 64 for z in sizes])
    gbuf = torch.zeros(int(offs[-1]), device=dev)
    views = [gbuf[int(o):int(o) + z].view(sh) for o, z, sh in zip(offs[:-1], sizes, shapes)]
    d_attr, d_proj, grads = views[0], views[1], views[2:]
    mlp_s = dm.struct()
    grad_s = G.make_mlp_grad(*grads[5:])
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    launches_per_step = 0
    ev = {}
    render_fwd = G.gsparc_render_fwd_tc if args.render == "tc" else G.gsparc_render_fwd
    # tensor-core configuration: the backward scheduled over the SMs (walk lengths, then the
    # longest work items first, long walks split in two), its front chunks fed by the fused
    # forward's s_tot and its schedule by the forward's tile walks
    s_tot = r.s_tot_buffer(B) if args.render == "tc" else None
    walks = r.walk_buffer(B) if args.render == "tc" else None
    bwd_ws = torch.zeros(G.gsparc_render_bwd_tc_workspace(r.view, r.band, B), dtype=torch.uint8, device=dev)

    def render_bwd():
        if args.render == "tc":
            G.gsparc_render_bwd_tc_balanced(r.view, r.band, B, n, r.proj, r.tile_ranges, r.sorted_ids, attr,
                                            None, s_tot, logT, nc, d_spec, bwd_ws, d_attr, d_proj, tile_walk=walks)
        else:
            G.gsparc_render_bwd(r.view, r.band, B, n, r.proj, r.tile_ranges, r.sorted_ids, attr, logT, nc,
                                d_spec, d_attr, d_proj)
    # the tensor-core configuration runs the attribute network forward and backward on the tensor
    # cores as well (split-BF16, the same products in both, so the ReLU masks agree)
    mlp_tc = args.render == "tc" and hidden in (16, 32)
    mlp_prec = G.GSPARC_BF16X2 if mlp_tc else G.GSPARC_FP32

    def mlp_bwd(scene):
        if mlp_tc:
            G.gsparc_attr_mlp_bwd_tc(txd, r.rx, scene.means, scene.opacity_logit, scene.latent, mlp_s,
                                     G.GSPARC_BF16X2, d_attr, grads[0], grads[3], grads[4], grad_s)
        else:
            G.gsparc_attr_mlp_bwd(txd, r.rx, scene.means, scene.opacity_logit, scene.latent, mlp_s,
                                  d_attr, grads[0], grads[3], grads[4], grad_s)

    def stage(name, fn):
        if name in ev:
            ev[name][0].record(stream)
        fn()
        if name in ev:
            ev[name][1].record(stream)

    side = torch.cuda.Stream(dev)

    def step(scene: DeviceScene, tgt, concurrent=False):
        """One training step.  concurrent: the gradient zeroing and the attribute network run on
        a side stream beside projection and bin/sort (they need neither), and the projection
        backward beside the network backward (both only add into the gradients); used for the
        graph, while the eager per-kernel timing keeps one stream."""
        cur = torch.cuda.current_stream(dev)   # the capture stream while a graph is captured
        if concurrent:
            fork = torch.cuda.Event()
            fork.record(cur)
            side.wait_event(fork)
            with torch.cuda.stream(side):
                gbuf.zero_()   # the gradients are first written by the compositing backward
            G.gsparc_attr_mlp(txd, r.rx, scene.means, scene.opacity_logit, scene.latent, mlp_s, mlp_prec,
                              attr, side)
            joined = torch.cuda.Event()
            joined.record(side)
        else:
            gbuf.zero_()
        stage("project", lambda: G.gsparc_project(r.view, scene.means, scene.log_scales, scene.quats,
                                                  r.proj))
        stage("bin_sort", lambda: G.gsparc_bin_sort(r.view, n, r.proj, r.capacity, r.ws, r.sorted_ids,
                                                    None, r.tile_ranges, r.n_pairs, r.status))
        if concurrent:
            cur.wait_event(joined)
        else:
            stage("attr_mlp", lambda: G.gsparc_attr_mlp(txd, r.rx, scene.means, scene.opacity_logit,
                                                        scene.latent, mlp_s, mlp_prec, attr))
        if args.render == "tc":
            # the loss fused into the forward's epilogue: it writes dL/dz, not the spectrum
            stage("render_fwd", lambda: G.gsparc_render_fwd_l2_tc(r.view, r.band, B, n, r.proj, r.tile_ranges,
                                                                  r.sorted_ids, attr, tgt, loss, d_spec, None,
                                                                  logT, nc, n_used, s_tot=s_tot,
                                                                  tile_walk=walks))
        else:
            stage("render_fwd", lambda: render_fwd(r.view, r.band, B, n, r.proj, r.tile_ranges,
                                                   r.sorted_ids, attr, spec, logT, nc, n_used))
            stage("l2_loss", lambda: G.gsparc_l2_loss(spec, tgt, loss, d_spec))
        stage("render_bwd", render_bwd)

        def proj_bwd(s=None):
            G.gsparc_project_bwd(r.view, scene.means, scene.log_scales, scene.quats, d_proj, grads[0],
                                 grads[1], grads[2], s)

        if concurrent:
            fork2 = torch.cuda.Event()
            fork2.record(cur)
            side.wait_event(fork2)
            proj_bwd(side)
            joined2 = torch.cuda.Event()
            joined2.record(side)
            mlp_bwd(scene)
            cur.wait_event(joined2)
        else:
            stage("attr_mlp_bwd", lambda: mlp_bwd(scene))
            stage("project_bwd", proj_bwd)

    copy_s = torch.cuda.Stream(dev)
    spec_e2e = spec

    def step_e2e(scene: DeviceScene, tgt):
        """The tensor-core step with host-resident inputs, its copies captured with it: scene,
        network and transmitters first, then the 16.6 MB target spectrum on a third stream,
        overlapping projection, binning and the forward.  The forward therefore writes the
        spectrum and gsparc_l2_loss forms the loss and dL/dz once the target is in (the fused
        form would hold the forward until the whole target had crossed the host link); the
        backward's front chunks form s_tot from the spectrum.  Same loss, same gradients."""
        cur = torch.cuda.current_stream(dev)
        inp.upload(0, len(inp.views) - 1)
        scene_in = torch.cuda.Event()
        scene_in.record(cur)
        copy_s.wait_event(scene_in)
        with torch.cuda.stream(copy_s):
            inp.upload(len(inp.views) - 1)
        tgt_in = torch.cuda.Event()
        tgt_in.record(copy_s)
        side.wait_event(scene_in)
        with torch.cuda.stream(side):
            gbuf.zero_()
        G.gsparc_attr_mlp(txd, r.rx, scene.means, scene.opacity_logit, scene.latent, mlp_s, mlp_prec, attr, side)
        joined = torch.cuda.Event()
        joined.record(side)
        G.gsparc_project(r.view, scene.means, scene.log_scales, scene.quats, r.proj)
        G.gsparc_bin_sort(r.view, n, r.proj, r.capacity, r.ws, r.sorted_ids, None, r.tile_ranges, r.n_pairs,
                          r.status)
        cur.wait_event(joined)
        G.gsparc_render_fwd_tc(r.view, r.band, B, n, r.proj, r.tile_ranges, r.sorted_ids, attr, spec_e2e, logT,
                               nc, n_used)
        cur.wait_event(tgt_in)
        G.gsparc_l2_loss(spec_e2e, tgt, loss, d_spec)
        G.gsparc_render_bwd_tc_balanced(r.view, r.band, B, n, r.proj, r.tile_ranges, r.sorted_ids, attr, spec_e2e,
                                        None, logT, nc, d_spec, bwd_ws, d_attr, d_proj)
        fork2 = torch.cuda.Event()
        fork2.record(cur)
        side.wait_event(fork2)
        G.gsparc_project_bwd(r.view, scene.means, scene.log_scales, scene.quats, d_proj, grads[0], grads[1],
                             grads[2], side)
        joined2 = torch.cuda.Event()
        joined2.record(side)
        mlp_bwd(scene)
        cur.wait_event(joined2)

    # kernels of ours launched per step: project 1, bin/sort 3 (count + scan, emit, per-tile
    # sort), network 1, render 1, loss 1 (fused into the tensor-core forward), render bwd 1
    # (+ its schedule in the tensor-core form), network bwd 1, projection bwd 1
    launches_per_step = 1 + 3 + 1 + 1 + (1 if args.render != "tc" else 0) + (2 if args.render == "tc" else 1) + 1 + 1

    for _ in range(args.warmup):
        step(ds, target)
    torch.cuda.synchronize(dev)
    st = r.check()
    if st != 0:
        raise RuntimeError("device status %d after warm-up" % st)
    units = int(n_used.sum().item()) * K
    n_pairs = int(r.n_pairs.item())

    dist = world > 1
    if dist:
        import torch.distributed as tdist
    names = ["project", "bin_sort", "attr_mlp", "render_fwd"] + (["l2_loss"] if args.render != "tc" else []) + \
        ["render_bwd", "attr_mlp_bwd", "project_bwd"]
    # per-kernel durations: eager steps with CUDA events around every stage (kernel time does not
    # depend on how it was launched); the headline times the whole step as one CUDA graph
    per_kernel = {k: [] for k in names}
    for _ in range(min(args.steps, 50)):
        flush.fill_(1.0)
        for k in names:
            ev[k] = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
        step(ds, target)
        torch.cuda.synchronize(dev)
        for k in names:
            per_kernel[k].append(ev[k][0].elapsed_time(ev[k][1]))
    ev.clear()
    # the step as one CUDA graph: the library only enqueues stream-ordered work, so it captures
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        step(ds, target, concurrent=True)
    for _ in range(3):
        graph.replay()
    torch.cuda.synchronize(dev)
    if r.check() != 0:
        raise RuntimeError("device status after graph warm-up")
    step_ms = []
    sampler = ClockSampler(local_rank)
    if dist:
        tdist.barrier()
    torch.cuda.synchronize(dev)
    sampler.start()
    sampler.wait_first()
    for _ in range(args.steps):
        flush.fill_(1.0)                      # evict L2 between timed steps (not timed)
        s0 = torch.cuda.Event(enable_timing=True)
        s1 = torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        graph.replay()
        s1.record(stream)
        s1.synchronize()
        step_ms.append(s0.elapsed_time(s1))
    torch.cuda.synchronize(dev)
    # whole job: the units all ranks processed over the slowest rank's time
    job_units, total_ms = job_totals(units * args.steps, sum(step_ms), device=dev)
    if dist:
        tdist.barrier()

    # end to end: host (pinned) inputs copied into the buffers the graph reads, the step, the loss
    # read back -- all inside the timed region
    # (the packed inputs' pinned mirror holds the scene, network, transmitters and target)
    host_loss = torch.empty(1).pin_memory()
    h2d = inp.nbytes
    d2h = host_loss.numel() * host_loss.element_size()
    # every input copied from the pinned mirror inside the timed step.  The host link moves
    # ~165 GB/s (measured), so the 22 MB take ~0.13 ms: the tensor-core step overlaps the
    # target's copy with projection, binning and the forward (step_e2e, one graph); the FP32
    # configuration copies first, then replays its step graph.
    graph_e2e = None
    e2e_agree = None
    e2e_copies = "one pinned host-to-device copy of all inputs (scene, network, transmitters, target), " \
                 "then the step's graph"
    if args.render == "tc":
        graph_e2e = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph_e2e):
            step_e2e(ds, target)
        for _ in range(3):
            graph_e2e.replay()
        torch.cuda.synchronize(dev)
        if r.check() != 0:
            raise RuntimeError("device status after the end-to-end graph's warm-up")
        # the two step graphs compute the same loss and gradients (not timed)
        graph.replay()
        torch.cuda.synchronize(dev)
        loss_a, grad_a = float(loss), gbuf.clone()
        graph_e2e.replay()
        torch.cuda.synchronize(dev)
        loss_b, grad_b = float(loss), gbuf.clone()
        e2e_agree = {"loss_rel": abs(loss_a - loss_b) / abs(loss_a),
                     "grad_rel_l2": float((grad_a - grad_b).norm() / grad_a.norm())}
        if e2e_agree["loss_rel"] > 1e-5 or e2e_agree["grad_rel_l2"] > 1e-4:
            raise RuntimeError("end-to-end step disagrees with the step graph: %s" % e2e_agree)
        e2e_copies = "inside the step's graph: scene, network and transmitters first, the target spectrum " \
                     "on a third stream beside projection, binning and the forward (spectrum written, " \
                     "loss by gsparc_l2_loss once the target is in)"
    e2e_ms = []
    for it in range(args.warmup + args.steps):
        flush.fill_(1.0)
        if dist and it == args.warmup:
            tdist.barrier()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        if graph_e2e is not None:
            graph_e2e.replay()
        else:
            inp.upload()
            graph.replay()
        host_loss.copy_(loss, non_blocking=True)
        torch.cuda.current_stream(dev).synchronize()
        if it >= args.warmup:
            e2e_ms.append((time.perf_counter() - t0) * 1e3)
    clocks = sampler.stop()   # sampled over both timed regions (device-timed and end to end)
    job_units_e2e, e2e_total = job_totals(units * len(e2e_ms), sum(e2e_ms), device=dev)

    # dominant kernel and its roofline
    avg = {k: statistics.mean(v) for k, v in per_kernel.items()}
    top = max(avg, key=avg.get)
    peaks = measured_peaks()
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    fp32_peak = sms * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12      # TFLOP/s
    unit_flop = {"render_bwd": FLOP_BWD_UNIT, "render_fwd": FLOP_FWD_UNIT}
    # DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of the tensor-core
    # compositing kernels in this step (50k Gaussians, 64 subcarriers, 360x90, one transmitter),
    # from one ncu capture of each current kernel (the forward with its fused loss)
    traffic = {"render_bwd": 17510912, "render_fwd": 17157888} if args.render == "tc" else {}
    if top in unit_flop:
        achieved = units * unit_flop[top] / (avg[top] * 1e-3) / 1e12
        roofline = {"kernel": top, "bound": "alu", "achieved": achieved, "peak": fp32_peak,
                    "unit": "TFLOP/s", "frac": achieved / fp32_peak, "traffic": traffic.get(top),
                    "traffic_unit": "bytes per launch (DRAM read + write)",
                    "peak_note": "%d SMs x 128 FP32 lanes x 2 flop x %.0f MHz (max SM clock)"
                                 % (sms, sm_max)}
        if clocks and clocks.get("sm_mhz"):
            # the same peak at the median SM clock sampled under load
            roofline["frac_at_measured_clock"] = achieved / (fp32_peak * float(clocks["sm_mhz"]) / sm_max)
    else:
        roofline = {"kernel": top, "bound": "hbm", "achieved": None,
                    "peak": float(peaks.get("hbm_gbs", 6800.0)), "unit": "GB/s", "frac": None,
                    "traffic": None}

    value = throughput(job_units, total_ms)
    e2e_value = throughput(job_units_e2e, e2e_total)
    sorted_ms = sorted(step_ms)
    latency = query_latency(dev, queries=max(50, min(args.steps, 400)))
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded)",
        "config": {"workload": wl["name"], "n_gaussians": n, "subcarriers": K, "H": H, "W": W,
                   "hidden": hidden, "transmitters_per_step": B, "pairs": n_pairs,
                   "units_per_step": job_units // args.steps, "l2": "flushed (256 MiB write) between timed steps",
                   "compositing": "subcarrier sums on tensor cores (split-BF16 products, FP32 "
                                  "accumulation), transmittance and gradients FP32"
                                  if args.render == "tc" else "FP32 CUDA cores",
                   "attribute_network": "tensor cores, split-BF16 products, FP32 accumulation "
                                        "(forward and backward)" if mlp_tc else "FP32 CUDA cores",
                   "parallelism": "replicas x%d" % world},
        "latency_ms": {"p50": float(np.percentile(step_ms, 50)), "p99": float(np.percentile(step_ms, 99)),
                       "min": sorted_ms[0]},
        "kernels_ms": avg,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "ms_per_step": e2e_total / args.steps, "copies": e2e_copies,
                "agrees_with_step_graph": e2e_agree},
        "gpu_launches": launches_per_step * args.steps,
        "launch": "whole step captured once as a CUDA graph (gradient zeroing and network forward "
                  "beside projection and bin/sort, projection backward beside network backward, on a "
                  "second stream), replayed per timed step",
        "query_latency": latency,
        "roofline": roofline,
        "clocks": clocks,
    }
    return out, units, sc, mlp, tx


def query_latency(dev, queries=200):
    """Single-query forward latency (1,024 Gaussians, 1 subcarrier, 360x90, hidden 32, FP32):
    the plain one-query path (projection, bin/sort, network, render) and the query part alone
    when the receiver is fixed and the geometry is cached (network + render), each timed per
    query with CUDA events, L2 not flushed (a serving loop keeps the scene hot)."""
    import torch

    from paper_2511_22793_gb300 import synth
    from paper_2511_22793_gb300.pipeline import DeviceMLP, DeviceScene, Renderer

    n, K, H, W = 1024, 1, 90, 360
    sc = synth.make_scene(n, seed=0)
    mlp = synth.make_mlp(32, seed=3)
    txs = torch.tensor(synth.make_tx(queries, seed=2), device=dev)
    r = Renderer(H, W, K, n, device=dev)
    ds = DeviceScene.from_host(sc, dev)
    dm = DeviceMLP.from_host(mlp, dev)
    attr = torch.empty((1, n, 4), device=dev)
    outs = r.alloc_outputs(1)
    stream = torch.cuda.current_stream(dev)

    tx_buf = torch.empty((1, 3), device=dev)

    def full():
        r.geometry(ds)
        r.attributes(ds, dm, tx_buf, out=attr)
        r.render(attr, out=outs)

    def cached():
        r.attributes(ds, dm, tx_buf, out=attr)
        r.render(attr, out=outs)

    res = {}
    for name, fn in (("full_path", full), ("cached_geometry", cached)):
        tx_buf.copy_(txs[0:1])
        for _ in range(3):
            fn()
        torch.cuda.synchronize(dev)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            fn()
        ms = []
        for q in range(queries):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            tx_buf.copy_(txs[q:q + 1])          # the query's transmitter (device to device)
            graph.replay()
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        res[name] = {"p50_ms": float(np.percentile(ms, 50)), "p99_ms": float(np.percentile(ms, 99))}
    res["workload"] = ("1,024 Gaussians, 1 subcarrier, 360x90, hidden 32, FP32, one query at a time, "
                       "each query's launches replayed as one CUDA graph")
    res["queries"] = queries
    return res


def run_batched(args):
    """Batched inference: 200,000 Gaussians, 64 transmitters in one launch, 256 subcarriers,
    720x180, hidden 64; BF16X2 tensor-core network + FP32 compositing, against the plain path
    (FP32 network, one transmitter per launch) on the same queries."""
    import torch

    from paper_2511_22793_gb300 import gsparc as G
    from paper_2511_22793_gb300 import synth
    from paper_2511_22793_gb300.pipeline import DeviceMLP, DeviceScene, Renderer

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    n, B, K, H, W, hd = 200_000, 64, 256, 180, 720, 64
    sc = synth.make_scene(n, seed=0, bf16_latent=True)
    mlp = synth.make_mlp(hd, seed=3, bf16_weights=True)
    tx = torch.tensor(synth.make_tx(B, seed=2), device=dev)
    r = Renderer(H, W, K, n, device=dev)
    ds = DeviceScene.from_host(sc, dev)
    dm = DeviceMLP.from_host(mlp, dev)
    r.geometry(ds)
    assert r.check() == 0
    attr = torch.empty((B, n, 4), device=dev)
    spec, logT, nc = r.alloc_outputs(B)
    n_used = torch.empty((B, H, W), dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def batched():
        r.attributes(ds, dm, tx, G.GSPARC_BF16X2, out=attr)
        r.render(attr, out=(spec, logT, nc), n_used=n_used)

    attr1 = torch.empty((1, n, 4), device=dev)
    out1 = r.alloc_outputs(1)

    def plain():
        for b in range(B):
            r.attributes(ds, dm, tx[b:b + 1], G.GSPARC_FP32, out=attr1)
            r.render(attr1, out=out1)

    batched()
    torch.cuda.synchronize(dev)
    units = int(n_used.sum().item()) * K
    res = {}
    for name, fn, reps in (("batched_bf16x2", batched, args.steps), ("plain_fp32_one_query", plain, 1)):
        fn()
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1) / reps
        res[name] = {"ms_per_64_queries": ms, "units_per_s": units / (ms * 1e-3)}
    out = {"metric": "Gaussian·pixel·subcarrier/s forward, batched", "value": res["batched_bf16x2"]["units_per_s"],
           "unit": UNIT, "n_gpus": 1, "higher_is_better": True, "dtype": "bf16x2 network, f32 compositing",
           "data": "synthetic (seeded)",
           "config": {"workload": "batched inference, 200k Gaussians, 64 transmitters per launch, 256 subcarriers, "
                                  "720x180, hidden 64", "units_per_launch": units, "pairs": int(r.n_pairs.item())},
           "forms": res,
           "speedup_vs_plain": res["plain_fp32_one_query"]["ms_per_64_queries"] / res["batched_bf16x2"]["ms_per_64_queries"]}
    print(json.dumps(out))


def run_emission(args):
    """Per-Gaussian emission network (Eq. 1 in the paper's own form, Sec. 4.1 and the Sec. 4.2
    implementation notes; the Sec. 7 width sweep and 1/d toggle): forward and backward of gsparc_emission_fwd/_bwd on 50k Gaussians at
    hidden widths 8, 16 and 64, one and 16 transmitters, CUDA events, L2 flushed between
    launches.  Each Gaussian has its own weights, so the pass is a stream over the flat
    buffer: the achieved HBM bandwidth (weights + means + logits in, attributes out; the
    backward also reads d_attr and reads and writes the weight gradients) is reported against
    the measured copy peak."""
    import torch

    from paper_2511_22793_gb300 import gsparc as G
    from paper_2511_22793_gb300 import synth

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    n = 50_000
    sc = synth.make_scene(n, seed=0)
    means = torch.tensor(sc.means, device=dev)
    ologit = torch.tensor(sc.opacity_logit, device=dev)
    flush = torch.empty(64 * 1024 * 1024, device=dev)
    peak = float(measured_peaks().get("hbm_gbs", 6800.0))
    rows = []
    for h in (8, 16, 64):
        stride = G.gsparc_emission_stride(h)
        rng = np.random.default_rng(h)
        w = np.zeros((n, stride), np.float32)
        w[:, :6 * h + 2] = rng.normal(size=(n, 6 * h + 2)) / np.sqrt(max(h, 3))
        wd = torch.tensor(w, device=dev)
        dw = torch.zeros_like(wd)
        dm, do = torch.zeros((n, 3), device=dev), torch.zeros(n, device=dev)
        for B in (1, 16):
            tx = torch.tensor(synth.make_tx(B, seed=2), device=dev)
            attr = torch.empty((B, n, 4), device=dev)
            d_attr = torch.randn((B, n, 4), device=dev)
            for inv_d in ((True, False) if (h == 16 and B == 1) else (True,)):
                def timed(fn, reps=30):
                    ts = []
                    for it in range(reps + 3):
                        flush.fill_(1.0)
                        e0 = torch.cuda.Event(enable_timing=True)
                        e1 = torch.cuda.Event(enable_timing=True)
                        e0.record()
                        fn()
                        e1.record()
                        e1.synchronize()
                        if it >= 3:
                            ts.append(e0.elapsed_time(e1) * 1e3)
                    return float(np.median(ts))
                fwd_us = timed(lambda: G.gsparc_emission_fwd(tx, (0.0, 0.0, 0.0), means, ologit, wd, h, attr,
                                                             inv_d=inv_d))
                bwd_us = timed(lambda: G.gsparc_emission_bwd(tx, (0.0, 0.0, 0.0), means, ologit, wd, h, d_attr,
                                                             dm, do, dw, inv_d=inv_d))
                fwd_bytes = n * (stride * 4 + 16) + B * n * 16
                bwd_bytes = n * (stride * 4 + 16) + B * n * 16 + n * (2 * stride * 4 + 32)
                rows.append({"hidden": h, "transmitters": B, "inv_d": inv_d,
                             "fwd_us": fwd_us, "bwd_us": bwd_us,
                             "fwd_gaussian_tx_per_s": n * B / (fwd_us * 1e-6),
                             "fwd_hbm_gbs": fwd_bytes / (fwd_us * 1e-6) / 1e9,
                             "fwd_hbm_frac": fwd_bytes / (fwd_us * 1e-6) / 1e9 / peak,
                             "bwd_hbm_gbs": bwd_bytes / (bwd_us * 1e-6) / 1e9,
                             "bwd_hbm_frac": bwd_bytes / (bwd_us * 1e-6) / 1e9 / peak})
    torch.cuda.synchronize(dev)
    out = {"metric": "per-Gaussian emission network forward and backward (Gaussian x transmitter / s)",
           "unit": "us", "n_gpus": 1, "dtype": "f32", "data": "synthetic (seeded)",
           "config": {"workload": "per-Gaussian emission network 3 -> h -> 2, 50k Gaussians, "
                                  "widths 8/16/64, 1 or 16 transmitters, L2 flushed between launches",
                      "hbm_peak_gbs": peak},
           "rows": rows}
    print(json.dumps(out))


def run_spectrum_loss(args):
    """Magnitude-spectrum loss (Eq. 4, L1 + SSIM) and its gradient on the default step's
    spectrum size (one transmitter, 64 subcarriers, 360x90): CUDA events, L2 flushed between
    launches; the effective bandwidth counts the algorithmic bytes of the four passes (44 B of
    maps written and read per pixel and plane, the spectrum and target read twice, dL/dz
    written: 132 B)."""
    import torch

    from paper_2511_22793_gb300 import gsparc as G

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    B, K, H, W = 1, 64, 90, 360
    g = torch.Generator(device=dev).manual_seed(0)
    z = torch.randn((B, K, H, W, 2), device=dev, generator=g)
    y = (z.square().sum(-1).sqrt() * (1 + 0.3 * torch.randn((B, K, H, W), device=dev, generator=g))).clamp_min(0)
    ws = torch.empty(G.gsparc_spectrum_loss_workspace(B, K, H, W), dtype=torch.uint8, device=dev)
    loss = torch.zeros(1, device=dev)
    dz = torch.empty_like(z)
    flush = torch.empty(64 * 1024 * 1024, device=dev)
    peak = float(measured_peaks().get("hbm_gbs", 6800.0))

    def timed(fn, reps=50):
        ts = []
        for it in range(reps + 3):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            e1.synchronize()
            if it >= 3:
                ts.append(e0.elapsed_time(e1) * 1e3)
        return float(np.median(ts))

    both = timed(lambda: G.gsparc_spectrum_loss(z, y, ws, loss, dz))
    fwd = timed(lambda: G.gsparc_spectrum_loss(z, y, ws, loss, None))
    n = B * K * H * W
    out = {"metric": "magnitude-spectrum loss (L1 + SSIM) and gradient", "unit": "us", "n_gpus": 1,
           "dtype": "f32", "data": "synthetic (seeded)",
           "config": {"workload": "Eq. 4 loss, 1 transmitter, 64 subcarriers, 360x90, L2 flushed"},
           "loss_and_grad_us": both, "loss_only_us": fwd,
           "effective_gbs": 132 * n / (both * 1e-6) / 1e9, "hbm_frac": 132 * n / (both * 1e-6) / 1e9 / peak}
    print(json.dumps(out))


def run_train_extras(args):
    """Training extras: one densification of 500k resident Gaussians with 16-float payloads
    (Algorithm 1: count, one-block scan, scatter), and the confidence objective of Eq. 5 at a
    training batch of 4 samples and at 4,096.  CUDA events, L2 flushed between launches; the
    densification's effective bandwidth counts every input once (84 + 4P B per Gaussian, the
    split draws included) and every output row once (48 + 4P B)."""
    import torch

    from paper_2511_22793_gb300 import gsparc as G
    from paper_2511_22793_gb300 import synth

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    N, P, H, W = 500_000, 16, 90, 360
    rng = np.random.default_rng(0)
    sc = synth.make_scene(N, seed=0)
    d = lambda a: torch.tensor(np.ascontiguousarray(a), device=dev)
    proj = d(synth.make_proj_records(N, H, W, seed=5))
    count = rng.integers(0, 5, size=N).astype(np.int32)
    norm = (count * 2e-4 * np.exp(rng.normal(0.0, 0.7, size=N))).astype(np.float32)
    xi = d(rng.normal(size=(N, 2, 3)).astype(np.float32))
    means, ls, quats, ologit, payload = (d(a) for a in (sc.means, sc.log_scales, sc.quats, sc.opacity_logit,
                                                        sc.latent))
    norm_t, count_t = d(norm), d(count)
    cap = 2 * N
    out = {"means": torch.empty((cap, 3), device=dev), "log_scales": torch.empty((cap, 3), device=dev),
           "quats": torch.empty((cap, 4), device=dev), "opacity_logit": torch.empty(cap, device=dev),
           "payload": torch.empty((cap, P), device=dev),
           "parent": torch.empty(cap, dtype=torch.int32, device=dev)}
    n_out = torch.zeros(1, dtype=torch.int32, device=dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    ws = torch.empty(G.gsparc_densify_workspace(N), dtype=torch.uint8, device=dev)
    params = G.densify_params()
    flush = torch.empty(64 * 1024 * 1024, device=dev)
    peak = float(measured_peaks().get("hbm_gbs", 6800.0))

    def timed(fn, reps=50):
        ts = []
        for it in range(reps + 3):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            e1.synchronize()
            if it >= 3:
                ts.append(e0.elapsed_time(e1) * 1e3)
        return float(np.median(ts))

    dens_us = timed(lambda: G.gsparc_densify(means, ls, quats, ologit, payload, proj, norm_t, count_t, xi, params,
                                             ws, out, n_out, status))
    rows = int(n_out.item())
    if int(status.item()) != 0:
        raise RuntimeError("densification status %d" % int(status.item()))
    nbytes = N * (84 + 4 * P) + rows * (48 + 4 * P)
    conf = {}
    for B in (4, 4096):
        pos = d(synth.make_tx(B, seed=2))
        L = d(rng.uniform(0.01, 0.6, size=B).astype(np.float32))
        w = d((0.3 * rng.normal(size=5 * 32 + 1)).astype(np.float32))
        obj = torch.zeros(1, device=dev)
        C, dL, dw = torch.empty(B, device=dev), torch.empty(B, device=dev), torch.zeros(5 * 32 + 1, device=dev)
        conf["batch_%d_us" % B] = timed(lambda: G.gsparc_confidence(pos, L, w, 32, obj, C, dL, dw))
    line = {"metric": "densification and confidence objective", "unit": "us", "n_gpus": 1, "dtype": "f32",
            "data": "synthetic (seeded)",
            "config": {"workload": "densify 500k Gaussians (payload 16 floats, 2 children per split); "
                                   "confidence 3->32->1 at batch 4 and 4096; L2 flushed"},
            "densify_us": dens_us, "rows_out": rows, "densify_effective_gbs": nbytes / (dens_us * 1e-6) / 1e9,
            "densify_hbm_frac": nbytes / (dens_us * 1e-6) / 1e9 / peak, "confidence": conf}
    print(json.dumps(line))


def run_csi(args):
    """CSI queries (Eq. 2): the 64-subcarrier channel estimate at unseen transmitter positions,
    50k Gaussians, 360x90, hidden 32, 16 transmitters per launch, receiver fixed (geometry
    cached).  The tensor-core forward with the spatial mean fused into its epilogue (no
    spectrum written) against the same forward writing the spectrum and gsparc_csi_head
    reducing it."""
    import torch

    from paper_2511_22793_gb300 import gsparc as G
    from paper_2511_22793_gb300 import synth
    from paper_2511_22793_gb300.pipeline import DeviceMLP, DeviceScene, Renderer

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    n, B, K, H, W, hd = 50_000, 16, 64, 90, 360, 32
    sc = synth.make_scene(n, seed=0)
    mlp = synth.make_mlp(hd, seed=3)
    tx = torch.tensor(synth.make_tx(B, seed=2), device=dev)
    r = Renderer(H, W, K, n, device=dev)
    ds = DeviceScene.from_host(sc, dev)
    dm = DeviceMLP.from_host(mlp, dev)
    r.geometry(ds)
    assert r.check() == 0
    attr = torch.empty((B, n, 4), device=dev)
    csi_f = torch.empty((B, K, 2), device=dev)
    csi_u = torch.empty((B, K, 2), device=dev)
    out = r.alloc_outputs(B)
    stream = torch.cuda.current_stream(dev)

    def fused():
        r.attributes(ds, dm, tx, G.GSPARC_BF16X2, out=attr)
        r.render_csi(attr, csi=csi_f)

    def unfused():
        r.attributes(ds, dm, tx, G.GSPARC_BF16X2, out=attr)
        r.render(attr, out=out, tensor_cores=True)
        G.gsparc_csi_head(out[0], csi_u, 1.0 / (H * W))

    res = {}
    reps = max(10, min(args.steps, 200))
    for name, fn in (("fused_csi_head", fused), ("spectrum_then_csi_head", unfused)):
        for _ in range(max(3, args.warmup)):
            fn()
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1) / reps
        res[name] = {"ms_per_launch": ms, "queries_per_s": B / (ms * 1e-3)}
    assert r.check() == 0
    a, b = csi_f.double(), csi_u.double()
    agree = float((a - b).norm() / b.norm())
    out_line = {"metric": "CSI queries/s (64-subcarrier channel estimates)",
                "value": res["fused_csi_head"]["queries_per_s"], "unit": "queries/s", "n_gpus": 1,
                "higher_is_better": True, "dtype": "bf16x2 network and subcarrier sums, f32 accumulation",
                "data": "synthetic (seeded)",
                "config": {"workload": "CSI queries, 50k Gaussians, 16 transmitters per launch, 64 subcarriers, "
                                       "360x90, hidden 32, geometry cached",
                           "spectrum_bytes_not_written": B * K * H * W * 8},
                "forms": res, "fused_vs_unfused_rel_l2": agree,
                "speedup_vs_unfused": res["spectrum_then_csi_head"]["ms_per_launch"] / res["fused_csi_head"]["ms_per_launch"]}
    print(json.dumps(out_line))


def run_train(args):
    """Training loop: 100,000 Gaussians fitted to spectra of a 20,000-Gaussian ground-truth scene
    at 2,000 training transmitters (uniform in the cube), 128 subcarriers, 360x90, hidden 32,
    split-BF16 tensor-core network with FP32 master weights, Adam; held-out error on 200 other
    transmitters before and after."""
    import torch

    from paper_2511_22793_gb300 import synth
    from paper_2511_22793_gb300.train import Trainer

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    gt = synth.make_scene(20_000, seed=1)
    gt_mlp = synth.make_mlp(32, seed=7)
    train_tx = synth.make_tx(2000, seed=2)
    held = synth.make_tx(200, seed=8)
    steps = args.steps
    tr = Trainer(100_000, gt, gt_mlp, train_tx, H=90, W=360, K=128, hidden=32, batch=4,
                 total_steps=steps, device=dev)
    e0 = tr.evaluate(held)
    for _ in range(args.warmup):
        tr.step()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    losses = []
    for i in range(steps):
        loss = tr.step()
        if i % 50 == 0 or i == steps - 1:
            losses.append(float(loss))
    torch.cuda.synchronize(dev)
    dt = time.perf_counter() - t0
    e1 = tr.evaluate(held)
    out = {"metric": "training steps/s", "value": steps / dt, "unit": "steps/s", "n_gpus": 1,
           "higher_is_better": True, "steps": steps, "warmup": args.warmup,
           "config": {"workload": "training: 100k Gaussians fit to a 20k-Gaussian scene, 2000 training "
                                  "transmitters, batch 4, 128 subcarriers, 360x90, hidden 32",
                      "network": "split-BF16 tensor cores forward and backward, FP32 master weights",
                      "compositing_fwd": "tensor cores"},
           "heldout_rel_error": {"before": e0, "after": e1, "transmitters": 200},
           "loss_trace": losses}
    print(json.dumps(out))


def run_serve(args):
    """Serving: 500,000-Gaussian resident scene; Poisson streams of queries (transmitters uniform
    in the cube, resolutions from {180x45, 360x90, 720x180}, subcarriers from {1, 64, 256, 1024})
    at fractions of the plain path's saturated rate; continuous batching (split-BF16 tensor-core
    network, tensor-core compositing) against the plain one-query-at-a-time FP32 path."""
    import torch

    from paper_2511_22793_gb300 import synth
    from paper_2511_22793_gb300.pipeline import DeviceMLP, DeviceScene
    from paper_2511_22793_gb300.serve import Request, Server, latency_stats, serve_plain

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    res = [(45, 180), (90, 360), (180, 720)]
    Ks = [1, 64, 256, 1024]
    sc = synth.make_scene(500_000, seed=0, bf16_latent=True)
    mlp = synth.make_mlp(32, seed=3, bf16_weights=True)
    ds = DeviceScene.from_host(sc, dev)
    dm = DeviceMLP.from_host(mlp, dev)
    n_req = max(100, args.requests)
    rng = np.random.default_rng(4)

    def make(n):
        tx = rng.uniform(-synth.CUBE_HALF, synth.CUBE_HALF, size=(n, 3))
        return [Request(i, tuple(float(v) for v in tx[i]), res[rng.integers(3)], Ks[rng.integers(4)])
                for i in range(n)]

    # saturated rate of the plain path: the same kind of requests back to back
    probe = make(100)
    serve_plain(ds, dm, probe, np.zeros(len(probe)), res, device=dev, keep_results=False)
    for q in probe:
        q.spectrum = None
    st = latency_stats(probe)
    sat = st["spectra_per_s"]
    out_rows = []
    srv = Server(ds, dm, res, mem_budget_bytes=24 << 30, max_batch=8, n_streams=4, device=dev, keep_results=False)
    for frac in (0.25, 0.5, 0.75, 0.9, 1.25, 2.0):
        lam = frac * sat
        reqs = make(n_req)
        arr = np.cumsum(rng.exponential(1.0 / lam, size=n_req))
        srv.done = []
        srv.run(reqs, arr)
        torch.cuda.synchronize(dev)
        for q in reqs:
            q.spectrum = None
        a = latency_stats(reqs)
        plain = [Request(q.rid, q.tx, q.res, q.K) for q in reqs]
        serve_plain(ds, dm, plain, arr, res, device=dev, keep_results=False)
        for q in plain:
            q.spectrum = None
        b = latency_stats(plain)
        out_rows.append({"load": frac, "rate_per_s": lam, "batched": a, "plain": b})
    # saturated: every request queued at once
    burst = make(n_req)
    srv.done = []
    srv.run(burst, np.zeros(n_req))
    torch.cuda.synchronize(dev)
    for q in burst:
        q.spectrum = None
    burst_plain = [Request(q.rid, q.tx, q.res, q.K) for q in burst]
    serve_plain(ds, dm, burst_plain, np.zeros(n_req), res, device=dev, keep_results=False)
    for q in burst_plain:
        q.spectrum = None
    out_rows.append({"load": "burst", "batched": latency_stats(burst), "plain": latency_stats(burst_plain)})
    # moving receiver: every request carries its own pose (position in the cube, random heading),
    # so its projection and bin/sort run per request; one burst, both paths
    n_mov = min(n_req, 200)

    def make_moving(n):
        reqs = make(n)
        for q in reqs:
            rx = rng.uniform(-synth.CUBE_HALF, synth.CUBE_HALF, size=3)
            yaw = rng.uniform(-np.pi, np.pi)
            c, s_ = np.cos(yaw), np.sin(yaw)
            q.rx = tuple(float(v) for v in rx)
            q.V = (c, 0.0, s_, 0.0, 1.0, 0.0, -s_, 0.0, c)
        return reqs

    mov = make_moving(n_mov)
    srv.done = []
    srv.run(mov, np.zeros(n_mov))
    torch.cuda.synchronize(dev)
    for q in mov:
        q.spectrum = None
    mov_plain = [Request(q.rid, q.tx, q.res, q.K, rx=q.rx, V=q.V) for q in mov]
    serve_plain(ds, dm, mov_plain, np.zeros(n_mov), res, device=dev, keep_results=False)
    for q in mov_plain:
        q.spectrum = None
    out_rows.append({"load": "burst, moving receiver", "requests": n_mov, "batched": latency_stats(mov),
                     "plain": latency_stats(mov_plain)})
    out = {"metric": "query latency p50/p99 and spectra/s under Poisson load", "unit": "ms",
           "n_gpus": 1, "requests_per_load": n_req, "plain_saturated_spectra_per_s": sat,
           "config": {"workload": "serving: 500k-Gaussian resident scene, resolutions {180x45, 360x90, "
                                  "720x180}, subcarriers {1, 64, 256, 1024}, transmitters uniform in the cube",
                      "server": "continuous batching, up to 8 queries per launch, 4 streams, 24 GiB budget, "
                                "split-BF16 tensor-core network, tensor-core compositing",
                      "plain": "one query at a time, FP32 network, FP32 compositing"},
           "loads": out_rows}
    print(json.dumps(out))


def cpu_baseline(sample_pixels, seed=0, threads=0, sc=None, mlp=None, tx=None):
    """FP64 oracle, fwd + bwd, on a seeded pixel sample of the same workload, on `threads`
    host threads (0: every core), both for its C renderer and its PyTorch CPU parts."""
    import torch

    from oracle import pipeline as opl
    from oracle import render as orender
    from paper_2511_22793_gb300 import synth

    wl = WORKLOAD
    n, K, H, W, hidden = wl["n"], wl["K"], wl["H"], wl["W"], wl["hidden"]
    if sc is None:
        sc = synth.make_scene(n, seed=0)
        mlp = synth.make_mlp(hidden, seed=3)
        tx = synth.make_tx(1, seed=2)
    orender.build()
    sample_pixels = min(sample_pixels, H * W)
    rng = np.random.default_rng(seed)
    pix = np.sort(rng.choice(H * W, size=sample_pixels, replace=False)).astype(np.int32)
    view, band = synth.View(H=H, W=W), synth.Band(K=K, f_c=wl["f_c"], df=wl["df"])
    cores = threads if threads > 0 else (os.cpu_count() or 1)
    torch_threads = torch.get_num_threads()
    torch.set_num_threads(cores)
    try:
        # unit count of the sample (untimed): Gaussians composited per pixel x K
        counted = opl.forward(sc, mlp, view, band, tx[:1], pixels=pix, threads=cores)
        units = int(counted["n_used"].sum()) * K
        target = np.zeros((1, sample_pixels, K), dtype=np.complex128)
        t0 = time.perf_counter()
        opl.loss_and_grad(sc, mlp, view, band, tx[:1], target, pixels=pix, threads=cores)
        dt = time.perf_counter() - t0
    finally:
        torch.set_num_threads(torch_threads)
    what = "the full %dx%d image" % (W, H) if sample_pixels == H * W else \
        "%d seeded pixels of the %dx%d image" % (sample_pixels, W, H)
    return {"value": units / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "%s, one transmitter, forward + FP64 analytic backward (loss and all "
                      "parameter gradients)" % what, "seconds": dt, "units": units}


def run_reference(args):
    """Reference arm: the FP64 CPU oracle as it stands, on bounded pixel samples."""
    from paper_2511_22793_gb300 import synth

    wl = WORKLOAD
    sc = synth.make_scene(wl["n"], seed=0)
    mlp = synth.make_mlp(wl["hidden"], seed=3)
    tx = synth.make_tx(1, seed=2)
    per_step = 1024
    for i in range(args.warmup):
        cpu_baseline(per_step, seed=100 + i, sc=sc, mlp=mlp, tx=tx)
    secs, units = 0.0, 0
    for i in range(args.steps):
        r = cpu_baseline(per_step, seed=i, sc=sc, mlp=mlp, tx=tx)
        secs += r["seconds"]
        units += r["units"]
    value = units / secs
    cores = os.cpu_count() or 1
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": secs / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded)",
        "config": {"workload": wl["name"], "n_gaussians": wl["n"], "subcarriers": wl["K"], "H": wl["H"],
                   "W": wl["W"], "hidden": wl["hidden"], "sample_pixels_per_step": per_step},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": "%d seeded pixels per step, forward + FP64 analytic backward" % per_step},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-sample", type=int, default=90 * 360,
                    help="pixels in the oracle CPU baseline (default: the whole image)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--requests", type=int, default=2000,
                    help="serving workload: Poisson requests per load level")
    ap.add_argument("--render", default="tc", choices=["tc", "fp32"],
                    help="forward compositing: tcgen05 (default) or FP32 CUDA cores")
    ap.add_argument("--workload", default="fwdbwd",
                    choices=["fwdbwd", "batched", "train", "serve", "csi", "emission", "spectrum_loss",
                             "train_extras"],
                    help="fwdbwd: the default step; batched: 64-transmitter inference with the "
                         "tensor-core network against the plain one-query path; train: the training "
                         "loop; serve: the continuous-batching query server; csi: channel-estimate "
                         "queries with the fused CSI head; emission: the per-Gaussian emission "
                         "network's width sweep; spectrum_loss: the L1 + SSIM loss of Eq. 4; train_extras: "
                         "densification (Algorithm 1) and the confidence objective (Eq. 5)")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)

    rank = _env_int("RANK", 0)
    world = _env_int("WORLD_SIZE", 1)
    local_rank = _env_int("LOCAL_RANK", 0)

    if args.impl == "reference":
        if rank == 0:
            run_reference(args)
        return
    if args.workload == "batched":
        if rank == 0:
            run_batched(args)
        return
    if args.workload == "csi":
        if rank == 0:
            run_csi(args)
        return
    if args.workload == "emission":
        if rank == 0:
            run_emission(args)
        return
    if args.workload == "spectrum_loss":
        if rank == 0:
            run_spectrum_loss(args)
        return
    if args.workload == "train_extras":
        if rank == 0:
            run_train_extras(args)
        return
    if args.workload == "train":
        if rank == 0:
            run_train(args)
        return
    if args.workload == "serve":
        if rank == 0:
            run_serve(args)
        return

    if world > 1:
        import torch
        import torch.distributed as tdist
        torch.cuda.set_device(local_rank)
        tdist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    out, units, sc, mlp, tx = run_ours(args, rank, world, local_rank)
    if rank == 0:
        if world == 1 and not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline(args.cpu_sample, sc=sc, mlp=mlp, tx=tx)
            out["cpu_baseline"].pop("units", None)
            out["cpu_baseline"]["seconds"] = round(out["cpu_baseline"]["seconds"], 3)
            # the same oracle on one host thread, on a smaller sample
            one = cpu_baseline(min(args.cpu_sample, 1024), seed=1, threads=1, sc=sc, mlp=mlp, tx=tx)
            out["cpu_baseline"]["single_thread"] = {"value": one["value"], "unit": UNIT, "cores": 1,
                                                    "sample": one["sample"],
                                                    "seconds": round(one["seconds"], 3)}
        else:
            out["cpu_baseline"] = None
        print(json.dumps(out))
    if world > 1:
        import torch.distributed as tdist
        tdist.barrier()
        tdist.destroy_process_group()


if __name__ == "__main__":
    main()
