"""Benchmark of the splatting hot path on one GB300 (or N independent replicas).

Headline workload (one step = one pass of the whole path over one query):
  50,000 Gaussians (seeded synthetic scene: means uniform in a 10 m cube around the receiver,
  upper hemisphere; log-scales N(-1.5, 0.5); random unit quaternions; opacity logits N(0,1);
  16-dim latents N(0,1)), one transmitter, 64 subcarriers 312.5 kHz apart about 2.4 GHz,
  360x90 hemisphere (1-degree bins, 16x16 tiles), attribute network 20 -> 32 -> 32 -> 3.
  Step = project -> bin/sort -> attribute network -> render forward -> complex L2 loss against a
  target spectrum (rendered once, outside the timed region, from a second seeded scene) ->
  render backward -> network backward -> projection backward.  The headline arithmetic is FP32
  on the CUDA cores throughout (`--render fp32`, the default); the tensor-core form (split-BF16
  products with FP32 accumulation for the subcarrier contractions and the network, FP32
  transmittance) is timed beside it and reported under `forms`.

Metric: Gaussian-pixel-subcarrier units per second, where a unit is one Gaussian composited at
one pixel (counted up to termination by the forward kernel's per-pixel counter) for one
subcarrier; fwd+bwd per step.

`value` times the step on the device with inputs resident in HBM (CUDA events on the launching
stream, L2 flushed by a 256 MiB write between timed steps).  `e2e` times the same step through
the C ABI with the scene, network, transmitters and target copied from pinned host memory and
the loss read back, inside the timed region (the target's copy overlaps projection, binning and
the forward).  `roofline` reports the dominant kernel against the FP32 ALU peak; `cpu_baseline`
times the FP64 oracle on a bounded pixel sample and reports the GPU spectra's error against it.
The default line also carries the other configurations: `c1_query_latency` (single query),
`c3_batched` (64 transmitters per launch vs the plain path), `c4_train` (training loop steps/s
and held-out error), `c5_serve` (continuous batching vs the plain path under Poisson load) and
`probes` (FMA and ex2 throughput measured on this GPU).

Multi-GPU: queries are independent, so N ranks run N replicas on their own transmitters (weak
scaling) with no data-path collective; timing is the max over ranks.  `--impl reference` times
the FP64 CPU oracle as the reference arm.
"""
from __future__ import annotations

import argparse
import ctypes
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
# Algorithmic work per unit (one Gaussian composited at one pixel for one subcarrier), as the
# scope table counts it: forward ~10 flop (the complex product of w = T alpha with the emission
# a e^{j psi} and its accumulation), backward ~20 flop (the conjugate products of dL/dz with
# the emission for the alpha, amplitude, phase and path-length derivatives).  The kernels hoist
# the per-(Gaussian, subcarrier) phasor out of the pixel loop and execute 2 and 6 FP32 lane
# operations per unit on the FMA pipe (forward one paired FMA; backward two paired FMAs and one
# paired add).
FLOP_FWD_UNIT = 10
FLOP_BWD_UNIT = 20
FMA_FWD_UNIT, FMA_BWD_UNIT = 2, 6
FP32_LANES_PER_SM = 128
# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of the compositing
# kernels on this workload, from one `ncu --set full --clock-control none` capture of the
# kernels as they are now (one launch each, L2 flushed before the step); set an entry to None
# when its kernel changes until it is captured again.  Algorithmic bytes for comparison: the
# 16.6 MB upstream gradient (backward) or target (forward) read once, plus per-pixel state.
NCU_TRAFFIC = {("fp32", "render_bwd"): 17_885_696, ("fp32", "render_fwd"): 17_186_560,
               ("tc", "render_bwd"): 17_511_936, ("tc", "render_fwd"): 17_186_304}


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


def probe_peaks(dev, local_rank):
    """FMA and ex2 throughput of this GPU (libgsparc_probe.so): 8 independent chains per thread,
    8 blocks of 256 threads per SM, best of 5 launches of ~20 ms, CUDA events; the SM clock is
    sampled meanwhile.  Returns per-second rates, their value per SM per clock at the sampled
    clock, and the FP32 peak they imply at the maximum clock."""
    import torch

    path = os.path.join(ROOT, "paper_2511_22793_gb300", "libgsparc_probe.so")
    if not os.path.exists(path):
        raise RuntimeError("libgsparc_probe.so is not built; run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    lib.gsparc_probe_launch.restype = ctypes.c_int64
    lib.gsparc_probe_launch.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    blocks = sms * 8
    out = torch.empty(blocks * 256, device=dev)
    stream = torch.cuda.current_stream(dev)
    sampler = ClockSampler(local_rank)
    sampler.start()
    sampler.wait_first()
    res = {}
    for kind, name, iters in ((0, "fma", 6000), (1, "ex2", 1500)):
        best = None
        for rep in range(6):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ops = lib.gsparc_probe_launch(kind, blocks, iters, ctypes.c_void_p(out.data_ptr()),
                                          ctypes.c_void_p(stream.cuda_stream))
            e1.record(stream)
            e1.synchronize()
            if ops < 0:
                raise RuntimeError("probe launch failed")
            if rep == 0:
                continue
            rate = ops / (e0.elapsed_time(e1) * 1e-3)
            best = rate if best is None else max(best, rate)
        res[name] = best
    clocks = sampler.stop()
    mhz = float(clocks["sm_mhz"]) if clocks else None
    peaks = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    out_d = {"fma_per_s": res["fma"], "ex2_per_s": res["ex2"], "clocks": clocks, "sms": sms,
             "method": "8 independent chains per thread, %d blocks x 256 threads, best of 5 launches, CUDA events"
                       % blocks}
    if mhz:
        out_d["fma_per_sm_per_clk"] = res["fma"] / (sms * mhz * 1e6)
        out_d["ex2_per_sm_per_clk"] = res["ex2"] / (sms * mhz * 1e6)
        out_d["fp32_tflops_at_max_clock"] = 2 * out_d["fma_per_sm_per_clk"] * sms * sm_max * 1e6 / 1e12
    return out_d


# --------------------------------------------------------------------------------------------
# our arm: the headline training step
# --------------------------------------------------------------------------------------------

def _make_inputs(dev, rank, world):
    """Seeded scene, network, transmitter of this rank and the target spectrum (rendered by the
    FP32 path from the seed-1 scene, not timed), as views of one device allocation with a pinned
    host mirror (the end-to-end step copies them from there)."""
    import torch

    from paper_2511_22793_gb300 import synth
    from paper_2511_22793_gb300.pipeline import DeviceMLP, DeviceScene, PackedInputs, Renderer
    from paper_2511_22793_gb300.replicas import rank_queries

    wl = WORKLOAD
    n, K, H, W, hidden, B = wl["n"], wl["K"], wl["H"], wl["W"], wl["hidden"], wl["B"]
    sc = synth.make_scene(n, seed=0)
    mlp = synth.make_mlp(hidden, seed=3)
    tx = rank_queries(synth.make_tx(B * world, seed=2), B, rank, world)
    sc_t = synth.make_scene(n, seed=1)
    rt = Renderer(H, W, K, n, f_c=wl["f_c"], df=wl["df"], device=dev)
    dst = DeviceScene.from_host(sc_t, dev)
    dm = DeviceMLP.from_host(mlp, dev)
    txd = torch.tensor(tx, device=dev)
    rt.geometry(dst)
    target = rt.render(rt.attributes(dst, dm, txd))[0].clone()
    torch.cuda.synchronize(dev)
    if rt.check() != 0:
        raise RuntimeError("target render failed")
    del rt, dst
    arrays = list(sc.arrays()) + list(mlp.arrays()) + [txd, target]
    inp = PackedInputs([tuple(np.shape(a)) if not isinstance(a, torch.Tensor) else tuple(a.shape)
                        for a in arrays], dev)
    for i, a in enumerate(arrays):
        inp.set_host(i, a)
    inp.upload()
    torch.cuda.synchronize(dev)
    return sc, mlp, tx, inp


def entries_visited(st, r, composited):
    """Tile-list entries the compositing walks per algorithmic unit (the Gaussians composited at a
    pixel, per subcarrier): at the pixel (entries up to the pixel's last composited one), at the
    tile (its CTA walks until every pixel of the tile has stopped) and the whole tile lists."""
    H, W = r.H, r.W
    TW, TH = (W + 15) // 16, (H + 15) // 16
    rows = np.minimum(16, H - 16 * np.arange(TH))
    cols = np.minimum(16, W - 16 * np.arange(TW))
    px = np.outer(rows, cols).reshape(-1).astype(np.float64)                  # pixels of tile t
    walks = st.walks.double().cpu().numpy()                                    # [B, T]
    rng = r.tile_ranges.view(-1, 2).long().cpu().numpy()
    lists = (rng[:, 1] - rng[:, 0]).astype(np.float64)
    c = float(max(composited, 1))
    return {"per_pixel_walk": float(st.nc.double().sum().item()) / c,
            "per_tile_walk": float((walks * px[None, :]).sum()) / c,
            "per_tile_list": float((lists * px).sum()) * st.B / c,
            "note": "tile-list entries per composited (Gaussian, pixel); the units count only the "
                    "composited ones"}


def time_form(args, dev, form, inp, steps, flush, sampler=None, dist=False):
    """Build the step of `form` on the packed inputs, check it, time its kernels (eager, per
    stage), the step graph (device-resident inputs) and the host-input graph (end to end)."""
    import torch

    from paper_2511_22793_gb300 import gsparc as G
    from paper_2511_22793_gb300.pipeline import DeviceMLP, DeviceScene, Renderer
    from paper_2511_22793_gb300.step import TrainStep

    wl = WORKLOAD
    n, K, H, W, hidden = wl["n"], wl["K"], wl["H"], wl["W"], wl["hidden"]
    ds = DeviceScene(*inp.views[0:5])
    dm = DeviceMLP(hidden, *inp.views[5:11])
    txd, target = inp.views[11], inp.views[12]
    r = Renderer(H, W, K, n, f_c=wl["f_c"], df=wl["df"], device=dev)
    st = TrainStep(r, ds, dm, txd, target, form=form)
    stream = torch.cuda.current_stream(dev)
    for _ in range(args.warmup):
        st.enqueue()
    torch.cuda.synchronize(dev)
    if r.check() != 0:
        raise RuntimeError("device status %d after warm-up (%s)" % (r.check(), form))
    units = int(st.n_used.sum().item()) * K
    n_pairs = int(r.n_pairs.item())
    visited = entries_visited(st, r, units // K)
    # per-kernel durations: eager steps with CUDA events around every stage (one stream)
    per_kernel = {k: [] for k in st.stages}
    for _ in range(min(steps, 50)):
        flush.fill_(1.0)
        ev = {k: (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for k in st.stages}
        st.enqueue(events=ev)
        torch.cuda.synchronize(dev)
        for k in st.stages:
            per_kernel[k].append(ev[k][0].elapsed_time(ev[k][1]))
    graph = st.capture()
    for _ in range(3):
        graph.replay()
    torch.cuda.synchronize(dev)
    if r.check() != 0:
        raise RuntimeError("device status after graph warm-up (%s)" % form)
    if dist:
        import torch.distributed as tdist
        tdist.barrier()
    torch.cuda.synchronize(dev)
    if sampler is not None:
        sampler.start()
        sampler.wait_first()
    step_ms = []
    for _ in range(steps):
        flush.fill_(1.0)                      # evict L2 between timed steps (not timed)
        s0 = torch.cuda.Event(enable_timing=True)
        s1 = torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        graph.replay()
        s1.record(stream)
        s1.synchronize()
        step_ms.append(s0.elapsed_time(s1))
    torch.cuda.synchronize(dev)
    loss_a, grad_a = float(st.loss), st.gbuf.clone()
    # end to end: host (pinned) inputs copied inside the step's graph, the loss read back
    graph_e2e = st.capture(inp)
    for _ in range(3):
        graph_e2e.replay()
    torch.cuda.synchronize(dev)
    if r.check() != 0:
        raise RuntimeError("device status after the end-to-end graph's warm-up (%s)" % form)
    loss_b, grad_b = float(st.loss), st.gbuf.clone()
    if float(st.host_loss[0]) != loss_b:
        raise RuntimeError("the end-to-end graph's host copy of the loss differs from the device loss (%s)" % form)
    agree = {"loss_rel": abs(loss_a - loss_b) / abs(loss_a),
             "grad_rel_l2": float((grad_a - grad_b).norm() / grad_a.norm())}
    if agree["loss_rel"] > 1e-5 or agree["grad_rel_l2"] > 1e-4:
        raise RuntimeError("end-to-end step disagrees with the step graph (%s): %s" % (form, agree))
    host_loss = st.host_loss                  # the graph copies the loss here during the backward
    e2e_ms = []
    for it in range(args.warmup + steps):
        flush.fill_(1.0)
        if dist and it == args.warmup:
            import torch.distributed as tdist
            tdist.barrier()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        graph_e2e.replay()
        torch.cuda.current_stream(dev).synchronize()
        _ = float(host_loss[0])
        if it >= args.warmup:
            e2e_ms.append((time.perf_counter() - t0) * 1e3)
    clocks = sampler.stop() if sampler is not None else None
    # the step's spectrum (its fused forward does not store it), for the accuracy comparison
    spec = st.spectrum().detach().cpu()
    torch.cuda.synchronize(dev)
    return {"st": st, "r": r, "units": units, "n_pairs": n_pairs, "visited": visited, "step_ms": step_ms,
            "e2e_ms": e2e_ms,
            "kernels_ms": {k: statistics.mean(v) for k, v in per_kernel.items()}, "agree": agree,
            "clocks": clocks, "spec": spec, "h2d": inp.nbytes, "d2h": host_loss.numel() * host_loss.element_size()}


def roofline(form_res, dev, probes, form="fp32"):
    """Dominant kernel of the step against the FP32 ALU peak (SMs x 128 lanes x 2 flop x the
    maximum SM clock), with the scope table's flop per unit; also against the FMA rate the probe
    measured on this GPU, and as FMA-pipe issue (the FMAs the kernel executes per unit)."""
    import torch

    avg = form_res["kernels_ms"]
    top = max(avg, key=avg.get)
    peaks = measured_peaks()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    fp32_peak = sms * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12      # TFLOP/s
    units = form_res["units"]
    flop = {"render_bwd": FLOP_BWD_UNIT, "render_fwd": FLOP_FWD_UNIT}
    fma = {"render_bwd": FMA_BWD_UNIT, "render_fwd": FMA_FWD_UNIT}
    out = {}
    for k in ("render_bwd", "render_fwd"):
        ms = avg[k]
        achieved = units * flop[k] / (ms * 1e-3) / 1e12
        d = {"kernel": k, "bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
             "frac": achieved / fp32_peak, "kernel_ms": ms,
             "flop_per_unit": flop[k], "units_per_launch": units,
             "peak_note": "%d SMs x 128 FP32 lanes x 2 flop x %.0f MHz (max SM clock)" % (sms, sm_max),
             "traffic": NCU_TRAFFIC.get((form, k)), "traffic_unit": "B per launch (ncu DRAM read + write)"}
        if probes and probes.get("fp32_tflops_at_max_clock"):
            d["peak_probe"] = probes["fp32_tflops_at_max_clock"]
            d["frac_vs_probe"] = achieved / probes["fp32_tflops_at_max_clock"]
        # FMA-pipe issue: the FMAs executed per unit against the pipe's lane rate
        d["fma_issue_frac"] = units * fma[k] / (ms * 1e-3) / (sms * FP32_LANES_PER_SM * sm_max * 1e6)
        out[k] = d
    dom = dict(out[top]) if top in out else {"kernel": top, "bound": "hbm", "achieved": None,
                                             "peak": float(peaks.get("hbm_gbs", 6800.0)), "unit": "GB/s",
                                             "frac": None, "traffic": None}
    return dom, out


def run_ours(args, rank, world, local_rank):
    import torch

    from paper_2511_22793_gb300.replicas import job_totals, throughput

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    wl = WORKLOAD
    dist = world > 1
    sc, mlp, tx, inp = _make_inputs(dev, rank, world)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    head = time_form(args, dev, args.render, inp, args.steps, flush, sampler=ClockSampler(local_rank), dist=dist)
    units, step_ms, e2e_ms = head["units"], head["step_ms"], head["e2e_ms"]
    # whole job: the units all ranks processed over the slowest rank's time
    job_units, total_ms = job_totals(units * args.steps, sum(step_ms), device=dev)
    job_units_e2e, e2e_total = job_totals(units * len(e2e_ms), sum(e2e_ms), device=dev)
    value = throughput(job_units, total_ms)
    e2e_value = throughput(job_units_e2e, e2e_total)
    probes = probe_peaks(dev, local_rank) if world == 1 else None
    dom, rl = roofline(head, dev, probes, args.render)
    st = head["st"]
    tc_head = args.render == "tc"
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded)",
        "config": {"workload": wl["name"], "n_gaussians": wl["n"], "subcarriers": wl["K"], "H": wl["H"],
                   "W": wl["W"], "hidden": wl["hidden"], "transmitters_per_step": wl["B"],
                   "pairs": head["n_pairs"], "units_per_step": job_units // args.steps,
                   "entries_visited_per_unit": head["visited"],
                   "l2": "flushed (256 MiB write) between timed steps",
                   "compositing": ("subcarrier sums on tensor cores (split-BF16 products, FP32 accumulation), "
                                   "transmittance and gradients FP32") if tc_head else "FP32 CUDA cores",
                   "attribute_network": ("tensor cores, split-BF16 products, FP32 accumulation"
                                         if tc_head else "FP32 CUDA cores"),
                   "target": "spectrum of a second seeded scene rendered by the FP32 path (not timed)",
                   "parallelism": "replicas x%d" % world},
        "latency_ms": {"p50": float(np.percentile(step_ms, 50)), "p99": float(np.percentile(step_ms, 99)),
                       "min": float(min(step_ms))},
        "kernels_ms": head["kernels_ms"],
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": head["h2d"],
                "d2h_bytes_per_step": head["d2h"], "ms_per_step": e2e_total / args.steps,
                "copies": "inside the step's graph: means, log-scales and quaternions first (projection's "
                          "inputs), the rest of the scene, the network and the transmitters on the second "
                          "stream ahead of the network forward, the target spectrum on a third stream after "
                          "them, beside projection, binning and the forward (spectrum written, loss by "
                          "gsparc_l2_loss once the target is in, copied to pinned host memory on the third "
                          "stream while the backward runs)",
                "agrees_with_step_graph": head["agree"]},
        "gpu_launches": st.launches * args.steps,
        "launch": "whole step captured once as a CUDA graph (gradient zeroing and network forward beside "
                  "projection and bin/sort, projection backward beside network backward, on a second "
                  "stream), replayed per timed step; launch overlap %s (tile emit and sort, the backward's "
                  "schedule and walks and the network backward launched as programmatic dependents of the "
                  "kernel before them)" % args.launch_overlap,
        "roofline": dom,
        "roofline_kernels": rl,
        "clocks": head["clocks"],
    }
    spectra = {args.render: head["spec"]}
    if world == 1:
        other = "fp32" if tc_head else "tc"
        res_o = time_form(args, dev, other, inp, min(args.steps, 100), flush)
        tot_o = sum(res_o["step_ms"])
        dom_o, _ = roofline(res_o, dev, probes, other)
        spectra[other] = res_o["spec"]
        d_head = head["spec"].double()
        d_o = res_o["spec"].double()
        out["forms"] = {
            ("tc_split_bf16" if other == "tc" else "fp32"): {
                "value": res_o["units"] * len(res_o["step_ms"]) / (tot_o * 1e-3),
                "unit": UNIT, "ms_per_step": tot_o / len(res_o["step_ms"]),
                "e2e_ms_per_step": statistics.mean(res_o["e2e_ms"]),
                "dtype": "split-BF16 operands (hi + lo, three products), FP32 accumulation" if other == "tc"
                         else "f32",
                "compositing": "subcarrier sums on tcgen05 tensor cores, alpha / transmittance / recursions FP32"
                               if other == "tc" else "FP32 CUDA cores",
                "attribute_network": "tcgen05, split-BF16, forward and backward" if other == "tc"
                                     else "FP32 CUDA cores",
                "kernels_ms": res_o["kernels_ms"], "roofline": dom_o,
                "spectrum_rel_l2_vs_headline_form": float((d_o - d_head).norm() / d_head.norm()),
                "gpu_launches_per_step": res_o["st"].launches,
                "speedup_vs_headline": (total_ms / args.steps) / (tot_o / len(res_o["step_ms"])),
            }}
        del res_o
        out["probes"] = probes
        out["c1_query_latency"] = query_latency(dev, queries=max(50, min(args.steps, 400)))
        if not args.quick:
            out["c3_batched"] = run_batched(args, dev, emit=False)
            out["c4_train"] = run_train(args, dev, emit=False)
            out["c5_serve"] = run_serve(args, dev, emit=False, loads=(0.25, 0.5, 0.75, 0.9))
            out["c5_binsort"] = run_binsort_scale(args, dev, emit=False)
    return out, spectra, sc, mlp, tx


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
    if r.check() != 0:
        raise RuntimeError("single-query path status")
    res["workload"] = ("1,024 Gaussians, 1 subcarrier, 360x90, hidden 32, FP32, one query at a time, "
                       "each query's launches replayed as one CUDA graph")
    res["queries"] = queries
    return res


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


def _pix_sample(H, W, npix, seed):
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(H * W, size=npix, replace=False)).astype(np.int64)


def _spec_at(spec_b, pix, W):
    """[K, H, W, 2] device tensor -> [npix, K] complex128 (host) at linear pixel ids pix."""
    import torch

    ys = torch.as_tensor(pix // W, device=spec_b.device)
    xs = torch.as_tensor(pix % W, device=spec_b.device)
    z = spec_b[:, ys, xs].double().cpu().numpy()          # [K, npix, 2]
    return (z[..., 0] + 1j * z[..., 1]).T


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def run_batched(args, dev=None, emit=True):
    """Batched inference: 200,000 Gaussians, 64 transmitters in one launch, 256 subcarriers,
    720x180, hidden 64; BF16X2 tensor-core network + tensor-core compositing, against the plain
    path (FP32 network and FP32 compositing, one transmitter per launch) on the same queries.
    Accuracy: every batched spectrum against the plain path's on the whole image, and (the
    oracle leg, timed as a CPU baseline) both against the FP64 oracle on 128 seeded pixels of
    8 of the transmitters."""
    import torch

    from paper_2511_22793_gb300 import gsparc as G
    from paper_2511_22793_gb300 import synth
    from paper_2511_22793_gb300.pipeline import DeviceMLP, DeviceScene, Renderer

    if dev is None:
        dev = torch.device("cuda", 0)
        torch.cuda.set_device(dev)
    n, B, K, H, W, hd = 200_000, 64, 256, 180, 720, 64
    sc = synth.make_scene(n, seed=0, bf16_latent=True)
    mlp = synth.make_mlp(hd, seed=3, bf16_weights=True)
    txh = synth.make_tx(B, seed=2)
    tx = torch.tensor(txh, device=dev)
    r = Renderer(H, W, K, n, device=dev)
    ds = DeviceScene.from_host(sc, dev)
    dm = DeviceMLP.from_host(mlp, dev)
    r.geometry(ds)
    if r.check() != 0:
        raise RuntimeError("batched geometry status")
    attr = torch.empty((B, n, 4), device=dev)
    spec, logT, nc = r.alloc_outputs(B)
    n_used = torch.empty((B, H, W), dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def batched():
        r.attributes(ds, dm, tx, G.GSPARC_BF16X2, out=attr)
        r.render(attr, out=(spec, logT, nc), n_used=n_used, tensor_cores=True)

    attr1 = torch.empty((1, n, 4), device=dev)
    out1 = r.alloc_outputs(1)

    def plain(check=None):
        for b in range(B):
            r.attributes(ds, dm, tx[b:b + 1], G.GSPARC_FP32, out=attr1)
            r.render(attr1, out=out1)
            if check is not None:
                check(b)

    batched()
    torch.cuda.synchronize(dev)
    units = int(n_used.sum().item()) * K
    res = {}
    for name, fn, reps in (("batched_bf16x2", batched, 10), ("plain_fp32_one_query", plain, 2)):
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
    if r.check() != 0:
        raise RuntimeError("batched status")
    # accuracy: each batched spectrum against the plain FP32 path's, whole image
    batched()
    torch.cuda.synchronize(dev)
    sel = list(range(0, B, B // 8))
    pix = _pix_sample(H, W, 128, seed=30)
    rel_plain, z_b, z_p = [], {}, {}

    def check(b):
        d = (spec[b].double() - out1[0][0].double()).norm() / out1[0][0].double().norm()
        rel_plain.append(float(d))
        if b in sel:
            z_b[b] = _spec_at(spec[b], pix, W)
            z_p[b] = _spec_at(out1[0][0], pix, W)

    plain(check)
    torch.cuda.synchronize(dev)
    # the oracle leg: FP64 oracle spectra of 8 transmitters on 128 seeded pixels (host cores)
    from oracle import attributes as oattr
    from oracle import projection as oproj
    from oracle import render as orender

    orender.build()
    view, band = synth.View(H=H, W=W), synth.Band(K=K)
    f64 = lambda a: torch.tensor(np.asarray(a), dtype=torch.float64)
    t0 = time.perf_counter()
    geo = oproj.project(f64(sc.means), f64(sc.log_scales), f64(sc.quats), view)
    g = {k: geo[k].numpy() for k in ("px", "py", "cxx", "cxy", "cyy", "r", "valid")}
    weights = [f64(a) for a in mlp.arrays()]
    err_b, err_p, n_units = [], [], 0
    for b in sel:
        at = oattr.attributes(f64(sc.means), f64(sc.opacity_logit), f64(sc.latent), weights, f64(txh[b]), view.rx)
        at = {k: at[k].numpy() for k in ("sigma", "a", "phi0", "L")}
        z_or, _, nu = orender.render_fwd(g, at, H, W, K, band.f_c, band.df, pixels=pix.astype(np.int32))
        n_units += int(nu.sum()) * K
        err_b.append(_rel(z_b[b], z_or))
        err_p.append(_rel(z_p[b], z_or))
    oracle_s = time.perf_counter() - t0
    out = {"metric": "Gaussian·pixel·subcarrier/s forward, batched", "value": res["batched_bf16x2"]["units_per_s"],
           "unit": UNIT, "n_gpus": 1, "higher_is_better": True,
           "dtype": "bf16x2 network and compositing products, f32 accumulation and transmittance",
           "data": "synthetic (seeded)",
           "config": {"workload": "batched inference, 200k Gaussians, 64 transmitters per launch, 256 subcarriers, "
                                  "720x180, hidden 64", "units_per_launch": units, "pairs": int(r.n_pairs.item())},
           "forms": res,
           "speedup_vs_plain": res["plain_fp32_one_query"]["ms_per_64_queries"] / res["batched_bf16x2"]["ms_per_64_queries"],
           "rel_l2_vs_plain_per_spectrum": {"max": max(rel_plain), "median": float(np.median(rel_plain)),
                                            "spectra": len(rel_plain), "pixels": "whole image"},
           "rel_l2_vs_oracle_per_spectrum": {"batched_max": max(err_b), "batched_median": float(np.median(err_b)),
                                             "plain_max": max(err_p), "plain_median": float(np.median(err_p)),
                                             "spectra": len(sel), "pixels": 128},
           "cpu_baseline": {"value": n_units / oracle_s, "unit": UNIT, "cores": os.cpu_count() or 1, "kind": "oracle",
                            "sample": "128 seeded pixels of 8 transmitters (forward, projection and network "
                                      "of all 200k Gaussians included)", "seconds": oracle_s}}
    if emit:
        print(json.dumps(out))
    return out


def run_train(args, dev=None, emit=True):
    """Training loop: 100,000 Gaussians fitted to spectra of a 20,000-Gaussian ground-truth scene
    at 2,000 training transmitters (uniform in the cube, their targets resident in HBM), 128
    subcarriers, 360x90, hidden 32, split-BF16 tensor-core network with FP32 master weights, Adam,
    recompute in the backward, the paper's loss for spectrum targets (Eq. 4: L1 + SSIM on
    magnitudes).  steps/s over the timed steps; held-out relative error (of |z|, and of z) on 200
    other transmitters against the ground truth rendered by the FP32 path (whole images) and, in
    the oracle leg, against the FP64 oracle's render of the ground truth on 64 seeded pixels,
    before and after.  A second run adds Algorithm 1's densification (every 100 steps) and the
    Eq. 5 confidence objective."""
    import torch

    from paper_2511_22793_gb300 import synth
    from paper_2511_22793_gb300.train import Trainer

    if dev is None:
        dev = torch.device("cuda", 0)
        torch.cuda.set_device(dev)
    H, W, K = 90, 360, 128
    gt = synth.make_scene(20_000, seed=1)
    gt_mlp = synth.make_mlp(32, seed=7)
    train_tx = synth.make_tx(2000, seed=2)
    held = synth.make_tx(200, seed=8)
    steps = args.c4_steps
    pix = _pix_sample(H, W, 64, seed=31)

    def make(**kw):
        return Trainer(100_000, gt, gt_mlp, train_tx, H=H, W=W, K=K, hidden=32, batch=4,
                       total_steps=steps + args.warmup, device=dev, loss="l1ssim", **kw)

    def predict_at(tr):
        txs = torch.tensor(np.asarray(held, dtype=np.float32), device=dev)
        out = []
        for s in range(0, txs.shape[0], tr.batch):
            (spec, _, _), _ = tr.forward(txs[s:s + tr.batch])
            for b in range(spec.shape[0]):
                out.append(_spec_at(spec[b], pix, W))
        return np.stack(out)

    def timed_run(tr, n_steps, checkpoints):
        trace, t_train, done = [], 0.0, 0
        for _ in range(args.warmup):
            tr.step()
        torch.cuda.synchronize(dev)
        chunk = max(1, n_steps // checkpoints)
        while done < n_steps:
            m = min(chunk, n_steps - done)
            t0 = time.perf_counter()
            for _ in range(m):
                loss = tr.step()
            torch.cuda.synchronize(dev)
            t_train += time.perf_counter() - t0
            done += m
            trace.append({"step": done + args.warmup, "loss": float(loss), "gaussians": tr.n,
                          "heldout_rel_error_magnitude": tr.evaluate(held, magnitude=True)})
        if tr.r.check() != 0:
            raise RuntimeError("training status")
        return n_steps / t_train, trace

    tr = make()
    e0 = {"magnitude": tr.evaluate(held, magnitude=True), "complex": tr.evaluate(held)}
    p0 = predict_at(tr)
    rate, trace = timed_run(tr, steps, 5)
    e1 = {"magnitude": trace[-1]["heldout_rel_error_magnitude"], "complex": tr.evaluate(held)}
    p1 = predict_at(tr)
    del tr
    torch.cuda.empty_cache()
    # the same loop with densification and the confidence objective
    ex_steps = max(200, steps // 3)
    tr = make(densify_every=100, confidence=True)
    x0 = tr.evaluate(held, magnitude=True)
    ex_rate, ex_trace = timed_run(tr, ex_steps, 2)
    del tr
    torch.cuda.empty_cache()
    # the oracle leg: ground-truth spectra of the held-out transmitters on 64 seeded pixels
    from oracle import pipeline as opl

    t0 = time.perf_counter()
    ref = opl.forward(gt, gt_mlp, synth.View(H=H, W=W), synth.Band(K=K), held, pixels=pix.astype(np.int32))
    oracle_s = time.perf_counter() - t0
    z_or = ref["z"]
    oracle_units = int(ref["n_used"].sum()) * K
    err_c = lambda p: float(np.linalg.norm(p - z_or) / np.linalg.norm(z_or))
    err_m = lambda p: float(np.linalg.norm(np.abs(p) - np.abs(z_or)) / np.linalg.norm(np.abs(z_or)))
    out = {"metric": "training steps/s", "value": rate, "unit": "steps/s", "n_gpus": 1,
           "higher_is_better": True, "steps": steps, "warmup": args.warmup,
           "config": {"workload": "training: 100k Gaussians fit to a 20k-Gaussian scene, 2000 training "
                                  "transmitters, batch 4, 128 subcarriers, 360x90, hidden 32",
                      "network": "split-BF16 tensor cores forward and backward, FP32 master weights",
                      "compositing": "tensor cores forward and scheduled backward",
                      "loss": "Eq. 4, L1 + SSIM on magnitude spectra (lambda_1 = 0.2)",
                      "init": "geometry-agnostic (uniform centres, isotropic 0.2 m, opacity 0.1)",
                      "training_targets": "ground truth rendered by the FP32 path once, resident in HBM "
                                          "(2000 x 128 x 360 x 90 magnitudes, 33 GB)"},
           "heldout_rel_error": {"before": e0, "after": e1, "transmitters": 200, "pixels": "whole image",
                                 "against": "FP32-path render of the ground truth"},
           "trace": trace,
           "with_densification_and_confidence": {
               "value": ex_rate, "unit": "steps/s", "steps": ex_steps, "densify_every": 100,
               "objective": "Eq. 5 over the batch of Eq. 4 losses", "heldout_rel_error_magnitude_before": x0,
               "trace": ex_trace},
           "cpu_baseline": {"value": oracle_units / oracle_s, "unit": UNIT, "cores": os.cpu_count() or 1,
                            "kind": "oracle",
                            "sample": "ground truth (20k Gaussians) at the 200 held-out transmitters, 64 seeded "
                                      "pixels, forward (projection and network of every Gaussian included)",
                            "seconds": oracle_s,
                            "heldout_rel_error_vs_oracle": {
                                "magnitude": {"before": err_m(p0), "after": err_m(p1)},
                                "complex": {"before": err_c(p0), "after": err_c(p1)},
                                "transmitters": 200, "pixels": 64}}}
    if emit:
        print(json.dumps(out))
    return out


def run_binsort_scale(args, dev=None, emit=True, reps=20):
    """Projection and tile binning + directional sort at serving scale: the 500,000-Gaussian
    resident scene at 180x45, 360x90 and 720x180, each pass timed with CUDA events on its stream
    (L2 flushed before each), achieved bandwidth on the algorithmic bytes: projection 40 B read
    (mean, log-scales, quaternion) + 32 B written per Gaussian; bin/sort 36 B read per Gaussian
    (the footprint box twice, the distance once) + 8 B written per pair (the keys), 8 B read + 4 B
    written per pair (the per-tile sort)."""
    import torch

    from paper_2511_22793_gb300 import gsparc as G
    from paper_2511_22793_gb300 import synth
    from paper_2511_22793_gb300.pipeline import DeviceScene, Renderer

    if dev is None:
        dev = torch.device("cuda", 0)
        torch.cuda.set_device(dev)
    n = 500_000
    ds = DeviceScene.from_host(synth.make_scene(n, seed=0, bf16_latent=True), dev)
    peak = float(measured_peaks().get("hbm_gbs", 6800.0))
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    rows = []
    for (H, W) in ((45, 180), (90, 360), (180, 720)):
        r = Renderer(H, W, 1, n, device=dev)
        proj_fn = lambda: G.gsparc_project(r.view, ds.means, ds.log_scales, ds.quats, r.proj, d_status=r.status)
        bin_fn = lambda: G.gsparc_bin_sort(r.view, n, r.proj, r.capacity, r.ws, r.sorted_ids, None, r.tile_ranges,
                                           r.n_pairs, r.status)
        for _ in range(3):
            proj_fn()
            bin_fn()
        torch.cuda.synchronize(dev)
        if r.check() != 0:
            raise RuntimeError("bin/sort status at %dx%d" % (W, H))
        pairs = int(r.n_pairs.item())
        t = {}
        for name, fn in (("project", proj_fn), ("bin_sort", bin_fn)):
            ms = []
            for _ in range(reps):
                flush.fill_(1.0)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                fn()
                e1.record(stream)
                e1.synchronize()
                ms.append(e0.elapsed_time(e1))
            t[name] = statistics.median(ms)
        b_proj = 72 * n
        b_bin = 36 * n + 20 * pairs
        rows.append({"resolution": "%dx%d" % (W, H), "pairs": pairs,
                     "project": {"ms": t["project"], "bytes": b_proj, "gbs": b_proj / (t["project"] * 1e6),
                                 "frac": b_proj / (t["project"] * 1e6) / peak},
                     "bin_sort": {"ms": t["bin_sort"], "bytes": b_bin, "gbs": b_bin / (t["bin_sort"] * 1e6),
                                  "frac": b_bin / (t["bin_sort"] * 1e6) / peak, "launches": 3}})
        del r
    out = {"metric": "projection and bin/sort bandwidth", "unit": "GB/s", "n_gaussians": n, "peak_gbs": peak,
           "peak_note": "measured copy bandwidth (MEASURED_PEAKS.json)", "resolutions": rows}
    if emit:
        print(json.dumps(out))
    return out


def run_serve(args, dev=None, emit=True, loads=(0.25, 0.5, 0.75, 0.9, 1.25, 2.0)):
    """Serving: 500,000-Gaussian resident scene; Poisson streams of queries (transmitters uniform
    in the cube, resolutions from {180x45, 360x90, 720x180}, subcarriers from {1, 64, 256, 1024})
    at fractions of the plain path's saturated rate; continuous batching (split-BF16 tensor-core
    network, tensor-core compositing) against the plain one-query-at-a-time FP32 path."""
    import torch

    from paper_2511_22793_gb300 import synth
    from paper_2511_22793_gb300.pipeline import DeviceMLP, DeviceScene
    from paper_2511_22793_gb300.serve import Request, Server, latency_stats, serve_plain

    if dev is None:
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
    st = latency_stats(probe)
    sat = st["spectra_per_s"]
    out_rows = []
    srv = Server(ds, dm, res, mem_budget_bytes=24 << 30, max_batch=8, n_streams=4, device=dev, keep_results=False)
    srv.run(make(50), np.zeros(50))          # warm-up: every (resolution, subcarrier count) seen once
    torch.cuda.synchronize(dev)
    for frac in loads:
        lam = frac * sat
        reqs = make(n_req)
        arr = np.cumsum(rng.exponential(1.0 / lam, size=n_req))
        srv.done = []
        srv.run(reqs, arr)
        torch.cuda.synchronize(dev)
        a = latency_stats(reqs)
        plain = [Request(q.rid, q.tx, q.res, q.K) for q in reqs]
        serve_plain(ds, dm, plain, arr, res, device=dev, keep_results=False)
        b = latency_stats(plain)
        out_rows.append({"load": frac, "rate_per_s": lam, "batched": a, "plain": b})
    # saturated: every request queued at once
    burst = make(n_req)
    srv.done = []
    srv.run(burst, np.zeros(n_req))
    torch.cuda.synchronize(dev)
    burst_plain = [Request(q.rid, q.tx, q.res, q.K) for q in burst]
    serve_plain(ds, dm, burst_plain, np.zeros(n_req), res, device=dev, keep_results=False)
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
    mov_plain = [Request(q.rid, q.tx, q.res, q.K, rx=q.rx, V=q.V) for q in mov]
    serve_plain(ds, dm, mov_plain, np.zeros(n_mov), res, device=dev, keep_results=False)
    out_rows.append({"load": "burst, moving receiver", "requests": n_mov, "batched": latency_stats(mov),
                     "plain": latency_stats(mov_plain)})
    out = {"metric": "query latency p50/p99 and spectra/s under Poisson load", "unit": "ms",
           "n_gpus": 1, "requests_per_load": n_req, "plain_saturated_spectra_per_s": sat,
           "config": {"workload": "serving: 500k-Gaussian resident scene, resolutions {180x45, 360x90, "
                                  "720x180}, subcarriers {1, 64, 256, 1024}, transmitters uniform in the cube",
                      "server": "continuous batching, up to 8 queries per launch, 4 streams, 24 GiB budget, "
                                "split-BF16 tensor-core network, tensor-core compositing",
                      "plain": "one query at a time, FP32 network, FP32 compositing",
                      "latency": "arrival to the host observing the completion event"},
           "loads": out_rows}
    if emit:
        print(json.dumps(out))
    return out


def cpu_baseline(sample_pixels, seed=0, threads=0, sc=None, mlp=None, tx=None, spectra=None):
    """FP64 oracle, fwd + bwd, on a seeded pixel sample of the same workload, on `threads`
    host threads (0: every core), both for its C renderer and its PyTorch CPU parts.  spectra:
    optional form -> [1, K, H, W, 2] GPU spectrum (host tensor) of the same scene and
    transmitter, each compared with the oracle's on the sample."""
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
        _, g = opl.loss_and_grad(sc, mlp, view, band, tx[:1], target, pixels=pix, threads=cores)
        dt = time.perf_counter() - t0
    finally:
        torch.set_num_threads(torch_threads)
    what = "the full %dx%d image" % (W, H) if sample_pixels == H * W else \
        "%d seeded pixels of the %dx%d image" % (sample_pixels, W, H)
    out = {"value": units / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": "%s, one transmitter, forward + FP64 analytic backward (loss and all "
                     "parameter gradients)" % what, "seconds": dt, "units": units}
    if spectra:
        z_or = g["z"][0]
        out["gpu_spectrum_rel_l2_vs_oracle"] = {}
        for form, s in spectra.items():
            z = s[0].double().numpy()
            zc = (z[..., 0] + 1j * z[..., 1]).transpose(1, 2, 0).reshape(H * W, K)[pix]
            out["gpu_spectrum_rel_l2_vs_oracle"]["tc_split_bf16" if form == "tc" else form] = _rel(zc, z_or)
    return out


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
    ap.add_argument("--quick", action="store_true",
                    help="headline step (both forms), probes and the single-query latency only")
    ap.add_argument("--requests", type=int, default=2000,
                    help="serving workload: Poisson requests per load level")
    ap.add_argument("--c4-steps", type=int, default=1500, help="training workload: timed steps")
    ap.add_argument("--render", default="fp32", choices=["fp32", "tc"],
                    help="headline arithmetic: FP32 CUDA cores (default) or the tensor-core form")
    ap.add_argument("--workload", default="fwdbwd",
                    choices=["fwdbwd", "batched", "train", "serve", "binsort", "csi", "emission", "spectrum_loss",
                             "train_extras"],
                    help="fwdbwd: the default line (headline step and every configuration); batched: "
                         "64-transmitter inference against the plain one-query path; train: the training "
                         "loop; serve: the continuous-batching query server; csi: channel-estimate "
                         "queries with the fused CSI head; emission: the per-Gaussian emission "
                         "network's width sweep; spectrum_loss: the L1 + SSIM loss of Eq. 4; train_extras: "
                         "densification (Algorithm 1) and the confidence objective (Eq. 5)")
    ap.add_argument("--launch-overlap", default="on", choices=["on", "off"],
                    help="programmatic dependent launch of the library's follow-on kernels (gsparc_set_launch_overlap)")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    if args.impl != "reference":
        from paper_2511_22793_gb300 import gsparc as G
        G.gsparc_set_launch_overlap(args.launch_overlap == "on")

    rank = _env_int("RANK", 0)
    world = _env_int("WORLD_SIZE", 1)
    local_rank = _env_int("LOCAL_RANK", 0)

    if args.impl == "reference":
        if rank == 0:
            run_reference(args)
        return
    single = {"batched": run_batched, "csi": run_csi, "emission": run_emission, "binsort": run_binsort_scale,
              "spectrum_loss": run_spectrum_loss, "train_extras": run_train_extras, "train": run_train,
              "serve": run_serve}
    if args.workload in single:
        if rank == 0:
            single[args.workload](args)
        return

    if world > 1:
        import torch
        import torch.distributed as tdist
        torch.cuda.set_device(local_rank)
        tdist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    out, spectra, sc, mlp, tx = run_ours(args, rank, world, local_rank)
    if rank == 0:
        if world == 1 and not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline(args.cpu_sample, sc=sc, mlp=mlp, tx=tx, spectra=spectra)
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
