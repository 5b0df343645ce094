#!/usr/bin/env python
"""Benchmark: encode + decode throughput of the SLRME dual-layer lossless
RGBE coder on one GB300 (or N independent replicas, one per GPU).

Workload (one "step", the default ``--workload 8k``): the 7680x4320 synthetic
RGBE image (fBm luminance over 8 decades with a smooth sky band in the top
third, exponents within 100..150; seed 3) coded at base quality 90:
rgbe_split, sdri_base_roundtrip, slr_fit, residual_encode, then
residual_decode, with the decoded words checked against the input.  The
step's C-ABI calls are captured once as a CUDA graph and the timed steps
replay it; per-call times come from replays of a copy of that graph with
event-record nodes between the calls (timed apart, since each node adds a
few microseconds to the step).  The input is resident in HBM when timing
starts; L2 is flushed (a 256 MiB write) between timed steps, outside the
step events.

The same JSON line carries, measured in the same process outside the timed
steps: the batch form on 64 images of uneven sizes (``batch64``), the
enhancement-layer rate of the learned estimator against the regression on
the 2048x1536 image at qualities 50/75/90 (``bits_per_px_2k``), the
enhancement-layer coder, the base-layer rate and a quality sweep.
``--workload 2k`` times the 2048x1536 image at qualities 50/75/90 instead
(one concurrent branch per quality), ``--workload batch64`` the batch form
alone.

Prints one JSON line.  ``--impl reference`` times the CPU oracle instead
(rank 0 only) on the same workload, on every host core: each step codes the
image as one horizontal band per core, the bands concurrently.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "encode+decode MPixel/s (bit-exact); enh.-layer bits/px, learned vs SLR, 1 GB300"
UNIT = "MPixel/s"

# Algorithmic HBM bytes per pixel of each C-ABI call (reads + writes of the
# planes it must touch once): split 4+4, base 4+3, fit 7, residual 7+6,
# decode 10+4.
BYTES_PER_PX = {"rgbe_split": 8, "sdri_base_roundtrip": 7, "slr_fit": 7, "residual_encode": 13,
                "residual_decode": 14}
# DRAM bytes per pixel measured by ncu (dram__bytes_read.sum + dram__bytes_write.sum
# over one launch, divided by its pixels) with the sha256 of the kernel source the
# counters were taken on; a changed source reports null.  See profiles/.
TRAFFIC = {"slr_fit": {"bytes_per_px": (235972864 + 6271488) / (7680 * 4320), "sha": "6eb8a3a613e98b85"},
           "sdri_base_roundtrip": {"bytes_per_px": (132826112 + 62897920) / (7680 * 4320), "sha": "db4407c559a0ae81"}}
# The base round trip is bound by instruction issue, not by memory: its
# roofline counts the arithmetic operations its definition needs per pixel
# (tone mapping 24; four 8-point integer DCT passes per channel, 36 butterfly
# operations and 8 rounding shifts per 8 values and pass, 66; quantiser 15;
# clamp and pack 3) against the issue peak of the GPU's SMs x 128 lanes x the
# maximum SM clock.
ALU_OPS_PER_PX = {"sdri_base_roundtrip": 108}
KERNEL_SOURCE = {"rgbe_split": "split.cu", "sdri_base_roundtrip": "base.cu", "slr_fit": "slr.cu",
                 "residual_encode": "slr.cu", "residual_decode": "slr.cu"}


def _sha(name: str) -> str:
    p = os.path.join(ROOT, "paper_2309_11072_gb300", "csrc", name)
    return hashlib.sha256(open(p, "rb").read()).hexdigest()[:16]


def load_peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return {"hbm_gbs": float(d["hbm_gbs"]), "sm_max_mhz": float(d.get("sm_max_mhz", 2070.0)), "src": "measured"}
    return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0, "src": "fallback"}


class ClockSampler:
    """nvidia-smi clock / throttle samples while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = os.path.join("/tmp", f"slrme_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.idx)], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return None
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for name, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def max_over_ranks(ms: float, dist, device: str) -> float:
    """The whole job's time for a region every rank timed: the slowest rank's
    (one all-reduce of a float64 on `device`), or `ms` itself on one rank."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_mpx_per_s(world: int, px_per_step: int, steps: int, ms: float) -> float:
    """Whole-job throughput of `world` replicas that each coded `px_per_step`
    pixels per step for `steps` steps, the slowest within `ms` milliseconds."""
    return world * px_per_step * steps / (ms / 1e3) / 1e6


def run_ours(args) -> None:
    import numpy as np
    import torch

    from paper_2309_11072_gb300 import codec, native, synth
    from paper_2309_11072_gb300.metrics import enhancement_bits_per_pixel

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    native.lib()

    wl = synth.workload_8k() if args.workload == "8k" else synth.workload_2k()
    (h, w), = wl.sizes
    img = synth.make_workload_images(wl)[0]
    n = h * w
    qualities = wl.qualities
    stream = torch.cuda.current_stream()
    rgbe = torch.from_numpy(img.view(np.int32).reshape(-1).copy()).cuda()
    # one set of device buffers per quality: the qualities are independent
    # encodes, so the step runs their chains of calls as concurrent branches
    cq = {q: codec.Codec(h, w, "cuda", gf_on=True) for q in qualities}
    c = cq[qualities[0]]
    side = {q: torch.cuda.Stream() for q in qualities}
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    calls = ["rgbe_split", "sdri_base_roundtrip", "slr_fit", "residual_encode", "residual_decode"]

    def chain(q, st, ev=None):
        b = cq[q]
        if ev is not None:
            ev[q][0].record(st)
        native.rgbe_split(rgbe, h, w, b.m3, b.e, b.stats, st)
        if ev is not None:
            ev[q][1].record(st)
        native.sdri_base_roundtrip(b.m3, b.e, h, w, b.stats, q, b.s3, None, st)
        if ev is not None:
            ev[q][2].record(st)
        native.slr_fit(b.s3, b.m3, b.e, h, w, 1, b.sums, b.params, st)
        if ev is not None:
            ev[q][3].record(st)
        native.residual_encode(b.s3, b.m3, b.e, h, w, 1, b.params, b.r3, b.hist, st)
        if ev is not None:
            ev[q][4].record(st)
        native.residual_decode(b.s3, b.e, b.r3, h, w, 1, b.params, b.out, st)
        if ev is not None:
            ev[q][5].record(st)

    def step(ev=None, st=None):
        # the qualities one after another on one stream (per-call timing)
        st = stream if st is None else st
        for q in qualities:
            chain(q, st, ev)

    def step_par(st):
        # the qualities as concurrent branches forked from and joined to `st`
        fork = torch.cuda.Event()
        fork.record(st)
        for q in qualities:
            side[q].wait_event(fork)
            chain(q, side[q])
        for q in qualities:
            done = torch.cuda.Event()
            done.record(side[q])
            st.wait_event(done)

    for _ in range(args.warmup):
        step()
        flush.zero_()
    torch.cuda.synchronize()

    # bit-exact check and rates at each quality (outside the timed region)
    from paper_2309_11072_gb300 import learned as Lr
    net_dev = Lr.upload_net(Lr.load_net(Lr.default_weights())) if os.path.exists(Lr.default_weights()) else None
    bpp, bit_exact = learned_vs_slr(c, rgbe, qualities, net_dev, stream)
    torch.cuda.synchronize()

    # the step's C-ABI calls, captured once into a CUDA graph and replayed.
    # A second graph of the same calls carries event-record nodes between the
    # calls (external events, where this torch has them) and times each call;
    # event nodes add a few microseconds each, so the step time comes from the
    # graph without them.
    try:
        gev = {q: [torch.cuda.Event(enable_timing=True, external=True) for _ in range(6)] for q in qualities}
    except TypeError:
        gev = None
    cap = torch.cuda.Stream()
    cap.wait_stream(stream)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=cap, capture_error_mode="thread_local"):
        step_par(torch.cuda.current_stream())
    egraph = None
    if gev is not None:
        egraph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(egraph, stream=cap, capture_error_mode="thread_local"):
            step(gev, torch.cuda.current_stream())
    stream.wait_stream(cap)
    for _ in range(args.warmup):
        graph.replay()
        flush.zero_()
    torch.cuda.synchronize()

    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    step_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    per_call = {name: [] for name in calls}
    with ClockSampler(local) as clocks:
        wall0 = time.perf_counter()
        for k in range(args.steps):
            step_ev[k][0].record(stream)
            graph.replay()
            step_ev[k][1].record(stream)
            flush.zero_()
        torch.cuda.synchronize()
        wall = time.perf_counter() - wall0
        if egraph is not None:
            # per-call times: the same steps replayed with event nodes between
            # the calls, L2 flushed between steps as above; the in-graph events
            # are rewritten by every replay, so they are read after each one
            for _ in range(args.warmup):
                egraph.replay()
                flush.zero_()
            for k in range(args.steps):
                egraph.replay()
                flush.zero_()
                stream.synchronize()
                for q in qualities:
                    for i, name in enumerate(calls):
                        per_call[name].append(gev[q][i].elapsed_time(gev[q][i + 1]))
    if dist is not None:
        dist.barrier()
    step_ms = [a.elapsed_time(b) for a, b in step_ev]
    total_ms = sum(step_ms)
    out_ok = all(bool(torch.equal(cq[q].out, rgbe)) for q in qualities)

    call_timing = "event-record nodes between the calls in replays of the same step graph (L2 flushed between steps)"
    if gev is None:
        # no external events in this torch: the same step launched call by call
        # with events between the calls (not part of the timed steps above)
        call_timing = "separate call-by-call pass (no in-graph events in this torch)"
        call_ev = [{q: [torch.cuda.Event(enable_timing=True) for _ in range(6)] for q in qualities}
                   for _ in range(args.steps)]
        for k in range(args.steps):
            step(call_ev[k])
            flush.zero_()
        torch.cuda.synchronize()
        for k in range(args.steps):
            for q in qualities:
                ev = call_ev[k][q]
                for i, name in enumerate(calls):
                    per_call[name].append(ev[i].elapsed_time(ev[i + 1]))
    total_ms = max_over_ranks(total_ms, dist, "cuda")

    px_per_step = n * len(qualities)
    value = job_mpx_per_s(world, px_per_step, args.steps, total_ms)

    # roofline of the dominant call (its own bound: HBM bytes, or ALU operations)
    peaks = load_peaks()
    avg_us = {name: 1e3 * statistics.mean(v) for name, v in per_call.items()}
    alu_peak = torch.cuda.get_device_properties(local).multi_processor_count * 128 * peaks["sm_max_mhz"] * 1e6 / 1e12

    def call_roofline(name):
        t = avg_us[name] * 1e-6
        if name in ALU_OPS_PER_PX:
            a = ALU_OPS_PER_PX[name] * n / t / 1e12
            return {"bound": "alu", "achieved": round(a, 2), "peak": round(alu_peak, 2), "unit": "Tops/s",
                    "frac": round(a / alu_peak, 4), "algorithmic_ops": ALU_OPS_PER_PX[name] * n,
                    "peak_source": "SMs x 128 lanes x max SM clock"}
        a = BYTES_PER_PX[name] * n / t / 1e9
        return {"bound": "hbm", "achieved": round(a, 1), "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": round(a / peaks["hbm_gbs"], 4), "algorithmic_bytes": BYTES_PER_PX[name] * n,
                "peak_source": peaks["src"]}

    dom = max(avg_us, key=lambda k: avg_us[k])
    roofline = call_roofline(dom)
    tr = TRAFFIC.get(dom)
    roofline["traffic"] = tr["bytes_per_px"] * n if tr and tr["sha"] == _sha(KERNEL_SOURCE[dom]) else None
    roofline["kernel"] = dom
    roofline["timing"] = call_timing
    stage_roofline = {name: {k: v for k, v in call_roofline(name).items() if k in ("bound", "achieved", "unit", "frac")}
                      for name in calls}
    stage_us = {name: round(v, 2) for name, v in avg_us.items()}
    stage_frac = {name: round(BYTES_PER_PX[name] * n / (avg_us[name] * 1e-6) / 1e9 / peaks["hbm_gbs"], 4)
                  for name in calls}

    # end to end through the public API with host buffers: the K steps run as
    # one job (HostCodec's slots take the calls in turn on their own streams,
    # so one call's copies back overlap the next call's copy in and coding);
    # every step copies its input words in and its layers and decoded words
    # back inside the timed region, and its input comes from host memory, so
    # no L2 flush is needed between steps
    hc = codec.HostCodec(h, w, "cuda", gf_on=True)
    h_rgbe = torch.from_numpy(img.view(np.int32).reshape(-1).copy()).pin_memory()
    for _ in range(args.warmup):
        for q in qualities:
            hc.roundtrip(h_rgbe, q)
    torch.cuda.synchronize()
    side = hc.streams()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for s_ in side:
        s_.wait_stream(stream)
    for k in range(args.steps):
        for q in qualities:
            hc.roundtrip(h_rgbe, q)
    for s_ in side:
        stream.wait_stream(s_)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1)
    e2e_ok = bool(torch.equal(hc.h_out, h_rgbe))
    e2e_ms = max_over_ranks(e2e_ms, dist, "cuda")
    e2e_value = job_mpx_per_s(world, px_per_step, args.steps, e2e_ms)

    enh = enhancement_coder(c, rgbe, qualities, n, args, flush, stream)

    extras = {}
    if args.workload == "8k" and not args.no_extras:
        # the 2048x1536 image: learned estimator against the regression at q 50/75/90
        wl2 = synth.workload_2k()
        (h2, w2), = wl2.sizes
        img2 = synth.make_workload_images(wl2)[0]
        c2 = codec.Codec(h2, w2, "cuda", gf_on=True)
        rgbe2 = torch.from_numpy(img2.view(np.int32).reshape(-1).copy()).cuda()
        bpp2, ok2 = learned_vs_slr(c2, rgbe2, wl2.qualities, net_dev, stream)
        extras["bits_per_px_2k"] = {"image": f"{w2}x{h2}", "workload": wl2.name, "rates": bpp2, "bit_exact": ok2}
        bit_exact &= ok2
        del c2, rgbe2
        if world == 1:
            extras["batch64"] = measure_batch(args)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(img, qualities, budget_s=args.cpu_seconds)

    step_bytes = sum(BYTES_PER_PX.values()) * px_per_step
    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(total_ms / args.steps, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": {"workload": f"{wl.name} q{{{','.join(map(str, qualities))}}} encode+decode, SLR, "
                                   "gaussian restoration on",
                       "pixels_per_step": px_per_step, "image": f"{w}x{h}", "qualities": list(qualities),
                       "l2": "flushed between timed steps (256 MiB write)", "parallelism": f"replicas{world}",
                       "launch": f"the step's {5 * len(qualities)} C-ABI calls captured once as a CUDA graph (one "
                                 "branch of five calls per quality, the branches concurrent), replayed per step"},
            "bit_exact": bit_exact and e2e_ok and out_ok,
            "bits_per_px": bpp,
            "e2e": {"value": round(e2e_value, 2), "unit": UNIT,
                    "h2d_bytes_per_step": hc.h2d_bytes() * len(qualities),
                    "d2h_bytes_per_step": hc.d2h_bytes() * len(qualities)},
            "gpu_launches": args.steps * len(qualities) * 6,
            "roofline": roofline, "stage_us": stage_us, "stage_roofline": stage_roofline,
            "stage_hbm_frac": stage_frac,
            "step_hbm_frac": {"bytes_per_px": sum(BYTES_PER_PX.values()),
                              "achieved_gbs": round(step_bytes / (total_ms / args.steps * 1e-3) / 1e9, 1),
                              "frac": round(step_bytes / (total_ms / args.steps * 1e-3) / 1e9 / peaks["hbm_gbs"], 4),
                              "peak_source": peaks["src"]},
            "clocks": clocks.summary(), "cpu_baseline": cpu, "wall_s_timed": round(wall, 3),
            **extras,
            "enhancement_coder": enh,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def learned_vs_slr(c, rgbe, qualities, net_dev, stream):
    """Enhancement-layer bits per pixel (order-0 entropy of the residuals plus
    side information) at each quality: the regression (SLRME), no estimator
    (M* = S), and the learned estimator refining the regression with the
    per-image pick; every decode checked against the input words.  Returns
    (rates per quality, bit_exact)."""
    import numpy as np
    import torch

    from paper_2309_11072_gb300 import codec, native
    from paper_2309_11072_gb300 import learned as Lr
    from paper_2309_11072_gb300.metrics import enhancement_bits_per_pixel

    h, w = c.h, c.w
    n = h * w
    bit_exact = True
    bpp = {}
    ident = torch.from_numpy(codec.params_from_numpy(np.full((3, 256), 1 / 16, np.float32),
                                                     np.zeros((3, 256), np.float32))).cuda()
    for q in qualities:
        L = c.encode(rgbe, q)
        out = c.decode(L.s3, L.e, L.r3, L.params)
        bit_exact &= bool(torch.equal(out, rgbe))
        slr = c.bits_per_pixel()
        native.residual_encode(c.s3, c.m3, c.e, h, w, 0, ident, c.r3, c.hist, stream)
        # without SLRME nothing but the residual planes is sent (M* = S)
        plain = enhancement_bits_per_pixel(c.hist.view(3, 511).cpu().numpy().view(np.uint32), 0, n) - 256.0 / n
        bpp[str(q)] = {"slr": round(slr, 4), "without_slrme": round(plain, 4), "learned": None}
        if net_dev is not None:
            # the learned estimator (refining this image's regression), picked only if cheaper
            native.residual_encode(c.s3, c.m3, c.e, h, w, 1, c.params, c.r3, c.hist, stream)
            hist_slr = c.hist.view(3, 511).cpu().numpy().view(np.uint32).copy()
            J = native.rgbe_key_scale(c.stats.cpu().numpy())[0]
            r3c = torch.empty_like(c.r3)
            hc = torch.empty_like(c.hist)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            Lr.cnn_residual_encode(c.s3, c.m3, c.e, h, w, J, net_dev, c.params, 1, r3c, hc, stream)
            e1.record(stream)
            Lr.cnn_residual_decode(c.s3, c.e, r3c, h, w, J, net_dev, c.params, 1, c.out, stream)
            torch.cuda.synchronize()
            bit_exact &= bool(torch.equal(c.out, rgbe))
            pk = Lr.pick_image(hist_slr, codec.params_to_numpy(c.params)["n_used"],
                               hc.view(3, 511).cpu().numpy().view(np.uint32), n)
            bpp[str(q)].update(learned=round(pk.bits_cnn, 4), picked="learned" if pk.use_cnn else "slr",
                               with_pick=round(pk.bits, 4), learned_encode_us=round(1e3 * e0.elapsed_time(e1), 1),
                               learned_mpx_s=round(n / (1e3 * e0.elapsed_time(e1)), 1))
    return bpp, bit_exact


def enhancement_coder(c, rgbe, qualities, n, args, flush, stream) -> dict:
    """The enhancement layer's entropy coding on this image's residuals at
    each quality, outside the timed step, in two forms: interleaved rANS over
    the residual planes (a table per channel), and the same coder over the
    coefficients of a three-level reversible 5/3 wavelet (a table per band).
    Reports the coded size against the zeroth-order entropy, the lossless
    round trip, and the device time of each call: the calls of each form are
    captured once as a CUDA graph with event-record nodes between them and
    replayed (L2 flushed between replays), so host submission gaps do not
    enter the times."""
    import numpy as np
    import torch

    from paper_2309_11072_gb300 import native
    from paper_2309_11072_gb300.metrics import entropy_bits

    nres = native.SLRME_NRES
    h, w = c.h, c.w
    levels = 3
    nb = 1 + 3 * levels
    bands = native.dwt53_bands(h, w, levels)
    lengths = [a * b for a, b in bands] * 3
    # plain form buffers
    freq = torch.empty(3 * nres, dtype=torch.int32, device="cuda")
    words = torch.empty(native.rans_words_capacity(n), dtype=torch.int16, device="cuda")
    counts = torch.empty(native.rans_counts_capacity(n), dtype=torch.int32, device="cuda")
    r_back = torch.empty_like(c.r3)
    # wavelet form buffers
    coef = torch.empty(3 * n, dtype=torch.int16, device="cuda")
    bhist = torch.empty(3 * nb * nres, dtype=torch.int32, device="cuda")
    bfreq = torch.empty(3 * nb * nres, dtype=torch.int32, device="cuda")
    ws = torch.empty(native.dwt53_workspace_bytes(3, h, w), dtype=torch.uint8, device="cuda")
    nw, nc = native.rans_segments_capacity(lengths)
    wwords = torch.empty(nw, dtype=torch.int16, device="cuda")
    wcounts = torch.empty(nc, dtype=torch.int32, device="cuda")
    coef_back = torch.empty_like(coef)
    w_back = torch.empty_like(c.r3)

    plain_names = ("rans_tables", "rans_encode", "rans_decode")
    wave_names = ("dwt53_forward", "rans_tables_n", "rans_encode_segments", "rans_decode_segments", "dwt53_inverse")

    def plain_calls(st, ev=None):
        steps = [lambda: native.rans_tables(c.hist, freq, st),
                 lambda: native.rans_encode(c.r3, n, freq, words, counts, st),
                 lambda: native.rans_decode(words, counts, n, freq, r_back, st)]
        for i, f in enumerate(steps):
            if ev is not None:
                ev[i].record(st)
            f()
        if ev is not None:
            ev[len(steps)].record(st)

    def wave_calls(st, ev=None):
        steps = [lambda: native.dwt53_forward(c.r3, 3, h, w, levels, coef, bhist, ws, st),
                 lambda: native.rans_tables_n(bhist, 3 * nb, bfreq, st),
                 lambda: native.rans_encode_segments(coef, lengths, bfreq, wwords, wcounts, st),
                 lambda: native.rans_decode_segments(wwords, wcounts, lengths, bfreq, coef_back, st),
                 lambda: native.dwt53_inverse(coef_back, 3, h, w, levels, w_back, ws, st)]
        for i, f in enumerate(steps):
            if ev is not None:
                ev[i].record(st)
            f()
        if ev is not None:
            ev[len(steps)].record(st)

    c.encode(rgbe, qualities[0])
    plain_calls(stream)                # first calls set up the kernels before capture
    wave_calls(stream)
    torch.cuda.synchronize()
    forms = {}
    try:
        for name, fn, k in (("plain", plain_calls, len(plain_names)), ("wavelet", wave_calls, len(wave_names))):
            gev = [torch.cuda.Event(enable_timing=True, external=True) for _ in range(k + 1)]
            cap = torch.cuda.Stream()
            cap.wait_stream(stream)
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph, stream=cap, capture_error_mode="thread_local"):
                fn(torch.cuda.current_stream(), gev)
            stream.wait_stream(cap)
            forms[name] = (graph, gev)
        timing = "event-record nodes between the calls in replays of one CUDA graph per form, L2 flushed between replays"
    except TypeError:
        forms = {}
        timing = "events between the calls launched one by one (host gaps included), L2 flushed between repetitions"

    def timed(name, fn, names):
        t = {k: [] for k in names}
        for rep in range(args.warmup + args.steps):
            if name in forms:
                forms[name][0].replay()
                ev = forms[name][1]
            else:
                ev = [torch.cuda.Event(enable_timing=True) for _ in range(len(names) + 1)]
                fn(stream, ev)
            flush.zero_()
            torch.cuda.synchronize()
            if rep >= args.warmup:
                for i, k in enumerate(names):
                    t[k].append(ev[i].elapsed_time(ev[i + 1]) * 1e3)
        return {k: round(statistics.mean(v), 2) for k, v in t.items()}

    out = {"coder": "static rANS, M = 2^14, 32 interleaved 16-bit streams per 8192 symbols; plain: a table per "
                    "channel over the residual planes; wavelet: three-level reversible 5/3 transform, a table "
                    "per band (30), chunks with values beyond +-255 stored raw",
           "timing": timing}
    ok = True
    for q in qualities:
        c.encode(rgbe, q)
        native.device_status(clear=True)
        us = timed("plain", plain_calls, plain_names)
        ok &= bool(torch.equal(r_back, c.r3))
        wus = timed("wavelet", wave_calls, wave_names)
        ok &= bool(torch.equal(w_back, c.r3)) and native.device_status(clear=True) == 0
        cnt = counts.cpu().numpy().view(np.uint32).astype(np.int64)
        hist = c.hist.view(3, nres).cpu().numpy().view(np.uint32)
        h0 = sum(entropy_bits(hist[ch]) for ch in range(3))
        wc = wcounts.cpu().numpy().view(np.uint32)
        raw = wc == 0xFFFFFFFF
        raw_chunks = int(raw.sum()) // 32
        wbits = 16.0 * wc[~raw].astype(np.int64).sum() + 16.0 * 8192 * raw_chunks
        bh = bhist.view(3 * nb, nres).cpu().numpy().view(np.uint32)
        wh0 = sum(entropy_bits(bh[i]) * bh[i].sum() for i in range(3 * nb)) / n
        out[str(q)] = {"coded_bits_per_px": round(16.0 * cnt.sum() / n, 4), "h0_bits_per_px": round(h0, 4),
                       "table_bits": 3 * nres * 15, "us": us,
                       "encode_msym_s": round(3 * n / us["rans_encode"], 1),
                       "decode_msym_s": round(3 * n / us["rans_decode"], 1),
                       "wavelet": {"coded_bits_per_px": round(wbits / n, 4), "h0_bits_per_px": round(wh0, 4),
                                   "raw_chunks": raw_chunks, "table_bits": 3 * nb * nres * 15, "us": wus}}
    out["lossless"] = ok
    out["base_layer"] = base_layer_bits(c, rgbe, qualities, n, args, flush, stream, out)
    out["quality_sweep"] = quality_sweep(c, rgbe, n, stream)
    return out


def quality_sweep(c, rgbe, n, stream) -> dict:
    """Bits per pixel against the base layer's JPEG quality Q, in the manner of
    Fig. 4: the base layer's Huffman-coded levels plus the enhancement layer
    coded by the wavelet form, with the SLRME (the fitted parameters) and
    without it (M* = S: slope 1/16 per grey level of x = 16 S*, intercept 0,
    no restoration), at Q = 10, 20, ..., 100 and 85 (Table I's quality)."""
    import numpy as np
    import torch

    from paper_2309_11072_gb300 import codec, native

    h, w = c.h, c.w
    levels_n = 3
    nb = 1 + 3 * levels_n
    lengths = [a * b for a, b in native.dwt53_bands(h, w, levels_n)] * 3
    bh, bw = (h + 7) // 8, (w + 7) // 8
    lv = torch.empty(3 * bh * bw * 64, dtype=torch.int16, device="cuda")
    s3 = torch.empty_like(c.s3)
    bits3 = torch.empty(3, dtype=torch.int64, device="cuda")
    coef = torch.empty(3 * n, dtype=torch.int16, device="cuda")
    bhist = torch.empty(3 * nb * 511, dtype=torch.int32, device="cuda")
    bfreq = torch.empty_like(bhist)
    ws = torch.empty(native.dwt53_workspace_bytes(3, h, w), dtype=torch.uint8, device="cuda")
    nw, nc = native.rans_segments_capacity(lengths)
    words = torch.empty(nw, dtype=torch.int16, device="cuda")
    counts = torch.empty(nc, dtype=torch.int32, device="cuda")
    r_plain = torch.empty_like(c.r3)
    ident = torch.from_numpy(codec.params_from_numpy(np.full((3, 256), 1 / 16, np.float32),
                                                     np.zeros((3, 256), np.float32))).cuda()

    def enh_bits(r3):
        native.dwt53_forward(r3, 3, h, w, levels_n, coef, bhist, ws, stream)
        native.rans_tables_n(bhist, 3 * nb, bfreq, stream)
        native.rans_encode_segments(coef, lengths, bfreq, words, counts, stream)
        cnt = counts.cpu().numpy().view(np.uint32)
        raw = cnt == 0xFFFFFFFF
        return (16.0 * cnt[~raw].astype(np.int64).sum() + 16.0 * 8192 * (int(raw.sum()) // 32)) / n

    # the YCbCr 4:2:0 base layer: its own levels, sizes, fit and residuals
    nbY = ((h + 7) // 8) * ((w + 7) // 8)
    nbC = (((h + 1) // 2 + 7) // 8) * (((w + 1) // 2 + 7) // 8)
    lv420 = torch.empty((nbY + 2 * nbC) * 64, dtype=torch.int16, device="cuda")
    ws420 = torch.empty(native.sdri_base_420_workspace_bytes(h, w), dtype=torch.uint8, device="cuda")
    s420 = torch.empty_like(c.s3)
    r420 = torch.empty_like(c.r3)
    sums = torch.empty_like(c.sums)
    params = torch.empty_like(c.params)

    out = {"form": "base: JPEG baseline Huffman of the quantised levels (4:4:4: each RGB plane with the luminance "
                   "tables; 4:2:0: Y with the luminance, Cb and Cr with the chrominance tables); enhancement: "
                   "three-level 5/3 wavelet + rANS (a table per band); bits per pixel"}
    native.device_status(clear=True)
    for q in list(range(10, 101, 10)) + [85]:
        c.encode(rgbe, q)
        native.sdri_base_levels(c.m3, c.e, h, w, c.stats, q, s3, lv, stream)
        native.jpeg_huffman_bits(lv, h, w, bits3, None, stream)
        base = float(bits3.cpu().numpy().sum()) / n
        slr = enh_bits(c.r3)
        native.residual_encode(c.s3, c.m3, c.e, h, w, 0, ident, r_plain, None, stream)
        plain = enh_bits(r_plain)
        native.sdri_base_roundtrip_420(c.m3, c.e, h, w, c.stats, q, s420, lv420, ws420, stream)
        native.jpeg_huffman_bits_planes(lv420, [nbY, nbC, nbC], [0, 1, 1], bits3, None, stream)
        base420 = float(bits3.cpu().numpy().sum()) / n
        native.slr_fit(s420, c.m3, c.e, h, w, 1, sums, params, stream)
        native.residual_encode(s420, c.m3, c.e, h, w, 1, params, r420, None, stream)
        slr420 = enh_bits(r420)
        out[str(q)] = {"base": round(base, 4), "enh_slr": round(slr, 4), "enh_without_slrme": round(plain, 4),
                       "total_slr": round(base + slr, 4), "total_without_slrme": round(base + plain, 4),
                       "base_420": round(base420, 4), "enh_slr_420": round(slr420, 4),
                       "total_slr_420": round(base420 + slr420, 4)}
    out["status"] = native.device_status(clear=True)
    return out


def base_layer_bits(c, rgbe, qualities, n, args, flush, stream, enh) -> dict:
    """The base layer's coded size at each quality: the quantised levels of
    the round trip (sdri_base_levels) and the JPEG baseline Huffman size of
    their coding (jpeg_huffman_bits, luminance tables of T.81 Annex K.3,
    entropy-coded bits before byte stuffing and markers), the total with the
    enhancement layer's wavelet form, and the same base size for the YCbCr
    4:2:0 layer (sdri_base_roundtrip_420, jpeg_huffman_bits_planes), in bits
    per pixel; device times by CUDA events around each call (host gaps
    included, L2 flushed between repetitions)."""
    import numpy as np
    import torch

    from paper_2309_11072_gb300 import native

    h, w = c.h, c.w
    bh, bw = (h + 7) // 8, (w + 7) // 8
    levels = torch.empty(3 * bh * bw * 64, dtype=torch.int16, device="cuda")
    s3 = torch.empty_like(c.s3)
    bits = torch.empty(3, dtype=torch.int64, device="cuda")
    out = {"coder": "JPEG baseline Huffman (T.81 Annex K.3 luminance tables), each plane its own scan; "
                    "entropy-coded bits without byte stuffing, markers or headers"}
    nbY = bh * bw
    nbC = (((h + 1) // 2 + 7) // 8) * (((w + 1) // 2 + 7) // 8)
    lv420 = torch.empty((nbY + 2 * nbC) * 64, dtype=torch.int16, device="cuda")
    ws420 = torch.empty(native.sdri_base_420_workspace_bytes(h, w), dtype=torch.uint8, device="cuda")
    bits420 = torch.empty(3, dtype=torch.int64, device="cuda")
    names = ("sdri_base_levels", "jpeg_huffman_bits", "sdri_base_roundtrip_420", "jpeg_huffman_bits_planes")
    for q in qualities:
        c.encode(rgbe, q)
        t = {k: [] for k in names}
        for rep in range(args.warmup + args.steps):
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
            ev[0].record(stream)
            native.sdri_base_levels(c.m3, c.e, h, w, c.stats, q, s3, levels, stream)
            ev[1].record(stream)
            native.jpeg_huffman_bits(levels, h, w, bits, None, stream)
            ev[2].record(stream)
            native.sdri_base_roundtrip_420(c.m3, c.e, h, w, c.stats, q, s3, lv420, ws420, stream)
            ev[3].record(stream)
            native.jpeg_huffman_bits_planes(lv420, [nbY, nbC, nbC], [0, 1, 1], bits420, None, stream)
            ev[4].record(stream)
            flush.zero_()
            torch.cuda.synchronize()
            if rep >= args.warmup:
                for i, k in enumerate(names):
                    t[k].append(ev[i].elapsed_time(ev[i + 1]) * 1e3)
        base = float(bits.cpu().numpy().sum()) / n
        wav = enh[str(q)]["wavelet"]["coded_bits_per_px"]
        out[str(q)] = {"base_bits_per_px": round(base, 4), "total_bits_per_px": round(base + wav, 4),
                       "base_420_bits_per_px": round(float(bits420.cpu().numpy().sum()) / n, 4),
                       "us": {k: round(statistics.mean(v), 2) for k, v in t.items()}}
    return out


def measure_batch(args) -> dict:
    """The batch form on the 64-image uneven workload: plan, autotune, capture
    encode + decode as one CUDA graph, time graph launches with CUDA events
    (inputs larger than L2), check every image against its input words."""
    import numpy as np
    import torch

    from paper_2309_11072_gb300 import batch as Bm
    from paper_2309_11072_gb300 import synth

    wl = synth.workload_batch()
    imgs = synth.make_workload_images(wl)
    bc = Bm.BatchCodec(wl.sizes, list(wl.qualities) * len(wl.sizes))
    bc.load(imgs)
    tiles = bc.autotune(reps=3)
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        bc.graph_build(side)
        for _ in range(args.warmup):
            bc.graph_launch(side)
        side.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        for a, b in ev:
            a.record(side)
            bc.graph_launch(side)
            b.record(side)
        side.synchronize()
    ms = [a.elapsed_time(b) for a, b in ev]
    total = sum(ms)
    px = sum(h * w for h, w in wl.sizes)
    ok = all(np.array_equal(bc.image_layers(i)["out"].cpu().numpy().view(np.uint32), img)
             for i, img in enumerate(imgs))
    peaks = load_peaks()
    bpp = sum(BYTES_PER_PX.values())
    gbs = bpp * px / (total / args.steps * 1e-3) / 1e9
    bc.close()
    del bc
    torch.cuda.empty_cache()
    return {"workload": f"{wl.name}: {len(imgs)} images, {px / 1e6:.1f} MP, q90, one CUDA graph of persistent "
                        "stage kernels", "value": round(px * args.steps / (total / 1e3) / 1e6, 2), "unit": UNIT,
            "ms_per_step": round(total / args.steps, 4), "pixels_per_step": px, "steps": args.steps,
            "tiles": tiles, "l2": "inputs larger than L2", "bit_exact": ok,
            "roofline": {"bound": "hbm", "achieved": round(gbs, 1), "peak": peaks["hbm_gbs"], "unit": "GB/s",
                         "frac": round(gbs / peaks["hbm_gbs"], 4), "traffic": None,
                         "kernel": "whole encode+decode graph", "bytes_per_px": bpp, "peak_source": peaks["src"]}}


def run_batch(args) -> None:
    """The batch form alone, as its own JSON line."""
    import torch
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    m = measure_batch(args)
    line = {"metric": METRIC, "value": m["value"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": m["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": {"workload": m["workload"], "tiles": m["tiles"], "l2": m["l2"]},
            "bit_exact": m["bit_exact"], "roofline": m["roofline"]}
    print(json.dumps(line), flush=True)


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the machine type)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=20).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.machine()


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def image_bands(img, parts: int):
    """The image cut into `parts` horizontal bands of whole rows (at least 8
    rows each), as independent images."""
    import numpy as np
    h = img.shape[0]
    parts = max(1, min(parts, h // 8 if h >= 8 else 1))
    edges = np.linspace(0, h, parts + 1).astype(int)
    return [np.ascontiguousarray(img[edges[k]:edges[k + 1]]) for k in range(parts)]


def _oracle_pass(band, q) -> bool:
    """One full encode + decode of one image by the CPU oracle (the oracle's
    C calls release the GIL, so threads run them on separate cores)."""
    from oracle import oracle as O
    o = O.encode(band, q)
    d = O.decode(o["s3"], o["e"], o["r3"], o["a"], o["b"])
    return bool((d == band).all())


def cpu_baseline(img, qualities, budget_s: float) -> dict:
    """The CPU oracle, as it stands, on bands of the same image: a single
    thread coding one band repeatedly for about budget_s / 2 seconds, then one
    thread per host core, each coding its own band repeatedly for about as
    long (full encode + decode per pass, qualities cycling)."""
    from concurrent.futures import ThreadPoolExecutor

    from oracle import oracle as O
    O.lib()
    cores = host_cores()
    bands = image_bands(img, cores)

    def worker(band, seconds):
        done, i, t0 = 0, 0, time.perf_counter()
        while True:
            _oracle_pass(band, qualities[i % len(qualities)])
            done += band.size
            i += 1
            if time.perf_counter() - t0 >= seconds:
                return done, i

    t0 = time.perf_counter()
    px1, passes1 = worker(bands[0], budget_s / 2)
    dt1 = time.perf_counter() - t0
    with ThreadPoolExecutor(max_workers=len(bands)) as ex:
        t0 = time.perf_counter()
        res = list(ex.map(lambda b: worker(b, budget_s / 2), bands))
        dtn = time.perf_counter() - t0
    pxn = sum(r[0] for r in res)
    hb, wb = bands[0].shape
    return {"value": round(pxn / dtn / 1e6, 4), "unit": UNIT, "cores": len(bands), "kind": "oracle",
            "cpu_model": cpu_model(), "host_cores": cores,
            "sample": f"{len(bands)} threads, each coding its own horizontal band ({wb} columns, about {hb} "
                      f"rows) of the {img.shape[1]}x{img.shape[0]} image repeatedly with the single-threaded C "
                      f"oracle (full encode + decode, q cycling {list(qualities)}), {dtn:.1f} s, "
                      f"{sum(r[1] for r in res)} passes",
            "single_core": {"value": round(px1 / dt1 / 1e6, 4), "unit": UNIT, "cores": 1,
                            "sample": f"{passes1} passes over one {wb}x{hb} band, {dt1:.1f} s"}}


def run_reference(args) -> None:
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from concurrent.futures import ThreadPoolExecutor

    from oracle import oracle as O
    from paper_2309_11072_gb300 import synth
    O.build()
    O.lib()
    wl = synth.workload_8k() if args.workload == "8k" else synth.workload_2k()
    img = synth.make_workload_images(wl)[0]
    qualities = wl.qualities
    cores = host_cores()
    bands = image_bands(img, cores)

    def one(ex, k):
        q = qualities[k % len(qualities)]
        return all(ex.map(lambda b: _oracle_pass(b, q), bands))

    ok = True
    with ThreadPoolExecutor(max_workers=len(bands)) as ex:
        for k in range(args.warmup):
            one(ex, k)
        t0 = time.perf_counter()
        for k in range(args.steps):
            ok &= one(ex, k)
        dt = time.perf_counter() - t0
    value = img.size * args.steps / dt / 1e6
    sample = (f"each step: the whole {img.shape[1]}x{img.shape[0]} image as {len(bands)} horizontal bands, one "
              f"thread per band running the single-threaded C oracle (full encode + decode), the bands concurrently")
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": 0,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * dt / args.steps, 2),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": {"workload": f"{wl.name} q{{{','.join(map(str, qualities))}}} encode+decode, SLR, "
                                   "gaussian restoration on",
                       "pixels_per_step": int(img.size), "qualities": list(qualities),
                       "step": "one full-image encode+decode over all host cores, quality cycling"},
            "bit_exact": ok,
            "cpu_baseline": {"value": round(value, 4), "unit": UNIT, "cores": len(bands), "kind": "oracle",
                             "cpu_model": cpu_model(), "sample": sample},
            "e2e": {"value": round(value, 4), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", choices=["2k", "8k", "batch64"], default="8k",
                    help="8k: the benchmark line, the 7680x4320 image (q90); 2k: the 2048x1536 image "
                         "(q 50/75/90); batch64: the batch form on 64 uneven images alone")
    ap.add_argument("--no-extras", action="store_true",
                    help="8k: skip the 2048x1536 rates and the batch form")
    args = ap.parse_args()
    if args.impl == "ours":
        args.warmup = max(3, args.warmup)   # at least three untimed warm-up steps on the GPU
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch64":
        run_batch(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
