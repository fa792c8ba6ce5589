"""Benchmark: clamp-to-edge conv2d on 8192 x 8192 x 3 FP32 images.

One step = the four filter passes of that workload over the resident image:
3x3, 7x7 and 15x15 direct (normalised U[0,1) weights) and a 15x15 Gaussian
(sigma 3) through the separable kernel.  `value` is output Gpixel/s of the
whole job (all ranks); `e2e` is the same metric through the plain C-ABI calls
with pinned HOST buffers, so host<->device copies are inside its timed region.
Extra keys report the other workloads (Jacobi 8192^2 x 100 sweeps, the FP16
storage variant) measured the same way.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun (N > 1) each rank runs the same workload on its own GPU
(independent images: weak scaling, no data-path collective).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "conv2d/Jacobi Gpixel/s and % of HBM peak; served vs plain at p50/p99 latency"
C, H, W = 3, 8192, 8192
DIRECT_K = (3, 7, 15)
GAUSS_R, GAUSS_SIGMA = 7, 3.0
PX_PER_PASS = C * H * W
PASSES = len(DIRECT_K) + 1
PX_PER_STEP = PX_PER_PASS * PASSES
SM_COUNT = 152
FP32_LANES_PER_SM = 128
SM_MAX_MHZ = 2070.0
SERVE_SECONDS = 60.0
WORKLOAD = ("conv2d clamp-to-edge, 3 planar channels of 8192x8192 FP32, filters 3x3/7x7/15x15 "
            "direct (normalised U[0,1) weights) + 15x15 Gaussian sigma=3 separable")


def config(extra=None):
    cfg = {"workload": WORKLOAD, "channels": C, "h": H, "w": W,
           "filters": ["3x3", "7x7", "15x15", "gauss15x15-separable"],
           "seed": synth.SEEDS["conv8192x3"],
           "l2": "inputs larger than L2 (768 MiB image vs 129 MB L2); no flush between steps"}
    if extra:
        cfg.update(extra)
    return cfg


def fp32_peak_tflops():
    """FP32 (non-tensor) FMA peak from unit counts and the maximum SM clock."""
    return SM_COUNT * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


KERNEL_SOURCES = ["paper_1302_5586_gb300/csrc/conv2d.cu", "paper_1302_5586_gb300/csrc/conv_tile.cuh",
                  "paper_1302_5586_gb300/csrc/internal.cuh", "paper_1302_5586_gb300/csrc/tma.cuh"]


def sources_sha(paths=KERNEL_SOURCES):
    hsh = hashlib.sha256()
    for p in paths:
        with open(os.path.join(ROOT, p), "rb") as f:
            hsh.update(f.read())
    return hsh.hexdigest()[:16]


def traffic_record(kernel_key):
    """DRAM bytes per launch from the committed ncu summary, if the kernel
    sources have not changed since it was taken."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f).get(kernel_key)
    except (OSError, ValueError):
        return None
    if not rec:
        return None
    return rec.get("bytes_per_launch") if rec.get("source_sha") == sources_sha() else None


class Clocks:
    """nvidia-smi samples (200 ms) while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.f = None

    def __enter__(self):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        self.f.flush()

    def summary(self):
        self.f.seek(0)
        rows = [r.split(", ") for r in self.f.read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        sm, mx, reasons = [], [], set()
        for r in rows:
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except ValueError:
                continue
            for n, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def max_over_ranks(ms, dist, device):
    """The slowest rank's elapsed time (every rank gets it)."""
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_gpx(px_per_step, world, steps, ms):
    """Output Gpixel/s of all ranks: every rank processes its own images."""
    return px_per_step * world * steps / (ms * 1e-3) / 1e9


# ------------------------------------------------------------------ our arm
def run_ours(args, rank, world, local_rank):
    import torch

    import paper_1302_5586_gb300 as pg

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    seed = synth.SEEDS["conv8192x3"]
    img = synth.image_f32(seed + rank * 7919, C, H, W)  # each rank: its own images
    ks = [synth.filter_f32(seed + K, K, K) for K in DIRECT_K]
    g = synth.gaussian_taps_f32(GAUSS_R, GAUSS_SIGMA)
    d_img = torch.from_numpy(img).to(dev)
    d_ks = [torch.from_numpy(k).to(dev) for k in ks]
    d_g = torch.from_numpy(g).to(dev)
    d_out = [torch.empty_like(d_img) for _ in range(PASSES)]
    stream = torch.cuda.Stream(dev)
    sraw = stream.cuda_stream

    def step(ev15=None):
        for n, (K, dk) in enumerate(zip(DIRECT_K, d_ks)):
            if K == 15 and ev15 is not None:
                ev15[0].record(stream)
            pg.pencil_conv2d_ex(C, H, W, d_img, K, K, dk, d_out[n], pg.PENCIL_F32, 0, sraw)
            if K == 15 and ev15 is not None:
                ev15[1].record(stream)
        pg.pencil_conv2d_sep_ex(C, H, W, d_img, 15, d_g, 15, d_g, d_out[-1], pg.PENCIL_F32, 0, sraw)

    def barrier():
        torch.cuda.synchronize(dev)
        if dist is not None:
            dist.barrier()

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
    barrier()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = Clocks(local_rank)
    with clocks:
        with torch.cuda.stream(stream):
            t0.record(stream)
            for i in range(args.steps):
                step(ev[i])
            t1.record(stream)
        barrier()
    ms = t0.elapsed_time(t1)
    k15_ms = sum(a.elapsed_time(b) for a, b in ev) / args.steps
    if dist is not None:
        ms = max_over_ranks(ms, dist, dev)
    ms_per_step = ms / args.steps
    value = whole_job_gpx(PX_PER_STEP, world, args.steps, ms)

    # dominant kernel roofline: 15x15 direct conv is FP32-pipe bound
    flops_15 = 2 * 15 * 15 * PX_PER_PASS
    achieved = flops_15 / (k15_ms * 1e-3) / 1e12
    peak = fp32_peak_tflops()
    traffic = traffic_record("conv2d_direct_f32_15x15_8192x8192x3")
    roofline = {"bound": "alu", "kernel": "conv2d_direct_tma_kernel<float,15,15,16,8,4,2,3,false,true>",
                "achieved": round(achieved, 3),
                "peak": round(peak, 2), "unit": "TFLOP/s", "frac": round(achieved / peak, 4),
                "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz",
                "launch_ms": round(k15_ms, 4), "algorithmic_bytes": 8 * PX_PER_PASS, "traffic": traffic}
    clk = clocks.summary()

    extras = {}
    if rank == 0 and not args.no_extras:
        extras = measure_extras(torch, pg, dev, stream, d_img, d_out, ks, g, args.serve_seconds)
    e2e = measure_e2e(torch, pg, img, ks, g, max(2, min(args.steps // 50, 5))) if not args.no_e2e else None

    del d_out, d_img
    if dist is not None:
        dist.barrier()
    if rank == 0:
        cpu = None if (world > 1 or args.no_cpu) else cpu_baseline(img, ks, g, budget_s=args.cpu_seconds)
        launches = PASSES * args.steps
        line = {"metric": METRIC, "value": round(value, 3), "unit": "Gpixel/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_per_step, 4),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic (seeded SplitMix64 U[0,1) images; normalised U[0,1) and Gaussian filters)",
                "config": config({"parallelism": f"replicas x{world} (independent images per GPU)"}),
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
                "clocks": clk, "hbm_peak_gbs": measured_peaks().get("hbm_gbs")}
        line.update(extras)
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


def _time_stream(torch, stream, fn, reps):
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        fn()
        torch.cuda.synchronize()
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def measure_extras(torch, pg, dev, stream, d_img, d_out, ks, g, serve_seconds=SERVE_SECONDS):
    """Per-pass kernel times of the workload, the FP16-storage variant, and
    the 8192^2 x 100-sweep Jacobi run (residual every 10 sweeps)."""
    sraw = stream.cuda_stream
    hbm = measured_peaks().get("hbm_gbs") or 6800.0
    out = {}
    per = {}
    d_ks = [torch.from_numpy(k).to(dev) for k in ks]
    d_g = torch.from_numpy(g).to(dev)
    for K, dk in zip(DIRECT_K, d_ks):
        ms = _time_stream(torch, stream, lambda: pg.pencil_conv2d_ex(C, H, W, d_img, K, K, dk, d_out[0],
                                                                     pg.PENCIL_F32, 0, sraw), 10)
        per[f"{K}x{K}"] = {"ms": round(ms, 4), "gpx_s": round(PX_PER_PASS / ms / 1e6, 2),
                           "hbm_frac": round(8 * PX_PER_PASS / (ms * 1e-3) / 1e9 / hbm, 4),
                           "fp32_frac": round(2 * K * K * PX_PER_PASS / (ms * 1e-3) / 1e12 / fp32_peak_tflops(), 4)}
    ms = _time_stream(torch, stream, lambda: pg.pencil_conv2d_sep_ex(C, H, W, d_img, 15, d_g, 15, d_g, d_out[0],
                                                                     pg.PENCIL_F32, 0, sraw), 10)
    per["gauss15-sep"] = {"ms": round(ms, 4), "gpx_s": round(PX_PER_PASS / ms / 1e6, 2),
                          "hbm_frac": round(8 * PX_PER_PASS / (ms * 1e-3) / 1e9 / hbm, 4)}
    out["passes_f32"] = per
    # FP16 storage, same filters
    d16 = d_img.half()
    o16 = torch.empty_like(d16)
    per16 = {}
    for K, dk in zip(DIRECT_K, d_ks):
        ms = _time_stream(torch, stream, lambda: pg.pencil_conv2d_ex(C, H, W, d16, K, K, dk, o16,
                                                                     pg.PENCIL_F16, 0, sraw), 10)
        per16[f"{K}x{K}"] = {"ms": round(ms, 4), "gpx_s": round(PX_PER_PASS / ms / 1e6, 2),
                             "hbm_frac": round(4 * PX_PER_PASS / (ms * 1e-3) / 1e9 / hbm, 4)}
    ms = _time_stream(torch, stream, lambda: pg.pencil_conv2d_sep_ex(C, H, W, d16, 15, d_g, 15, d_g, o16,
                                                                     pg.PENCIL_F16, 0, sraw), 10)
    per16["gauss15-sep"] = {"ms": round(ms, 4), "gpx_s": round(PX_PER_PASS / ms / 1e6, 2),
                            "hbm_frac": round(4 * PX_PER_PASS / (ms * 1e-3) / 1e9 / hbm, 4)}
    out["passes_f16"] = per16
    del d16, o16
    # Jacobi 8192^2, 100 sweeps, residual after every 10 sweeps
    n = 8192
    u0 = torch.from_numpy(synth.jacobi_init_f32(synth.SEEDS["jacobi8192"], n, n)).to(dev)
    u = u0.clone()
    wsb = pg.pencil_jacobi2d_workspace_size(n, n)
    ws = torch.empty(wsb, dtype=torch.uint8, device=dev)
    res = torch.empty(10, dtype=torch.float64, device=dev)
    jac = {}
    for t in (1, 0):
        def run():
            u.copy_(u0)
            pg.pencil_jacobi2d_ex(n, n, u, 100, 10, res, ws, wsb, t, sraw)
        ms_copy = _time_stream(torch, stream, lambda: u.copy_(u0), 3)
        ms = _time_stream(torch, stream, run, 3) - ms_copy
        pts = (n - 2) * (n - 2) * 100
        jac[f"temporal_t={t or 'auto'}"] = {
            "ms": round(ms, 3), "gpt_sweeps_s": round(pts / ms / 1e6, 2),
            "effective_hbm_frac": round(8 * n * n * 100 / (ms * 1e-3) / 1e9 / hbm, 4)}
    jac["residuals"] = [float(x) for x in res.cpu()]
    out["jacobi_8192x8192_100sweeps"] = jac
    # red-black SOR, omega 1.9, in place: per sweep each point is read twice and
    # its float4 written twice (16 B per point-sweep)
    wsr = pg.pencil_rbsor2d_workspace_size(n, n)

    def sor():
        u.copy_(u0)
        pg.pencil_rbsor2d_ex(n, n, u, 100, 1.9, 10, res, ws, wsr, sraw)
    ms_copy = _time_stream(torch, stream, lambda: u.copy_(u0), 3)
    ms = _time_stream(torch, stream, sor, 3) - ms_copy
    out["rbsor_8192x8192_100sweeps"] = {
        "ms": round(ms, 3), "gpt_sweeps_s": round((n - 2) * (n - 2) * 100 / ms / 1e6, 2),
        "hbm_frac_16B_per_point_sweep": round(16 * n * n * 100 / (ms * 1e-3) / 1e9 / hbm, 4),
        "residuals": [float(x) for x in res.cpu()]}
    del u0, u, ws
    out["plain_512x512_5x5"] = measure_small(torch, pg, dev, stream)
    out["batched_512"] = measure_batched(torch, pg, dev, stream)
    out["op2_inc_2048x2048_cells"] = measure_op2(torch, pg, dev, stream)
    out["chain_8192x8192x3"] = measure_chain(torch, pg, dev, stream, d_img, d_out)
    out["serving"] = measure_serving(torch, pg, dev, serve_seconds)
    return out



def measure_serving(torch, pg, dev, seconds):
    """Open-loop Poisson replay, FP16 storage, sides log-uniform [128, 4096],
    odd filter sides 3..15, 8 GiB arena budget: continuous batching against
    one launch per request, at 2000 req/s (latency) and at a saturating rate
    (throughput)."""
    from paper_1302_5586_gb300 import serve, tune

    res = {}
    seed = synth.SEEDS["serve"]
    for label, rate, dur in (("2000_req_s", 2000.0, seconds), ("saturation_40000_req_s", 40000.0, 0.5)):
        tr = serve.make_trace(seed, rate, dur)
        pool = serve.host_pool(tr, pg.PENCIL_F16, seed + 1)
        bank = torch.from_numpy(tr.filters).to(dev)
        srv = serve.Server(dtype=pg.PENCIL_F16, budget_bytes=8 << 30, streams=4, max_wave=64, max_inflight=256)
        try:
            srv.set_variants(tune.cached_variants(pg.PENCIL_F16))
            served, _ = srv.run(tr, pool, bank, mode="served")
            plain, _ = srv.run(tr, pool, bank, mode="plain")
        finally:
            srv.close()
        res[label] = {"offered_req_s": rate, "seconds": dur,
                      "offered_gpx_s": round(sum(r.h * r.w for r in tr.requests) / dur / 1e9, 3),
                      "served": served.summary(), "plain": plain.summary()}
        del pool, bank
    return res


def measure_chain(torch, pg, dev, stream, d_img, d_out):
    """Two filters in a row on the 3 x 8192^2 FP32 image: the fused chain
    kernel (forced) against two conv2d passes through a temporary (same bits),
    and what pencil_conv2d_chain picks by default.  HBM basis: 8 B per pixel
    fused (read in, write out), 16 B for two passes."""
    hbm = measured_peaks().get("hbm_gbs") or 6800.0
    sraw = stream.cuda_stream
    tmp = torch.empty_like(d_img)
    res = {}
    for k1s, k2s in ((3, 3), (5, 5), (7, 7)):
        k1 = torch.from_numpy(synth.filter_f32(60 + k1s, k1s, k1s)).to(dev)
        k2 = torch.from_numpy(synth.gaussian_2d_f32(k2s // 2, 1.0)).to(dev)
        ms_f = _time_stream(torch, stream, lambda: pg.pencil_conv2d_chain(C, H, W, d_img, k1s, k1s, k1, k2s, k2s, k2,
                                                                          d_out[0], pg.PENCIL_F32,
                                                                          pg.PENCIL_CHAIN_FUSED, sraw), 10)
        ms_l = _time_stream(torch, stream, lambda: pg.pencil_conv2d_chain(C, H, W, d_img, k1s, k1s, k1, k2s, k2s, k2,
                                                                          d_out[0], pg.PENCIL_F32, 0, sraw), 10)

        def two():
            pg.pencil_conv2d_ex(C, H, W, d_img, k1s, k1s, k1, tmp, pg.PENCIL_F32, 0, sraw)
            pg.pencil_conv2d_ex(C, H, W, tmp, k2s, k2s, k2, d_out[0], pg.PENCIL_F32, 0, sraw)
        ms_t = _time_stream(torch, stream, two, 10)
        flop = 2 * (k1s * k1s + k2s * k2s) * PX_PER_PASS
        res[f"{k1s}x{k1s}->{k2s}x{k2s}"] = {
            "fused_ms": round(ms_f, 4), "two_pass_ms": round(ms_t, 4), "speedup": round(ms_t / ms_f, 3),
            "library_choice_ms": round(ms_l, 4),
            "fused_hbm_frac": round(8 * PX_PER_PASS / (ms_f * 1e-3) / 1e9 / hbm, 4),
            "fused_fp32_frac": round(flop / (ms_f * 1e-3) / 1e12 / fp32_peak_tflops(), 4)}
    del tmp
    return res


def measure_op2(torch, pg, dev, stream):
    """The OP2 edge-to-cell increment on a 2048 x 2048-cell mesh with shuffled
    labels (8.4 M edges): the ordered kernel (the sequential loop's bits)
    against FP64 atomics.  Algorithmic bytes per call: each edge's value and
    two cell indices once (16 B), each cell read and written once (16 B)."""
    hbm = measured_peaks().get("hbm_gbs") or 6800.0
    ncells, e2c = synth.mesh_edges(synth.SEEDS["op2mesh"], 2048, 2048)
    nedges = len(e2c)
    edge = torch.from_numpy(2.0 * synth.u01_f64(synth.SEEDS["op2mesh"] ^ 0x0E, nedges) - 1.0).to(dev)
    cell = torch.from_numpy(synth.u01_f64(synth.SEEDS["op2mesh"] ^ 0x0C, ncells)).to(dev)
    plan = pg.pencil_op2_plan_create(ncells, nedges, e2c)
    alg = 16 * nedges + 16 * ncells
    res = {"cells": ncells, "edges": nedges, "algorithmic_bytes": alg}
    try:
        for name, mode in (("ordered", pg.PENCIL_OP2_ORDERED), ("atomic", pg.PENCIL_OP2_ATOMIC)):
            ms = _time_stream(torch, stream, lambda: pg.pencil_op2_inc(plan, edge, cell, mode, stream.cuda_stream), 20)
            res[name] = {"ms": round(ms, 4), "gedges_s": round(nedges / ms / 1e6, 2),
                         "hbm_frac": round(alg / (ms * 1e-3) / 1e9 / hbm, 4)}
    finally:
        pg.pencil_op2_plan_destroy(plan)
    return res


def measure_small(torch, pg, dev, stream):
    """The small plain case: one 512 x 512 FP32 image, 5 x 5 normalised
    filter (1 MiB in, 1 MiB out: resident in the 129 MB L2, so launch latency
    and L2 bandwidth bound it, not HBM).  Device time per launch (events
    around 200 back-to-back launches, median of 5) and host wall time of the
    synchronous plain call on device pointers."""
    n, K = 512, 5
    x = torch.from_numpy(synth.image_f32(synth.SEEDS["conv512"], 1, n, n)).to(dev)
    k = torch.from_numpy(synth.filter_f32(synth.SEEDS["conv512"] + 1, K, K)).to(dev)
    y = torch.empty_like(x)
    sraw = stream.cuda_stream
    reps = []
    for _ in range(5):
        reps.append(_time_stream(torch, stream, lambda: pg.pencil_conv2d_ex(1, n, n, x, K, K, k, y, pg.PENCIL_F32,
                                                                            0, sraw), 200))
    us = statistics.median(reps) * 1e3
    # the same 200 launches captured once and replayed from a CUDA graph: the
    # device time per launch without the host's per-call cost
    graph_us = None
    try:
        g = torch.cuda.CUDAGraph()
        cap = torch.cuda.Stream(dev)
        cap.wait_stream(torch.cuda.current_stream(dev))
        with torch.cuda.graph(g, stream=cap):
            for _ in range(200):
                pg.pencil_conv2d_ex(1, n, n, x, K, K, k, y, pg.PENCIL_F32, 0, cap.cuda_stream)
        greps = []
        with torch.cuda.stream(stream):  # replay and events on the same stream
            g.replay()
            for _ in range(5):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                g.replay()
                b.record(stream)
                b.synchronize()
                greps.append(a.elapsed_time(b) / 200 * 1e3)
        graph_us = statistics.median(greps)
    except RuntimeError as e:  # capture not possible here: report the stream-launched number only
        graph_us = f"not captured: {e}"
    for _ in range(20):
        pg.pencil_conv2d(n, n, x, K, K, k, y)
    t = time.perf_counter()
    for _ in range(500):
        pg.pencil_conv2d(n, n, x, K, K, k, y)
    call_us = (time.perf_counter() - t) / 500 * 1e6
    px = n * n
    best = graph_us if isinstance(graph_us, float) else us
    return {"device_us_per_launch": round(best, 2), "gpx_s": round(px / best / 1e3, 2),
            "l2_resident_gb_s": round(8 * px / best / 1e3, 1), "graph_replay_us": graph_us if not isinstance(
                graph_us, float) else round(graph_us, 2), "stream_launch_us": round(us, 2),
            "plain_call_us": round(call_us, 2),
            "note": "fits in L2: launch-latency bound; GB/s is L2-resident, not HBM"}


def measure_batched(torch, pg, dev, stream):
    """512 uneven images (sides log-uniform in [64, 4096], odd filter sides
    3..15): one persistent launch per batch (graph replay, autotuned tiles)
    against one standalone launch per image, FP32 and FP16 storage."""
    from paper_1302_5586_gb300 import tune

    seed = synth.SEEDS["batch512"]
    h, w, k = synth.batch_spec(seed, 512, 64, 4096)
    hbm = (measured_peaks().get("hbm_gbs") or 6800.0) * 1e9
    fp32 = fp32_peak_tflops() * 1e12
    px = int(np.sum(h.astype(np.int64) * w))
    res = {"images": 512, "pixels": px, "mean_flop_per_px": round(float(np.sum(2.0 * k * k * h * w) / px), 1)}
    for dtype, name, esz in ((pg.PENCIL_F32, "f32", 4), (pg.PENCIL_F16, "f16", 2)):
        items = []
        for i in range(512):
            img = synth.image_f32(seed + 17 * i, 1, int(h[i]), int(w[i]))
            t = torch.from_numpy(img).to(dev)
            if dtype == pg.PENCIL_F16:
                t = t.half()
            kk = torch.from_numpy(synth.filter_f32(seed + 17 * i + 1, int(k[i]), int(k[i]))).to(dev)
            items.append((t, torch.empty_like(t), kk, int(h[i]), int(w[i]), int(k[i])))
        plan = pg.pencil_batch_create(dtype, 512, 1 << 22)
        with torch.cuda.stream(stream):
            chosen = tune.autotune(plan, dtype, items, reps=3)
            imgs = pg.make_images(items)
            ms_b = _time_stream(torch, stream, lambda: pg.pencil_batch_run(plan, imgs, stream.cuda_stream), 5)

            def per_image():
                for it in items:
                    pg.pencil_conv2d_ex(1, it[3], it[4], it[0], it[5], it[5], it[2], it[1], dtype, 0,
                                        stream.cuda_stream)
            ms_p = _time_stream(torch, stream, per_image, 3)
        pg.pencil_batch_destroy(plan)
        # roofline time: per image the larger of its HBM time and FP32 time
        roof = float(np.sum(np.maximum(2 * esz * h * w / hbm, 2.0 * k * k * h * w / fp32))) * 1e3
        res[name] = {"batched_ms": round(ms_b, 3), "batched_gpx_s": round(px / ms_b / 1e6, 2),
                     "per_image_launch_ms": round(ms_p, 3), "per_image_gpx_s": round(px / ms_p / 1e6, 2),
                     "roofline_ms": round(roof, 3), "frac_of_roofline": round(roof / ms_b, 4),
                     "variants": {str(a): v for a, (v, _) in chosen.items()}}
        del items
    return res


def measure_e2e(torch, pg, img, ks, g, steps):
    """Plain C-ABI calls with pinned host buffers: each call copies its input
    in, runs the kernel, and copies its output back before returning."""
    h_in = torch.from_numpy(img).pin_memory()
    h_out = torch.empty_like(h_in).pin_memory()
    h_ks = [np.ascontiguousarray(k) for k in ks]

    def step():
        for K, k in zip(DIRECT_K, h_ks):
            for ch in range(C):
                pg.pencil_conv2d(H, W, h_in[ch], K, K, k, h_out[ch])
        for ch in range(C):
            pg.pencil_conv2d_sep(H, W, h_in[ch], 15, g, 15, g, h_out[ch])

    step()
    torch.cuda.synchronize()
    t = time.perf_counter()
    for _ in range(steps):
        step()
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t) / steps
    per_call = 4 * H * W
    return {"value": round(PX_PER_STEP / dt / 1e9, 3), "unit": "Gpixel/s",
            "h2d_bytes_per_step": PASSES * C * per_call, "d2h_bytes_per_step": PASSES * C * per_call,
            "steps": steps, "ms_per_step": round(dt * 1e3, 2),
            "api": "pencil_conv2d / pencil_conv2d_sep, pinned host buffers, one call per channel and filter"}


# ------------------------------------------------------------- CPU oracle
def _oracle_band(oracle, img, ks, g, rows, r0):
    """Oracle over rows [r0, r0+rows) of all channels for every pass of the step."""
    t = time.perf_counter()
    for K, k in zip(DIRECT_K, ks):
        a = K // 2
        lo, hi = max(0, r0 - a), min(H, r0 + rows + a)
        oracle.conv2d(img[:, lo:hi, :], k, want_bound=False)
    lo, hi = max(0, r0 - GAUSS_R), min(H, r0 + rows + GAUSS_R)
    oracle.conv2d_sep(img[:, lo:hi, :], g, g, want_bound=False)
    return time.perf_counter() - t


def cpu_baseline(img, ks, g, budget_s=15.0):
    import oracle

    probe = 32
    _oracle_band(oracle, img, ks, g, 8, 0)  # start the thread pool
    t_probe = _oracle_band(oracle, img, ks, g, probe, 4096)
    rows = int(max(probe, min(H, probe * budget_s / max(t_probe, 1e-6))))
    dt = _oracle_band(oracle, img, ks, g, rows, 4096 - rows // 2 if rows < H else 0)
    px = rows * W * C * PASSES
    return {"value": round(px / dt / 1e9, 6), "unit": "Gpixel/s", "cores": oracle.num_threads(),
            "kind": "oracle",
            "sample": f"FP64 oracle, all 4 passes over rows {rows} of 8192 (x3 channels) of the same image, {dt:.1f} s"}


def run_reference(args, rank, world):
    """The FP64 oracle on the host cores, on this workload: each step is a
    band of rows sized so the whole run stays within a few minutes."""
    if rank != 0:
        return
    import oracle

    img = synth.image_f32(synth.SEEDS["conv8192x3"], C, H, W)
    ks = [synth.filter_f32(synth.SEEDS["conv8192x3"] + K, K, K) for K in DIRECT_K]
    g = synth.gaussian_taps_f32(GAUSS_R, GAUSS_SIGMA)
    _oracle_band(oracle, img, ks, g, 8, 0)  # start the thread pool
    t_probe = _oracle_band(oracle, img, ks, g, 8, 4096)
    per_step_budget = max(0.01, args.ref_seconds / max(args.steps + args.warmup, 1))
    rows = int(max(1, min(H, 8 * per_step_budget / max(t_probe, 1e-6))))
    for i in range(args.warmup):
        _oracle_band(oracle, img, ks, g, rows, (i * rows) % (H - rows + 1))
    total = 0.0
    for i in range(args.steps):
        total += _oracle_band(oracle, img, ks, g, rows, (i * rows) % (H - rows + 1))
    px = rows * W * C * PASSES * args.steps
    value = px / total / 1e9
    cores = oracle.num_threads()
    sample = f"each step: FP64 oracle, all 4 passes over {rows} rows x 8192 x 3 channels"
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": "Gpixel/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(total / args.steps * 1e3, 2), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config({"parallelism": "host cores (OpenMP)"}),
            "cpu_baseline": {"value": round(value, 6), "unit": "Gpixel/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(value, 6), "unit": "Gpixel/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def run_case(name, reps):
    """One kernel on a reduced workload, for profiler captures: inputs still
    larger than L2, a few launches, a few hundred MB on the device."""
    import torch

    import paper_1302_5586_gb300 as pg

    dev = torch.device("cuda", 0)
    if name.startswith("conv"):
        f16 = name.endswith("h")
        K = int(name[4:].rstrip("h").split("-")[0])
        c, h, w = 2, 4096, 4096
        img = torch.from_numpy(synth.image_f32(1, c, h, w)).to(dev)
        if f16:  # binary16 storage: twice the pixels, so the image is still larger than L2
            c = 4
            img = torch.from_numpy(synth.to_f16(synth.image_f32(1, c, h, w))).to(dev)
        k = torch.from_numpy(synth.filter_f32(2, K, K)).to(dev)
        out = torch.empty_like(img)
        for _ in range(reps):
            pg.pencil_conv2d_ex(c, h, w, img, K, K, k, out, pg.PENCIL_F16 if f16 else pg.PENCIL_F32)
    elif name == "sep15":
        c, h, w = 2, 4096, 4096
        img = torch.from_numpy(synth.image_f32(1, c, h, w)).to(dev)
        g = torch.from_numpy(synth.gaussian_taps_f32(7, 3.0)).to(dev)
        out = torch.empty_like(img)
        for _ in range(reps):
            pg.pencil_conv2d_sep_ex(c, h, w, img, 15, g, 15, g, out, pg.PENCIL_F32)
    elif name == "batch":
        seed = synth.SEEDS["batch512"]
        h, w, k = synth.batch_spec(seed, 128, 64, 2048)
        items = []
        for i in range(128):
            t = torch.from_numpy(synth.image_f32(seed + i, 1, int(h[i]), int(w[i]))).to(dev)
            kk = torch.from_numpy(synth.filter_f32(seed + 500 + i, int(k[i]), int(k[i]))).to(dev)
            items.append((t, torch.empty_like(t), kk, int(h[i]), int(w[i]), int(k[i])))
        plan = pg.pencil_batch_create(pg.PENCIL_F32, 128, 1 << 20)
        imgs = pg.make_images(items)
        for _ in range(reps):
            pg.pencil_batch_run(plan, imgs)
        torch.cuda.synchronize()
        pg.pencil_batch_destroy(plan)
    elif name.startswith("chain"):
        K = int(name[5:])
        c, h, w = 2, 4096, 4096
        img = torch.from_numpy(synth.image_f32(1, c, h, w)).to(dev)
        k = torch.from_numpy(synth.filter_f32(2, K, K)).to(dev)
        out = torch.empty_like(img)
        for _ in range(reps):
            pg.pencil_conv2d_chain(c, h, w, img, K, K, k, K, K, k, out, pg.PENCIL_F32)
    elif name.startswith("op2"):
        ncells, e2c = synth.mesh_edges(synth.SEEDS["op2mesh"], 2048, 2048)
        edge = torch.from_numpy(synth.u01_f64(1, len(e2c))).to(dev)
        cell = torch.zeros(ncells, dtype=torch.float64, device=dev)
        plan = pg.pencil_op2_plan_create(ncells, len(e2c), e2c)
        mode = pg.PENCIL_OP2_ATOMIC if name == "op2-atomic" else pg.PENCIL_OP2_ORDERED
        for _ in range(reps):
            pg.pencil_op2_inc(plan, edge, cell, mode)
        torch.cuda.synchronize()
        pg.pencil_op2_plan_destroy(plan)
    elif name.startswith("jacobi"):
        t = int(name.split("t")[-1]) if "t" in name[6:] else 1
        n = 8192
        u = torch.from_numpy(synth.jacobi_init_f32(3, n, n)).to(dev)
        wsb = pg.pencil_jacobi2d_workspace_size(n, n)
        ws = torch.empty(wsb, dtype=torch.uint8, device=dev)
        res = torch.empty(reps, dtype=torch.float64, device=dev)
        pg.pencil_jacobi2d_ex(n, n, u, 10 * reps, 10, res, ws, wsb, t)
    else:
        raise SystemExit(f"unknown case {name}")
    torch.cuda.synchronize()
    print(f"case {name} done")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--case", default=None,
                    help="profile one kernel on a reduced workload: conv3, conv7, conv15, conv3h (binary16), sep15, batch, jacobi, jacobi-tN (N sweeps per pass), op2-ordered, op2-atomic, chain3, chain5, chain7")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=600)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--ref-seconds", type=float, default=150.0,
                    help="approximate host time of a --impl reference run (warm-up and timed steps)")
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--serve-seconds", type=float, default=SERVE_SECONDS)
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    if args.case:
        run_case(args.case, args.reps)
        return
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
