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
SM_COUNT = 152            # GB300; the run reads the device's own count
FP32_LANES_PER_SM = 128
SM_MAX_MHZ = 2070.0       # GB300; the run reads nvidia-smi's clocks.max.sm
TOL_F32 = 1e-6            # |gpu - oracle| <= TOL_F32 * sum|k||x| per pixel
TOL_F16 = 2.0 ** -10      # the same against the oracle on the binary16 input
TOL_JACOBI = 1e-5         # max |u_gpu - u_oracle| after 100 sweeps
SERVE_SECONDS = 60.0
WORKLOAD = ("conv2d clamp-to-edge, 3 planar channels of 8192x8192 FP32, filters 3x3/7x7/15x15 "
            "direct (normalised U[0,1) weights) + 15x15 Gaussian sigma=3 separable")


def config():
    """The workload both arms measure (the same dict for either)."""
    return {"workload": WORKLOAD, "channels": C, "h": H, "w": W,
            "filters": ["3x3", "7x7", "15x15", "gauss15x15-separable"],
            "seed": synth.SEEDS["conv8192x3"],
            "l2": "inputs larger than L2 (768 MiB image vs 129 MB L2); no flush between steps",
            "parallelism": "one image set per process (independent images: replicas, no collective)"}


_PEAK = {"sms": SM_COUNT, "mhz": SM_MAX_MHZ, "source": "nominal GB300 counts"}


def fp32_peak_tflops(sms=None, mhz=None):
    """FP32 (non-tensor) FMA peak from unit counts and the maximum SM clock:
    SMs x 128 FP32 lanes x 2 flops per FMA x MHz (the device's own SM count and
    maximum clock once set_fp32_peak has read them)."""
    sms = _PEAK["sms"] if sms is None else sms
    mhz = _PEAK["mhz"] if mhz is None else mhz
    return sms * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12


def set_fp32_peak(sms, mhz, source):
    _PEAK.update(sms=int(sms), mhz=float(mhz), source=source)


def max_sm_mhz(index):
    """clocks.max.sm of a GPU from nvidia-smi, or None."""
    try:
        r = subprocess.run(["nvidia-smi", "-i", str(index), "--query-gpu=clocks.max.sm",
                            "--format=csv,noheader,nounits"], capture_output=True, text=True, timeout=30)
        return float(r.stdout.strip().splitlines()[0])
    except (OSError, ValueError, IndexError, subprocess.TimeoutExpired):
        return None


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


KERNEL_SOURCES = ["paper_1302_5586_gb300/csrc/conv2d.cu", "paper_1302_5586_gb300/csrc/conv_kernels.cuh",
                  "paper_1302_5586_gb300/csrc/conv_tile.cuh", "paper_1302_5586_gb300/csrc/internal.cuh",
                  "paper_1302_5586_gb300/csrc/tma.cuh"]


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
    _, sms, _ = pg.pencil_device_info()
    mhz = max_sm_mhz(local_rank) or measured_peaks().get("sm_max_mhz") or SM_MAX_MHZ
    set_fp32_peak(sms, mhz, f"derived: {sms} SMs (device count) x 128 FP32 lanes x 2 flop x {mhz:.0f} MHz "
                            "(clocks.max.sm)")
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
    roofline = {"bound": "alu", "kernel": "conv2d_direct_tma_kernel<float,15,15,16,8,2,1,3,false,true,1,12>",
                "achieved": round(achieved, 3),
                "peak": round(peak, 2), "unit": "TFLOP/s", "frac": round(achieved / peak, 4),
                "peak_source": _PEAK["source"],
                "launch_ms": round(k15_ms, 4), "algorithmic_bytes": 8 * PX_PER_PASS, "traffic": traffic}
    clk = clocks.summary()

    extras, keep = {}, {}
    if rank == 0 and not args.no_extras:
        extras, keep = measure_extras(torch, pg, dev, stream, d_img, d_out, ks, g, args.serve_seconds)
    e2e = measure_e2e(torch, pg, img, ks, g, max(3, min(args.steps // 20, 24))) if not args.no_e2e else None

    if dist is not None:
        dist.barrier()
    if rank == 0:
        cpu, precision = None, None
        if world == 1 and not args.no_cpu:
            cpu, precision = cpu_baseline(torch, img, ks, g, d_out, keep, budget_s=args.cpu_seconds)
        del d_out, d_img, keep
        launches = PASSES * args.steps
        line = {"metric": METRIC, "value": round(value, 3), "unit": "Gpixel/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_per_step, 4),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic (seeded SplitMix64 U[0,1) images; normalised U[0,1) and Gaussian filters)",
                "config": config(), "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": launches, "clocks": clk, "hbm_peak_gbs": measured_peaks().get("hbm_gbs")}
        line.update(ordered_extras(extras, precision))
        print(json.dumps(line))
    else:
        del d_out, d_img
    if dist is not None:
        dist.destroy_process_group()


# Keys printed last, in this order: the per-config summary the reader needs
# most sits at the end of the line, where a truncated log keeps it.
SUMMARY_KEYS = ("batched_512", "serving_2000_req_s", "passes_f16", "passes_f32", "jacobi_8192x8192_100sweeps")


def ordered_extras(extras, precision):
    out = {k: v for k, v in extras.items() if k not in SUMMARY_KEYS}
    out.update({k: extras[k] for k in SUMMARY_KEYS if k in extras})
    if precision is not None:
        out["precision"] = precision
    return out


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


def _pass_entry(ms, bytes_per_px, flop_per_px, hbm):
    e = {"ms": round(ms, 4), "gpx_s": round(PX_PER_PASS / ms / 1e6, 1),
         "hbm": round(bytes_per_px * PX_PER_PASS / (ms * 1e-3) / 1e9 / hbm, 3)}
    if flop_per_px:
        e["fp32"] = round(flop_per_px * PX_PER_PASS / (ms * 1e-3) / 1e12 / fp32_peak_tflops(), 3)
    return e


def measure_extras(torch, pg, dev, stream, d_img, d_out, ks, g, serve_seconds=SERVE_SECONDS):
    """Per-pass kernel times of the workload (FP32 and binary16 storage), the
    8192^2 x 100-sweep Jacobi run (residual every 10 sweeps) and the other
    workloads.  Returns (results, keep): keep holds the outputs the CPU leg
    compares with the oracle (binary16 outputs per filter, the Jacobi iterate,
    sampled batch and served results)."""
    sraw = stream.cuda_stream
    hbm = measured_peaks().get("hbm_gbs") or 6800.0
    out, keep = {}, {}
    per = {}
    d_ks = [torch.from_numpy(k).to(dev) for k in ks]
    d_g = torch.from_numpy(g).to(dev)
    for K, dk in zip(DIRECT_K, d_ks):
        ms = _time_stream(torch, stream, lambda: pg.pencil_conv2d_ex(C, H, W, d_img, K, K, dk, d_out[0],
                                                                     pg.PENCIL_F32, 0, sraw), 10)
        per[f"{K}x{K}"] = _pass_entry(ms, 8, 2 * K * K, hbm)
    ms = _time_stream(torch, stream, lambda: pg.pencil_conv2d_sep_ex(C, H, W, d_img, 15, d_g, 15, d_g, d_out[0],
                                                                     pg.PENCIL_F32, 0, sraw), 10)
    per["gauss15-sep"] = _pass_entry(ms, 8, 0, hbm)
    # d_out[0] holds the 3x3 result again, as the timed steps left it
    pg.pencil_conv2d_ex(C, H, W, d_img, 3, 3, d_ks[0], d_out[0], pg.PENCIL_F32, 0, sraw)
    out["passes_f32"] = per
    # binary16 storage, same filters; each output kept for the precision check
    d16 = d_img.half()
    per16, o16s = {}, []
    for K, dk in zip(DIRECT_K, d_ks):
        o16 = torch.empty_like(d16)
        ms = _time_stream(torch, stream, lambda: pg.pencil_conv2d_ex(C, H, W, d16, K, K, dk, o16,
                                                                     pg.PENCIL_F16, 0, sraw), 10)
        per16[f"{K}x{K}"] = _pass_entry(ms, 4, 2 * K * K, hbm)
        o16s.append(o16)
    o16 = torch.empty_like(d16)
    ms = _time_stream(torch, stream, lambda: pg.pencil_conv2d_sep_ex(C, H, W, d16, 15, d_g, 15, d_g, o16,
                                                                     pg.PENCIL_F16, 0, sraw), 10)
    per16["gauss15-sep"] = _pass_entry(ms, 4, 0, hbm)
    o16s.append(o16)
    # the 7x7 and 15x15 passes again on the tensor cores (PENCIL_CONV_TENSOR:
    # within the binary16 tolerance, not the same bits); outputs checked too
    o16ts = {}
    for K, dk in zip(DIRECT_K, d_ks):
        if K < 7:
            continue
        o16t = torch.empty_like(d16)
        ms = _time_stream(torch, stream, lambda: pg.pencil_conv2d_ex(C, H, W, d16, K, K, dk, o16t, pg.PENCIL_F16,
                                                                     pg.PENCIL_CONV_TENSOR, sraw), 10)
        per16[f"{K}x{K}-tensor"] = _pass_entry(ms, 4, 2 * K * K, hbm)
        o16ts[K] = o16t
    out["passes_f16"] = per16
    keep["f16"] = (d16, o16s)
    keep["f16_tensor"] = o16ts
    # Jacobi 8192^2, 100 sweeps, residual after every 10 sweeps
    n = 8192
    u0h = synth.jacobi_init_f32(synth.SEEDS["jacobi8192"], n, n)
    u0 = torch.from_numpy(u0h).to(dev)
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
        jac[f"t{t}" if t else "auto"] = {
            "ms": round(ms, 3), "gpt_sweeps_s": round(pts / ms / 1e6, 1),
            "hbm_effective": round(8 * n * n * 100 / (ms * 1e-3) / 1e9 / hbm, 3)}
    jac["note"] = "t1: one sweep per pass; auto: the library's temporal tiling; hbm on 8 B per point-sweep"
    out["jacobi_8192x8192_100sweeps"] = jac
    keep["jacobi"] = (u0h, u, res)
    # red-black SOR, omega 1.9, in place: per sweep each point is read twice and
    # its float4 written twice (16 B per point-sweep)
    u2 = torch.empty_like(u0)
    res2 = torch.empty(10, dtype=torch.float64, device=dev)
    wsr = pg.pencil_rbsor2d_workspace_size(n, n)
    if wsr > wsb:
        ws = torch.empty(wsr, dtype=torch.uint8, device=dev)

    def sor():
        u2.copy_(u0)
        pg.pencil_rbsor2d_ex(n, n, u2, 100, 1.9, 10, res2, ws, wsr, sraw)
    ms_copy = _time_stream(torch, stream, lambda: u2.copy_(u0), 3)
    ms = _time_stream(torch, stream, sor, 3) - ms_copy
    out["rbsor_8192x8192_100sweeps"] = {
        "ms": round(ms, 3), "gpt_sweeps_s": round((n - 2) * (n - 2) * 100 / ms / 1e6, 1),
        "hbm_frac_16B_per_point_sweep": round(16 * n * n * 100 / (ms * 1e-3) / 1e9 / hbm, 3),
        "residuals": [float(f"{x:.6g}") for x in res2.cpu()]}
    del u0, u2, ws
    out["plain_512x512_5x5"], keep["plain512"] = measure_small(torch, pg, dev, stream)
    out["op2_inc_2048x2048_cells"] = measure_op2(torch, pg, dev, stream)
    out["chain_8192x8192x3"] = measure_chain(torch, pg, dev, stream, d_img, d_out)
    out["conv_jacobi_8192x8192x3"] = measure_conv_jacobi(torch, pg, dev, stream, d_img, d_out)
    out["passes_f32_interleaved_8192x8192x3"] = measure_interleaved(torch, pg, dev, stream, d_img, ks, g)
    # the chain runs overwrote d_out[0]: the 3x3 result again for the precision check
    pg.pencil_conv2d_ex(C, H, W, d_img, 3, 3, d_ks[0], d_out[0], pg.PENCIL_F32, 0, sraw)
    out["batched_512"], keep["batch"] = measure_batched(torch, pg, dev, stream)
    serving, keep["served"] = measure_serving(torch, pg, dev, serve_seconds)
    out["serving_saturation_40000_req_s"] = serving.pop("saturation_40000_req_s")
    out["serving_2000_req_s"] = serving["2000_req_s"]
    torch.cuda.synchronize(dev)
    return out, keep


SERVE_SAMPLE_EVERY = 97  # every 97th request of the 2000 req/s replay is kept and checked


def _serve_brief(st):
    d = st.summary()
    return {k: d[k] for k in ("requests", "rejected", "p50_ms", "p99_ms", "max_ms", "gpx_s", "req_s", "mean_wave",
                              "batched_waves", "peak_inflight", "peak_arena_mib")}


def measure_serving(torch, pg, dev, seconds):
    """Open-loop Poisson replay, FP16 storage, sides log-uniform [128, 4096],
    odd filter sides 3..15, 8 GiB arena budget: continuous batching against
    one launch per request, at 2000 req/s (latency) and at a saturating rate
    (throughput).  Returns (results, kept): the served results of every 97th
    request of the 2000 req/s replay, with what the CPU leg needs to check
    them (their pinned buffers are allocated before the replay starts)."""
    from paper_1302_5586_gb300 import serve, tune

    res, kept = {}, None
    seed = synth.SEEDS["serve"]
    for label, rate, dur in (("2000_req_s", 2000.0, seconds), ("saturation_40000_req_s", 40000.0, 0.5)):
        tr = serve.make_trace(seed, rate, dur)
        pool = serve.host_pool(tr, pg.PENCIL_F16, seed + 1)
        bank = torch.from_numpy(tr.filters).to(dev)
        srv = serve.Server(dtype=pg.PENCIL_F16, budget_bytes=8 << 30, streams=4, max_wave=64, max_inflight=256)
        sample = range(0, len(tr.requests), SERVE_SAMPLE_EVERY) if label == "2000_req_s" else ()
        try:
            srv.set_variants(tune.cached_variants(pg.PENCIL_F16))
            served, outs = srv.run(tr, pool, bank, mode="served", keep_ids=sample)
            plain, _ = srv.run(tr, pool, bank, mode="plain")
        finally:
            srv.close()
        res[label] = {"offered_req_s": rate, "seconds": dur,
                      "offered_gpx_s": round(sum(r.h * r.w for r in tr.requests) / dur / 1e9, 3),
                      "served": _serve_brief(served), "plain": _serve_brief(plain)}
        if sample:
            kept = {"trace": tr, "pool": pool, "outputs": {i: outs[i] for i in sample if outs[i] is not None}}
        del bank
    return res, kept


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


def measure_conv_jacobi(torch, pg, dev, stream, d_img, d_out):
    """A filter pass then 10 Jacobi smoothing sweeps on every channel of the
    3 x 8192^2 FP32 image: the fused kernel (the filtered window goes straight
    into the register sweeps) against a conv2d pass followed by the library's
    tiled sweeps (same bits).  HBM basis: 8 B per pixel fused."""
    hbm = measured_peaks().get("hbm_gbs") or 6800.0
    sraw = stream.cuda_stream
    n = 10
    wsb = pg.pencil_jacobi2d_workspace_size(H, W)
    ws = torch.empty(wsb, dtype=torch.uint8, device=dev)
    res = {}
    for K in (3, 5, 7):
        k = torch.from_numpy(synth.gaussian_2d_f32(K // 2, 1.0)).to(dev)
        ms_f = _time_stream(torch, stream, lambda: pg.pencil_conv2d_jacobi(C, H, W, d_img, K, K, k, n, d_out[0],
                                                                           pg.PENCIL_CHAIN_FUSED, sraw), 10)

        def two():
            pg.pencil_conv2d_ex(C, H, W, d_img, K, K, k, d_out[0], pg.PENCIL_F32, 0, sraw)
            for ch in range(C):
                pg.pencil_jacobi2d_ex(H, W, d_out[0][ch], n, 0, None, ws, wsb, 0, sraw)
        ms_t = _time_stream(torch, stream, two, 10)
        res[f"{K}x{K}+{n}sweeps"] = {"fused_ms": round(ms_f, 4), "two_pass_ms": round(ms_t, 4),
                                     "speedup": round(ms_t / ms_f, 3),
                                     "fused_gpx_s": round(PX_PER_PASS / ms_f / 1e6, 1),
                                     "fused_hbm_frac": round(8 * PX_PER_PASS / (ms_f * 1e-3) / 1e9 / hbm, 4)}
    del ws
    return res


def measure_interleaved(torch, pg, dev, stream, d_img, ks, g):
    """The step's four passes on the same image stored interleaved
    [8192][8192][3] (PENCIL_LAYOUT_HWC): per-pass times next to the planar
    ones (same pixels, same bits per channel)."""
    hbm = measured_peaks().get("hbm_gbs") or 6800.0
    sraw = stream.cuda_stream
    x = d_img.permute(1, 2, 0).contiguous()
    y = torch.empty_like(x)
    d_ks = [torch.from_numpy(k).to(dev) for k in ks]
    d_g = torch.from_numpy(g).to(dev)
    res = {}
    for K, dk in zip(DIRECT_K, d_ks):
        ms = _time_stream(torch, stream, lambda: pg.pencil_conv2d_ex(C, H, W, x, K, K, dk, y, pg.PENCIL_F32,
                                                                     pg.PENCIL_LAYOUT_HWC, sraw), 10)
        res[f"{K}x{K}"] = _pass_entry(ms, 8, 2 * K * K, hbm)
    ms = _time_stream(torch, stream, lambda: pg.pencil_conv2d_sep_ex(C, H, W, x, 15, d_g, 15, d_g, y, pg.PENCIL_F32,
                                                                     pg.PENCIL_LAYOUT_HWC, sraw), 10)
    res["gauss15-sep"] = _pass_entry(ms, 8, 0, hbm)
    del x, y
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
    xh = synth.image_f32(synth.SEEDS["conv512"], 1, n, n)
    kh = synth.filter_f32(synth.SEEDS["conv512"] + 1, K, K)
    x = torch.from_numpy(xh).to(dev)
    k = torch.from_numpy(kh).to(dev)
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
    return ({"device_us_per_launch": round(best, 2), "gpx_s": round(px / best / 1e3, 2),
             "l2_resident_gb_s": round(8 * px / best / 1e3, 1), "graph_replay_us": graph_us if not isinstance(
                 graph_us, float) else round(graph_us, 2), "stream_launch_us": round(us, 2),
             "plain_call_us": round(call_us, 2),
             "note": "fits in L2: launch-latency bound; GB/s is L2-resident, not HBM"},
            (xh, kh, y))


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
    keep = {}
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
            # the batched results of every 8th image, for the precision check
            keep[name] = [(i, items[i][0].cpu().numpy(), items[i][2].cpu().numpy().reshape(items[i][5], items[i][5]),
                           items[i][1].cpu().numpy()) for i in range(0, 512, 8)]

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
    return res, keep


def measure_e2e(torch, pg, img, ks, g, steps, down_streams=1):
    """The step end to end from pinned HOST memory through the public
    stream-ordered calls: every step uploads its 3 x 8192^2 input image once
    (768 MiB), runs the four passes (pencil_conv2d_ex x3, pencil_conv2d_sep_ex)
    and reads each pass's output back (4 x 768 MiB) while the next pass
    computes.  Three streams (upload, compute, download) with events; device
    buffers are double-buffered across steps so the next step's upload
    overlaps this step's downloads.  Timed by wall clock around `steps` steps
    after one warm-up step, ending with a full synchronisation."""
    dev = torch.device("cuda", torch.cuda.current_device())
    h_in = torch.from_numpy(img).pin_memory()
    h_out = [torch.empty_like(h_in).pin_memory() for _ in range(PASSES)]
    d_in = [torch.empty_like(h_in, device=dev) for _ in range(2)]
    d_out = [[torch.empty_like(h_in, device=dev) for _ in range(PASSES)] for _ in range(2)]
    d_ks = [torch.from_numpy(k).to(dev) for k in ks]
    d_g = torch.from_numpy(g).to(dev)
    up, comp = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    downs = [torch.cuda.Stream(dev) for _ in range(down_streams)]  # pass n downloads on downs[n % len]
    in_free = [torch.cuda.Event() for _ in range(2)]            # compute done reading d_in[b]
    out_free = [[torch.cuda.Event() for _ in range(PASSES)] for _ in range(2)]  # download of d_out[b][n] done
    for b in range(2):
        in_free[b].record(comp)
        for n in range(PASSES):
            out_free[b][n].record(downs[n % len(downs)])

    def step(i):
        bb = i & 1
        up.wait_event(in_free[bb])
        with torch.cuda.stream(up):
            d_in[bb].copy_(h_in, non_blocking=True)
        loaded = torch.cuda.Event()
        loaded.record(up)
        comp.wait_event(loaded)
        for n in range(PASSES):
            comp.wait_event(out_free[bb][n])
            if n < len(DIRECT_K):
                pg.pencil_conv2d_ex(C, H, W, d_in[bb], DIRECT_K[n], DIRECT_K[n], d_ks[n], d_out[bb][n],
                                    pg.PENCIL_F32, 0, comp.cuda_stream)
            else:
                pg.pencil_conv2d_sep_ex(C, H, W, d_in[bb], 15, d_g, 15, d_g, d_out[bb][n], pg.PENCIL_F32, 0,
                                        comp.cuda_stream)
            done = torch.cuda.Event()
            done.record(comp)
            down = downs[n % len(downs)]
            down.wait_event(done)
            with torch.cuda.stream(down):
                h_out[n].copy_(d_out[bb][n], non_blocking=True)
            out_free[bb][n].record(down)
        in_free[bb].record(comp)

    step(0)
    torch.cuda.synchronize(dev)
    t = time.perf_counter()
    for i in range(steps):
        step(i + 1)
    torch.cuda.synchronize(dev)
    dt = (time.perf_counter() - t) / steps
    nbytes = 4 * C * H * W
    del d_in, d_out
    return {"value": round(PX_PER_STEP / dt / 1e9, 3), "unit": "Gpixel/s",
            "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": PASSES * nbytes,
            "steps": steps, "ms_per_step": round(dt * 1e3, 2),
            "api": "pencil_conv2d_ex / pencil_conv2d_sep_ex from pinned host buffers: one upload of the image "
                   "and four output downloads per step, overlapped with compute on three streams"}


# ------------------------------------------------------------- CPU oracle
def _oracle_band(oracle, img, ks, g, rows, r0, keep=False):
    """Oracle over rows [r0, r0+rows) of all channels for every pass of the
    step: each pass reads its halo rows too (cut at the image edges, where the
    sub-image's clamp is the image's), so the band rows are exact.  Returns the
    seconds taken and, with keep, each pass's band rows."""
    outs = []
    t = time.perf_counter()
    for K, k in zip(DIRECT_K, ks):
        a = K // 2
        lo, hi = max(0, r0 - a), min(H, r0 + rows + a)
        o, _ = oracle.conv2d(img[:, lo:hi, :], k, want_bound=False)
        if keep:
            outs.append(o[:, r0 - lo:r0 - lo + rows, :])
    lo, hi = max(0, r0 - GAUSS_R), min(H, r0 + rows + GAUSS_R)
    o, _ = oracle.conv2d_sep(img[:, lo:hi, :], g, g, want_bound=False)
    if keep:
        outs.append(o[:, r0 - lo:r0 - lo + rows, :])
    dt = time.perf_counter() - t
    return (dt, outs) if keep else dt


def _ratio_max(got, want, bound):
    """max |got - want| / bound over the elements (0 where both are 0)."""
    got = np.asarray(got, dtype=np.float64)
    err = np.abs(got - want)
    return float(np.max(np.where(err == 0, 0.0, err / np.maximum(bound, 1e-300)))) if err.size else 0.0


def _edge_and_random_points(seed, c, h, w, n):
    """n random (ch, i, j) points plus every pixel of the outer rows and
    columns of channel 0 (where the clamp acts)."""
    r = np.random.default_rng(seed)
    pts = [np.stack([r.integers(0, c, n), r.integers(0, h, n), r.integers(0, w, n)], axis=1)]
    for i in (0, h - 1):
        pts.append(np.stack([np.zeros(w, np.int64), np.full(w, i), np.arange(w)], axis=1))
    for j in (0, w - 1):
        pts.append(np.stack([np.zeros(h, np.int64), np.arange(h), np.full(h, j)], axis=1))
    return np.concatenate(pts).astype(np.int64)


def _gather(t, pts):
    import torch
    p = torch.from_numpy(pts).to(t.device)
    return t[p[:, 0], p[:, 1], p[:, 2]].double().cpu().numpy()


def cpu_baseline(torch, img, ks, g, d_out=None, keep=None, budget_s=15.0):
    """The CPU leg: the FP64 oracle as it stands, on all host cores.

    (1) Timed: all four passes over a band of rows of the benchmark image,
        sized to about budget_s seconds -- the cpu_baseline value.
    (2) Each result's error: that band's oracle rows and the oracle at every
        edge pixel of channel 0 plus 4096 random pixels, against the GPU
        outputs of this run; then the oracle on bounded samples of the other
        workloads (a band of the binary16 image, the whole Jacobi grid after
        100 sweeps, every 8th batched image, every 97th served request, the
        512 x 512 case), each against the GPU's result.
    Returns (cpu_baseline, precision)."""
    import oracle

    probe = 32
    _oracle_band(oracle, img, ks, g, 8, 0)  # start the thread pool
    t_probe = _oracle_band(oracle, img, ks, g, probe, H // 2)
    rows = int(max(probe, min(H, probe * budget_s / max(t_probe, 1e-6))))
    r0 = H // 2 - rows // 2 if rows < H else 0
    got_band = _oracle_band(oracle, img, ks, g, rows, r0, keep=d_out is not None)
    dt, bands = got_band if d_out is not None else (got_band, None)
    px = rows * W * C * PASSES
    cpu = {"value": round(px / dt / 1e9, 6), "unit": "Gpixel/s", "cores": oracle.num_threads(), "kind": "oracle",
           "sample": f"FP64 oracle, all 4 passes over rows {rows} of 8192 (x3 channels) of the same image, "
                     f"{dt:.1f} s"}
    if d_out is None:
        return cpu, None
    keep = keep or {}
    t0 = time.perf_counter()
    # every pixel and weight of the benchmark is >= 0, so sum |k||x| is the value itself
    assert img.min() >= 0 and all(k.min() >= 0 for k in ks) and g.min() >= 0
    names = [f"{K}x{K}" for K in DIRECT_K] + ["gauss15-sep"]
    pts = _edge_and_random_points(5, C, H, W, 4096)
    f32 = {}
    for n, name in enumerate(names):
        got = d_out[n][:, r0:r0 + rows, :].cpu().numpy()
        r = max(_ratio_max(got[:, i:i + 512], bands[n][:, i:i + 512], bands[n][:, i:i + 512])
                for i in range(0, rows, 512))
        if n < len(DIRECT_K):
            want, bound = oracle.conv2d_points(img, ks[n], pts)
        else:
            want, bound = oracle.conv2d_sep_points(img, g, g, pts)
        f32[name] = max(r, _ratio_max(_gather(d_out[n], pts), want, bound))
    prec = {"tol": {"f32": TOL_F32, "f16": TOL_F16, "jacobi_abs": TOL_JACOBI},
            "conv_f32_err_over_bound": {k: float(f"{v:.3g}") for k, v in f32.items()}}
    worst = max(f32.values()) / TOL_F32
    if keep.get("f16"):
        d16, o16s = keep["f16"]
        x16 = d16.cpu().numpy()
        rows16 = min(256, H // 2)
        r16 = H // 2 - rows16 // 2
        f16 = {}
        for n, (name, o16) in enumerate(zip(names, o16s)):
            a = GAUSS_R if n == len(DIRECT_K) else DIRECT_K[n] // 2
            sub = x16[:, r16 - a:r16 + rows16 + a, :]
            if n < len(DIRECT_K):
                want, bound = oracle.conv2d(sub, ks[n])
                pw, pb = oracle.conv2d_points(x16, ks[n], pts)
            else:
                want, bound = oracle.conv2d_sep(sub, g, g)
                pw, pb = oracle.conv2d_sep_points(x16, g, g, pts)
            got = o16[:, r16:r16 + rows16, :].cpu().numpy()
            f16[name] = max(_ratio_max(got, want[:, a:a + rows16], bound[:, a:a + rows16]),
                            _ratio_max(_gather(o16, pts), pw, pb))
        for K, o16t in (keep.get("f16_tensor") or {}).items():  # the tensor-core passes, same bound
            kk = ks[DIRECT_K.index(K)]
            a = K // 2
            sub = x16[:, r16 - a:r16 + rows16 + a, :]
            want, bound = oracle.conv2d(sub, kk)
            pw, pb = oracle.conv2d_points(x16, kk, pts)
            got = o16t[:, r16:r16 + rows16, :].cpu().numpy()
            f16[f"{K}x{K}-tensor"] = max(_ratio_max(got, want[:, a:a + rows16], bound[:, a:a + rows16]),
                                         _ratio_max(_gather(o16t, pts), pw, pb))
        prec["conv_f16_err_over_bound"] = {k: float(f"{v:.3g}") for k, v in f16.items()}
        worst = max(worst, max(f16.values()) / TOL_F16)
    if keep.get("plain512"):
        xh, kh, y = keep["plain512"]
        want, bound = oracle.conv2d(xh, kh)
        r = _ratio_max(y.cpu().numpy().reshape(want.shape), want, bound)
        prec["plain_512x512_5x5_err_over_bound"] = float(f"{r:.3g}")
        worst = max(worst, r / TOL_F32)
    if keep.get("batch"):
        for name, tol in (("f32", TOL_F32), ("f16", TOL_F16)):
            r = 0.0
            for i, x, k, y in keep["batch"].get(name, []):
                hh, ww = x.shape[-2:]
                x, y = x.reshape(hh, ww), y.reshape(hh, ww)
                p = _edge_and_random_points(i, 1, hh, ww, 1024)
                want, bound = oracle.conv2d_points(x, k, p)
                r = max(r, _ratio_max(y[p[:, 1], p[:, 2]], want, bound))
            prec[f"batched_{name}_err_over_bound"] = float(f"{r:.3g}")
            worst = max(worst, r / tol)
    if keep.get("served"):
        sv = keep["served"]
        tr, pool, r = sv["trace"], sv["pool"], 0.0
        for rid, y in sv["outputs"].items():
            q = tr.requests[rid]
            x = pool[q.src:q.src + q.h * q.w].numpy().reshape(1, q.h, q.w)
            k = tr.filters[q.filt:q.filt + q.ks * q.ks].reshape(q.ks, q.ks)
            p = _edge_and_random_points(rid, 1, q.h, q.w, 256)
            want, bound = oracle.conv2d_points(x, k, p)
            r = max(r, _ratio_max(y.numpy()[p[:, 1], p[:, 2]], want, bound))
        prec["served_f16_err_over_bound"] = float(f"{r:.3g}")
        prec["served_checked"] = len(sv["outputs"])
        worst = max(worst, r / TOL_F16)
    if keep.get("jacobi"):
        u0h, u, res = keep["jacobi"]
        u_ref, res_ref = oracle.jacobi2d(u0h, 100, 10)
        du = float(np.max(np.abs(u.cpu().numpy().astype(np.float64) - u_ref)))
        rr = float(np.max(np.abs(res.cpu().numpy() - res_ref) / res_ref))
        prec["jacobi_max_abs_du"] = float(f"{du:.3g}")
        prec["jacobi_residual_rel_err"] = float(f"{rr:.3g}")
        worst = max(worst, du / TOL_JACOBI)
    prec["worst_err_over_tol"] = float(f"{worst:.3g}")
    prec["oracle_check_s"] = round(time.perf_counter() - t0, 1)
    return cpu, prec


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
            "config": config(),
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
        unaligned = name.endswith("u")  # rows of 4095 elements: not 16-byte aligned
        name = name.rstrip("u")
        tensor = name.endswith("t")  # binary16 on the tensor cores
        f16 = name.endswith("h") or tensor
        K = int(name[4:].rstrip("ht").split("-")[0])
        c, h, w = 2, 4096, 4095 if unaligned else 4096
        img = torch.from_numpy(synth.image_f32(1, c, h, w)).to(dev)
        if f16:  # binary16 storage: twice the pixels, so the image is still larger than L2
            c = 4
            img = torch.from_numpy(synth.to_f16(synth.image_f32(1, c, h, w))).to(dev)
        k = torch.from_numpy(synth.filter_f32(2, K, K)).to(dev)
        out = torch.empty_like(img)
        for _ in range(reps):
            pg.pencil_conv2d_ex(c, h, w, img, K, K, k, out, pg.PENCIL_F16 if f16 else pg.PENCIL_F32,
                                pg.PENCIL_CONV_TENSOR if tensor else 0)
    elif name in ("sep15", "sep15h"):
        f16 = name.endswith("h")
        c, h, w = (4 if f16 else 2), 4096, 4096  # binary16: twice the pixels, still larger than L2
        img = torch.from_numpy(synth.image_f32(1, c, h, w)).to(dev)
        if f16:
            img = img.half()
        g = torch.from_numpy(synth.gaussian_taps_f32(7, 3.0)).to(dev)
        out = torch.empty_like(img)
        for _ in range(reps):
            pg.pencil_conv2d_sep_ex(c, h, w, img, 15, g, 15, g, out, pg.PENCIL_F16 if f16 else pg.PENCIL_F32)
    elif name.startswith("cj"):
        K = int(name[2:])
        c, h, w = 2, 4096, 4096
        img = torch.from_numpy(synth.image_f32(1, c, h, w)).to(dev)
        k = torch.from_numpy(synth.filter_f32(2, K, K)).to(dev)
        out = torch.empty_like(img)
        for _ in range(reps):
            pg.pencil_conv2d_jacobi(c, h, w, img, K, K, k, 10, out, pg.PENCIL_CHAIN_FUSED)
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
                    help="profile one kernel on a reduced workload: conv3, conv7, conv15, conv3h (binary16), conv15t "
                         "(binary16 on the tensor cores), conv15u (any conv case with rows of 4095 elements, not "
                         "16-byte aligned), sep15, sep15h "
                         "(binary16), batch, jacobi, jacobi-tN (N sweeps per pass), op2-ordered, op2-atomic, "
                         "chain3, chain5, chain7, cj3, cj5, cj7 (filter then 10 Jacobi sweeps, fused)")
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
