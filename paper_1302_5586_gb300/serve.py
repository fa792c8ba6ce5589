"""Continuous-batching conv2d serving on one GPU.

Requests (image size, filter side, input window, filter) arrive open-loop on
a Poisson trace.  The scheduler loop:

* admits arrived requests in arrival order while a slot is free
  (`max_inflight`) and the arena (one device buffer of `budget_bytes`, offsets
  kept by the native pencil_arena) has room for the request's input and
  output; a request that does not fit waits until completions free memory,
  and one that could not fit even an empty arena is rejected on arrival;
* packs requests admitted in one pass into a wave and issues it on one of
  `streams` CUDA streams -- an idle stream if there is one, the pending
  requests spread evenly over the idle streams (so at low load a request
  runs alone, with the latency of a plain launch), else the next stream in
  turn with up to `max_wave` requests (batching grows with the queue): host-to-device copies of the inputs (from
  pinned host memory into the arena), ONE batched persistent conv2d launch
  (pencil_batch_run, graph replay; one plan per stream) -- or, for a wave of
  a single request, its one standalone launch, which costs the host less
  than building a batch table and gives the same bits -- device-to-host
  copies of the outputs, and an event;
* polls the events of the waves in flight; a finished wave's requests are
  timestamped (latency = completion - arrival) and their arena blocks freed.

Waves on different streams overlap on the device (copies of one wave with the
kernel of another), and requests that arrive while others run join the next
wave -- continuous batching.  `mode="plain"` replays the same trace with one
standalone pencil_conv2d_ex launch per request (same copies, same admission)
for comparison.  Every result is the same bits in either mode and alone.

The paper has no serving layer; this is the serving pattern built on the
batched kernel (the tuned launch of the independent image loop, Sec. 2.2.3).
"""
from __future__ import annotations

import collections
import dataclasses
import time

import numpy as np

import synth

from . import _binding as b


@dataclasses.dataclass
class Request:
    rid: int
    arrival: float   # seconds after the start of the replay
    h: int
    w: int
    ks: int
    src: int         # element offset of the input window in the host pool
    filt: int        # element offset of the filter in the filter bank


@dataclasses.dataclass
class Trace:
    requests: list
    pool_elems: int
    filters: np.ndarray  # all filters, concatenated FP32


def make_trace(seed: int, rate: float, duration: float, lo: int = 128, hi: int = 4096,
               klo: int = 3, khi: int = 15, pool_elems: int = 1 << 25) -> Trace:
    """Poisson arrivals at `rate` per second for `duration` seconds; sides
    log-uniform in [lo, hi]; odd filter sides uniform in [klo, khi]; inputs
    are windows of a seeded noise pool at seed-derived offsets."""
    t = synth.poisson_arrivals(seed, rate, duration)
    n = len(t)
    h = synth.loguniform_sides(seed ^ 0xA1, n, lo, hi)
    w = synth.loguniform_sides(seed ^ 0xA2, n, lo, hi)
    ks = synth.odd_ksizes(seed ^ 0xA3, n, klo, khi)
    pool_elems = max(pool_elems, int(np.max(h * w)) if n else 1)
    z = synth.splitmix64(seed ^ 0xA4, n) if n else np.zeros(0, np.uint64)
    span = (pool_elems - h * w + 1).astype(np.uint64)
    src = (z % np.maximum(span, 1)).astype(np.int64)
    filts, reqs, off = [], [], 0
    for i in range(n):
        k = synth.filter_f32(seed * 7919 + i, int(ks[i]), int(ks[i])).ravel()
        filts.append(k)
        reqs.append(Request(i, float(t[i]), int(h[i]), int(w[i]), int(ks[i]), int(src[i]), off))
        off += k.size
    bank = np.concatenate(filts) if filts else np.zeros(1, np.float32)
    return Trace(reqs, pool_elems, bank)


ARENA_ALIGN = 256  # bytes; the arena rounds blocks up and its capacity down to this


def fits_alone(h: int, w: int, esz: int, budget: int, align: int = ARENA_ALIGN) -> bool:
    """Whether a request's input and output blocks fit an empty arena of
    `budget` bytes (each block rounded up to `align`, the capacity rounded
    down); a request that does not is rejected on arrival instead of waiting
    for memory that can never be freed."""
    need = -(-h * w * esz // align) * align
    return 2 * need <= budget // align * align


class Admission:
    """The serving loop's host-side admission (no CUDA calls).

    Arrived requests queue in arrival order.  `wave` takes requests from the
    head of the queue while fewer than `max_inflight` are in flight and the
    arena takes the head's input block and then its output block; when either
    allocation fails the head waits (the input block is given back), so a
    request is never reordered past an earlier one.  A request that could
    never fit even an empty arena is rejected on arrival; a cancelled request
    and one whose deadline (seconds after its arrival) has passed are dropped
    when they reach the head, before any memory is taken.  `release` gives a
    finished request's blocks back.  `alloc(nbytes) -> offset | None` and
    `free(offset)` are the arena's calls (a test may pass failing ones)."""

    def __init__(self, alloc, free, budget: int, esz: int, max_inflight: int, deadline_s: float | None = None):
        self.alloc, self.free = alloc, free
        self.budget, self.esz, self.max_inflight = budget, esz, max_inflight
        self.deadline_s = deadline_s
        self.pending = collections.deque()
        self.cancelled_ids = set()
        self.inflight = 0
        self.rejected = self.cancelled = self.expired = 0

    @property
    def dropped(self) -> int:
        """Requests that will never run: rejected, cancelled or expired."""
        return self.rejected + self.cancelled + self.expired

    def arrive(self, r) -> bool:
        """Queue an arrived request; False if it is rejected or was cancelled."""
        if r.rid in self.cancelled_ids:
            self.cancelled_ids.discard(r.rid)
            self.cancelled += 1
            return False
        if not fits_alone(r.h, r.w, self.esz, self.budget):
            self.rejected += 1
            return False
        self.pending.append(r)
        return True

    def cancel(self, rid: int) -> None:
        """Cancel a request that has not been admitted (no effect afterwards)."""
        self.cancelled_ids.add(rid)

    def wave(self, limit: int, now: float) -> list:
        """Admit up to `limit` requests at time `now`: [(request, in_offset, out_offset)]."""
        out = []
        while self.pending and len(out) < limit and self.inflight + len(out) < self.max_inflight:
            r = self.pending[0]
            if r.rid in self.cancelled_ids:
                self.pending.popleft()
                self.cancelled_ids.discard(r.rid)
                self.cancelled += 1
                continue
            if self.deadline_s is not None and now - r.arrival > self.deadline_s:
                self.pending.popleft()
                self.expired += 1
                continue
            nb = r.h * r.w * self.esz
            oi = self.alloc(nb)
            if oi is None:
                break
            oo = self.alloc(nb)
            if oo is None:
                self.free(oi)
                break
            self.pending.popleft()
            out.append((r, oi, oo))
        self.inflight += len(out)
        return out

    def release(self, items) -> None:
        """A wave's requests finished: give their blocks back."""
        for _, oi, oo in items:
            self.free(oi)
            self.free(oo)
        self.inflight -= len(items)


def wave_limit(mode: str, pending: int, idle_streams: int, max_wave: int) -> int:
    """Requests the next wave may take.  Plain mode: one.  Served: with idle
    streams, the pending requests spread evenly over them (a lone request
    goes alone); with every stream busy, up to max_wave."""
    if mode != "served":
        return 1
    if idle_streams > 0:
        return max(1, min(max_wave, -(-pending // idle_streams)))
    return max_wave


@dataclasses.dataclass
class Stats:
    mode: str
    requests: int
    rejected: int
    pixels: int
    wall_s: float
    latency_ms: np.ndarray
    waves: int
    peak_inflight: int
    peak_arena_bytes: int
    cancelled: int = 0
    expired: int = 0
    batched_waves: int = 0

    def summary(self) -> dict:
        lat = self.latency_ms
        ok = lat[np.isfinite(lat)]
        return {
            "mode": self.mode, "requests": self.requests, "rejected": self.rejected,
            "cancelled": self.cancelled, "expired": self.expired,
            "p50_ms": round(float(np.percentile(ok, 50)), 3) if ok.size else None,
            "p99_ms": round(float(np.percentile(ok, 99)), 3) if ok.size else None,
            "mean_ms": round(float(ok.mean()), 3) if ok.size else None,
            "max_ms": round(float(ok.max()), 3) if ok.size else None,
            "gpx_s": round(self.pixels / self.wall_s / 1e9, 3) if self.wall_s > 0 else None,
            "req_s": round(ok.size / self.wall_s, 1) if self.wall_s > 0 else None,
            "waves": self.waves, "batched_waves": self.batched_waves,
            "mean_wave": round(ok.size / max(self.waves, 1), 2),
            "peak_inflight": self.peak_inflight, "peak_arena_mib": round(self.peak_arena_bytes / 2**20, 1),
        }


class Server:
    """One GPU, `streams` CUDA streams, one batch plan per stream, one arena."""

    def __init__(self, dtype: int = b.PENCIL_F16, budget_bytes: int = 8 << 30, streams: int = 4,
                 max_wave: int = 64, max_inflight: int = 256, max_tiles: int = 1 << 20, device=None):
        import torch

        self.torch = torch
        self.dev = device or torch.device("cuda", torch.cuda.current_device())
        self.dtype = dtype
        self.tdtype = torch.float16 if dtype == b.PENCIL_F16 else torch.float32
        self.esz = 2 if dtype == b.PENCIL_F16 else 4
        self.budget = budget_bytes
        self.pool = torch.empty(budget_bytes, dtype=torch.uint8, device=self.dev)
        self.arena = b.pencil_arena_create(budget_bytes, ARENA_ALIGN)
        self.streams = [torch.cuda.Stream(self.dev) for _ in range(streams)]
        self.plans = [b.pencil_batch_create(dtype, max_wave, max_tiles) for _ in range(streams)]
        self.max_wave = max_wave
        self.max_inflight = max_inflight
        self.warm_up()

    def warm_up(self):
        """Before serving: load every filter side's kernels (batched and
        standalone) and build each plan's launch graph for every set of filter
        sides a wave can hold (255 sets), on tiny images, so no request waits
        behind a one-time kernel load or graph instantiation on the serving
        thread."""
        torch = self.torch
        imgs = torch.zeros((8, 16, 16), dtype=self.tdtype, device=self.dev)
        outs = torch.empty_like(imgs)
        k = torch.zeros(15 * 15, dtype=torch.float32, device=self.dev)
        for s, plan in zip(self.streams, self.plans):
            for ks in range(1, 16, 2):
                b.pencil_conv2d_ex(1, 16, 16, imgs[0], ks, ks, k, outs[0], self.dtype, 0, s.cuda_stream)
            for mask in range(1, 256):
                sides = [2 * i + 1 for i in range(8) if mask >> i & 1]
                b.pencil_batch_run(plan, b.make_images([(imgs[j], outs[j], k, 16, 16, ks)
                                                        for j, ks in enumerate(sides)]), s.cuda_stream)
        torch.cuda.synchronize(self.dev)

    def close(self):
        self.torch.cuda.synchronize(self.dev)
        for p in self.plans:
            b.pencil_batch_destroy(p)
        self.plans = []
        if self.arena:
            b.pencil_arena_destroy(self.arena)
            self.arena = None

    def set_variants(self, variants: dict):
        """Tile variant per filter side (a change drops the plans' captured
        graphs, so the warm-up runs again before any request is served)."""
        for p in self.plans:
            for ks, v in variants.items():
                b.pencil_batch_set_variant(p, int(ks), int(v))
        self.warm_up()

    def _view(self, off: int, n: int):
        return self.pool[off:off + n * self.esz].view(self.tdtype)

    def run(self, trace: Trace, host_pool, filters_dev, mode: str = "served", keep_outputs: bool = False,
            sink_bytes: int = 1 << 29, deadline_ms: float | None = None, cancel=(), keep_ids=()) -> tuple:
        """Replay `trace` open-loop.  host_pool: pinned host tensor of the
        storage dtype (trace.pool_elems elements); filters_dev: device FP32
        tensor holding trace.filters.  Requests still queued `deadline_ms`
        after their arrival, and those whose ids are in `cancel`, are dropped
        unrun (latency NaN).  keep_outputs keeps every result; keep_ids keeps
        only those requests' results, in pinned buffers allocated before the
        replay starts (so checking a sample costs the replay no allocation).
        Returns (Stats, outputs: a list with None for results not kept, or
        None when nothing is kept)."""
        torch = self.torch
        reqs = trace.requests
        n = len(reqs)
        lat = np.full(n, np.nan)
        outputs = [None] * n if (keep_outputs or keep_ids) else None
        for rid in keep_ids if not keep_outputs else ():
            r = reqs[int(rid)]
            outputs[r.rid] = torch.empty(r.h * r.w, dtype=self.tdtype, pin_memory=True)
        largest = max((r.h * r.w for r in reqs), default=1)
        sink = None if keep_outputs else torch.empty(max(sink_bytes // self.esz, largest), dtype=self.tdtype,
                                                     pin_memory=True)
        sink_pos = 0
        adm = Admission(lambda nb: b.pencil_arena_alloc(self.arena, nb),
                        lambda off: b.pencil_arena_free(self.arena, off), self.budget, self.esz,
                        self.max_inflight, None if deadline_ms is None else deadline_ms * 1e-3)
        for rid in cancel:
            adm.cancel(int(rid))
        inflight = [collections.deque() for _ in self.streams]
        peak_inflight = 0
        peak_arena = 0
        waves = 0
        batched = 0
        done = 0
        pix = 0
        nxt = 0
        rr = 0
        kbase = filters_dev.data_ptr()
        t0 = time.perf_counter()
        last_done = t0
        while done + adm.dropped < n:
            now = time.perf_counter() - t0
            while nxt < n and reqs[nxt].arrival <= now:
                adm.arrive(reqs[nxt])
                nxt += 1
            progressed = False
            # completions
            for q in inflight:
                while q and q[0][0].query():
                    ev, items = q.popleft()
                    tdone = time.perf_counter()
                    for r, _, _ in items:
                        lat[r.rid] = (tdone - t0 - r.arrival) * 1e3
                        pix += r.h * r.w
                    adm.release(items)
                    done += len(items)
                    last_done = tdone
                    progressed = True
            # admission: arrival order, while a slot and arena memory are free
            dropped = adm.dropped
            # batch only under load: with idle streams the queue is spread over them
            # (a lone request runs alone, as fast as a plain launch); when every
            # stream is busy the whole queue, up to max_wave, forms the next wave
            idle = [i for i, fq in enumerate(inflight) if not fq]
            limit = wave_limit(mode, len(adm.pending), len(idle), self.max_wave)
            wave = adm.wave(limit, time.perf_counter() - t0)
            progressed = progressed or adm.dropped != dropped
            if wave:
                si = idle[0] if idle else rr % len(self.streams)
                if not idle:
                    rr += 1
                s = self.streams[si]
                plan = self.plans[si]
                q = inflight[si]
                with torch.cuda.stream(s):
                    for r, oi, _ in wave:
                        hw = r.h * r.w
                        self._view(oi, hw).copy_(host_pool[r.src:r.src + hw], non_blocking=True)
                    if mode == "served" and len(wave) > 1:
                        imgs = b.make_images([(self.pool.data_ptr() + oi, self.pool.data_ptr() + oo,
                                               kbase + 4 * r.filt, r.h, r.w, r.ks) for r, oi, oo in wave])
                        b.pencil_batch_run(plan, imgs, s.cuda_stream)
                        batched += 1
                    else:
                        for r, oi, oo in wave:
                            b.pencil_conv2d_ex(1, r.h, r.w, self.pool.data_ptr() + oi, r.ks, r.ks,
                                               kbase + 4 * r.filt, self.pool.data_ptr() + oo, self.dtype, 0,
                                               s.cuda_stream)
                    for r, _, oo in wave:
                        hw = r.h * r.w
                        src = self._view(oo, hw)
                        if keep_outputs:
                            outputs[r.rid] = torch.empty(hw, dtype=self.tdtype, pin_memory=True)
                            outputs[r.rid].copy_(src, non_blocking=True)
                        elif outputs is not None and outputs[r.rid] is not None:
                            outputs[r.rid].copy_(src, non_blocking=True)
                        else:
                            if sink_pos + hw > sink.numel():
                                sink_pos = 0
                            sink[sink_pos:sink_pos + hw].copy_(src, non_blocking=True)
                            sink_pos += hw
                    ev = torch.cuda.Event()
                    ev.record(s)
                q.append((ev, wave))
                waves += 1
                peak_inflight = max(peak_inflight, adm.inflight)
                peak_arena = max(peak_arena, self.budget - b.pencil_arena_free_bytes(self.arena))
                progressed = True
            if not progressed:
                # nothing to do until the next arrival or completion
                wait = (reqs[nxt].arrival - (time.perf_counter() - t0)) if nxt < n else 0.0
                if wait > 2e-4 and not any(inflight):
                    time.sleep(min(wait, 0.01) - 1e-4)
        torch.cuda.synchronize(self.dev)
        first = reqs[0].arrival if n else 0.0
        wall = (last_done - t0) - first
        st = Stats(mode, n, adm.rejected, pix, wall, lat, waves, peak_inflight, peak_arena, adm.cancelled,
                   adm.expired, batched)
        if outputs is not None:
            outputs = [o.view(r.h, r.w) if o is not None else None for o, r in zip(outputs, reqs)]
        return st, outputs


def host_pool(trace: Trace, dtype: int, seed: int):
    """The pinned host noise pool the trace's input windows come from."""
    import torch

    vals = synth.u01_f32(seed, trace.pool_elems)
    t = torch.from_numpy(vals)
    if dtype == b.PENCIL_F16:
        t = t.half()
    return t.pin_memory()


def percentile_summary(stats_list):
    return {s.mode: s.summary() for s in stats_list}


__all__ = ["Request", "Trace", "Stats", "Server", "Admission", "make_trace", "fits_alone", "host_pool",
           "percentile_summary"]
