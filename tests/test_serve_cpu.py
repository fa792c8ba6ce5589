"""The serving loop's admission on the CPU (no CUDA): arrival order without
overtaking, the slot and wave limits, reject-on-arrival, allocator failures
injected on the host (the request waits and no block leaks), cancellation
and deadlines, and a simulated replay with random completion order against
the native arena."""
import ctypes
import random
import sys

import numpy as np
import pytest
import torch

import paper_1302_5586_gb300 as pg
from paper_1302_5586_gb300 import build as pg_build
from paper_1302_5586_gb300.serve import ARENA_ALIGN, Admission, Request


@pytest.fixture(scope="module", autouse=True)
def built():
    pg_build.build()


@pytest.fixture
def arena():
    a = pg.pencil_arena_create(1 << 20, ARENA_ALIGN)
    yield a
    pg.pencil_arena_destroy(a)


def adm_for(a, max_inflight=64, deadline_s=None, alloc=None, esz=4):
    return Admission(alloc or (lambda nb: pg.pencil_arena_alloc(a, nb)), lambda off: pg.pencil_arena_free(a, off),
                     1 << 20, esz, max_inflight, deadline_s)


def req(rid, h, w, t=0.0):
    return Request(rid, t, h, w, 3, 0, 0)


def test_arrival_order_is_kept(arena):
    """A head that does not fit now blocks the smaller requests behind it."""
    ad = adm_for(arena)
    big = req(1, 256, 256)          # 2 x 256 KiB
    for r in (req(0, 256, 256), big, req(2, 8, 8)):
        assert ad.arrive(r)
    first = ad.wave(64, 0.0)
    assert [r.rid for r, _, _ in first] == [0, 1]   # the whole 1 MiB is taken: the small one waits
    ad.release(first)
    assert pg.pencil_arena_free_bytes(arena) == 1 << 20
    ad2 = adm_for(arena)
    for r in (req(0, 300, 300), req(1, 300, 300), req(2, 4, 4)):
        ad2.arrive(r)
    w1 = ad2.wave(64, 0.0)
    assert [r.rid for r, _, _ in w1] == [0]          # rid 1 does not fit beside rid 0 ...
    assert [r.rid for r in ad2.pending] == [1, 2]    # ... and rid 2 does not overtake it
    ad2.release(w1)
    assert [r.rid for r, _, _ in ad2.wave(64, 0.0)] == [1, 2]


def test_slot_and_wave_limits(arena):
    ad = adm_for(arena, max_inflight=5)
    for i in range(12):
        ad.arrive(req(i, 4, 4))
    w1 = ad.wave(3, 0.0)
    w2 = ad.wave(3, 0.0)
    assert (len(w1), len(w2), ad.inflight) == (3, 2, 5)
    assert ad.wave(3, 0.0) == []
    ad.release(w1)
    assert [r.rid for r, _, _ in ad.wave(8, 0.0)] == [5, 6, 7]


def test_never_fits_is_rejected_on_arrival(arena):
    ad = adm_for(arena)
    assert not ad.arrive(req(0, 512, 513))   # 2 x ~1 MiB > 1 MiB
    assert ad.arrive(req(1, 256, 256))       # exactly half the budget each
    assert ad.rejected == 1 and ad.dropped == 1 and len(ad.pending) == 1


def test_injected_allocator_failure_waits_and_leaks_nothing(arena):
    """The arena's alloc fails (as if out of memory) on chosen calls: the head
    waits, an input block taken before a failed output block is given back,
    and a later wave admits the same request."""
    calls = {"n": 0}
    fail = {2, 3}                              # the 2nd request's output, then its retry's input

    def alloc(nb):
        calls["n"] += 1
        return None if calls["n"] in fail else pg.pencil_arena_alloc(arena, nb)

    ad = adm_for(arena, alloc=alloc)
    for i in range(3):
        ad.arrive(req(i, 16, 16))
    w1 = ad.wave(64, 0.0)                        # call 1 ok (in 0), call 2 fails (out 0)
    assert w1 == [] and [r.rid for r in ad.pending] == [0, 1, 2]
    assert pg.pencil_arena_free_bytes(arena) == 1 << 20   # the input block was given back
    assert ad.wave(64, 0.0) == []              # call 3 fails (in 0)
    w3 = ad.wave(64, 0.0)
    assert [r.rid for r, _, _ in w3] == [0, 1, 2]
    ad.release(w3)
    assert pg.pencil_arena_free_bytes(arena) == 1 << 20 and ad.inflight == 0


def test_cancellation(arena):
    ad = adm_for(arena)
    ad.cancel(3)                                 # before it arrives
    assert not ad.arrive(req(3, 4, 4))
    for i in range(3):
        ad.arrive(req(i, 4, 4))
    ad.cancel(1)                                 # while queued
    w = ad.wave(64, 0.0)
    assert [r.rid for r, _, _ in w] == [0, 2] and ad.cancelled == 2
    ad.cancel(0)                                 # after admission: no effect on the running request
    ad.release(w)
    assert ad.cancelled == 2 and ad.dropped == 2
    assert pg.pencil_arena_free_bytes(arena) == 1 << 20


def test_deadline_drops_only_what_waited_too_long(arena):
    ad = adm_for(arena, deadline_s=0.010)
    ad.arrive(req(0, 4, 4, t=0.000))
    ad.arrive(req(1, 4, 4, t=0.005))
    ad.arrive(req(2, 4, 4, t=0.0125))
    w = ad.wave(64, 0.0149)                      # waited 14.9, 9.9 and 2.4 ms
    assert [r.rid for r, _, _ in w] == [1, 2] and ad.expired == 1
    ad.release(w)
    assert pg.pencil_arena_free_bytes(arena) == 1 << 20


@pytest.mark.parametrize("seed", range(4))
def test_simulated_replay_against_the_arena(seed, arena):
    """Random sizes, waves completed in random order: every request runs once
    or is dropped, admission follows arrival order, the arena and the slots
    never overflow, and the arena is whole at the end."""
    rng = random.Random(seed)
    n = 400
    reqs = [req(i, rng.randint(1, 300), rng.randint(1, 300), t=i * 1e-4) for i in range(n)]
    cancel = set(rng.sample(range(n), 20))
    ad = adm_for(arena, max_inflight=24, deadline_s=0.004)
    for rid in cancel:
        ad.cancel(rid)
    inflight, ran, admitted, nxt, now = [], set(), [], 0, 0.0
    while len(ran) + ad.dropped < n:
        now += 1e-4
        while nxt < n and reqs[nxt].arrival <= now:
            ad.arrive(reqs[nxt])
            nxt += 1
        if inflight and rng.random() < 0.3:
            items = inflight.pop(rng.randrange(len(inflight)))
            ad.release(items)
            ran.update(r.rid for r, _, _ in items)
        w = ad.wave(rng.randint(1, 8), now)
        assert ad.inflight <= 24
        assert 1 << 20 >= (1 << 20) - pg.pencil_arena_free_bytes(arena) >= 0
        admitted += [r.rid for r, _, _ in w]
        if w:
            inflight.append(w)
        assert now < 10.0, "replay did not finish"
    assert admitted == sorted(admitted) and len(set(admitted)) == len(admitted)
    assert not (set(admitted) & cancel)
    assert len(ran) + ad.rejected + ad.cancelled + ad.expired == n
    assert ad.cancelled == len(cancel) and ad.inflight == 0 and not inflight
    assert ad.expired > 0 and len(ran) > n // 4  # the memory limit made requests wait, some too long
    assert pg.pencil_arena_free_bytes(arena) == 1 << 20


# ---- the whole Server.run loop on the CPU, with a fake device layer ---------

class _Stream:
    def __init__(self, i):
        self.cuda_stream = 1000 + i


class _Event:
    """Completes on the second query, so waves stay in flight for a while."""

    def __init__(self):
        self.polls = 0

    def record(self, s):
        pass

    def query(self):
        self.polls += 1
        return self.polls > 1


def _fake_torch():
    import contextlib
    import itertools
    import types

    ids = itertools.count()
    cuda = types.SimpleNamespace(
        Stream=lambda dev=None: _Stream(next(ids)), stream=lambda s: contextlib.nullcontext(), Event=_Event,
        synchronize=lambda dev=None: None, current_device=lambda: 0)
    return types.SimpleNamespace(
        float16=torch.float16, float32=torch.float32, uint8=torch.uint8, cuda=cuda,
        device=lambda *a: "cpu",
        empty=lambda *shape, dtype=None, device=None, pin_memory=False: torch.empty(*shape, dtype=dtype),
        zeros=lambda shape, dtype=None, device=None: torch.zeros(shape, dtype=dtype),
        empty_like=torch.empty_like)


class _FakeLib:
    """The binding with the CUDA calls replaced: the "convolution" copies its
    input to its output, so every output must equal its request's window."""

    def __init__(self, real):
        self.real = real
        self.batch_runs = 0

    def __getattr__(self, name):  # constants, make_images and the host-only arena calls
        return getattr(self.real, name)

    def pencil_batch_create(self, dtype, max_images, max_tiles):
        self.esz = 2 if dtype == self.real.PENCIL_F16 else 4
        return 1

    def pencil_batch_destroy(self, plan):
        pass

    def pencil_batch_set_variant(self, plan, ks, v):
        pass

    def pencil_batch_run(self, plan, imgs, stream):
        self.batch_runs += 1
        for im in imgs:
            ctypes.memmove(im.out, im.in_, im.h * im.w * self.esz)

    def pencil_conv2d_ex(self, c, h, w, in_, kh, kw, k, out, dtype, flags=0, stream=None):
        ctypes.memmove(self.real._ptr(out), self.real._ptr(in_), c * h * w * self.esz)


@pytest.fixture
def fake_server(monkeypatch):
    from paper_1302_5586_gb300 import _binding, serve
    fake = _FakeLib(_binding)
    monkeypatch.setattr(serve, "b", fake)
    monkeypatch.setitem(sys.modules, "torch", _fake_torch())
    srv = serve.Server(dtype=pg.PENCIL_F32, budget_bytes=1 << 20, streams=3, max_wave=8, max_inflight=24)
    yield srv, fake
    srv.close()


@pytest.mark.parametrize("mode", ["served", "plain"])
def test_server_loop_on_a_fake_device(fake_server, mode):
    from paper_1302_5586_gb300 import serve
    srv, fake = fake_server
    tr = serve.make_trace(11, rate=20000.0, duration=0.01, lo=8, hi=200, klo=3, khi=7, pool_elems=1 << 18)
    n = len(tr.requests)
    for r in tr.requests:  # all at once: the fake device is instant, so only a burst is sure to batch
        r.arrival = 0.0
    pool = torch.arange(tr.pool_elems, dtype=torch.float32)
    cancel = {3, 17, n - 1}
    runs0 = fake.batch_runs  # the server's warm-up runs
    st, outs = srv.run(tr, pool, torch.zeros(1), mode=mode, keep_outputs=True, cancel=cancel)
    assert st.cancelled == len(cancel) and st.rejected == 0 and st.expired == 0
    for r in tr.requests:
        if r.rid in cancel:
            assert outs[r.rid] is None and np.isnan(st.latency_ms[r.rid])
        else:
            assert torch.equal(outs[r.rid], pool[r.src:r.src + r.h * r.w].view(r.h, r.w)), r
            assert np.isfinite(st.latency_ms[r.rid])
    assert pg.pencil_arena_free_bytes(srv.arena) == 1 << 20
    assert st.peak_inflight <= 24 and 0 < st.peak_arena_bytes <= 1 << 20
    assert (st.waves < n - len(cancel)) if mode == "served" else (st.waves == n - len(cancel))
    # waves of several requests take one batched launch, single requests their own launch
    assert fake.batch_runs - runs0 == st.batched_waves and (0 < st.batched_waves <= st.waves if mode == "served"
                                                    else st.batched_waves == 0)
    # without kept outputs the results go through the wrapping host sink; a
    # zero deadline drops every request that was not admitted the moment it arrived
    st2, none = srv.run(tr, pool, torch.zeros(1), mode=mode, sink_bytes=4096, deadline_ms=0.0)
    assert none is None and st2.expired > 0
    assert st2.expired + int(np.isfinite(st2.latency_ms).sum()) == n
    assert pg.pencil_arena_free_bytes(srv.arena) == 1 << 20


def test_waves_batch_only_under_load():
    from paper_1302_5586_gb300 import serve
    assert serve.wave_limit("plain", 50, 4, 64) == 1
    assert serve.wave_limit("served", 1, 4, 64) == 1        # a lone request goes alone
    assert serve.wave_limit("served", 3, 4, 64) == 1        # fewer requests than idle streams
    assert serve.wave_limit("served", 10, 4, 64) == 3       # spread over the idle streams
    assert serve.wave_limit("served", 10, 0, 64) == 64      # every stream busy: the queue forms a wave
    assert serve.wave_limit("served", 500, 2, 64) == 64     # never beyond max_wave
    assert serve.wave_limit("served", 0, 4, 64) == 1
