"""Multi-rank paths on CPU with gloo (world sizes 2 and 3): the row-band
Jacobi decomposition equals the undivided grid bit for bit, the row-band
split of one image's conv2d (halo rows, no exchange) equals the undivided
image bit for bit, the benchmark's cross-rank timing takes the slowest
rank, and a rank that dies between steps makes its neighbour's next halo
exchange fail with an error instead of hanging."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
import synth
from paper_1302_5586_gb300 import shard


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _init(rank, world, port):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)


def _band_worker(rank, world, port, h, w, halo, iters, ce, out):
    _init(rank, world, port)
    try:
        u0 = synth.jacobi_init_f32(41, h, w).astype(np.float64)
        bj = shard.BandJacobi(h, w, rank, world, halo, dist)
        lo, hi = bj.local_slice()
        local = torch.from_numpy(u0[lo:hi].copy())

        def sweep(loc, n):
            arr = loc.numpy()
            arr[...] = oracle.jacobi2d(arr, n)[0]

        def resid(sub):
            return oracle.residual2d(np.ascontiguousarray(sub.numpy()))

        res = bj.run(local, iters, ce, sweep, resid)
        out[rank] = (bj.r0, bj.r1, bj.owned(local).numpy().copy(), res)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,halo,h,w,iters,ce", [(2, 1, 37, 23, 23, 5), (3, 3, 41, 19, 20, 10),
                                                      (2, 4, 30, 30, 13, 4), (3, 1, 12, 9, 9, 3)])
def test_band_jacobi_equals_single_domain(world, halo, h, w, iters, ce):
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_band_worker, args=(r, world, port, h, w, halo, iters, ce, out))
             for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    u0 = synth.jacobi_init_f32(41, h, w).astype(np.float64)
    ref, ref_res = oracle.jacobi2d(u0, iters, ce)
    got = np.zeros_like(ref)
    for r in range(world):
        r0, r1, rows, res = out[r]
        got[r0:r1] = rows
        np.testing.assert_allclose(res, ref_res, rtol=1e-13, atol=1e-300)
    np.testing.assert_array_equal(got, ref)


def test_band_bounds_cover_the_grid():
    for h in (3, 10, 97):
        for world in (1, 2, 5):
            if h - 2 < world:
                continue
            b = [shard.band_bounds(h, r, world) for r in range(world)]
            assert b[0][0] == 0 and b[-1][1] == h
            assert all(b[i][1] == b[i + 1][0] for i in range(world - 1))
    with pytest.raises(ValueError):
        shard.BandJacobi(10, 10, 0, 4, 3, dist)


def _timing_worker(rank, world, port, out):
    _init(rank, world, port)
    try:
        import bench
        ms = [10.0, 25.0, 17.0][rank]
        slowest = bench.max_over_ranks(ms, dist, torch.device("cpu"))
        out[rank] = (slowest, bench.whole_job_gpx(1e9, world, 4, slowest))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_bench_takes_the_slowest_rank(world):
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_timing_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    slowest = 25.0
    for r in range(world):
        assert out[r][0] == slowest
        assert out[r][1] == pytest.approx(1e9 * world * 4 / (slowest * 1e-3) / 1e9)


def _conv_worker(rank, world, port, c, h, w, kh, kw, out):
    _init(rank, world, port)
    try:
        img = synth.image_f32(51, c, h, w)
        k = synth.filter_f32(52, kh, kw)
        bc = shard.BandConv2d(h, kh, rank, world)
        mine = bc.run(img, lambda sub: oracle.conv2d(np.ascontiguousarray(sub), k, want_bound=False)[0])
        # one all-gather of the owned bands (padded to the largest band)
        rows = torch.tensor([bc.r1 - bc.r0])
        sizes = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
        dist.all_gather(sizes, rows)
        m = max(int(t) for t in sizes)
        pad = torch.zeros((c, m, w), dtype=torch.float64)
        pad[:, :bc.r1 - bc.r0] = torch.from_numpy(np.ascontiguousarray(mine))
        parts = [torch.zeros_like(pad) for _ in range(world)]
        dist.all_gather(parts, pad)
        full = np.concatenate([p[:, :int(n)].numpy() for p, n in zip(parts, sizes)], axis=1)
        out[rank] = full
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,c,h,w,kh,kw", [(2, 2, 37, 23, 5, 3), (3, 1, 41, 19, 15, 15), (3, 1, 4, 9, 7, 7),
                                                (2, 1, 1, 16, 3, 3)])
def test_band_conv2d_equals_single_image(world, c, h, w, kh, kw):
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_conv_worker, args=(r, world, port, c, h, w, kh, kw, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    img = synth.image_f32(51, c, h, w)
    ref = oracle.conv2d(img, synth.filter_f32(52, kh, kw), want_bound=False)[0]
    for r in range(world):
        np.testing.assert_array_equal(out[r].view(np.uint64), ref.view(np.uint64))


def test_conv_band_bounds_cover_the_rows():
    for h in (1, 2, 7, 64, 1001):
        for world in (1, 2, 3, 8):
            spans = [shard.conv_band_bounds(h, r, world) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == h
            assert all(a[1] == b[0] for a, b in zip(spans, spans[1:]))
            assert all(z - a in (h // world, h // world + 1) for a, z in spans)


def _dying_worker(rank, world, port, die_after, out):
    """Rank 1 raises between steps (after `die_after` sweeps, with nothing of
    its own in flight); rank 0 keeps iterating and must get an error from its
    next halo exchange, within the process group's timeout, not hang."""
    import datetime
    import time

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=5))
    h, w = 40, 16
    u0 = synth.jacobi_init_f32(43, h, w).astype(np.float64)
    bj = shard.BandJacobi(h, w, rank, world, 1, dist)
    lo, hi = bj.local_slice()
    local = torch.from_numpy(u0[lo:hi].copy())
    sweeps = {"n": 0}

    def sweep(loc, n):
        if rank == 1 and sweeps["n"] >= die_after:
            raise RuntimeError("injected rank failure")
        arr = loc.numpy()
        arr[...] = oracle.jacobi2d(arr, n)[0]
        sweeps["n"] += n

    t0 = time.monotonic()
    try:
        bj.run(local, 1000, 0, sweep, lambda sub: 0.0)
        out[rank] = ("finished", sweeps["n"], time.monotonic() - t0)
    except Exception as e:  # the failure, as each rank sees it
        out[rank] = (type(e).__name__, sweeps["n"], time.monotonic() - t0)
    finally:
        try:
            dist.destroy_process_group()
        except Exception:
            pass


def test_a_rank_that_dies_is_detected_by_the_others():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_dying_worker, args=(r, 2, port, 3, out)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        for p in procs:
            p.join(120)
            assert p.exitcode is not None, "a rank hung after its peer died"
    finally:
        for p in procs:
            if p.exitcode is None:
                p.kill()
    what1, n1, _ = out[1]
    assert what1 == "RuntimeError" and n1 == 3           # the injected failure, between steps
    what0, n0, t0 = out[0]
    assert what0 != "finished" and n0 <= 4              # the survivor stopped at the next exchange ...
    assert t0 < 60                                       # ... with an error, not a hang
