"""Multi-rank paths on CPU with gloo (world sizes 2 and 3): the row-band
Jacobi decomposition equals the undivided grid bit for bit, and the
benchmark's cross-rank timing takes the slowest rank."""
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
