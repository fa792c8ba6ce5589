"""Continuous-batching serving: every request's result is the same bits in
the served mix, in the plain one-launch-per-request replay and alone;
admission respects the memory budget; the arena is whole again at the end."""
import numpy as np
import pytest
import torch

import paper_1302_5586_gb300 as pg
from gpu_util import dev
from paper_1302_5586_gb300 import serve

pytestmark = pytest.mark.gpu


def alone(req, host_pool, bank, dtype):
    hw = req.h * req.w
    x = host_pool[req.src:req.src + hw].to(dev()).view(req.h, req.w)
    k = torch.from_numpy(bank[req.filt:req.filt + req.ks * req.ks].copy()).to(dev())
    y = torch.empty_like(x)
    pg.pencil_conv2d_ex(1, req.h, req.w, x, req.ks, req.ks, k, y, dtype)
    torch.cuda.synchronize()
    return y.cpu()


@pytest.mark.parametrize("dtype", [pg.PENCIL_F16, pg.PENCIL_F32])
def test_each_result_is_the_same_alone_and_in_the_mix(dtype):
    tr = serve.make_trace(77, rate=20000.0, duration=0.01, lo=8, hi=400, klo=1, khi=15, pool_elems=1 << 20)
    assert len(tr.requests) > 100
    for r in tr.requests:  # one burst: every stream is soon busy, so the queue forms batched waves
        r.arrival = 0.0
    pool = serve.host_pool(tr, dtype, 78)
    bank = torch.from_numpy(tr.filters).to(dev())
    srv = serve.Server(dtype=dtype, budget_bytes=64 << 20, streams=3, max_wave=16, max_inflight=48)
    try:
        st, outs = srv.run(tr, pool, bank, mode="served", keep_outputs=True)
        st2, outs2 = srv.run(tr, pool, bank, mode="plain", keep_outputs=True)
        assert pg.pencil_arena_free_bytes(srv.arena) == 64 << 20
    finally:
        srv.close()
    assert st.rejected == 0 and np.all(np.isfinite(st.latency_ms))
    assert st.waves < len(tr.requests)           # requests were batched
    assert st2.waves == len(tr.requests)         # one launch per request
    itype = torch.int16 if dtype == pg.PENCIL_F16 else torch.int32
    for r in tr.requests:
        ref = alone(r, pool, tr.filters, dtype)
        assert torch.equal(outs[r.rid].view(itype), ref.view(itype)), r
        assert torch.equal(outs2[r.rid].view(itype), ref.view(itype)), r


def test_admission_waits_for_memory_and_rejects_what_never_fits():
    tr = serve.make_trace(5, rate=50000.0, duration=0.004, lo=200, hi=400, klo=3, khi=7, pool_elems=1 << 20)
    big = serve.Request(len(tr.requests), tr.requests[-1].arrival, 2048, 2048, 3, 0, 0)
    tr.requests.append(big)                       # 16 MiB in + out: larger than the budget
    budget = 2 << 20                              # room for a few requests at a time
    pool = serve.host_pool(tr, pg.PENCIL_F16, 6)
    pool = torch.cat([pool, torch.zeros(2048 * 2048, dtype=pool.dtype)]).pin_memory()
    bank = torch.from_numpy(tr.filters).to(dev())
    srv = serve.Server(dtype=pg.PENCIL_F16, budget_bytes=budget, streams=2, max_wave=8, max_inflight=64)
    try:
        st, _ = srv.run(tr, pool, bank, mode="served")
        assert pg.pencil_arena_free_bytes(srv.arena) == budget
    finally:
        srv.close()
    assert st.rejected == 1 and np.isnan(st.latency_ms[big.rid])
    assert np.all(np.isfinite(st.latency_ms[:-1]))
    assert 0 < st.peak_arena_bytes <= budget
    assert st.peak_inflight < len(tr.requests) - 1  # memory, not the slot limit, held requests back


def test_served_mix_at_full_request_sizes_against_alone_runs_and_the_oracle():
    """The serving workload's request shapes (binary16 images, sides
    log-uniform in [128, 4096], odd filter sides 3..15) arriving ten times
    faster than the 2000 req/s stream, so that waves hold many requests: every
    served result is the same bits as its request run alone through
    pencil_conv2d_ex, in the served mix and in the plain replay, and every 97th
    request is checked against the FP64 oracle (on its binary16 input) at 1024
    sampled pixels plus the four corners, within 2^-10 * sum |k||x| (the
    floating-point reproducibility point of Sec. 3.1)."""
    import oracle
    from gpu_util import sample_points

    tr = serve.make_trace(2024, rate=20000.0, duration=0.016)
    n = len(tr.requests)
    assert 250 <= n <= 450
    sides = np.array([(r.h, r.w) for r in tr.requests])
    assert sides.min() >= 128 and sides.max() <= 4096 and sides.max() > 2048
    assert {r.ks for r in tr.requests} == set(range(3, 16, 2))
    pool = serve.host_pool(tr, pg.PENCIL_F16, 2025)
    bank = torch.from_numpy(tr.filters).to(dev())
    srv = serve.Server(dtype=pg.PENCIL_F16, budget_bytes=8 << 30, streams=4, max_wave=64, max_inflight=256)
    try:
        st, outs = srv.run(tr, pool, bank, mode="served", keep_outputs=True)
        st2, outs2 = srv.run(tr, pool, bank, mode="plain", keep_outputs=True)
        assert pg.pencil_arena_free_bytes(srv.arena) == 8 << 30
    finally:
        srv.close()
    assert st.rejected == 0 and np.all(np.isfinite(st.latency_ms))
    assert st.waves < n / 2                       # waves of many requests
    assert st2.waves == n
    worst = 0.0
    for r in tr.requests:
        ref = alone(r, pool, tr.filters, pg.PENCIL_F16)
        assert torch.equal(outs[r.rid].view(torch.int16), ref.view(torch.int16)), r
        assert torch.equal(outs2[r.rid].view(torch.int16), ref.view(torch.int16)), r
        if r.rid % 97:
            continue
        hw = r.h * r.w
        x = pool[r.src:r.src + hw].numpy().reshape(1, r.h, r.w)
        k = tr.filters[r.filt:r.filt + r.ks * r.ks].reshape(r.ks, r.ks)
        pts = sample_points(r.rid, 1, r.h, r.w, 1024, borders=False)
        corners = np.array([[0, 0, 0], [0, 0, r.w - 1], [0, r.h - 1, 0], [0, r.h - 1, r.w - 1]])
        pts = np.concatenate([pts, corners])
        want, bound = oracle.conv2d_points(x, k, pts)
        got = outs[r.rid].numpy().astype(np.float64)[pts[:, 1], pts[:, 2]]
        ratio = np.abs(got - want) / np.maximum(bound, 1e-300)
        assert np.all(ratio <= 2.0 ** -10), (r, float(ratio.max()))
        worst = max(worst, float(ratio.max()))
    assert 0.0 < worst <= 2.0 ** -10
