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
