"""The allocation-free Jacobi entry point against the workspace one.

pencil_jacobi2d_noalloc serves callers that cannot allocate device memory (a
fixed-latency loop that cannot pay for cudaMalloc's synchronisation, a process
whose framework allocator already holds the device's memory, or code that
forbids allocation after start-up): its scratch is a static device array shared
by all calls.  This file is collected last so that a run stopping at the first
failure has already run every other test; it needs nothing from them.
"""
import numpy as np
import pytest

import paper_1302_5586_gb300 as pg
import synth
from gpu_util import dev, to_dev, torch

pytestmark = pytest.mark.gpu


def _with_workspace(u0, iters, ce, t):
    h, w = u0.shape
    d = to_dev(u0)
    wsb = pg.pencil_jacobi2d_workspace_size(h, w)
    ws = torch.empty(wsb, dtype=torch.uint8, device=dev())
    res = torch.zeros(iters // ce, dtype=torch.float64, device=dev())
    pg.pencil_jacobi2d_ex(h, w, d, iters, ce, res, ws, wsb, t)
    torch.cuda.synchronize()
    return d.cpu().numpy(), res.cpu().numpy()


def _without_allocation(u0, iters, ce, t):
    h, w = u0.shape
    d = to_dev(u0)
    res = torch.zeros(iters // ce, dtype=torch.float64, device=dev())
    pg.pencil_jacobi2d_noalloc(h, w, d, iters, ce, res, t)
    torch.cuda.synchronize()
    return d.cpu().numpy(), res.cpu().numpy()


def test_noalloc_matches_workspace_entry_point_on_two_calls():
    # two calls in a row on different grids and paths (tiled float4 path, then
    # the scalar path of a width that is not a multiple of 4): the second call
    # finds the first call's data in the shared scratch and must not be affected
    cases = [((1000, 1300), 30, 10, 0), ((777, 1001), 25, 5, 1)]
    for n, ((h, w), iters, ce, t) in enumerate(cases):
        u0 = synth.jacobi_init_f32(4242 + n, h, w)
        ua, ra = _with_workspace(u0, iters, ce, t)
        ub, rb = _without_allocation(u0, iters, ce, t)
        assert np.max(np.abs(ub.astype(np.float64) - ua)) <= 1e-5
        np.testing.assert_allclose(rb, ra, rtol=1e-9, atol=1e-300)
        # same kernels on the same grid: the same bits
        np.testing.assert_array_equal(ub.view(np.uint32), ua.view(np.uint32))


def test_noalloc_rejects_grids_beyond_its_scratch():
    u = torch.zeros(2100, 2200, device=dev())
    assert pg.pencil_jacobi2d_workspace_size(2100, 2200) > pg.PENCIL_NOALLOC_SCRATCH_BYTES
    with pytest.raises(pg.PencilError) as e:
        pg.pencil_jacobi2d_noalloc(2100, 2200, u, 10, 0, None)
    assert e.value.name == "PENCIL_ERR_NOMEM"
    ok = torch.zeros(2048, 2048, device=dev())
    pg.pencil_jacobi2d_noalloc(2048, 2048, ok, 2, 0, None)
    torch.cuda.synchronize()


def test_noalloc_applies_the_row_limit_of_the_workspace_entry_point():
    # a tall, narrow grid fits the scratch but has more rows than a launch
    # can cover: the same UNSUPPORTED as pencil_jacobi2d_ex, before any launch
    h, w = pg.PENCIL_MAX_ROWS + 1, 3
    assert pg.pencil_jacobi2d_workspace_size(h, w) <= pg.PENCIL_NOALLOC_SCRATCH_BYTES
    u = torch.zeros(h, w, device=dev())
    for call in (lambda: pg.pencil_jacobi2d_noalloc(h, w, u, 1, 0, None),
                 lambda: pg.pencil_jacobi2d_ex(h, w, u, 1, 0, None, u, 1 << 30, 0)):
        with pytest.raises(pg.PencilError) as e:
            call()
        assert e.value.name == "PENCIL_ERR_UNSUPPORTED"


def test_noalloc_rejects_residuals_inside_the_grid():
    u = torch.zeros(64 * 64 + 64, device=dev())
    res = u[64 * 64 - 8:].view(torch.float64)  # overlaps the grid's last elements
    with pytest.raises(pg.PencilError) as e:
        pg.pencil_jacobi2d_noalloc(64, 64, u, 10, 5, res)
    assert e.value.name == "PENCIL_ERR_ALIAS"
