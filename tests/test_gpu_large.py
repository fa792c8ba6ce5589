"""Images and grids past 2^31 elements (50000 x 50000 = 2.5e9): every index
into them must be 64-bit.  Convolutions are checked on sampled pixels --
random ones, the border rows and columns, and pixels whose linear index is
above 2^31 -- against the FP64 oracle; the Jacobi tiles against the
one-sweep kernel bit for bit, and a window against the oracle."""
import numpy as np
import pytest

import oracle
import paper_1302_5586_gb300 as pg
import synth
from gpu_util import dev, torch

pytestmark = pytest.mark.gpu

N = 50000  # N * N > 2^31


def _points(seed, h, w, n=4000):
    r = np.random.default_rng(seed)
    pts = [np.stack([np.zeros(n, np.int64), r.integers(0, h, n), r.integers(0, w, n)], axis=1)]
    lo = (1 << 31) // w + 1  # rows whose first pixel is past index 2^31
    pts.append(np.stack([np.zeros(n, np.int64), r.integers(lo, h, n), r.integers(0, w, n)], axis=1))
    for i in (0, 1, h - 2, h - 1):
        cols = r.integers(0, w, 200)
        pts.append(np.stack([np.zeros(200, np.int64), np.full(200, i), cols], axis=1))
    for j in (0, 1, w - 2, w - 1):
        rows = r.integers(0, h, 200)
        pts.append(np.stack([np.zeros(200, np.int64), rows, np.full(200, j)], axis=1))
    return np.concatenate(pts)


@pytest.fixture(scope="module")
def big_image():
    dev()
    return synth.image_f32(synth.SEEDS["conv8192x3"] ^ 0x77, 1, N, N)


def _gather(t, pts):
    p = torch.from_numpy(pts).to(t.device)
    return t[p[:, 0], p[:, 1], p[:, 2]].double().cpu().numpy()


@pytest.mark.parametrize("K", [3, 15])
def test_direct_f32_past_2_31(big_image, K):
    k = synth.filter_f32(500 + K, K, K)
    d_in = torch.from_numpy(big_image).to(dev())
    d_out = torch.empty_like(d_in)
    pg.pencil_conv2d_ex(1, N, N, d_in, K, K, torch.from_numpy(k).to(dev()), d_out, pg.PENCIL_F32)
    torch.cuda.synchronize()
    pts = _points(K, N, N)
    ref, bound = oracle.conv2d_points(big_image, k, pts)
    got = _gather(d_out, pts)
    assert np.all(np.abs(got - ref) <= 1e-6 * bound)


def test_f16_and_separable_past_2_31(big_image):
    img16 = synth.to_f16(big_image)
    d_in = torch.from_numpy(img16).to(dev())
    d_out = torch.empty_like(d_in)
    k = synth.filter_f32(77, 7, 7)
    pg.pencil_conv2d_ex(1, N, N, d_in, 7, 7, torch.from_numpy(k).to(dev()), d_out, pg.PENCIL_F16)
    torch.cuda.synchronize()
    pts = _points(7, N, N)
    ref, bound = oracle.conv2d_points(img16, k, pts)
    got = _gather(d_out, pts)
    assert np.all(np.abs(got - ref) <= 2.0 ** -10 * bound)
    del d_in, d_out
    g = synth.gaussian_taps_f32(7, 3.0)
    d_in = torch.from_numpy(big_image).to(dev())
    d_out = torch.empty_like(d_in)
    dg = torch.from_numpy(g).to(dev())
    pg.pencil_conv2d_sep_ex(1, N, N, d_in, 15, dg, 15, dg, d_out, pg.PENCIL_F32)
    torch.cuda.synchronize()
    ref, bound = oracle.conv2d_sep_points(big_image, g, g, pts)
    got = _gather(d_out, pts)
    assert np.all(np.abs(got - ref) <= 1e-6 * bound)


def test_jacobi_tiles_past_2_31():
    dev()
    u0 = synth.jacobi_init_f32(17, N, N)
    wsb = pg.pencil_jacobi2d_workspace_size(N, N)
    ws = torch.empty(wsb, dtype=torch.uint8, device=dev())
    a = torch.from_numpy(u0).to(dev())
    pg.pencil_jacobi2d_ex(N, N, a, 3, 0, None, ws, wsb, 1)
    b = torch.from_numpy(u0).to(dev())
    pg.pencil_jacobi2d_ex(N, N, b, 3, 0, None, ws, wsb, 0)
    torch.cuda.synchronize()
    assert torch.equal(a.view(torch.int32), b.view(torch.int32))
    # a window near the far corner: 3 sweeps are exact 3 points inside it
    i0, j0 = N - 40, N - 50
    win = u0[i0 - 3:, j0 - 3:].astype(np.float64)
    ref, _ = oracle.jacobi2d(win, 3)
    got = b[i0:, j0:].double().cpu().numpy()
    np.testing.assert_allclose(got, ref[3:, 3:], atol=1e-5, rtol=0)
    del a, b, ws
