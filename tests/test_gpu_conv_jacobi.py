"""A filter pass followed by Jacobi smoothing (pencil_conv2d_jacobi), through
the C ABI.

The call is defined as pencil_conv2d_ex into out followed by
pencil_jacobi2d_ex on each channel of out, so it must return those bits
exactly, fused or not.  Against the composed FP64 oracle (the oracle's
correlation, then the oracle's sweeps from its exact result) the error is
bounded by the arithmetic: the filter pass leaves at most 1e-6 * sum|k||x| per
pixel (the FP32 tolerance of every conv2d result), a Jacobi sweep is a
convex combination so it never enlarges the largest error, and each FP32
sweep adds at most 2 * 2^-24 * max|u| (three roundings of the sum of four
neighbours, |sum| <= 4 max|u|, then an exact multiply by 1/4).
"""
import numpy as np
import pytest

import oracle
import paper_1302_5586_gb300 as pg
import synth
from gpu_util import to_dev, torch

pytestmark = pytest.mark.gpu

F32_TOL = 1e-6
U = 2.0 ** -24


def two_calls(img, k, sweeps):
    c, h, w = img.shape
    d_in = to_dev(img)
    out = torch.empty_like(d_in)
    pg.pencil_conv2d_ex(c, h, w, d_in, k.shape[0], k.shape[1], to_dev(k), out, pg.PENCIL_F32)
    wsb = pg.pencil_jacobi2d_workspace_size(h, w)
    ws = torch.empty(max(wsb, 1), dtype=torch.uint8, device=out.device)
    for ch in range(c):
        pg.pencil_jacobi2d_ex(h, w, out[ch], sweeps, 0, None, ws, wsb, 0)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def fused_call(img, k, sweeps, flags=0):
    c, h, w = img.shape
    d_in = to_dev(img)
    out = torch.empty_like(d_in)
    pg.pencil_conv2d_jacobi(c, h, w, d_in, k.shape[0], k.shape[1], to_dev(k), sweeps, out, flags)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def composed_oracle(img, k, sweeps):
    y, bound = oracle.conv2d(img, k)
    ref = np.stack([oracle.jacobi2d(y[ch], sweeps)[0] for ch in range(img.shape[0])])
    return ref, bound


def check_oracle(got, img, k, sweeps):
    ref, bound = composed_oracle(img, k, sweeps)
    m = np.max(np.abs(ref)) * (1 + 1e-6) + F32_TOL * np.max(bound)
    tol = F32_TOL * np.max(bound) + sweeps * 2 * U * m
    err = np.max(np.abs(got.astype(np.float64) - ref))
    assert err <= tol, (err, tol)
    return err / tol


# w % 4 == 0 (fused) and not (a filter pass, then the sweeps); several 128 x
# 128 windows with ragged tails; grids smaller than one window
SHAPES = [(2, 300, 260), (1, 130, 132), (1, 77, 101), (1, 5, 8), (3, 40, 36), (1, 257, 4)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("K", [1, 3, 5, 7])
def test_same_bits_as_two_calls_and_within_the_composed_oracle(shape, K):
    c, h, w = shape
    img = synth.image_f32(1000 + h + K, c, h, w)
    k = synth.filter_f32(1010 + K, K, K)
    for sweeps in (0, 1, 2, 3, 4, 5, 9, 10, 13, 25):
        got = fused_call(img, k, sweeps)
        np.testing.assert_array_equal(got.view(np.uint32), two_calls(img, k, sweeps).view(np.uint32),
                                      err_msg=f"{shape} K={K} sweeps={sweeps}")
        if sweeps in (0, 4, 13):
            check_oracle(got, img, k, sweeps)


def test_larger_or_uneven_filters_take_two_passes():
    img = synth.image_f32(1020, 2, 90, 120)
    for k in (synth.filter_f32(1021, 9, 9), synth.filter_f32(1022, 3, 5), synth.filter_f32(1023, 15, 15)):
        got = fused_call(img, k, 6)
        np.testing.assert_array_equal(got.view(np.uint32), two_calls(img, k, 6).view(np.uint32))
        check_oracle(got, img, k, 6)


def test_fused_flag_refuses_what_cannot_fuse():
    img = synth.image_f32(1030, 1, 40, 42)  # w % 4 != 0
    k = synth.filter_f32(1031, 3, 3)
    with pytest.raises(pg.PencilError) as e:
        fused_call(img, k, 5, pg.PENCIL_CHAIN_FUSED)
    assert e.value.name == "PENCIL_ERR_UNSUPPORTED"
    ok = synth.image_f32(1032, 1, 40, 44)
    np.testing.assert_array_equal(fused_call(ok, k, 5, pg.PENCIL_CHAIN_FUSED).view(np.uint32),
                                  two_calls(ok, k, 5).view(np.uint32))


def test_linear_field_survives_a_centred_symmetric_filter_and_the_sweeps():
    """A linear field away from the edges is kept by a point-symmetric filter
    of weights summing to 1 (correlation with a symmetric filter reproduces
    a ramp) and is a fixed point of every sweep; near the edges the clamp bends
    it.  Dyadic values, so the interior rows far from the edges are exact."""
    h, w = 64, 64
    ii, jj = np.meshgrid(np.arange(h), np.arange(w), indexing="ij")
    img = (0.25 * ii + 0.5 * jj + 0.125).astype(np.float32)[None]
    k = np.array([[0, 0.125, 0], [0.125, 0.5, 0.125], [0, 0.125, 0]], dtype=np.float32)
    got = fused_call(img, k, 10)
    # the clamp changes the rows and columns at the edge; their effect moves
    # inward one point per sweep
    core = (slice(12, h - 12), slice(12, w - 12))
    np.testing.assert_array_equal(got[0][core], img[0][core])


def test_full_size_band_against_the_composed_oracle():
    """The benchmark's image, 8192 x 8192 x 3 FP32, a 5 x 5 filter and 10
    sweeps: rows 4000..4063 of every channel against the composed oracle run
    on a band of rows wide enough that its own edges cannot reach them (the
    sweeps' dependence reaches 10 rows, the filter 2 more)."""
    c, h, w, K, n = 3, 8192, 8192, 5, 10
    img = synth.image_f32(1040, c, h, w)
    k = synth.filter_f32(1041, K, K)
    d_in = to_dev(img)
    out = torch.empty_like(d_in)
    pg.pencil_conv2d_jacobi(c, h, w, d_in, K, K, to_dev(k), n, out)
    torch.cuda.synchronize()
    r0, r1 = 4000, 4064
    lo, hi = r0 - n - 1, r1 + n + 1           # the band's own fixed ring sits n + 1 rows out
    y, bound = oracle.conv2d(img[:, lo - K // 2:hi + K // 2, :], k)
    y, bound = y[:, K // 2:-(K // 2)], bound[:, K // 2:-(K // 2)]
    ref = np.stack([oracle.jacobi2d(y[ch], n)[0] for ch in range(c)])[:, r0 - lo:r1 - lo]
    got = out[:, r0:r1, :].cpu().numpy().astype(np.float64)
    m = np.max(np.abs(ref)) * (1 + 1e-6) + F32_TOL * np.max(bound)
    tol = F32_TOL * np.max(bound) + n * 2 * U * m
    assert np.max(np.abs(got - ref)) <= tol
    # and the same bits as the two calls on those rows
    np.testing.assert_array_equal(got.astype(np.float32).view(np.uint32),
                                  two_calls(img, k, n)[:, r0:r1, :].view(np.uint32))
