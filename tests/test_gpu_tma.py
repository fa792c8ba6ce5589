"""The TMA-staged direct kernels (images whose rows are 16-byte aligned, clamp
and zero borders) and the bounded wait they use.

The TMA kernels share the tile body and the fixed per-pixel order of every
other conv2d kernel, so they must equal the generic kernel bit for bit; the
clamp border is rebuilt in shared memory from a box whose out-of-image
elements arrive as zeros, which the small and ragged shapes below exercise
on every edge.  The oracle check uses the tolerance of the other parity
tests (FP32: 1e-6 * sum|k||x|; binary16: 2^-10 * sum|k||x|).
"""
import numpy as np
import pytest

import oracle
import paper_1302_5586_gb300 as pg
import synth
from gpu_util import to_dev, torch

pytestmark = pytest.mark.gpu

F32_TOL = 1e-6
F16_TOL = 2.0 ** -10
# (channels, rows, columns): widths that keep FP32 and binary16 rows 16-byte
# aligned; single rows, images narrower and shorter than a tile and filter,
# ragged tile counts in both directions
SHAPES = [(1, 1, 8), (2, 5, 16), (1, 3, 8), (1, 33, 136), (3, 70, 264), (1, 40, 1032)]


def conv(img, k, dtype, flags):
    c, h, w = img.shape
    d_in = to_dev(img)
    d_out = torch.empty_like(d_in)
    pg.pencil_conv2d_ex(c, h, w, d_in, k.shape[0], k.shape[1], to_dev(k), d_out, dtype, flags)
    torch.cuda.synchronize()
    return d_out.cpu().numpy()


@pytest.mark.parametrize("dtype", [pg.PENCIL_F32, pg.PENCIL_F16])
@pytest.mark.parametrize("border", ["clamp", "zero"])
def test_tma_kernels_equal_generic_bitwise(dtype, border):
    flags = pg.PENCIL_BORDER(pg.BORDER_MODES[border])
    assert pg.pencil_device_status() == pg.PENCIL_OK  # nothing pending from earlier work
    for K in (1, 3, 5, 7, 9, 15):
        k = synth.filter_f32(900 + K, K, K)
        for shape in SHAPES:
            img = synth.image_f32(910 + K, *shape)
            if dtype == pg.PENCIL_F16:
                img = synth.to_f16(img)
            a = conv(img, k, dtype, flags)
            b = conv(img, k, dtype, flags | pg.PENCIL_CONV_GENERIC)
            view = np.uint16 if dtype == pg.PENCIL_F16 else np.uint32
            np.testing.assert_array_equal(a.view(view), b.view(view), err_msg=f"K={K} shape={shape}")
    assert pg.pencil_device_status() == pg.PENCIL_OK  # no wait ran out


@pytest.mark.parametrize("border", ["clamp", "zero"])
def test_tma_kernels_match_oracle(border):
    flags = pg.PENCIL_BORDER(pg.BORDER_MODES[border])
    for K, shape in ((3, (2, 37, 264)), (7, (1, 70, 136)), (15, (1, 45, 272))):
        k = synth.filter_f32(920 + K, K, K)
        img = synth.image_f32(930 + K, *shape)
        out = conv(img, k, pg.PENCIL_F32, flags)
        ref, bound = oracle.conv2d(img, k, border=border)
        assert np.all(np.abs(out - ref) <= F32_TOL * bound), f"f32 K={K} {border}"
        img16 = synth.to_f16(img)
        out16 = conv(img16, k, pg.PENCIL_F16, flags)
        ref16, bound16 = oracle.conv2d(img16, k, border=border)
        assert np.all(np.abs(out16.astype(np.float64) - ref16) <= F16_TOL * bound16), f"f16 K={K} {border}"


def test_bounded_wait_runs_out_and_is_reported():
    """A wait on an mbarrier that no copy completes gives up after its limit
    (the kernel returns instead of hanging) and the timeout is reported once."""
    assert pg.pencil_device_status() == pg.PENCIL_OK
    assert pg.pencil_selftest_wait_timeout(2000) == 0  # 2 ms limit: ran out
    assert pg.pencil_device_status() == pg.PENCIL_ERR_TIMEOUT
    assert pg.pencil_device_status() == pg.PENCIL_OK  # the report cleared the count
    # the context is still usable: a conv2d call afterwards is correct
    img = synth.image_f32(940, 1, 16, 64)
    k = synth.filter_f32(941, 3, 3)
    a = conv(img, k, pg.PENCIL_F32, 0)
    b = conv(img, k, pg.PENCIL_F32, pg.PENCIL_CONV_GENERIC)
    np.testing.assert_array_equal(a.view(np.uint32), b.view(np.uint32))


@pytest.mark.parametrize("dtype", [pg.PENCIL_F32, pg.PENCIL_F16])
@pytest.mark.parametrize("border", ["clamp", "zero"])
def test_tma_separable_matches_oracle(dtype, border):
    """The separable kernels' TMA staging on the same edge shapes.  Clamp: the
    separable oracle; zero: the 2-D oracle with the exact outer-product
    weights, plus the rounding slack of those weights in FP32."""
    flags = pg.PENCIL_BORDER(pg.BORDER_MODES[border])
    tol = F16_TOL if dtype == pg.PENCIL_F16 else F32_TOL
    for K in (3, 7, 9, 15):
        gx = synth.gaussian_taps_f32(K // 2, 1.0 + K / 5)
        gy = synth.filter_f32(950 + K, 1, K).ravel()
        for shape in SHAPES:
            c, h, w = shape
            img = synth.image_f32(960 + K, c, h, w)
            if dtype == pg.PENCIL_F16:
                img = synth.to_f16(img)
            d_in = to_dev(img)
            d_out = torch.empty_like(d_in)
            pg.pencil_conv2d_sep_ex(c, h, w, d_in, K, to_dev(gx), K, to_dev(gy), d_out, dtype, flags)
            torch.cuda.synchronize()
            out = d_out.cpu().numpy().astype(np.float64)
            if border == "clamp":
                ref, bound = oracle.conv2d_sep(img, gx, gy)
                slack = 0.0
            else:
                k2 = np.outer(gy.astype(np.float64), gx.astype(np.float64))
                ref, bound = oracle.conv2d(img, k2.astype(np.float32), border="zero")
                slack = np.abs(k2 - k2.astype(np.float32).astype(np.float64)).sum() * np.abs(img.astype(np.float64)).max()
            assert np.all(np.abs(out - ref) <= tol * bound + slack), f"K={K} shape={shape}"
    assert pg.pencil_device_status() == pg.PENCIL_OK


@pytest.mark.parametrize("w", [264, 262])
def test_conv2d_ex_in_a_cuda_graph(w):
    """pencil_conv2d_ex captured in a CUDA graph (TMA-staged for aligned rows,
    cp.async otherwise) replays to the bits of a plain stream launch."""
    img = synth.image_f32(970, 2, 45, w)
    k = to_dev(synth.filter_f32(971, 15, 15))
    d_in = to_dev(img)
    ref = torch.empty_like(d_in)
    pg.pencil_conv2d_ex(2, 45, w, d_in, 15, 15, k, ref, pg.PENCIL_F32)
    out = torch.full_like(d_in, float("nan"))
    g = torch.cuda.CUDAGraph()
    cap = torch.cuda.Stream()
    cap.wait_stream(torch.cuda.current_stream())
    with torch.cuda.graph(g, stream=cap):
        pg.pencil_conv2d_ex(2, 45, w, d_in, 15, 15, k, out, pg.PENCIL_F32, 0, cap.cuda_stream)
    assert torch.isnan(out).all()  # captured, not run
    g.replay()
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out.cpu().numpy().view(np.uint32), ref.cpu().numpy().view(np.uint32))
    assert pg.pencil_device_status() == pg.PENCIL_OK
