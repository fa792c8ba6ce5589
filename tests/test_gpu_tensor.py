"""GPU parity of the tensor-core binary16 correlation (PENCIL_CONV_TENSOR)
against the FP64 oracle, through the C ABI.

Tolerance: |gpu - oracle(binary16 input)| <= 2^-10 * sum |k| |x| per pixel,
the binary16 bound of the CUDA-core path.  The tensor-core path sums in
another order, so it is not the same bits as the CUDA-core kernels; where
the flag does not apply (FP32, sides below 7, rows not 16-byte aligned,
other borders, interleaved or generic) the call must give exactly the
CUDA-core bits.
"""
import numpy as np
import pytest

import oracle
import paper_1302_5586_gb300 as pg
import synth
from gpu_util import dev, gather, sample_points, to_dev, torch

pytestmark = pytest.mark.gpu

F16_TOL = 2.0 ** -10
TC = pg.PENCIL_CONV_TENSOR


def run(img, k, dtype, flags):
    c, h, w = img.shape
    d_in = to_dev(img)
    d_out = torch.empty_like(d_in)
    pg.pencil_conv2d_ex(c, h, w, d_in, k.shape[0], k.shape[1], to_dev(k), d_out, dtype, flags)
    torch.cuda.synchronize()
    return d_out


def check(out, ref, bound, what):
    err = np.abs(out.astype(np.float64) - ref)
    ratio = float(np.max(err / np.maximum(bound, 1e-300)))
    assert np.all(err <= F16_TOL * bound), f"{what}: max err/bound {ratio:.3e} > {F16_TOL:.3e}"
    return ratio


# w a multiple of 8 (rows 16-byte aligned); ragged tiles in both directions
SHAPES = [(1, 200, 520), (2, 75, 304), (1, 333, 136), (1, 1, 8), (3, 257, 1032)]


@pytest.mark.parametrize("K", [7, 9, 11, 13, 15])
@pytest.mark.parametrize("border", ["clamp", "zero"])
@pytest.mark.parametrize("shape", SHAPES)
def test_tensor_matches_oracle(K, border, shape):
    c, h, w = shape
    img = synth.to_f16(synth.image_f32(300 + K + w, c, h, w))
    k = synth.filter_f32(310 + K, K, K)
    m = pg.PENCIL_BORDER(pg.BORDER_MODES[border])
    out = run(img, k, pg.PENCIL_F16, m | TC).cpu().numpy()
    ref, bound = oracle.conv2d(img, k, border=border)
    check(out, ref, bound, f"K={K} {border} {shape}")
    assert pg.pencil_device_status() == pg.PENCIL_OK


@pytest.mark.parametrize("scale_exp", [-9, 0, 7])
def test_tensor_weight_scale_and_signs(scale_exp):
    """Weights far below (or above) 1 and of both signs: the power-of-two
    scale keeps the two binary16 terms normal, so the bound still holds."""
    img = synth.to_f16(synth.image_f32(41, 1, 150, 264))
    r = np.random.default_rng(42)
    k = (synth.filter_f32(43, 15, 15) * (r.integers(0, 2, (15, 15)) * 2 - 1)).astype(np.float32)
    k = np.ldexp(k, scale_exp).astype(np.float32)
    out = run(img, k, pg.PENCIL_F16, TC).cpu().numpy()
    ref, bound = oracle.conv2d(img, k)
    check(out, ref, bound, f"scale 2^{scale_exp}")


def test_tensor_zero_filter_gives_zeros():
    img = synth.to_f16(synth.image_f32(44, 1, 130, 136))
    out = run(img, np.zeros((11, 11), np.float32), pg.PENCIL_F16, TC).cpu().numpy()
    assert np.all(out == 0)


def test_tensor_full_size_sampled():
    """The bench's launch: 3 x 8192 x 8192 binary16, 15 x 15, sampled pixels
    (every pixel of the outer rows and columns of the last channel)."""
    C, H, W = 3, 8192, 8192
    img = synth.to_f16(synth.image_f32(1, C, H, W))
    k = synth.filter_f32(2, 15, 15)
    out = run(img, k, pg.PENCIL_F16, TC)
    pts = sample_points(5, C, H, W, 4000)
    ref, bound = oracle.conv2d_points(img, k, pts)
    err = np.abs(gather(out, pts) - ref)
    assert np.all(err <= F16_TOL * bound)
    # the tensor cores did run: their summation order differs from the CUDA cores'
    cc = run(img, k, pg.PENCIL_F16, 0)
    assert not torch.equal(out, cc)


@pytest.mark.parametrize("case", ["f32", "small_side", "unaligned", "reflect", "generic", "hwc", "nonsquare"])
def test_tensor_flag_falls_back_to_cuda_core_bits(case):
    c, h, w, K, kw = 2, 90, 264, 11, 11
    dtype, extra = pg.PENCIL_F16, 0
    if case == "f32":
        dtype = pg.PENCIL_F32
    elif case == "small_side":
        K = kw = 5
    elif case == "unaligned":
        w = 261
    elif case == "reflect":
        extra = pg.PENCIL_BORDER(pg.BORDER_MODES["reflect"])
    elif case == "generic":
        extra = pg.PENCIL_CONV_GENERIC
    elif case == "hwc":
        c, extra = 3, pg.PENCIL_LAYOUT_HWC
    elif case == "nonsquare":
        kw = 9
    img = synth.image_f32(50, c, h, w)
    if dtype == pg.PENCIL_F16:
        img = synth.to_f16(img)
    k = synth.filter_f32(51, K, kw)
    a = run(img, k, dtype, extra | TC).cpu().numpy()
    b = run(img, k, dtype, extra).cpu().numpy()
    view = np.uint16 if dtype == pg.PENCIL_F16 else np.uint32
    np.testing.assert_array_equal(a.view(view), b.view(view))
