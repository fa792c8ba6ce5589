"""Interleaved [h][w][c] images (PENCIL_LAYOUT_HWC) through the C ABI.

Each channel of an interleaved image is filtered on its own, exactly as the
planar layout filters it, so the results are checked three ways: against the
FP64 oracle's interleaved definition (FP32: 1e-6 * sum|k||x|; binary16
storage: 2^-10 * sum|k||x| against the oracle on the binary16 input), bit for
bit against the planar kernels on the transposed image, and bit for bit
between the tiled and the generic kernel.  Shapes cover rows whose w*c
elements are 16-byte aligned (tensor-memory-accelerator staging) and rows that
are not (cp.async staging), ragged tile tails, images smaller than the
filter, and every border mode.
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
HWC = pg.PENCIL_LAYOUT_HWC


def hwc_image(seed, h, w, c, f16=False):
    x = np.ascontiguousarray(np.moveaxis(synth.image_f32(seed, c, h, w), 0, 2))
    return synth.to_f16(x) if f16 else x


def run(img, k, dtype, flags):
    h, w, c = img.shape
    d_in = to_dev(img)
    d_out = torch.empty_like(d_in)
    pg.pencil_conv2d_ex(c, h, w, d_in, k.shape[0], k.shape[1], to_dev(k), d_out, dtype, flags)
    torch.cuda.synchronize()
    return d_out.cpu().numpy()


def run_planar(img, k, dtype, flags=0):
    """The planar kernels on the transposed image, transposed back."""
    pl = np.ascontiguousarray(np.moveaxis(img, 2, 0))
    c, h, w = pl.shape
    d_in = to_dev(pl)
    d_out = torch.empty_like(d_in)
    pg.pencil_conv2d_ex(c, h, w, d_in, k.shape[0], k.shape[1], to_dev(k), d_out, dtype, flags)
    torch.cuda.synchronize()
    return np.moveaxis(d_out.cpu().numpy(), 0, 2)


def check(got, ref, bound, tol, what):
    err = np.abs(got.astype(np.float64) - ref)
    assert np.all(err <= tol * bound), f"{what}: max err/bound {np.max(err / np.maximum(bound, 1e-300)):.3e}"


def bits(a):
    return a.view(np.uint16 if a.dtype == np.float16 else np.uint32)


# (h, w, c): w*c a multiple of 8 (aligned for both storage types), of 4 only,
# and of neither; tails of several tiles; tiny images
SHAPES = [(70, 128, 3), (33, 97, 4), (75, 301, 3), (40, 66, 4), (5, 3, 3), (1, 1, 4), (130, 43, 3)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("f16", [False, True])
def test_interleaved_matches_oracle_and_planar_bits(shape, f16):
    h, w, c = shape
    img = hwc_image(900 + h + w + c, h, w, c, f16)
    dtype = pg.PENCIL_F16 if f16 else pg.PENCIL_F32
    for K in (1, 3, 5, 7, 9, 15):
        k = synth.filter_f32(910 + K, K, K)
        got = run(img, k, dtype, HWC)
        ref, bound = oracle.conv2d_hwc(img, k)
        check(got, ref, bound, F16_TOL if f16 else F32_TOL, f"{shape} K={K} f16={f16}")
        np.testing.assert_array_equal(bits(got), bits(run_planar(img, k, dtype)), err_msg=f"K={K}")
        np.testing.assert_array_equal(bits(got), bits(run(img, k, dtype, HWC | pg.PENCIL_CONV_GENERIC)))


@pytest.mark.parametrize("border", ["zero", "reflect", "mirror", "wrap", "clamp"])
@pytest.mark.parametrize("shape", [(45, 130, 3), (31, 77, 4), (4, 6, 3)])
def test_interleaved_border_modes(border, shape):
    h, w, c = shape
    m = pg.BORDER_MODES[border]
    for f16 in (False, True):
        img = hwc_image(950 + m, h, w, c, f16)
        dtype = pg.PENCIL_F16 if f16 else pg.PENCIL_F32
        for K in (3, 7, 15):
            k = synth.filter_f32(960 + K, K, K)
            got = run(img, k, dtype, HWC | pg.PENCIL_BORDER(m))
            ref, bound = oracle.conv2d_hwc(img, k, border=border)
            check(got, ref, bound, F16_TOL if f16 else F32_TOL, f"{border} {shape} K={K} f16={f16}")
            np.testing.assert_array_equal(bits(got), bits(run_planar(img, k, dtype, pg.PENCIL_BORDER(m))))


@pytest.mark.parametrize("c", [2, 5, 8])
def test_other_channel_counts_take_the_generic_kernel(c):
    img = hwc_image(970 + c, 37, 51, c)
    for k in (synth.filter_f32(971, 5, 5), synth.filter_f32(972, 3, 6)):
        got = run(img, k, pg.PENCIL_F32, HWC)
        ref, bound = oracle.conv2d_hwc(img, k)
        check(got, ref, bound, F32_TOL, f"c={c} {k.shape}")
        np.testing.assert_array_equal(bits(got), bits(run_planar(img, k, pg.PENCIL_F32)))


def test_one_channel_interleaved_is_planar():
    img = hwc_image(975, 50, 70, 1)
    k = synth.filter_f32(976, 7, 7)
    np.testing.assert_array_equal(bits(run(img, k, pg.PENCIL_F32, HWC)), bits(run_planar(img, k, pg.PENCIL_F32)))


@pytest.mark.parametrize("shape", [(70, 128, 3), (75, 301, 3), (33, 97, 4), (29, 40, 5)])
@pytest.mark.parametrize("f16", [False, True])
def test_interleaved_separable(shape, f16):
    """The separable kernel on interleaved images: within tolerance of the
    separable oracle, the same bits as the planar separable kernel."""
    h, w, c = shape
    img = hwc_image(980 + h, h, w, c, f16)
    dtype = pg.PENCIL_F16 if f16 else pg.PENCIL_F32
    for K in (3, 7, 15):
        gx = synth.filter_f32(981 + K, 1, K).ravel()
        gy = synth.filter_f32(982 + K, 1, K).ravel()
        d_in = to_dev(img)
        d_out = torch.empty_like(d_in)
        pg.pencil_conv2d_sep_ex(c, h, w, d_in, K, to_dev(gx), K, to_dev(gy), d_out, dtype, HWC)
        torch.cuda.synchronize()
        got = d_out.cpu().numpy()
        ref, bound = oracle.conv2d_sep_hwc(img, gx, gy)
        check(got, ref, bound, F16_TOL if f16 else F32_TOL, f"sep {shape} K={K} f16={f16}")
        pl = to_dev(np.ascontiguousarray(np.moveaxis(img, 2, 0)))
        po = torch.empty_like(pl)
        pg.pencil_conv2d_sep_ex(c, h, w, pl, K, to_dev(gx), K, to_dev(gy), po, dtype)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(bits(got), bits(np.moveaxis(po.cpu().numpy(), 0, 2)))


@pytest.mark.parametrize("K", [3, 15])
def test_interleaved_full_size_sampled(K):
    """The benchmark's image size, 8192 x 8192 x 3 interleaved FP32, checked
    against the oracle at sampled pixels (every edge pixel of channel 1 and
    20000 random ones)."""
    h, w, c = 8192, 8192, 3
    img = hwc_image(990, h, w, c)
    k = synth.filter_f32(991 + K, K, K)
    d_in = to_dev(img)
    d_out = torch.empty_like(d_in)
    pg.pencil_conv2d_ex(c, h, w, d_in, K, K, to_dev(k), d_out, pg.PENCIL_F32, HWC)
    torch.cuda.synchronize()
    r = np.random.default_rng(K)
    pts = [np.stack([r.integers(0, c, 20000), r.integers(0, h, 20000), r.integers(0, w, 20000)], axis=1)]
    for i in (0, h - 1):
        pts.append(np.stack([np.ones(w, np.int64), np.full(w, i), np.arange(w)], axis=1))
    for j in (0, w - 1):
        pts.append(np.stack([np.ones(h, np.int64), np.arange(h), np.full(h, j)], axis=1))
    pts = np.concatenate(pts).astype(np.int64)
    want, bound = oracle.conv2d_hwc_points(img, k, pts)
    p = torch.from_numpy(pts).to(d_out.device)
    got = d_out[p[:, 1], p[:, 2], p[:, 0]].double().cpu().numpy()
    check(got, want, bound, F32_TOL, f"8192^2 x 3 interleaved K={K}")
