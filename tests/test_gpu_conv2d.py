"""GPU parity of the conv2d kernels against the FP64 oracle, through the C ABI.

Tolerances (per pixel, bound = sum |k| |x| from the oracle):
  FP32 storage: |gpu - oracle| <= 1e-6 * bound;
  FP16 storage: |gpu - oracle(binary16 input)| <= 2^-10 * bound.
Kernels that share the fixed per-pixel order must agree bit for bit.
"""
import numpy as np
import pytest

import oracle
import paper_1302_5586_gb300 as pg
import synth
from gpu_util import dev, gather, sample_points, to_dev, torch

pytestmark = pytest.mark.gpu

F32_TOL = 1e-6
F16_TOL = 2.0 ** -10


def run_conv(img, k, dtype=pg.PENCIL_F32, flags=0):
    c, h, w = img.shape
    d_in = to_dev(img)
    d_k = to_dev(k)
    d_out = torch.empty_like(d_in)
    pg.pencil_conv2d_ex(c, h, w, d_in, k.shape[0], k.shape[1], d_k, d_out, dtype, flags)
    torch.cuda.synchronize()
    return d_out


def assert_within(gpu, ref, bound, tol, what):
    err = np.abs(gpu.astype(np.float64) - ref)
    ratio = np.max(err / np.maximum(bound, 1e-300))
    assert np.all(err <= tol * bound), f"{what}: max err/bound {ratio:.3e} > {tol:.3e}"
    return ratio


SHAPES = [(2, 75, 301), (1, 200, 520), (3, 33, 128), (1, 1, 1), (1, 5, 3), (2, 1, 77), (1, 64, 1)]


@pytest.mark.parametrize("K", [1, 3, 5, 7, 9, 11, 13, 15])
@pytest.mark.parametrize("shape", SHAPES)
def test_direct_f32_matches_oracle(K, shape):
    c, h, w = shape
    img = synth.image_f32(1000 + K, c, h, w)
    k = synth.filter_f32(2000 + K, K, K)
    out = run_conv(img, k).cpu().numpy()
    ref, bound = oracle.conv2d(img, k)
    assert_within(out, ref, bound, F32_TOL, f"K={K} shape={shape}")


@pytest.mark.parametrize("K", [1, 3, 5, 7, 15])
@pytest.mark.parametrize("shape", [(2, 75, 301), (1, 200, 520), (1, 3, 2), (2, 40, 264)])
def test_specialised_and_generic_kernels_agree_bitwise(K, shape):
    c, h, w = shape
    img = synth.image_f32(31 + K, c, h, w)
    k = synth.filter_f32(41 + K, K, K)
    a = run_conv(img, k).cpu().numpy()
    b = run_conv(img, k, flags=pg.PENCIL_CONV_GENERIC).cpu().numpy()
    np.testing.assert_array_equal(a.view(np.uint32), b.view(np.uint32))
    img16 = synth.to_f16(img)
    a16 = run_conv(img16, k, pg.PENCIL_F16).cpu().numpy()
    b16 = run_conv(img16, k, pg.PENCIL_F16, pg.PENCIL_CONV_GENERIC).cpu().numpy()
    np.testing.assert_array_equal(a16.view(np.uint16), b16.view(np.uint16))


# Planar images of at least 2^20 elements whose rows are not 16-byte aligned
# (w % 4 = 1, 2, 3) take the row-staged TMA kernels (odd widths, sides up to
# 5) or the cp.async kernels compiled for unaligned rows (even widths, larger
# sides); the generic kernel shares the per-pixel order, so each agrees with
# it bit for bit, and the oracle checks both.
ROW_SHAPES = [(1, 1031, 1029), (2, 767, 1366), (1, 1100, 1023)]


@pytest.mark.parametrize("K", [1, 3, 5, 7, 9, 11, 13, 15])
@pytest.mark.parametrize("border", ["clamp", "zero"])
@pytest.mark.parametrize("shape", ROW_SHAPES)
def test_row_staged_unaligned_rows(K, border, shape):
    c, h, w = shape
    assert c * h * w >= 1 << 20 and w % 4 != 0
    img = synth.image_f32(900 + K + w, c, h, w)
    k = synth.filter_f32(910 + K, K, K)
    m = pg.PENCIL_BORDER(pg.BORDER_MODES[border])
    for dt, img_t, tol, view in ((pg.PENCIL_F32, img, F32_TOL, np.uint32),
                                 (pg.PENCIL_F16, synth.to_f16(img), F16_TOL, np.uint16)):
        a = run_conv(img_t, k, dt, m).cpu().numpy()
        b = run_conv(img_t, k, dt, m | pg.PENCIL_CONV_GENERIC).cpu().numpy()
        np.testing.assert_array_equal(a.view(view), b.view(view))
        ref, bound = oracle.conv2d(img_t, k, border=border)
        assert_within(a, ref, bound, tol, f"{border} K={K} {shape} dtype={dt}")


@pytest.mark.parametrize("kh,kw", [(4, 6), (2, 1), (1, 9), (31, 3), (17, 17), (3, 5)])
def test_generic_sizes_match_oracle(kh, kw):
    img = synth.image_f32(77, 2, 45, 70)
    k = synth.filter_f32(78, kh, kw)
    out = run_conv(img, k).cpu().numpy()
    ref, bound = oracle.conv2d(img, k)
    assert_within(out, ref, bound, F32_TOL, f"{kh}x{kw}")


@pytest.mark.parametrize("K", [1, 3, 5, 7, 9, 15])
@pytest.mark.parametrize("shape", [(2, 75, 304), (1, 130, 257)])
def test_direct_f16_matches_oracle(K, shape):
    c, h, w = shape
    img16 = synth.image_f16(300 + K, c, h, w)
    k = synth.filter_f32(400 + K, K, K)
    out = run_conv(img16, k, pg.PENCIL_F16).cpu().numpy()
    ref, bound = oracle.conv2d(img16, k)
    assert_within(out, ref, bound, F16_TOL, f"f16 K={K}")
    # the binary16 result is the rounding of an FP32 value close to the exact sum:
    # within one binary16 ulp of the exact sum rounded to nearest even
    want = oracle.f64_to_f16(ref).view(np.float16).astype(np.float64)
    ulp = np.spacing(np.abs(want).astype(np.float16)).astype(np.float64)
    assert np.all(np.abs(out.astype(np.float64) - want) <= ulp)


def test_delta_filter_is_identity_bitwise():
    img = synth.image_f32(5, 2, 67, 130)
    for K in (1, 3, 9, 15):
        k = np.zeros((K, K), dtype=np.float32)
        k[K // 2, K // 2] = 1.0
        out = run_conv(img, k).cpu().numpy()
        np.testing.assert_array_equal(out, img)
        img16 = synth.to_f16(img)
        out16 = run_conv(img16, k, pg.PENCIL_F16).cpu().numpy()
        np.testing.assert_array_equal(out16.view(np.uint16), img16.view(np.uint16))


@pytest.mark.parametrize("K,p,q", [(3, 0, 0), (7, 40, 129), (15, 13, 3), (15, 66, 131), (5, 33, 64)])
def test_nan_footprint_matches_oracle(K, p, q):
    """One NaN poisons exactly the pixels whose clamped window reads it."""
    img = synth.image_f32(9, 1, 67, 132)
    img[0, p, q] = np.nan
    k = synth.filter_f32(10, K, K)
    out = run_conv(img, k).cpu().numpy()
    ref, _ = oracle.conv2d(img, k)
    np.testing.assert_array_equal(np.isnan(out), np.isnan(ref))


@pytest.mark.parametrize("K", [3, 5, 7, 9, 11, 13, 15])
@pytest.mark.parametrize("shape", [(2, 75, 301), (1, 200, 520), (1, 2, 3), (1, 130, 258)])
def test_separable_matches_oracle(K, shape):
    c, h, w = shape
    gx = synth.gaussian_taps_f32(K // 2, 1.0 + K / 5)
    gy = synth.filter_f32(55 + K, 1, K).ravel()
    img = synth.image_f32(60 + K, c, h, w)
    d_in = to_dev(img)
    d_out = torch.empty_like(d_in)
    pg.pencil_conv2d_sep_ex(c, h, w, d_in, K, to_dev(gx), K, to_dev(gy), d_out, pg.PENCIL_F32)
    torch.cuda.synchronize()
    ref, bound = oracle.conv2d_sep(img, gx, gy)
    assert_within(d_out.cpu().numpy(), ref, bound, F32_TOL, f"sep K={K}")
    img16 = synth.to_f16(img)
    d16 = to_dev(img16)
    o16 = torch.empty_like(d16)
    pg.pencil_conv2d_sep_ex(c, h, w, d16, K, to_dev(gx), K, to_dev(gy), o16, pg.PENCIL_F16)
    torch.cuda.synchronize()
    ref16, bound16 = oracle.conv2d_sep(img16, gx, gy)
    assert_within(o16.cpu().numpy(), ref16, bound16, F16_TOL, f"sep f16 K={K}")


@pytest.mark.parametrize("kx,ky", [(3, 7), (1, 5), (15, 2)])
def test_separable_unequal_sides(kx, ky):
    gx = synth.filter_f32(1, 1, kx).ravel()
    gy = synth.filter_f32(2, 1, ky).ravel()
    img = synth.image_f32(3, 2, 70, 90)
    d_in = to_dev(img)
    d_out = torch.empty_like(d_in)
    pg.pencil_conv2d_sep_ex(2, 70, 90, d_in, kx, to_dev(gx), ky, to_dev(gy), d_out, pg.PENCIL_F32)
    torch.cuda.synchronize()
    ref, bound = oracle.conv2d_sep(img, gx, gy)
    assert_within(d_out.cpu().numpy(), ref, bound, F32_TOL, f"sep {kx}x{ky}")


@pytest.mark.parametrize("border", ["zero", "reflect", "mirror", "wrap", "clamp"])
@pytest.mark.parametrize("shape", [(2, 75, 301), (1, 5, 3), (1, 130, 264)])
def test_border_modes_match_oracle(border, shape):
    """Every border mode, specialised / generic / separable kernels, against the
    oracle's mode; specialised and generic agree bit for bit."""
    c, h, w = shape
    m = pg.BORDER_MODES[border]
    img = synth.image_f32(700 + m, c, h, w)
    for K in (3, 5, 7, 15):
        k = synth.filter_f32(710 + K, K, K)
        a = run_conv(img, k, flags=pg.PENCIL_BORDER(m)).cpu().numpy()
        b = run_conv(img, k, flags=pg.PENCIL_BORDER(m) | pg.PENCIL_CONV_GENERIC).cpu().numpy()
        np.testing.assert_array_equal(a.view(np.uint32), b.view(np.uint32))
        ref, bound = oracle.conv2d(img, k, border=border)
        assert_within(a, ref, bound, F32_TOL, f"{border} K={K}")
        img16 = synth.to_f16(img)
        a16 = run_conv(img16, k, pg.PENCIL_F16, pg.PENCIL_BORDER(m)).cpu().numpy()
        b16 = run_conv(img16, k, pg.PENCIL_F16, pg.PENCIL_BORDER(m) | pg.PENCIL_CONV_GENERIC).cpu().numpy()
        np.testing.assert_array_equal(a16.view(np.uint16), b16.view(np.uint16))
        ref16, bound16 = oracle.conv2d(img16, k, border=border)
        assert_within(a16, ref16, bound16, F16_TOL, f"f16 {border} K={K}")
    k = synth.filter_f32(720, 4, 6)
    g = run_conv(img, k, flags=pg.PENCIL_BORDER(m)).cpu().numpy()
    ref, bound = oracle.conv2d(img, k, border=border)
    assert_within(g, ref, bound, F32_TOL, f"{border} 4x6")
    for K in (5, 15):
        gx = synth.filter_f32(730 + K, 1, K).ravel()
        gy = synth.filter_f32(740 + K, 1, K).ravel()
        d_in = to_dev(img)
        d_out = torch.empty_like(d_in)
        pg.pencil_conv2d_sep_ex(c, h, w, d_in, K, to_dev(gx), K, to_dev(gy), d_out, pg.PENCIL_F32,
                                pg.PENCIL_BORDER(m))
        torch.cuda.synchronize()
        k2 = np.outer(gy.astype(np.float64), gx.astype(np.float64))
        # the separable definition under the border mode: the 2-D oracle with the
        # exact outer-product weights is the same sum (FP32 weights differ by
        # rounding, so compare with the separable oracle in clamp mode and with the
        # 2-D oracle of rounded weights plus the rounding slack otherwise)
        ref, bound = oracle.conv2d(img, k2.astype(np.float32), border=border)
        slack = np.abs(k2 - k2.astype(np.float32).astype(np.float64)).sum() * np.abs(img).max()
        err = np.abs(d_out.cpu().numpy().astype(np.float64) - ref)
        assert np.all(err <= F32_TOL * bound + slack), f"sep {border} K={K}"


def test_plain_call_accepts_host_and_device_memory():
    img = synth.image_f32(21, 1, 97, 203)[0]
    k = synth.filter_f32(22, 5, 5)
    out_host = np.empty_like(img)
    pg.pencil_conv2d(97, 203, img, 5, 5, k, out_host)
    d_in, d_k = to_dev(img), to_dev(k)
    d_out = torch.empty_like(d_in)
    pg.pencil_conv2d(97, 203, d_in, 5, 5, d_k, d_out)
    np.testing.assert_array_equal(out_host, d_out.cpu().numpy())
    pinned = torch.from_numpy(img).pin_memory()
    out_pinned = torch.empty_like(pinned).pin_memory()
    pg.pencil_conv2d(97, 203, pinned, 5, 5, k, out_pinned)
    np.testing.assert_array_equal(out_host, out_pinned.numpy())
    ref, bound = oracle.conv2d(img, k)
    assert_within(out_host[None], ref, bound, F32_TOL, "plain host")


def test_plain_separable_call_host_memory():
    img = synth.image_f32(24, 1, 90, 130)[0]
    g = synth.gaussian_taps_f32(7, 3.0)
    out = np.empty_like(img)
    pg.pencil_conv2d_sep(90, 130, img, 15, g, 15, g, out)
    d_in = to_dev(img[None])
    d_out = torch.empty_like(d_in)
    pg.pencil_conv2d_sep_ex(1, 90, 130, d_in, 15, to_dev(g), 15, to_dev(g), d_out, pg.PENCIL_F32)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out, d_out.cpu().numpy()[0])


@pytest.mark.parametrize("K", [3, 15])
def test_plain_call_banded_host_path_is_bitwise_the_single_launch(K):
    """Host buffers go through row bands pipelined over several streams; the
    result must be the same bits as one launch over the device image."""
    h, w = 1500, 8192                      # several bands and a ragged last band
    img = synth.image_f32(90 + K, 1, h, w)[0]
    k = synth.filter_f32(91 + K, K, K)
    d_in, d_k = to_dev(img), to_dev(k)
    d_out = torch.empty_like(d_in)
    pg.pencil_conv2d(h, w, d_in, K, K, d_k, d_out)
    ref = d_out.cpu().numpy()
    pinned = torch.from_numpy(img).pin_memory()
    out_p = torch.empty_like(pinned).pin_memory()
    pg.pencil_conv2d(h, w, pinned, K, K, k, out_p)
    np.testing.assert_array_equal(out_p.numpy().view(np.uint32), ref.view(np.uint32))
    out_m = np.empty_like(img)             # device input, pageable host output
    pg.pencil_conv2d(h, w, d_in, K, K, d_k, out_m)
    np.testing.assert_array_equal(out_m.view(np.uint32), ref.view(np.uint32))
    g = synth.gaussian_taps_f32(K // 2, 2.0)
    d_sep = torch.empty_like(d_in)
    pg.pencil_conv2d_sep(h, w, d_in, K, to_dev(g), K, to_dev(g), d_sep)
    out_s = torch.empty_like(pinned).pin_memory()
    pg.pencil_conv2d_sep(h, w, pinned, K, g, K, g, out_s)
    np.testing.assert_array_equal(out_s.numpy().view(np.uint32), d_sep.cpu().numpy().view(np.uint32))


def test_restrict_and_memory_kind_errors():
    d = torch.zeros(4, 64, 64, device=dev())
    k = torch.ones(3, 3, device=dev()) / 9
    with pytest.raises(pg.PencilError) as e:
        pg.pencil_conv2d_ex(1, 64, 64, d[0], 3, 3, k, d[0], pg.PENCIL_F32)
    assert e.value.name == "PENCIL_ERR_ALIAS"
    with pytest.raises(pg.PencilError) as e:  # partial overlap: out starts inside in
        pg.pencil_conv2d_ex(2, 64, 64, d[0], 3, 3, k, d[1], pg.PENCIL_F32)
    assert e.value.name == "PENCIL_ERR_ALIAS"
    host = np.zeros((64, 64), dtype=np.float32)
    with pytest.raises(pg.PencilError) as e:
        pg.pencil_conv2d_ex(1, 64, 64, host, 3, 3, k, d[1], pg.PENCIL_F32)
    assert e.value.name == "PENCIL_ERR_PTR"
    pg.pencil_conv2d_ex(1, 64, 64, d[0], 3, 3, k, d[1], pg.PENCIL_F32)  # disjoint: fine
    torch.cuda.synchronize()


def test_stream_ordered_on_a_side_stream():
    img = synth.image_f32(71, 3, 128, 256)
    k = synth.filter_f32(72, 7, 7)
    s = torch.cuda.Stream()
    d_in = to_dev(img)
    d_k = to_dev(k)
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        d_out = torch.empty_like(d_in)
        pg.pencil_conv2d_ex(3, 128, 256, d_in, 7, 7, d_k, d_out, pg.PENCIL_F32, 0, s)
    s.synchronize()
    ref = run_conv(img, k).cpu().numpy()
    np.testing.assert_array_equal(d_out.cpu().numpy(), ref)


@pytest.mark.parametrize("K", [3, 7, 15])
def test_full_size_8192x8192x3_sampled(K):
    """The 8192 x 8192 x 3 workload in the benchmark's launch configuration,
    checked at 50k random pixels plus every pixel of the outer two rows and
    columns of the last channel."""
    c, h, w = 3, 8192, 8192
    img = synth.image_f32(synth.SEEDS["conv8192x3"], c, h, w)
    k = synth.filter_f32(synth.SEEDS["conv8192x3"] + K, K, K)
    out = run_conv(img, k)
    pts = sample_points(K, c, h, w, 50000)
    ref, bound = oracle.conv2d_points(img, k, pts)
    assert_within(gather(out, pts), ref, bound, F32_TOL, f"full K={K}")


def test_full_size_gaussian_separable_sampled():
    c, h, w = 3, 8192, 8192
    img = synth.image_f32(synth.SEEDS["conv8192x3"], c, h, w)
    g = synth.gaussian_taps_f32(7, 3.0)
    d_in = to_dev(img)
    d_out = torch.empty_like(d_in)
    pg.pencil_conv2d_sep_ex(c, h, w, d_in, 15, to_dev(g), 15, to_dev(g), d_out, pg.PENCIL_F32)
    torch.cuda.synchronize()
    pts = sample_points(99, c, h, w, 50000)
    ref, bound = oracle.conv2d_sep_points(img, g, g, pts)
    assert_within(gather(d_out, pts), ref, bound, F32_TOL, "gaussian sep full")


def test_small_workload_512x512_5x5_whole_image():
    """The small plain workload exactly: one 512 x 512 FP32 image with pixels
    U[0,1) and a 5 x 5 filter of normalised U[0,1) weights, clamp-to-edge,
    every output pixel against the oracle (1e-6 * sum|k||x|), through the
    stream-ordered call and the synchronous plain call on host arrays (the
    same bits)."""
    img = synth.image_f32(synth.SEEDS["conv512"], 1, 512, 512)
    k = synth.filter_f32(synth.SEEDS["conv512"] + 1, 5, 5)
    got = run_conv(img, k).cpu().numpy()
    ref, bound = oracle.conv2d(img, k)
    assert_within(got, ref, bound, F32_TOL, "512x512 5x5")
    host_out = np.empty((512, 512), dtype=np.float32)
    pg.pencil_conv2d(512, 512, img[0], 5, 5, k, host_out)
    np.testing.assert_array_equal(host_out.view(np.uint32), got[0].view(np.uint32))
