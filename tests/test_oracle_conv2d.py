"""Pins of the FP64 conv2d oracle against things other than itself.

Each pin is chosen so that a plausible slip in the oracle (a flipped filter, a
wrong anchor, a transposed index, a dropped clamp, a lost term) fails at least
one of them.  Library routines used as references: scipy.ndimage.correlate
with mode='nearest' (clamp-to-edge correlation) and numpy edge padding.
"""
import json
import os

import numpy as np
import pytest
import scipy.ndimage as ndi
from numpy.lib.stride_tricks import sliding_window_view

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rng(seed):
    return np.random.default_rng(seed)


@pytest.mark.parametrize("seed", range(40))
def test_matches_scipy_nearest_correlate(seed):
    """scipy's clamp ('nearest') correlation on tiny random shapes, incl. even filter sides."""
    r = _rng(seed)
    h, w = r.integers(1, 10, size=2)
    kh, kw = r.integers(1, 8, size=2)
    img = r.standard_normal((h, w)).astype(np.float32)
    k = r.standard_normal((kh, kw)).astype(np.float32)
    out, bound = oracle.conv2d(img, k)
    ref = ndi.correlate(img.astype(np.float64), k.astype(np.float64), mode="nearest")
    assert np.all(np.abs(out[0] - ref) <= 1e-13 * bound[0] + 1e-300)


@pytest.mark.parametrize("seed", range(20))
def test_matches_edge_padding_brute_force(seed):
    """Edge-replicate padding then a 'valid' window sum: a second, independent route."""
    r = _rng(100 + seed)
    c = int(r.integers(1, 4))
    h, w = r.integers(1, 9, size=2)
    kh, kw = r.integers(1, 8, size=2)
    img = r.random((c, h, w)).astype(np.float32)
    k = r.random((kh, kw)).astype(np.float32)
    out, _ = oracle.conv2d(img, k)
    ah, aw = kh // 2, kw // 2
    pad = np.pad(img.astype(np.float64), ((0, 0), (ah, kh - 1 - ah), (aw, kw - 1 - aw)), mode="edge")
    win = sliding_window_view(pad, (kh, kw), axis=(1, 2))  # [c][h][w][kh][kw]
    ref = np.einsum("chwab,ab->chw", win, k.astype(np.float64))
    np.testing.assert_allclose(out, ref, rtol=1e-13, atol=1e-13)


def test_golden_hand_cases():
    with open(os.path.join(GOLDEN, "conv2d_hand.json")) as f:
        cases = json.load(f)["cases"]
    for cs in cases:
        img = np.array(cs["image"], dtype=np.float32)
        k = np.array(cs["filter"], dtype=np.float32)
        out, _ = oracle.conv2d(img, k)
        np.testing.assert_array_equal(out[0], np.array(cs["expected"], dtype=np.float64), err_msg=cs["name"])


@pytest.mark.parametrize("kh,kw", [(1, 1), (3, 3), (5, 3), (2, 4), (15, 15)])
def test_delta_filter_is_identity(kh, kw):
    """A unit weight at the anchor returns the input bit for bit (FP32 and binary16)."""
    img = synth.image_f32(7, 2, 13, 17)
    k = np.zeros((kh, kw), dtype=np.float32)
    k[kh // 2, kw // 2] = 1.0
    out, _ = oracle.conv2d(img, k)
    np.testing.assert_array_equal(out, img.astype(np.float64))
    img16 = synth.to_f16(img)
    out16, _ = oracle.conv2d(img16, k)
    np.testing.assert_array_equal(out16, img16.astype(np.float64))


def test_normalised_filter_preserves_constant():
    """Dyadic weights summing to 1 on a dyadic constant image give the constant exactly."""
    k = np.array([[0.125, 0.25, 0.125], [0.0625, 0.25, 0.0625], [0.0625, 0.0625, 0.0]], dtype=np.float32)
    assert k.astype(np.float64).sum() == 1.0
    img = np.full((1, 6, 5), 0.75, dtype=np.float32)
    out, _ = oracle.conv2d(img, k)
    np.testing.assert_array_equal(out, 0.75)
    # random normalised weights: constant within rounding
    k2 = synth.filter_f32(3, 7, 5)
    out2, _ = oracle.conv2d(np.full((1, 9, 4), 0.3, dtype=np.float32), k2)
    s = k2.astype(np.float64).sum()
    np.testing.assert_allclose(out2, np.float64(np.float32(0.3)) * s, rtol=1e-14)


@pytest.mark.parametrize("seed", range(6))
def test_separable_equals_two_1d_passes(seed):
    """outer(gy, gx) equals a 1 x kx pass followed by a ky x 1 pass (the clamp is per axis)."""
    r = _rng(200 + seed)
    h, w = r.integers(1, 12, size=2)
    kx, ky = r.integers(1, 9, size=2)
    gx = r.random(kx).astype(np.float32)
    gy = r.random(ky).astype(np.float32)
    img = r.random((h, w)).astype(np.float32)
    sep, _ = oracle.conv2d_sep(img, gx, gy)
    # pass 1 along rows with the FP32 image, pass 2 along columns on the FP64 result
    p1, _ = oracle.conv2d(img, gx[None, :])
    ah = ky // 2
    rows = np.clip(np.arange(h)[:, None] + np.arange(ky)[None, :] - ah, 0, h - 1)
    p2 = np.einsum("ia,iaj->ij", np.broadcast_to(gy.astype(np.float64), (h, ky)), p1[0][rows])
    np.testing.assert_allclose(sep[0], p2, rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("kh,kw,p,q", [(3, 3, 5, 6), (5, 3, 6, 4), (4, 6, 7, 7), (7, 1, 6, 3)])
def test_impulse_response_pins_orientation_and_anchor(kh, kw, p, q):
    """One 1 at (p,q): out[p-a+ah][q-b+aw] = k[a][b] (correlation, anchor floor(k/2))."""
    h, w = 14, 15
    img = np.zeros((h, w), dtype=np.float32)
    img[p, q] = 1.0
    k = (np.arange(kh * kw, dtype=np.float32) + 1.0).reshape(kh, kw)
    out, _ = oracle.conv2d(img, k)
    ah, aw = kh // 2, kw // 2
    expect = np.zeros((h, w))
    for a in range(kh):
        for b in range(kw):
            expect[p - a + ah, q - b + aw] = k[a, b]
    np.testing.assert_array_equal(out[0], expect)


@pytest.mark.parametrize("h,w,kh,kw,p,q", [(9, 8, 3, 3, 0, 0), (9, 8, 5, 3, 8, 3), (6, 11, 7, 5, 2, 10),
                                            (5, 5, 9, 9, 2, 2), (10, 10, 4, 2, 0, 9)])
def test_nan_footprint(h, w, kh, kw, p, q):
    """A NaN at (p,q) poisons exactly the outputs whose clamped window reads (p,q)."""
    img = np.ones((h, w), dtype=np.float32)
    img[p, q] = np.nan
    k = np.ones((kh, kw), dtype=np.float32)
    out, _ = oracle.conv2d(img, k)
    ah, aw = kh // 2, kw // 2
    expect = np.zeros((h, w), dtype=bool)
    for i in range(h):
        rows = {min(max(i + a - ah, 0), h - 1) for a in range(kh)}
        for j in range(w):
            cols = {min(max(j + b - aw, 0), w - 1) for b in range(kw)}
            expect[i, j] = p in rows and q in cols
    np.testing.assert_array_equal(np.isnan(out[0]), expect)


def test_single_pixel_image():
    """A 1x1 image is replicated everywhere: out = in * sum(k)."""
    k = synth.filter_f32(11, 5, 7) * np.float32(3.0)
    out, bound = oracle.conv2d(np.array([[0.5]], dtype=np.float32), k)
    assert out[0, 0, 0] == pytest.approx(0.5 * k.astype(np.float64).sum(), rel=1e-15)
    assert bound[0, 0, 0] == pytest.approx(out[0, 0, 0], rel=1e-15)


def test_linear_ramp_reproduced_by_point_symmetric_filter():
    """Away from the borders a point-symmetric normalised filter maps a ramp to itself."""
    h, w, kh, kw = 20, 23, 5, 7
    base = synth.filter_f32(5, kh, kw).astype(np.float64)
    k = (base + base[::-1, ::-1]) / 2
    k = (k / k.sum()).astype(np.float32)
    k = (k + k[::-1, ::-1]) / np.float32(2)  # exactly point symmetric in FP32
    i, j = np.mgrid[0:h, 0:w]
    img = (0.25 * i + 0.125 * j + 1.0).astype(np.float32)
    out, _ = oracle.conv2d(img, k)
    ah, aw = kh // 2, kw // 2
    inner = (slice(ah, h - ah), slice(aw, w - aw))
    s = k.astype(np.float64).sum()
    np.testing.assert_allclose(out[0][inner], img[inner].astype(np.float64) * s, rtol=1e-13)


def test_bound_equals_value_for_nonnegative_data():
    img = synth.image_f32(9, 2, 11, 7)
    k = synth.filter_f32(9, 3, 5)
    out, bound = oracle.conv2d(img, k)
    np.testing.assert_allclose(out, bound, rtol=1e-15)
    # and |out| <= bound with mixed signs
    img2 = (img - np.float32(0.5)).astype(np.float32)
    k2 = (k - np.float32(0.05)).astype(np.float32)
    out2, bound2 = oracle.conv2d(img2, k2)
    assert np.all(np.abs(out2) <= bound2 * (1 + 1e-15))


def test_linearity():
    r = _rng(5)
    x = r.random((2, 10, 9)).astype(np.float32)
    y = r.random((2, 10, 9)).astype(np.float32)
    k = r.random((3, 5)).astype(np.float32)
    ox, _ = oracle.conv2d(x, k)
    oy, _ = oracle.conv2d(y, k)
    oxy, _ = oracle.conv2d((x.astype(np.float64) + 2 * y.astype(np.float64)).astype(np.float32), k)
    # x + 2y rounded to FP32 first, so compare against the rounded input's own linear combination
    xy32 = (x.astype(np.float64) + 2 * y.astype(np.float64)).astype(np.float32).astype(np.float64)
    exact = ndi.correlate(xy32[0], k.astype(np.float64), mode="nearest")
    np.testing.assert_allclose(oxy[0], exact, rtol=1e-13)
    np.testing.assert_allclose(ox + 2 * oy, oxy, rtol=1e-6)


def test_channels_are_independent_planes():
    img = synth.image_f32(21, 3, 8, 9)
    k = synth.filter_f32(21, 3, 3)
    out, _ = oracle.conv2d(img, k)
    for c in range(3):
        oc, _ = oracle.conv2d(img[c], k)
        np.testing.assert_array_equal(out[c], oc[0])


def test_points_match_full_image():
    img = synth.image_f32(4, 2, 31, 29)
    k = synth.filter_f32(4, 7, 5)
    out, bound = oracle.conv2d(img, k)
    r = _rng(4)
    pts = np.stack([r.integers(0, 2, 50), r.integers(0, 31, 50), r.integers(0, 29, 50)], axis=1)
    po, pb = oracle.conv2d_points(img, k, pts)
    np.testing.assert_array_equal(po, out[pts[:, 0], pts[:, 1], pts[:, 2]])
    np.testing.assert_array_equal(pb, bound[pts[:, 0], pts[:, 1], pts[:, 2]])
    with pytest.raises(ValueError):
        oracle.conv2d_points(img, k, np.array([[0, 31, 0]]))


def test_separable_points_match_full_image():
    img = synth.image_f32(14, 2, 23, 19)
    gx = synth.filter_f32(15, 1, 5).ravel()
    gy = synth.filter_f32(16, 1, 3).ravel()
    out, bound = oracle.conv2d_sep(img, gx, gy)
    r = _rng(14)
    pts = np.stack([r.integers(0, 2, 40), r.integers(0, 23, 40), r.integers(0, 19, 40)], axis=1)
    po, pb = oracle.conv2d_sep_points(img, gx, gy, pts)
    np.testing.assert_array_equal(po, out[pts[:, 0], pts[:, 1], pts[:, 2]])
    np.testing.assert_array_equal(pb, bound[pts[:, 0], pts[:, 1], pts[:, 2]])


def test_binary16_input_is_widened_exactly():
    img = synth.image_f16(8, 1, 12, 10)
    k = synth.filter_f32(8, 3, 3)
    out, _ = oracle.conv2d(img, k)
    ref = ndi.correlate(img[0].astype(np.float64), k.astype(np.float64), mode="nearest")
    np.testing.assert_allclose(out[0], ref, rtol=1e-13)


def test_rejects_bad_arguments():
    with pytest.raises(ValueError):
        oracle.conv2d(np.zeros((1, 0, 3), dtype=np.float32), np.ones((3, 3), dtype=np.float32))
    with pytest.raises(ValueError):
        oracle.conv2d(np.zeros((1, 2, 3), dtype=np.float32), np.ones((0, 3), dtype=np.float32))


SCIPY_MODE = {"clamp": "nearest", "zero": "constant", "reflect": "reflect", "mirror": "mirror", "wrap": "wrap"}


@pytest.mark.parametrize("border", ["clamp", "zero", "reflect", "mirror", "wrap"])
@pytest.mark.parametrize("seed", range(12))
def test_border_modes_match_scipy(border, seed):
    """Each border mode against scipy.ndimage.correlate's mode of the same
    meaning, including filters larger than the image (repeated reflection)."""
    r = _rng(300 + seed)
    h, w = r.integers(1, 9, size=2)
    kh, kw = r.integers(1, 12, size=2)
    img = r.standard_normal((h, w)).astype(np.float32)
    k = r.standard_normal((kh, kw)).astype(np.float32)
    out, bound = oracle.conv2d(img, k, border=border)
    ref = ndi.correlate(img.astype(np.float64), k.astype(np.float64), mode=SCIPY_MODE[border], cval=0.0)
    assert np.all(np.abs(out[0] - ref) <= 1e-13 * bound[0] + 1e-300)


def test_border_modes_hand_row():
    """One row [1, 2, 3], filter [1, 10, 100, 1000, 10000] (anchor 2): the two
    columns past each edge read, per mode: clamp 1 1 | 3 3, zero 0 0 | 0 0,
    reflect 2 1 | 3 2, mirror 3 2 | 2 1, wrap 2 3 | 1 2."""
    img = np.array([[1, 2, 3]], dtype=np.float32)
    k = np.array([[1, 10, 100, 1000, 10000]], dtype=np.float32)
    ext = {"clamp": [1, 1, 1, 2, 3, 3, 3], "zero": [0, 0, 1, 2, 3, 0, 0], "reflect": [2, 1, 1, 2, 3, 3, 2],
           "mirror": [3, 2, 1, 2, 3, 2, 1], "wrap": [2, 3, 1, 2, 3, 1, 2]}
    for mode, e in ext.items():
        want = [sum(k[0, b] * e[j + b] for b in range(5)) for j in range(3)]
        out, _ = oracle.conv2d(img, k, border=mode)
        np.testing.assert_array_equal(out[0, 0], want, err_msg=mode)


# ------------------------------------------------ interleaved [h][w][c] layout

@pytest.mark.parametrize("border", ["clamp", "zero", "reflect", "mirror", "wrap"])
@pytest.mark.parametrize("seed", range(8))
def test_interleaved_layout_matches_scipy_per_channel(border, seed):
    """Channel ch of an interleaved image is scipy's correlation of the slice
    x[:, :, ch] under the same border mode (channels never mix)."""
    r = _rng(700 + seed)
    h, w = r.integers(1, 9, size=2)
    c = int(r.integers(1, 6))
    kh, kw = r.integers(1, 10, size=2)
    img = r.standard_normal((h, w, c)).astype(np.float32)
    k = r.standard_normal((kh, kw)).astype(np.float32)
    out, bound = oracle.conv2d_hwc(img, k, border=border)
    assert out.shape == (h, w, c)
    for ch in range(c):
        ref = ndi.correlate(img[:, :, ch].astype(np.float64), k.astype(np.float64), mode=SCIPY_MODE[border],
                            cval=0.0)
        assert np.all(np.abs(out[:, :, ch] - ref) <= 1e-13 * bound[:, :, ch] + 1e-300), (border, ch)


@pytest.mark.parametrize("seed", range(6))
def test_interleaved_layout_is_the_planar_definition_transposed(seed):
    """The interleaved result is the planar result of the transposed image,
    bit for bit (the same per-pixel sum), for FP32 and binary16 inputs."""
    r = _rng(800 + seed)
    h, w, c = int(r.integers(1, 12)), int(r.integers(1, 12)), int(r.integers(1, 5))
    k = r.standard_normal((3, 5)).astype(np.float32)
    for img in (r.standard_normal((h, w, c)).astype(np.float32),
                r.standard_normal((h, w, c)).astype(np.float16)):
        out, bound = oracle.conv2d_hwc(img, k)
        pl, pb = oracle.conv2d(np.ascontiguousarray(np.moveaxis(img, 2, 0)), k)
        np.testing.assert_array_equal(np.moveaxis(out, 2, 0), pl)
        np.testing.assert_array_equal(np.moveaxis(bound, 2, 0), pb)


def test_interleaved_impulse_stays_in_its_channel():
    """One 1 at (p, q) of channel 1 of a 3-channel image: channel 1 shows the
    filter (correlation orientation, anchor k/2), the other channels stay 0."""
    img = np.zeros((9, 11, 3), dtype=np.float32)
    img[4, 5, 1] = 1.0
    k = np.arange(1, 16, dtype=np.float32).reshape(3, 5)
    out, _ = oracle.conv2d_hwc(img, k)
    assert not out[:, :, 0].any() and not out[:, :, 2].any()
    for a in range(3):
        for b in range(5):
            assert out[4 - a + 1, 5 - b + 2, 1] == k[a, b]


def test_interleaved_separable_equals_two_1d_passes():
    r = _rng(901)
    img = r.standard_normal((13, 10, 3)).astype(np.float32)
    gx = r.standard_normal(5).astype(np.float32)
    gy = r.standard_normal(7).astype(np.float32)
    out, bound = oracle.conv2d_sep_hwc(img, gx, gy)
    x = img.astype(np.float64)
    ref = ndi.correlate1d(ndi.correlate1d(x, gx.astype(np.float64), axis=1, mode="nearest"),
                          gy.astype(np.float64), axis=0, mode="nearest")
    assert np.all(np.abs(out - ref) <= 1e-13 * bound + 1e-300)


def test_interleaved_points_match_full_image():
    r = _rng(902)
    img = r.standard_normal((17, 9, 4)).astype(np.float32)
    k = r.standard_normal((5, 3)).astype(np.float32)
    full, fb = oracle.conv2d_hwc(img, k)
    pts = np.array([[0, 0, 0], [3, 16, 8], [2, 7, 4], [1, 0, 8], [3, 16, 0]])
    v, b = oracle.conv2d_hwc_points(img, k, pts)
    np.testing.assert_array_equal(v, full[pts[:, 1], pts[:, 2], pts[:, 0]])
    np.testing.assert_array_equal(b, fb[pts[:, 1], pts[:, 2], pts[:, 0]])
