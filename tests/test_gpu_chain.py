"""The fused two-filter chain out = conv(conv(in, k1), k2) (one kernel, the
intermediate kept on chip) against two separate conv2d calls through a
temporary of the storage dtype -- bit for bit -- and against the FP64 oracle
composed the same way: y = oracle(in, k1) rounded to the storage type, then
oracle(y, k2).

Oracle tolerance: the chain's error is the second pass's own rounding
(<= tol * bound2, bound2 = sum |k2| |y|) plus the first pass's error carried
through k2 (<= tol * B12, B12 = sum |k2| bound1); tol as for one conv2d pass
(1e-6 FP32, 2^-10 binary16, which cover the intermediate's storage rounding).
"""
import numpy as np
import pytest

import oracle
import paper_1302_5586_gb300 as pg
import synth
from gpu_util import dev, to_dev, torch

pytestmark = pytest.mark.gpu

F32_TOL = 1e-6
F16_TOL = 2.0 ** -10


def chain(img, k1, k2, dtype=pg.PENCIL_F32, flags=0):
    c, h, w = img.shape
    d_in, d_k1, d_k2 = to_dev(img), to_dev(k1), to_dev(k2)
    out = torch.empty_like(d_in)
    pg.pencil_conv2d_chain(c, h, w, d_in, k1.shape[0], k1.shape[1], d_k1, k2.shape[0], k2.shape[1], d_k2, out,
                           dtype, flags)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def two_pass(img, k1, k2, dtype=pg.PENCIL_F32):
    c, h, w = img.shape
    d_in, d_k1, d_k2 = to_dev(img), to_dev(k1), to_dev(k2)
    tmp, out = torch.empty_like(d_in), torch.empty_like(d_in)
    pg.pencil_conv2d_ex(c, h, w, d_in, k1.shape[0], k1.shape[1], d_k1, tmp, dtype, 0)
    pg.pencil_conv2d_ex(c, h, w, tmp, k2.shape[0], k2.shape[1], d_k2, out, dtype, 0)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def bits(a):
    return a.view(np.uint16 if a.dtype == np.float16 else np.uint32)


SHAPES = [(2, 75, 301), (1, 200, 520), (3, 33, 128), (1, 1, 1), (1, 5, 3), (2, 1, 77), (1, 64, 1), (1, 130, 257)]


@pytest.mark.parametrize("k1s", [3, 5, 7])
@pytest.mark.parametrize("k2s", [3, 5, 7])
@pytest.mark.parametrize("shape", SHAPES)
def test_chain_equals_two_passes_f32(k1s, k2s, shape):
    dev()
    c, h, w = shape
    img = synth.image_f32(100 * k1s + k2s, c, h, w)
    k1 = synth.filter_f32(7 * k1s, k1s, k1s)
    k2 = synth.filter_f32(11 * k2s + 1, k2s, k2s)
    a = chain(img, k1, k2)
    np.testing.assert_array_equal(bits(a), bits(two_pass(img, k1, k2)))
    np.testing.assert_array_equal(bits(a), bits(chain(img, k1, k2, flags=pg.PENCIL_CHAIN_FUSED)))
    np.testing.assert_array_equal(bits(a), bits(chain(img, k1, k2, flags=pg.PENCIL_CONV_GENERIC)))


@pytest.mark.parametrize("k1s,k2s", [(3, 3), (5, 5), (7, 3), (3, 7), (5, 7), (7, 7)])
@pytest.mark.parametrize("shape", [(2, 75, 304), (1, 130, 257), (1, 3, 2), (1, 260, 136)])
def test_chain_equals_two_passes_f16(k1s, k2s, shape):
    dev()
    c, h, w = shape
    img = synth.image_f16(200 + k1s * k2s, c, h, w)
    k1 = synth.filter_f32(3 * k1s, k1s, k1s)
    k2 = synth.filter_f32(5 * k2s, k2s, k2s)
    a = chain(img, k1, k2, pg.PENCIL_F16)
    np.testing.assert_array_equal(bits(a), bits(two_pass(img, k1, k2, pg.PENCIL_F16)))
    np.testing.assert_array_equal(bits(a), bits(chain(img, k1, k2, pg.PENCIL_F16, pg.PENCIL_CHAIN_FUSED)))
    np.testing.assert_array_equal(bits(a), bits(chain(img, k1, k2, pg.PENCIL_F16, pg.PENCIL_CONV_GENERIC)))


@pytest.mark.parametrize("kk", [((4, 6), (2, 1)), ((1, 9), (9, 1)), ((15, 15), (3, 3)), ((3, 3), (11, 11)),
                                ((2, 2), (5, 5)), ((1, 1), (1, 1))])
def test_generic_pairs_equal_two_passes(kk):
    dev()
    (a1, b1), (a2, b2) = kk
    img = synth.image_f32(a1 * 31 + b2, 2, 45, 70)
    k1 = synth.filter_f32(a1 + 3 * b1, a1, b1)
    k2 = synth.filter_f32(a2 + 5 * b2 + 100, a2, b2)
    np.testing.assert_array_equal(bits(chain(img, k1, k2)), bits(two_pass(img, k1, k2)))
    np.testing.assert_array_equal(bits(chain(img, k1, k2, flags=pg.PENCIL_CHAIN_FUSED)), bits(two_pass(img, k1, k2)))


def _oracle_chain(img, k1, k2, store):
    y, b1 = oracle.conv2d(img, k1)
    z, b2 = oracle.conv2d(y.astype(store), k2)
    b12, _ = oracle.conv2d(b1.astype(np.float32), np.abs(k2), want_bound=False)
    return z, b2, b12


@pytest.mark.parametrize("k1s,k2s", [(3, 3), (5, 5), (7, 7), (3, 7)])
def test_chain_matches_oracle(k1s, k2s):
    dev()
    img = synth.image_f32(9 + k1s, 2, 150, 333)
    k1 = synth.filter_f32(91 + k1s, k1s, k1s)
    k2 = synth.filter_f32(93 + k2s, k2s, k2s)
    z, b2, b12 = _oracle_chain(img, k1, k2, np.float32)
    for fl in (0, pg.PENCIL_CHAIN_FUSED):
        got = chain(img, k1, k2, flags=fl).astype(np.float64)
        assert np.all(np.abs(got - z) <= F32_TOL * (b2 + b12))
    img16 = synth.to_f16(img)
    z, b2, b12 = _oracle_chain(img16, k1, k2, np.float16)
    for fl in (0, pg.PENCIL_CHAIN_FUSED):
        got = chain(img16, k1, k2, pg.PENCIL_F16, fl).astype(np.float64)
        assert np.all(np.abs(got - z) <= F16_TOL * (b2 + b12))


def test_delta_filters_compose_shifts():
    """Two one-hot filters: the chain is a shift by the sum of both offsets
    with the clamp applied after each (exact, no rounding)."""
    dev()
    img = synth.image_f32(5, 1, 40, 57)
    k1 = np.zeros((5, 5), np.float32); k1[0, 4] = 1.0   # reads x[i-2][j+2]
    k2 = np.zeros((3, 3), np.float32); k2[2, 0] = 1.0   # reads y[i+1][j-1]
    got = chain(img, k1, k2)[0]
    h, w = 40, 57
    ii = np.arange(h)[:, None]; jj = np.arange(w)[None, :]
    yi = np.clip(ii + 1, 0, h - 1); yj = np.clip(jj - 1, 0, w - 1)
    xi = np.clip(yi - 2, 0, h - 1); xj = np.clip(yj + 2, 0, w - 1)
    np.testing.assert_array_equal(got, img[0][xi, xj])


def test_full_size_whole_output():
    """3 x 8192 x 8192 FP32, 5x5 then a 5x5 Gaussian: the whole output against
    two separate passes, compared on the device."""
    dev()
    c, h, w = 3, 8192, 8192
    img = torch.from_numpy(synth.image_f32(synth.SEEDS["conv8192x3"], c, h, w)).to(dev())
    k1 = to_dev(synth.filter_f32(51, 5, 5))
    k2 = to_dev(synth.gaussian_2d_f32(2, 1.0))
    out = torch.empty_like(img)
    tmp = torch.empty_like(img)
    pg.pencil_conv2d_chain(c, h, w, img, 5, 5, k1, 5, 5, k2, out, pg.PENCIL_F32)
    pg.pencil_conv2d_ex(c, h, w, img, 5, 5, k1, tmp, pg.PENCIL_F32, 0)
    pg.pencil_conv2d_ex(c, h, w, tmp, 5, 5, k2, img, pg.PENCIL_F32, 0)  # img now holds the two-pass result
    torch.cuda.synchronize()
    assert torch.equal(out.view(torch.int32), img.view(torch.int32))


def test_errors():
    dev()
    x = torch.zeros(2, 16, 16, device=dev())
    k = torch.full((3, 3), 1.0 / 9, device=dev())
    o = torch.empty_like(x)
    with pytest.raises(pg.PencilError) as ei:
        pg.pencil_conv2d_chain(2, 16, 16, x, 3, 3, k, 3, 3, k, o, pg.PENCIL_F32, pg.PENCIL_BORDER(1))
    assert ei.value.status == -8
    with pytest.raises(pg.PencilError) as ei:
        pg.pencil_conv2d_chain(2, 16, 16, x, 3, 3, k, 3, 3, k, x, pg.PENCIL_F32)
    assert ei.value.status == -3
    with pytest.raises(pg.PencilError) as ei:
        pg.pencil_conv2d_chain(2, 16, 16, x, 0, 3, k, 3, 3, k, o, pg.PENCIL_F32)
    assert ei.value.status == -1
    with pytest.raises(pg.PencilError) as ei:
        pg.pencil_conv2d_chain(2, 16, 16, x, 3, 3, k, 3, 3, k, o, pg.PENCIL_F32, 4)
    assert ei.value.status == -1
    with pytest.raises(pg.PencilError) as ei:
        pg.pencil_conv2d_chain(2, 16, 16, x.cpu(), 3, 3, k, 3, 3, k, o, pg.PENCIL_F32)
    assert ei.value.status == -4
