"""The seeded input generators: published SplitMix64 values and recipe properties."""
import numpy as np

import synth


def test_splitmix64_published_vector():
    # first outputs of SplitMix64 from state 1234567 (the generator's reference test vector)
    want = [6457827717110365317, 3203168211198807973, 9817491932198370423,
            4593380528125082431, 16408922859458223821]
    assert [int(v) for v in synth.splitmix64(1234567, 5)] == want


def test_stream_is_counter_based():
    a = synth.splitmix64(42, 100)
    b = synth.splitmix64(42, 60, offset=40)
    np.testing.assert_array_equal(a[40:], b)
    big = synth.u01_f32(42, (1 << 22) + 1000)
    np.testing.assert_array_equal(big[(1 << 22):], synth.u01_f32(42, 1000, offset=1 << 22))


def test_uniform_ranges_and_exactness():
    u = synth.u01_f32(1, 100000)
    assert u.dtype == np.float32 and u.min() >= 0 and u.max() < 1
    z = synth.splitmix64(1, 100000)
    np.testing.assert_array_equal(u.astype(np.float64), (z >> np.uint64(40)).astype(np.float64) * 2.0 ** -24)
    d = synth.u01_f64(1, 1000)
    assert d.min() >= 0 and d.max() < 1


def test_filters_normalised():
    k = synth.filter_f32(5, 7, 3)
    assert k.shape == (7, 3) and k.dtype == np.float32
    assert abs(k.astype(np.float64).sum() - 1) < 1e-6
    g = synth.gaussian_taps_f32(7, 3.0)
    assert g.shape == (15,) and abs(g.astype(np.float64).sum() - 1) < 1e-6
    np.testing.assert_array_equal(g, g[::-1])
    g2 = synth.gaussian_2d_f32(7, 3.0)
    assert g2.shape == (15, 15) and abs(g2.astype(np.float64).sum() - 1) < 1e-6


def test_batch_and_stream_recipes():
    s = synth.loguniform_sides(3, 5000, 64, 4096)
    assert s.min() >= 64 and s.max() <= 4096
    k = synth.odd_ksizes(3, 5000)
    assert set(np.unique(k)) == {3, 5, 7, 9, 11, 13, 15}
    t = synth.poisson_arrivals(3, 2000.0, 2.0)
    assert abs(len(t) - 4000) < 400 and np.all(np.diff(t) > 0) and t[-1] < 2.0
