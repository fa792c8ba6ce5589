"""Pins of the oracle's binary16 codec against numpy's and torch's conversions."""
import numpy as np
import pytest
import torch

import oracle


def test_decode_all_65536_patterns():
    bits = np.arange(65536, dtype=np.uint32).astype(np.uint16)
    ours = oracle.f16_to_f64(bits)
    ref = bits.view(np.float16).astype(np.float64)
    nan = np.isnan(ref)
    np.testing.assert_array_equal(np.isnan(ours), nan)
    np.testing.assert_array_equal(ours[~nan], ref[~nan])
    # signed zeros keep their sign
    assert np.signbit(ours[0x8000]) and not np.signbit(ours[0])


def test_encode_round_trips_every_finite_half():
    bits = np.arange(65536, dtype=np.uint32).astype(np.uint16)
    vals = bits.view(np.float16).astype(np.float64)
    finite = np.isfinite(vals)
    back = oracle.f64_to_f16(vals[finite])
    np.testing.assert_array_equal(back, bits[finite])
    inf = ~finite & ~np.isnan(vals)
    np.testing.assert_array_equal(oracle.f64_to_f16(vals[inf]), bits[inf])
    assert (oracle.f64_to_f16(np.array([np.nan]))[0] & 0x7C00) == 0x7C00
    assert (oracle.f64_to_f16(np.array([np.nan]))[0] & 0x03FF) != 0


def test_ties_round_to_even():
    one = 1.0
    ulp = 2.0 ** -10
    cases = {
        one + ulp / 2: 0x3C00,          # tie, even stays at 1.0
        one + 3 * ulp / 2: 0x3C02,      # tie, rounds up to the even neighbour
        one + ulp / 2 + 2 ** -30: 0x3C01,
        65504.0: 0x7BFF,                # max finite
        65519.99: 0x7BFF,
        65520.0: 0x7C00,                # tie at the top rounds to infinity
        2.0 ** -24: 0x0001,             # smallest subnormal
        2.0 ** -25: 0x0000,             # tie to even (zero)
        3 * 2.0 ** -25: 0x0002,         # tie to even (2)
        2.0 ** -14 - 2.0 ** -25: 0x0400,  # rounds up into the smallest normal
        -0.0: 0x8000,
    }
    for x, want in cases.items():
        assert oracle.f64_to_f16(np.array([x]))[0] == want, x


@pytest.mark.parametrize("lib", ["numpy", "torch"])
def test_encode_matches_library_over_float32_sweep(lib):
    """2^24 FP32 values (every 256th bit pattern, all signs and exponents) against a library."""
    pats = (np.arange(1 << 24, dtype=np.uint64) * np.uint64(256) + np.uint64(0x5A)).astype(np.uint32)
    f = pats.view(np.float32)
    f = f[np.isfinite(f)]
    ours = oracle.f64_to_f16(f.astype(np.float64))
    if lib == "numpy":
        with np.errstate(over="ignore"):
            ref = f.astype(np.float16).view(np.uint16)
    else:
        ref = torch.from_numpy(f).to(torch.float16).view(torch.int16).numpy().view(np.uint16)
    np.testing.assert_array_equal(ours, ref)
