"""Pins for the oracle's 16-bit baselines (Sec. IV-C: values stored in FP16 or
BF16, widened to FP64 for the multiply-accumulate).

FP16 rounding is pinned to numpy's float64 -> float16 conversion (IEEE round to
nearest even, one rounding).  BF16 has no library routine here: it is pinned
by hand-worked values (ties, overflow threshold, subnormals) and by checking
that every result is a nearest representable value with ties to an even
mantissa, by enumerating the neighbouring BF16 values.
"""
import numpy as np
import pytest

import oracle


def _values(rng, n):
    v = rng.choice([-1.0, 1.0], n) * 2.0 ** rng.uniform(-30, 20, n)
    # exact ties and near-ties of the FP16 and BF16 grids
    base = 2.0 ** rng.integers(-20, 10, n)
    t16 = base * (1.0 + (2 * rng.integers(0, 512, n) + 1) * 2.0 ** -11)
    t8 = base * (1.0 + (2 * rng.integers(0, 64, n) + 1) * 2.0 ** -8)
    return np.concatenate([v, t16, t8, [0.0, -0.0, 65504.0, 65519.99, 65520.0, 1e30, -1e30, 2.0 ** -24, 2.0 ** -25,
                                        3 * 2.0 ** -26, 2.0 ** -14, 2.0 ** -15]])


def test_fp16_equals_numpy_conversion():
    rng = np.random.default_rng(0)
    v = _values(rng, 200000)
    bits, ov = oracle.round16(v, oracle.FP16)
    with np.errstate(over="ignore"):
        ref = v.astype(np.float16)
    assert np.array_equal(bits, ref.view(np.uint16))
    assert ov == int(np.sum(np.isinf(ref) & np.isfinite(v)))
    back = oracle.widen16(bits, oracle.FP16)
    assert np.array_equal(back, ref.astype(np.float64))


HAND_BF16 = [
    (1.0, 0x3F80), (-2.0, 0xC000), (1.0 / 3.0, 0x3EAB), (1.0 + 2.0 ** -8, 0x3F80),        # tie -> even
    (1.0 + 3 * 2.0 ** -8, 0x3F82), (1.0 + 2.0 ** -8 + 2.0 ** -30, 0x3F81),               # tie -> even; above the tie
    (3.3895313892515355e38, 0x7F7F), (3.4e38, 0x7F80), (-0.0, 0x8000), (0.0, 0x0000),    # max, overflow
    (2.0 ** -133, 0x0001), (2.0 ** -126, 0x0080), (2.0 ** -134, 0x0000),                  # subnormal, min normal, tie to 0
]


@pytest.mark.parametrize("v,bits", HAND_BF16)
def test_bf16_hand_worked(v, bits):
    b, _ = oracle.round16(np.array([v]), oracle.BF16)
    assert int(b[0]) == bits, hex(int(b[0]))


def test_bf16_nearest_even_by_enumeration():
    rng = np.random.default_rng(1)
    v = _values(rng, 50000)
    v = v[np.abs(v) < 3.38e38]
    b, ov = oracle.round16(v, oracle.BF16)
    assert ov == 0
    r = oracle.widen16(b, oracle.BF16)
    # neighbours on the BF16 grid: one code up and one code down (same sign)
    mag = b & np.uint16(0x7FFF)
    sign = b & np.uint16(0x8000)
    up = oracle.widen16(sign | np.minimum(mag + 1, 0x7F7F).astype(np.uint16), oracle.BF16)
    dn = oracle.widen16(sign | np.maximum(mag.astype(np.int32) - 1, 0).astype(np.uint16), oracle.BF16)
    err = np.abs(v - r)
    assert np.all(err <= np.abs(v - up)) and np.all(err <= np.abs(v - dn))
    ties = (err == np.abs(v - up)) | (err == np.abs(v - dn))
    ties &= err > 0
    assert np.all((b[ties] & 1) == 0)            # ties go to the even mantissa
    assert np.all(np.sign(r[r != 0]) == np.sign(v[r != 0]))


def test_overflow_count():
    v = np.array([1.0, 7e4, -1e5, 65504.0, np.inf])
    _, ov = oracle.round16(v, oracle.FP16)
    assert ov == 2                               # infinities already in the input are not overflows
    _, ov = oracle.round16(v, oracle.BF16)
    assert ov == 0


@pytest.mark.parametrize("kind", [oracle.FP16, oracle.BF16])
def test_nonfinite_values_keep_their_class(kind):
    """NaN stays a NaN (all-ones exponent, nonzero mantissa) and +-Inf stays
    +-Inf, in both 16-bit formats; FP16 agrees with numpy bit for bit."""
    v = np.array([np.nan, np.inf, -np.inf])
    b, ov = oracle.round16(v, kind)
    mb = 10 if kind == oracle.FP16 else 7
    exp_ones = (0xFFFF >> (16 - (15 - mb))) << mb & 0x7FFF
    assert (int(b[0]) & exp_ones) == exp_ones and int(b[0]) & ((1 << mb) - 1) != 0
    assert int(b[1]) == exp_ones and int(b[2]) == 0x8000 | exp_ones
    assert ov == 0                                  # none of them was a finite value
    back = oracle.widen16(b, kind)
    assert np.isnan(back[0]) and back[1] == np.inf and back[2] == -np.inf
    if kind == oracle.FP16:
        assert np.array_equal(b, v.astype(np.float16).view(np.uint16))
