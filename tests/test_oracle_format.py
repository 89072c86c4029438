"""Pins for the oracle's GSE encode/decode (Sec. III-B, Alg. 1, Alg. 2, Fig. 3).

Each check fixes the oracle against something other than itself: hand-worked
values, an independent restatement of Alg. 1 / Alg. 2 written here in numpy,
exact round trips, and the error bound of truncation.
"""
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "encode_handworked.txt")
SEG = (16, 16, 20)


def _bits(a):
    return np.ascontiguousarray(a, dtype=np.float64).view(np.uint64)


def test_handworked_group():
    rows = [l.split() for l in open(GOLDEN) if l.strip() and not l.startswith("#")]
    vals = np.array([float.fromhex(r[1]) for r in rows])
    head, t1, t2, gexp = oracle.encode(vals, 32, SEG)
    assert gexp.tolist() == [1024]
    for i, r in enumerate(rows):
        assert head[i] == int(r[2], 16), (i, hex(head[i]))
        assert t1[i] == int(r[3], 16), (i, hex(t1[i]))
        assert t2[i] == int(r[4], 16), (i, hex(t2[i]))
    for k in (1, 2, 3):
        dec = oracle.decode(head, t1, t2, gexp, k, 32, SEG)
        exp = np.array([float.fromhex(r[4 + k]) for r in rows])
        assert np.array_equal(_bits(dec), _bits(exp)), k


def _random_values(rng, n, lo=-12, hi=12):
    """Values spread over ~24 binades with random signs, a few exact zeros."""
    v = rng.choice([-1.0, 1.0], n) * 2.0 ** rng.uniform(lo, hi, n)
    v[rng.random(n) < 0.01] = 0.0
    return v


def _alg1_head(vals, G):
    """Alg. 1 restated for one shared exponent per group (numExp = 1, so the
    exponent index is 0 bits): the mantissa field is shifted right by the
    distance to the shared exponent, cut to the head width, and the explicit
    leading 1 is OR-ed in below the sign.  The shared exponent is the group's
    maximum exponent + 1 (Sec. III-B)."""
    b = _bits(vals)
    sign = ((b >> np.uint64(48)) & np.uint64(0x8000)).astype(np.uint64)
    e = ((b >> np.uint64(52)) & np.uint64(0x7FF)).astype(np.int64)
    frac = b & np.uint64((1 << 52) - 1)
    ng = (vals.size + G - 1) // G
    emax = np.zeros(ng, np.int64)
    np.maximum.at(emax, np.arange(vals.size) // G, e)
    shared = emax[np.arange(vals.size) // G] + 1
    min_diff = (shared - e).astype(np.uint64)   # exp + 1 == shared gives 1
    mant = (frac >> min_diff) >> np.uint64(37)
    lead = np.left_shift(np.uint64(1), (np.uint64(15) - min_diff))
    return (sign | mant | lead).astype(np.uint16), shared, e


def test_alg1_restated_matches_head():
    rng = np.random.default_rng(1)
    vals = _random_values(rng, 2_000_000)
    head, t1, t2, gexp = oracle.encode(vals, 32, SEG)
    ref, shared, e = _alg1_head(vals, 32)
    ok = (e > 0) & (shared - e <= 15)          # Alg. 1 is defined for these
    assert ok.mean() > 0.5
    assert np.array_equal(head[ok], ref[ok])
    # outside that range the head magnitude is 0 (a value that far below the
    # group maximum has no bit in the head), sign kept
    far = ~ok
    assert np.all((head[far] & 0x7FFF) == 0)
    assert np.array_equal(head[far] >> 15, (_bits(vals[far]) >> np.uint64(63)).astype(np.uint16))


def _alg2_decode(head, gexp, G):
    """Alg. 2 restated: sign from head bit 15; find the highest set bit `pos`
    among bits 14..0; exponent = shared exponent - (15 - pos); the bits below
    the leading one become the top of the 52-bit mantissa; no set bit -> 0."""
    h = head.astype(np.uint64)
    E = gexp.astype(np.int64)[np.arange(head.size) // G]
    mag = h & np.uint64(0x7FFF)
    out = np.zeros(head.size, np.uint64)
    nz = mag != 0
    pos = np.floor(np.log2(mag[nz].astype(np.float64))).astype(np.int64)   # exact for < 2^15
    expo = (E[nz] - (15 - pos)).astype(np.uint64)
    mant = ((mag[nz] << np.uint64(36)) << (np.uint64(16) - pos.astype(np.uint64))) & np.uint64((1 << 52) - 1)
    out[nz] = ((h[nz] & np.uint64(0x8000)) << np.uint64(48)) | (expo << np.uint64(52)) | mant
    out[~nz] = 0
    return out.view(np.float64)


def test_alg2_restated_matches_level1():
    rng = np.random.default_rng(2)
    vals = _random_values(rng, 2_000_000)
    head, t1, t2, gexp = oracle.encode(vals, 32, SEG)
    dec1 = oracle.decode(head, t1, t2, gexp, 1, 32, SEG)
    ref = _alg2_decode(head, gexp, 32)
    nz = (head & 0x7FFF) != 0
    assert np.array_equal(_bits(dec1[nz]), _bits(ref[nz]))
    assert np.all(dec1[~nz] == 0.0)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_exact_round_trip_of_representable_values(k):
    """v = +-M * 2^(E_g - 1023 - W_k) with M < 2^W_k survives encode/decode at
    level k and every level above it, bit for bit."""
    rng = np.random.default_rng(10 + k)
    W = {1: 15, 2: 31, 3: 51}[k]
    G, ng = 32, 4000
    Eg = rng.integers(900, 1100, ng)
    M = rng.integers(0, 2 ** W, (ng, G), dtype=np.int64).astype(np.uint64)
    M[:, 0] |= np.uint64(1 << (W - 1))     # group maximum has d = 1 -> fixes E_g
    sign = rng.choice([-1.0, 1.0], (ng, G))
    vals = (sign * np.ldexp(M.astype(np.float64), (Eg - 1023 - W)[:, None])).ravel()
    head, t1, t2, gexp = oracle.encode(vals, G, SEG)
    assert np.array_equal(gexp.astype(np.int64), Eg)
    for kk in range(k, 4):
        dec = oracle.decode(head, t1, t2, gexp, kk, G, SEG)
        assert np.array_equal(dec, vals), kk


def test_prefix_monotone_and_error_bound():
    rng = np.random.default_rng(3)
    vals = _random_values(rng, 1_000_000, -30, 30)
    G = 32
    head, t1, t2, gexp = oracle.encode(vals, G, SEG)
    d = [oracle.decode(head, t1, t2, gexp, k, G, SEG) for k in (1, 2, 3)]
    a = [np.abs(x) for x in d]
    assert np.all(a[0] <= a[1]) and np.all(a[1] <= a[2]) and np.all(a[2] <= np.abs(vals))
    for x in d:   # truncation toward zero never flips a sign
        assert np.all((x == 0) | (np.sign(x) == np.sign(vals)))
    Eg = gexp.astype(np.int64)[np.arange(vals.size) // G]
    for k, W in zip((1, 2, 3), (15, 31, 51)):
        ulp = np.ldexp(1.0, Eg - 1023 - W)
        assert np.all(np.abs(vals - d[k - 1]) < ulp), k
        # level k is level k+1 truncated to W_k bits (the prefix property)
        if k < 3:
            Mk1 = np.abs(d[k]) / np.ldexp(1.0, Eg - 1023 - (W + (16 if k == 1 else 20)))
            shift = 16 if k == 1 else 20
            Mk = np.floor(Mk1 / 2 ** shift)
            assert np.array_equal(np.abs(d[k - 1]), Mk * ulp)


def test_lossless_with_32bit_tail2():
    """With seg_bits 16/16/32 (the paper's 64-bit SEM example), level 3 keeps
    63 magnitude bits, so every value within 11 binades of its group maximum
    is reproduced exactly."""
    rng = np.random.default_rng(4)
    G = 32
    vals = rng.choice([-1.0, 1.0], (5000, G)) * rng.uniform(1.0, 2.0, (5000, G))
    vals *= 2.0 ** rng.integers(-10, 1, (5000, G))       # d <= 11
    vals[:, 0] = 1.999
    vals = vals.ravel()
    enc = oracle.encode(vals, G, (16, 16, 32))
    dec = oracle.decode(*enc, 3, G, (16, 16, 32))
    assert np.array_equal(dec, vals)


def test_zero_and_subnormal_groups_and_partial_group():
    vals = np.array([0.0] * 32 + [5e-324, -5e-324, 0.0] + [1.0] * 5)
    head, t1, t2, gexp = oracle.encode(vals, 32, SEG)
    assert gexp.tolist() == [0, 1024]
    assert head[32] == 0 and head[33] == 0x8000
    for k in (1, 2, 3):
        dec = oracle.decode(head, t1, t2, gexp, k, 32, SEG)
        assert np.all(dec[:35] == 0.0) and np.all(dec[35:] == 1.0)


def test_extreme_exponent_groups_closed_form():
    """The top and bottom of the exponent range, worked by hand (G = 4, 16/16/32,
    W = 15 / 31 / 63).  Group 0 holds DBL_MAX, so E_g = 2046 + 1 = 2047.  Group 1
    holds the smallest normal exponents, E_g = 2 + 1 = 3."""
    big = np.finfo(np.float64).max
    vals = np.array([big, 1.0, -2.0 ** 1000, 0.0,
                     2.0 ** -1022, 1.75 * 2.0 ** -1022, 5e-324, -2.0 ** -1021])
    seg = (16, 16, 32)
    enc = oracle.encode(vals, 4, seg)
    assert enc[3].tolist() == [2047, 3]
    lv = [oracle.decode(*enc, k, 4, seg) for k in (1, 2, 3)]
    # DBL_MAX: d = 1, M = (2^53 - 1) << 10; level 1 keeps the top 15 bits,
    # (2^15 - 1) * 2^(2047 - 1023 - 15) = 2^1024 - 2^1009; level 3 is exact (63 >= 53 + 1)
    assert lv[0][0] == (2.0 ** 15 - 1) * 2.0 ** 1009
    assert lv[2][0] == big
    # 1.0 is 1024 binades below E_g: M = 0 at every level
    assert all(l[1] == 0.0 for l in lv)
    # -2^1000: d = 24, M = 2^52 >> 13 = 2^39; level 1 keeps M >> 48 = 0, level 2
    # keeps M >> 32 = 2^7, i.e. 2^7 * 2^(2047 - 1023 - 31) = 2^1000
    assert lv[0][2] == 0.0 and lv[1][2] == -2.0 ** 1000 and lv[2][2] == -2.0 ** 1000
    # group 1: 2^-1022 (d = 2) and 1.75 * 2^-1022 (d = 2) fit in the head's 15 bits,
    # -2^-1021 has d = 1; the subnormal input gives M = 0 (R4)
    for l in lv:
        assert l[4] == 2.0 ** -1022 and l[5] == 1.75 * 2.0 ** -1022 and l[6] == 0.0 and l[7] == -2.0 ** -1021
    assert enc[0][4] == 1 << 13 and enc[0][5] == 14336 and enc[0][7] == 0x8000 | (1 << 14)


def test_nonfinite_rejected():
    for bad in (np.inf, -np.inf, np.nan):
        with pytest.raises(ValueError):
            oracle.encode(np.array([1.0, bad]), 32, SEG)
