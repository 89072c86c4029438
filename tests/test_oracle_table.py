"""Pins for the oracle's global shared-exponent table format (Sec. III-B
"Shared Exponents Extraction" and "Denormalized Representation", Alg. 1,
Alg. 2, Sec. III-C).

Fixed against: hand-worked values, an independent restatement of Alg. 1 with
the exponent index in the SEM word, closed forms (lossless level 3 when every
exponent is in the table), the truncation error bound, the single-entry case
(which is the group format over one group), and brute-force SpMV.
"""
import collections
import math
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table_handworked.txt")
SEG = (16, 16, 20)


def _bits(a):
    return np.ascontiguousarray(a, dtype=np.float64).view(np.uint64)


def _exps(v):
    return ((_bits(v) >> np.uint64(52)) & np.uint64(0x7FF)).astype(np.int64)


def _values(rng, n, lo=-20, hi=20):
    v = rng.choice([-1.0, 1.0], n) * 2.0 ** rng.uniform(lo, hi, n)
    v[rng.random(n) < 0.01] = 0.0
    return v


def test_handworked_table():
    lines = [l for l in open(GOLDEN) if l.strip() and not l.startswith("#")]
    rows = [l.split() for l in lines]
    vals = np.array([float.fromhex(r[0]) for r in rows])
    table = oracle.table_build(vals, 2)
    assert table.tolist() == [1025, 1027]
    head, t1, t2, idx = oracle.table_encode(vals, table, SEG)
    for i, r in enumerate(rows):
        assert idx[i] == int(r[1]), i
        assert head[i] == int(r[2], 16), (i, hex(head[i]))
    dec = oracle.table_decode(head, t1, t2, idx, table, 1, SEG)
    exp = np.array([float.fromhex(r[3]) for r in rows])
    assert np.array_equal(_bits(dec), _bits(exp))


def _alg1_sem(v, table, ei_bits):
    """Alg. 1 restated for one value: the 16-bit SEM word holds the sign, an
    exponent index of ei_bits bits and 15 - ei_bits mantissa bits.  The shared
    exponent is the entry equal to exp + 1 when there is one (distance 1), else
    the nearest entry above exp (the smallest positive distance).  The 52-bit
    fraction is shifted right by that distance, cut to the field width, and the
    explicit leading one is placed distance places below the field's top."""
    b = int(np.float64(v).view(np.uint64))
    sign = (b >> 48) & 0x8000
    e = (b >> 52) & 0x7FF
    candidates = [k for k, t in enumerate(table) if t == e + 1]
    if candidates:
        k, dist = candidates[0], 1
    else:
        above = [(int(t) - e, k) for k, t in enumerate(table) if int(t) - e > 0]
        dist, k = min(above)
    width = 15 - ei_bits
    if dist > width:
        return None, k, dist              # the explicit one falls out of the field
    frac = b & ((1 << 52) - 1)
    mant = (frac >> dist) >> (52 - width)
    mant |= 1 << (width - dist)
    return sign | (k << width) | mant, k, dist


@pytest.mark.parametrize("num_exp", [2, 4, 8, 16])
def test_alg1_restatement(num_exp):
    rng = np.random.default_rng(num_exp)
    vals = _values(rng, 4000, -8, 8)
    vals = vals[vals != 0.0]
    table = oracle.table_build(vals, num_exp)
    head, t1, t2, idx = oracle.table_encode(vals, table, SEG)
    ei = max(0, math.ceil(math.log2(len(table))))
    checked = 0
    for i, v in enumerate(vals):
        sem, k, dist = _alg1_sem(v, table, ei)
        assert idx[i] == k
        if dist > 15 - ei:
            continue                      # Alg. 1 shifts the explicit one out (reading R4: M = 0)
        width = 15 - ei
        assert (sem & 0x8000) == (head[i] & 0x8000)
        assert (sem & ((1 << width) - 1)) == (head[i] & 0x7FFF) >> ei, (i, v)
        checked += 1
    assert checked > 1000


def test_table_selection_rule():
    rng = np.random.default_rng(3)
    vals = _values(rng, 20000, -10, 6)
    cnt = collections.Counter(int(e) for e in _exps(vals) if e != 0)
    emax = max(cnt)
    for num_exp in (1, 2, 5, 8, 40):
        table = oracle.table_build(vals, num_exp)
        assert len(table) == min(num_exp, len(cnt))
        assert emax + 1 in table.tolist()
        kept = [int(t) - 1 for t in table]
        assert len(set(kept)) == len(kept)
        # every kept exponent (except a max(e) that was forced in) is at least as
        # frequent as every exponent left out
        left = [e for e in cnt if e not in kept]
        forced = emax if (len(kept) == num_exp and sorted(cnt, key=lambda e: (-cnt[e], -e)).index(emax) >= num_exp) else None
        for e in kept:
            if e == forced:
                continue
            assert all(cnt[e] >= cnt[o] for o in left)


def test_lossless_when_every_exponent_is_shared():
    # with 16/16/32 the level-3 magnitude has 63 bits; when e + 1 is in the table
    # the shift is 63 - 52 - 1 = 10 to the left, so every value is kept exactly
    rng = np.random.default_rng(5)
    vals = _values(rng, 5000, -30, 30)
    distinct = len(set(int(e) for e in _exps(vals) if e != 0))
    seg = (16, 16, 32)
    table = oracle.table_build(vals, distinct)
    enc = oracle.table_encode(vals, table, seg)
    dec = oracle.table_decode(*enc, table, 3, seg)
    assert np.array_equal(_bits(dec), _bits(vals))


def test_truncation_bound_and_prefix():
    rng = np.random.default_rng(6)
    vals = _values(rng, 5000, -12, 12)
    table = oracle.table_build(vals, 8)
    enc = oracle.table_encode(vals, table, SEG)
    T = table[enc[3]].astype(np.int64)
    prev = np.zeros_like(vals)
    for k, W in zip((1, 2, 3), (15, 31, 51)):
        a = oracle.table_decode(*enc, table, k, SEG)
        assert np.all(np.abs(a) <= np.abs(vals))
        assert np.all(np.sign(a[a != 0]) == np.sign(vals[a != 0]))
        assert np.all(np.abs(vals - a) < np.ldexp(1.0, (T - 1023 - W).astype(np.int32)))
        assert np.all(np.abs(a) >= np.abs(prev))
        prev = a


def test_single_entry_is_one_group():
    # numExp = 1 leaves only max(e) + 1: the group format over a single group
    rng = np.random.default_rng(7)
    vals = _values(rng, 1000, -6, 6)
    table = oracle.table_build(vals, 1)
    th, t1, t2, idx = oracle.table_encode(vals, table, SEG)
    gh, g1, g2, gexp = oracle.encode(vals, vals.size, SEG)
    assert table.tolist() == [int(gexp[0])]
    assert np.all(idx == 0)
    assert np.array_equal(th, gh) and np.array_equal(t1, g1) and np.array_equal(t2, g2)


def test_table_spmv_brute_force():
    rng = np.random.default_rng(8)
    n = 40
    dense = np.where(rng.random((n, n)) < 0.2, rng.integers(-9, 10, (n, n)) * 2.0 ** rng.integers(-3, 4, (n, n)), 0.0)
    rows, cols = np.nonzero(dense)
    val = dense[rows, cols]
    row_ptr = np.zeros(n + 1, np.int32)
    np.cumsum(np.bincount(rows, minlength=n), out=row_ptr[1:])
    table = oracle.table_build(val, 4)
    enc = oracle.table_encode(val, table, SEG)
    x = rng.integers(-5, 6, n).astype(np.float64)
    for k in (1, 2, 3):
        a = oracle.table_decode(*enc, table, k, SEG)
        y = oracle.spmv(row_ptr, cols.astype(np.int32), a, x)
        A = np.zeros((n, n))
        A[rows, cols] = a
        assert np.array_equal(y, A @ x)           # dyadic values: every sum is exact


def test_rejects_nonfinite():
    with pytest.raises(ValueError):
        oracle.table_build(np.array([1.0, np.inf]), 2)
