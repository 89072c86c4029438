"""Pins for two variants of the oracle's table format.

- The sampled extraction of Sec. III-B: one row per row block stands for the
  block's exponent distribution.
- The exponent index kept in the value instead of the column index
  (Sec. III-C, for column counts without spare bits).

Fixed against hand-worked values and an independent restatement of Alg. 1,
which keeps the index in the 16-bit SEM word.  Also against special cases
that reduce to the exact extraction: one row per block, and blocks of rows
with equal exponent multisets.  Also closed forms: lossless storage when
every exponent is shared, and the truncation bound with the b bits the index
takes.  And brute-force SpMV.
"""
import collections
import os

import numpy as np
import pytest

import oracle
import synth
from test_oracle_table import _alg1_sem, _bits, _exps, _values

GOLD = os.path.join(os.path.dirname(__file__), "golden")
SEG = (16, 16, 20)


def _rows_of(row_ptr, n_rows):
    return [slice(int(row_ptr[r]), int(row_ptr[r + 1])) for r in range(n_rows)]


# ---- sampled extraction ------------------------------------------------------

def test_sampled_handworked():
    rows, tables, full = [], {}, None
    for line in open(os.path.join(GOLD, "table_sampled_handworked.txt")):
        f = line.split()
        if not f or f[0].startswith("#"):
            continue
        if f[0] == "row":
            rows.append([float.fromhex(t) for t in f[1:]])
        elif f[0] == "block_rows":
            block_rows = int(f[1])
        elif f[0] == "sample":
            sample = np.array([int(t) for t in f[1:]], np.int64)
        elif f[0] == "table":
            tables[int(f[1])] = [int(t) for t in f[2:]]
        elif f[0] == "full":
            full = (int(f[1]), [int(t) for t in f[2:]])
    row_ptr = np.zeros(len(rows) + 1, np.int32)
    np.cumsum([len(r) for r in rows], out=row_ptr[1:])
    val = np.array([v for r in rows for v in r])
    for num_exp, want in tables.items():
        got = oracle.table_build_sampled(row_ptr, val, num_exp, block_rows, sample)
        assert got.tolist() == want, num_exp
    assert oracle.table_build(val, full[0]).tolist() == full[1]


@pytest.mark.parametrize("num_exp", [1, 3, 8, 64])
def test_one_row_per_block_is_the_full_count(num_exp):
    A = synth.powerlaw_random(3000, 8.0, 300, seed=4)
    sample = np.arange(A.n_rows, dtype=np.int64)
    assert (oracle.table_build_sampled(A.row_ptr, A.val, num_exp, 1, sample).tolist() ==
            oracle.table_build(A.val, num_exp).tolist())


def test_blocks_of_alike_rows_give_the_full_table():
    # every row of a block carries the same exponent multiset (the values differ),
    # so any sampled row describes its block exactly: the sample is the full count
    rng = np.random.default_rng(12)
    block_rows, n_blocks = 7, 40
    row_ptr, val = [0], []
    for _ in range(n_blocks):
        exps = rng.integers(-12, 12, rng.integers(1, 9))
        for _ in range(block_rows):
            val += list(rng.choice([-1.0, 1.0], exps.size) * rng.uniform(1.0, 2.0, exps.size) * 2.0 ** exps)
            row_ptr.append(len(val))
    row_ptr, val = np.array(row_ptr, np.int32), np.array(val)
    sample = np.array([b * block_rows + rng.integers(block_rows) for b in range(n_blocks)], np.int64)
    for num_exp in (2, 5, 8, 30):
        assert (oracle.table_build_sampled(row_ptr, val, num_exp, block_rows, sample).tolist() ==
                oracle.table_build(val, num_exp).tolist())


def test_sampled_counts_by_brute_force():
    # the selection's input, recounted here: the entries are the exponents with
    # the largest weighted counts (ties to the larger exponent), plus max + 1
    A = synth.powerlaw_random(5000, 6.0, 400, seed=7)
    rng = np.random.default_rng(3)
    block_rows = 64
    nb = (A.n_rows + block_rows - 1) // block_rows
    sample = np.array([min(b * block_rows + rng.integers(block_rows), A.n_rows - 1) for b in range(nb)], np.int64)
    cnt = collections.Counter()
    for b, r in enumerate(sample):
        w = min(block_rows, A.n_rows - b * block_rows)
        for e in _exps(A.val[A.row_ptr[r]:A.row_ptr[r + 1]]):
            if e:
                cnt[int(e)] += w
    emax = int(_exps(A.val).max())
    for num_exp in (1, 4, 8):
        got = oracle.table_build_sampled(A.row_ptr, A.val, num_exp, block_rows, sample).tolist()
        top = sorted(cnt, key=lambda e: (-cnt[e], -e))[:num_exp]
        want = [e + 1 for e in top]
        if emax not in top:
            want[-1] = emax + 1
        assert got == want, num_exp


def test_sampled_keeps_the_maximum_outside_the_sample():
    row_ptr = np.array([0, 2, 3, 4], np.int32)
    val = np.array([1.0, 2.0, 1.0, 2.0 ** 40])
    t = oracle.table_build_sampled(row_ptr, val, 4, 3, np.array([0], np.int64))
    assert int(_exps(np.array([2.0 ** 40]))[0]) + 1 in t.tolist()
    # every value is representable: nothing above the largest entry
    _, levels = oracle.table_levels(val, 4, SEG, table=t)
    assert np.array_equal(levels[2], val)


def test_sampled_rejects_bad_input():
    row_ptr = np.array([0, 1, 2, 3, 4], np.int32)
    val = np.array([1.0, 2.0, 3.0, 4.0])
    with pytest.raises(ValueError):                       # row 2 is not in block 0
        oracle.table_build_sampled(row_ptr, val, 2, 2, np.array([2, 3], np.int64))
    with pytest.raises(ValueError):                       # a sample row past the last row
        oracle.table_build_sampled(row_ptr, val, 2, 3, np.array([0, 4], np.int64))
    with pytest.raises(ValueError):                       # Inf outside the sampled rows
        oracle.table_build_sampled(row_ptr, np.array([1.0, np.inf, 3.0, 4.0]), 2, 2, np.array([0, 2], np.int64))


# ---- index in the value --------------------------------------------------------

def test_in_value_handworked():
    rows = [l.split() for l in open(os.path.join(GOLD, "table_in_value_handworked.txt"))
            if l.strip() and not l.startswith("#")]
    vals = np.array([float.fromhex(r[0]) for r in rows])
    table = np.array([1025, 1027], np.int16)
    head, t1, t2 = oracle.table_encode_in_value(vals, table, SEG)
    assert [int(h) for h in head] == [int(r[1], 16) for r in rows]
    dec = oracle.table_decode_in_value(head, t1, t2, table, 1, SEG)
    assert np.array_equal(_bits(dec), _bits(np.array([float.fromhex(r[2]) for r in rows])))


@pytest.mark.parametrize("num_exp", [2, 4, 8, 16, 64])
def test_in_value_head_is_the_alg1_sem_word(num_exp):
    rng = np.random.default_rng(20 + num_exp)
    vals = _values(rng, 4000, -24, 24)
    vals = vals[vals != 0.0]
    table = oracle.table_build(vals, num_exp)
    b = oracle.index_bits(len(table))
    head, _, _ = oracle.table_encode_in_value(vals, table, SEG)
    checked = 0
    for i, v in enumerate(vals):
        sem, k, dist = _alg1_sem(v, table, b)
        if sem is None:                   # the explicit one falls out: sign and index, magnitude 0
            assert head[i] == (int(np.float64(v).view(np.uint64)) >> 48 & 0x8000) | (k << (15 - b))
            continue
        assert head[i] == sem, (i, v, hex(head[i]), hex(sem))
        checked += 1
    assert checked > 1000


def test_in_value_lossless_when_every_exponent_is_shared():
    # 16/16/32 with b index bits leaves 63 - b magnitude bits; a value whose e + 1
    # is an entry needs 53 of them, so for b <= 10 nothing is cut
    rng = np.random.default_rng(21)
    vals = _values(rng, 5000, -30, 30)
    distinct = len(set(int(e) for e in _exps(vals) if e != 0))
    seg = (16, 16, 32)
    table = oracle.table_build(vals, distinct)
    assert oracle.index_bits(len(table)) == 6
    enc = oracle.table_encode_in_value(vals, table, seg)
    assert np.array_equal(_bits(oracle.table_decode_in_value(*enc, table, 3, seg)), _bits(vals))


def test_in_value_truncation_bound_and_prefix():
    rng = np.random.default_rng(22)
    vals = _values(rng, 5000, -12, 12)
    table = oracle.table_build(vals, 8)
    b = oracle.index_bits(len(table))
    assert b == 3
    enc = oracle.table_encode_in_value(vals, table, SEG)
    _, _, _, idx = oracle.table_encode(vals, table, SEG)   # the entry Alg. 1 picks does not move
    T = table[idx].astype(np.int64)
    assert np.array_equal((enc[0] >> (15 - b)) & ((1 << b) - 1), idx)
    prev = np.zeros_like(vals)
    for k, W in zip((1, 2, 3), (15, 31, 51)):
        a = oracle.table_decode_in_value(*enc, table, k, SEG)
        assert np.all(np.abs(a) <= np.abs(vals))
        assert np.all(np.sign(a[a != 0]) == np.sign(vals[a != 0]))
        assert np.all(np.abs(vals - a) < np.ldexp(1.0, (T - 1023 - (W - b)).astype(np.int32)))
        assert np.all(np.abs(a) >= np.abs(prev))
        prev = a


def test_in_value_spmv_brute_force():
    rng = np.random.default_rng(23)
    n = 40
    dense = np.where(rng.random((n, n)) < 0.2, rng.integers(-9, 10, (n, n)) * 2.0 ** rng.integers(-3, 4, (n, n)), 0.0)
    rows, cols = np.nonzero(dense)
    val = dense[rows, cols]
    row_ptr = np.zeros(n + 1, np.int32)
    np.cumsum(np.bincount(rows, minlength=n), out=row_ptr[1:])
    table = oracle.table_build(val, 4)
    enc = oracle.table_encode_in_value(val, table, SEG)
    x = rng.integers(-5, 6, n).astype(np.float64)
    for k in (1, 2, 3):
        a = oracle.table_decode_in_value(*enc, table, k, SEG)
        y = oracle.spmv(row_ptr, cols.astype(np.int32), a, x)
        A = np.zeros((n, n))
        A[rows, cols] = a
        assert np.array_equal(y, A @ x)


def test_in_value_rejects_too_many_index_bits():
    vals = 2.0 ** np.arange(-20, 20, dtype=np.float64)
    table = oracle.table_build(vals, 64)                   # 40 entries: 6 index bits
    with pytest.raises(ValueError):                        # a 6-bit head has no magnitude bit left
        oracle.table_encode_in_value(vals, table, (6, 16, 20))
    oracle.table_encode_in_value(vals, table, (8, 16, 20))
