"""Pins for the oracle's SpMV (Sec. III-C): brute force, exact rational sums,
the Dot2 error bound, and integer matrices with x = 1 (the Sec. IV-A setting)."""
from fractions import Fraction

import numpy as np

import oracle
import synth

U = 2.0 ** -53


def _tiny_random(rng, n, m, density=0.3):
    dense = np.where(rng.random((n, m)) < density,
                     rng.choice([-1.0, 1.0], (n, m)) * 10.0 ** rng.uniform(-3, 3, (n, m)), 0.0)
    dense[rng.integers(0, n)] = 0.0           # at least one empty row
    rows, cols = np.nonzero(dense)
    row_ptr = np.zeros(n + 1, np.int32)
    np.cumsum(np.bincount(rows, minlength=n), out=row_ptr[1:])
    return row_ptr, cols.astype(np.int32), dense[rows, cols], dense


def test_spmv_matches_dense_and_exact_sum():
    rng = np.random.default_rng(0)
    for trial in range(20):
        n, m = rng.integers(1, 40), rng.integers(1, 40)
        rp, col, val, dense = _tiny_random(rng, n, m)
        x = rng.uniform(-1, 1, m)
        y = oracle.spmv(rp, col, val, x)
        ya = np.abs(dense) @ np.abs(x)
        for i in range(n):
            exact = sum(Fraction(float(dense[i, j])) * Fraction(float(x[j])) for j in range(m))
            cnt = rp[i + 1] - rp[i]
            gamma = cnt * U / (1 - cnt * U)
            # standard bound for recursive summation of products
            assert abs(Fraction(float(y[i])) - exact) <= Fraction(gamma * ya[i] * 1.0000001), (trial, i)
            if cnt == 0:
                assert y[i] == 0.0
        assert np.allclose(y, dense @ x, rtol=0, atol=1e-12 * (ya.max() + 1))


def test_dot2_error_bound_against_exact():
    """Ogita-Rump-Oishi: |Dot2 - x'y| <= u |x'y| + gamma_n^2 sum|x_i y_i|."""
    rng = np.random.default_rng(1)
    # ill-conditioned rows: large cancelling terms
    n = 30
    rows = []
    for i in range(n):
        L = int(rng.integers(2, 60))
        big = rng.uniform(-1, 1, L // 2) * 1e8
        v = np.concatenate([big, -big * (1 + rng.uniform(-1e-9, 1e-9, L // 2)), rng.uniform(-1, 1, L % 2)])
        rows.append(v)
    m = max(len(v) for v in rows)
    rp = np.zeros(n + 1, np.int32)
    rp[1:] = np.cumsum([len(v) for v in rows])
    col = np.concatenate([np.arange(len(v)) for v in rows]).astype(np.int32)
    val = np.concatenate(rows)
    x = rng.uniform(0.5, 1.5, m)
    y2, ya = oracle.spmv_dot2(rp, col, val, x)
    for i in range(n):
        exact = sum(Fraction(float(a)) * Fraction(float(x[c])) for a, c in zip(rows[i], range(len(rows[i]))))
        L = len(rows[i])
        g = L * U / (1 - L * U)
        bound = U * abs(exact) + Fraction(g * g * ya[i] * 1.0001)
        assert abs(Fraction(float(y2[i])) - exact) <= bound, i


def test_gse_spmv_is_decode_then_fp64_spmv():
    rng = np.random.default_rng(2)
    A = synth.powerlaw_random(2000, 8.0, 300, seed=3)
    x = rng.uniform(-1, 1, A.n_cols)
    enc = oracle.encode(A.val)
    for k in (1, 2, 3):
        ak = oracle.decode(*enc, k)
        y = oracle.gse_spmv(A.row_ptr, A.col, enc, k, x)
        assert np.array_equal(y, oracle.spmv(A.row_ptr, A.col, ak, x))
        # and the dense product of the decoded matrix agrees to rounding
        rows = np.repeat(np.arange(A.n_rows), np.diff(A.row_ptr))
        yd = np.bincount(rows, weights=ak * x[A.col], minlength=A.n_rows)
        ya = np.bincount(rows, weights=np.abs(ak * x[A.col]), minlength=A.n_rows)
        assert np.all(np.abs(y - yd) <= 1e-13 * ya + 1e-300)


def test_integer_matrix_times_ones_is_exact():
    """Sec. IV-A sets the SpMV input vector to ones; with small-integer values
    every level is exact and so is every row sum."""
    A = synth.poisson2d(32)
    ones = np.ones(A.n_cols)
    enc = oracle.encode(A.val)
    for k in (1, 2, 3):
        y = oracle.gse_spmv(A.row_ptr, A.col, enc, k, ones)
        deg = np.diff(A.row_ptr) - 1
        assert np.array_equal(y, 4.0 - deg)


def test_row_scale_is_the_sum_of_absolute_products():
    """The parity scale sum_j |a_ij x_j| (returned beside Dot2) against exact
    rational sums: a sum of L nonnegative FP64 products is within
    gamma_(L+1) of the exact value, and a row with cancelling terms keeps its
    full magnitude."""
    rng = np.random.default_rng(7)
    rp, col, val, dense = _tiny_random(rng, 25, 30, density=0.5)
    x = rng.uniform(-1, 1, 30)
    _, ya = oracle.spmv_dot2(rp, col, val, x)
    for i in range(25):
        exact = sum(abs(Fraction(float(dense[i, j])) * Fraction(float(x[j]))) for j in range(30))
        L = int(rp[i + 1] - rp[i])
        g = (L + 1) * U / (1 - (L + 1) * U)
        assert abs(Fraction(float(ya[i])) - exact) <= Fraction(g) * exact, i
    # +a and -a in one row: y = 0, scale = 2|a|
    y2, ya2 = oracle.spmv_dot2(np.array([0, 2], np.int32), np.array([0, 1], np.int32),
                               np.array([3.0, -3.0]), np.array([0.5, 0.5]))
    assert y2[0] == 0.0 and ya2[0] == 3.0


def test_row_range_and_threads_sum_rows_as_the_full_spmv():
    """orc_gse_spmv_rows (the timed CPU baselines' routine: a row range, rows
    shared among threads) sums every row exactly as orc_gse_spmv does."""
    A = synth.powerlaw_random(6000, 16.0, 512, seed=4)
    x = synth.uniform_x(A.n_cols, seed=2)
    enc = oracle.encode(A.val)
    for k in (1, 2, 3):
        y = oracle.gse_spmv(A.row_ptr, A.col, enc, k, x)
        for threads in (1, 3):
            yr = oracle.gse_spmv_rows(A.row_ptr, A.col, enc, k, x, 0, A.n_rows, threads=threads)
            assert np.array_equal(y.view(np.uint64), yr.view(np.uint64))
        part = oracle.gse_spmv_rows(A.row_ptr, A.col, enc, k, x, 250, 4100, threads=2)
        assert np.array_equal(part[250:4100].view(np.uint64), y[250:4100].view(np.uint64))
        assert not part[:250].any() and not part[4100:].any()
