"""The input recipe: the seeded generators build the matrices, vectors and
system mixes that the tests and the benchmark describe (sizes, stencils,
row-length law, value ranges, determinism).  CPU only."""
import numpy as np
import pytest

import synth


def _check_csr(A):
    rp, col = A.row_ptr, A.col
    assert rp.dtype == np.int32 and col.dtype == np.int32 and A.val.dtype == np.float64
    assert rp[0] == 0 and np.all(np.diff(rp) >= 0) and rp[-1] == col.size == A.val.size
    assert col.size == 0 or (col.min() >= 0 and col.max() < A.n_cols)
    # columns strictly increasing inside every row
    inside = np.ones(col.size, bool)
    inside[rp[1:-1][rp[1:-1] < col.size]] = False
    if col.size:
        inside[0] = False
        assert np.all(np.diff(col.astype(np.int64))[inside[1:]] > 0)


@pytest.mark.parametrize("N", [1, 2, 5, 32])
def test_poisson2d_size_and_stencil(N):
    A = synth.poisson2d(N)
    _check_csr(A)
    assert A.n_rows == N * N and A.nnz == 5 * N * N - 4 * N
    D = A.dense()
    assert np.array_equal(D, D.T) and np.all(np.diag(D) == 4.0)
    assert set(np.unique(D)) <= {-1.0, 0.0, 4.0}


def test_grid_matrix_sizes_of_the_workloads():
    # 7N^3 - 6N^2 nonzeros for the 7-point stencil, 5N^2 - 4N for the 5-point
    for N in (2, 3, 7):
        assert synth.laplace3d(N).nnz == 7 * N ** 3 - 6 * N ** 2
    A = synth.laplace3d(128)
    _check_csr(A)
    assert (A.n_rows, A.nnz) == (2_097_152, 14_581_760)
    assert 7 * 192 ** 3 - 6 * 192 ** 2 == 49_324_032 and 192 ** 3 == 7_077_888
    C = synth.convdiff2d(1024)
    assert (C.n_rows, C.nnz) == (1_048_576, 5_238_784)
    assert synth.poisson2d(32).nnz == 4992


def test_laplace3d_anisotropy_and_shift_give_an_spd_stencil():
    A = synth.laplace3d(0, shift=1e-3, aniso=(0.2, 0.5, 1.0), dims=(4, 3, 5))
    _check_csr(A)
    D = A.dense()
    assert np.array_equal(D, D.T)
    assert np.allclose(np.diag(D), 2 * (0.2 + 0.5 + 1.0) + 1e-3)
    assert set(np.round(np.unique(D[D < 0]), 12)) == {-0.2, -0.5, -1.0}
    assert np.linalg.eigvalsh(D).min() > 1e-3 * 0.999          # shift plus a positive Laplacian


def test_convdiff_upwind_stencil():
    N, pe = 6, 10.0
    A = synth.convdiff2d(N, pe)
    _check_csr(A)
    D = A.dense()
    h = 1.0 / (N + 1)
    i = 2 * N + 3                                      # an interior point
    assert D[i, i] == 4.0 + h * 2 * pe
    assert D[i, i - 1] == -1.0 - h * pe and D[i, i - N] == -1.0 - h * pe
    assert D[i, i + 1] == -1.0 and D[i, i + N] == -1.0
    assert not np.array_equal(D, D.T)                   # nonsymmetric
    assert np.allclose(D.sum(axis=1)[[i]], 0.0)          # interior rows: upwind differences of a constant vanish


def test_powerlaw_matrix_recipe():
    A = synth.powerlaw_random(1_000_000, 16.0, 2048, seed=0)
    _check_csr(A)
    lens = np.diff(A.row_ptr)
    assert A.n_rows == A.n_cols == 1_000_000
    assert lens.min() >= 1 and lens.max() == 2048
    assert abs(lens.mean() - 16.0) < 0.5
    # heavy tail: most rows are short, a few are very long
    assert np.median(lens) <= 4 and np.sum(lens >= 512) > 10
    mag = np.abs(A.val)
    assert mag.min() >= 1e-3 and mag.max() <= 1e3
    assert abs(np.mean(A.val < 0) - 0.5) < 0.01
    # log-uniform magnitudes: each decade holds about a sixth of the values
    dec = np.histogram(np.log10(mag), bins=6, range=(-3, 3))[0] / mag.size
    assert np.all(np.abs(dec - 1 / 6) < 0.01)
    # the bisected exponent gives the requested mean of the discrete law
    a = synth._powerlaw_alpha(16.0, 2048)
    L = np.arange(1, 2049.0)
    assert abs((L * L ** -a).sum() / (L ** -a).sum() - 16.0) < 1e-9


def test_generators_are_seeded():
    a = synth.powerlaw_random(5000, 8.0, 300, seed=3)
    b = synth.powerlaw_random(5000, 8.0, 300, seed=3)
    c = synth.powerlaw_random(5000, 8.0, 300, seed=4)
    assert all(np.array_equal(getattr(a, f), getattr(b, f)) for f in ("row_ptr", "col", "val"))
    assert not np.array_equal(a.val[:100], c.val[:100])
    assert np.array_equal(synth.uniform_x(1000, 0), synth.uniform_x(1000, 0))
    x = synth.uniform_x(100000, 0)
    assert x.min() >= -1 and x.max() <= 1 and abs(x.mean()) < 0.01


def test_rhs_is_a_times_ones():
    A = synth.poisson2d(9)
    assert np.array_equal(synth.rhs_ones(A), A.dense() @ np.ones(A.n_cols))


@pytest.mark.parametrize("n_rows,block", [(1000, 64), (64, 64), (65, 64), (7, 1)])
def test_sample_rows_one_per_block(n_rows, block):
    s = synth.sample_rows(n_rows, block, seed=0)
    assert s.size == -(-n_rows // block)
    assert np.all(s // block == np.arange(s.size)) and np.all(s < n_rows)


def test_batch_mix_recipe():
    specs = synth.batch_specs(512, seed=0)
    n = np.array([s.n for s in specs], float)
    dims = np.array([s.dim for s in specs])
    # grid sides round(n^(1/d)) keep n within rounding of [1e3, 2.56e5]
    assert n.min() >= 0.75 * 1e3 and n.max() <= 1.3 * 2.56e5
    # log-uniform: the median of log n sits near the middle of the range
    assert abs(np.median(np.log(n)) - 0.5 * (np.log(1e3) + np.log(2.56e5))) < 0.4
    assert 0.4 < np.mean(dims == 2) < 0.6
    for s in specs:
        assert len(s.dims) == s.dim and len(s.aniso) == s.dim
        assert all(0.01 <= e <= 1.0 for e in s.aniso) and 1e-4 <= s.shift <= 1e-1
    A = specs[0].build()
    _check_csr(A)
    assert A.n_rows == specs[0].n
    # every system is SPD: symmetric and strictly diagonally dominant (the shift)
    small = next(s for s in specs if s.n <= 2000).build()
    D = small.dense()
    assert np.array_equal(D, D.T)
    assert np.all(np.diag(D) - (np.abs(D).sum(axis=1) - np.abs(np.diag(D))) > 0)


def test_sharding_partitions_the_systems():
    specs = synth.batch_specs(37, seed=1)
    parts = [synth.shard_specs(specs, r, 4) for r in range(4)]
    ids = sorted(id(s) for p in parts for s in p)
    assert ids == sorted(id(s) for s in specs)
    assert [specs.index(s) for s in parts[1]] == list(range(1, 37, 4))      # round robin
