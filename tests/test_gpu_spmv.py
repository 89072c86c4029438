"""GPU GSE-SpMV (Sec. III-C, Alg. 2 and its tail variants) and the FP64/FP32 CSR
baselines vs the oracle: every row within 1e-13 * sum_j |a_ij x_j| of the
compensated (Dot2) oracle sum over the same decoded values; empty rows exactly 0."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import check_spmv_rows

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2411_04686_gb300 as gse  # noqa: E402


def _with_empty_rows(seed):
    rng = np.random.default_rng(seed)
    n, m = 4000, 3000
    lens = rng.integers(0, 40, n)
    lens[:5] = 0
    lens[-7:] = 0
    lens[rng.random(n) < 0.2] = 0
    rp = np.zeros(n + 1, np.int64)
    np.cumsum(lens, out=rp[1:])
    col = np.concatenate([np.sort(rng.choice(m, L, replace=False)) for L in lens])
    val = rng.normal(size=rp[-1]) * 10.0 ** rng.uniform(-5, 5, rp[-1])
    return synth.CSR(rp.astype(np.int32), col.astype(np.int32), val, m, "empty_rows")


def _one_long_row():
    n_cols = 20000
    rng = np.random.default_rng(7)
    col = np.sort(rng.choice(n_cols, 9000, replace=False))
    rp = np.array([0, 3, 3, 3 + 9000, 3 + 9000 + 5], np.int32)
    cols = np.concatenate([[1, 5, 9], col, [0, 1, 2, 3, 4]]).astype(np.int32)
    val = rng.normal(size=cols.size)
    return synth.CSR(rp, cols, val, n_cols, "long_row")


def _extreme_range():
    """Magnitudes 2^U(-1022, 1015): groups from the smallest normal exponents up
    to E_g near the top, products down in the subnormal range (no row sum can
    overflow)."""
    rng = np.random.default_rng(13)
    n, m = 3000, 3000
    lens = rng.integers(1, 24, n)
    rp = np.zeros(n + 1, np.int64)
    np.cumsum(lens, out=rp[1:])
    col = np.concatenate([np.sort(rng.choice(m, L, replace=False)) for L in lens])
    val = rng.choice([-1.0, 1.0], rp[-1]) * 2.0 ** rng.uniform(-1022, 1015, rp[-1])
    return synth.CSR(rp.astype(np.int32), col.astype(np.int32), val, m, "extreme_range")


def _band41():
    """Rows of 41 nonzeros (|i - j| <= 20) with values in [1, 2): one group
    exponent, rows spanning two or three groups of 32, batches of 8 plus a
    remainder; n = 1481 is not a multiple of 32."""
    n = 1481
    i = np.arange(n)
    cols = i[:, None] + np.arange(-20, 21)[None, :]
    valid = (cols >= 0) & (cols < n)
    vals = 1.0 + ((i[:, None] * 7 + cols * 3) % 11) / 11.0
    lens = valid.sum(1)
    rp = np.zeros(n + 1, np.int64)
    np.cumsum(lens, out=rp[1:])
    return synth.CSR(rp.astype(np.int32), cols[valid].astype(np.int32), vals[valid], n, "band41")


MATS = {
    # off-diagonals 1e-6 of the diagonal: zero head magnitudes, the leading one
    # in tail1 (level 2) and tail2 (level 3), one exponent per group
    "aniso_tiny": lambda: synth.laplace2d(40, 37, shift=0.5, aniso=(1.0, 1e-6)),
    "band41": _band41,
    "poisson32": lambda: synth.poisson2d(32),
    "extreme_range": _extreme_range,
    "poisson32_third": lambda: synth.poisson2d(32, 1.0 / 3.0),
    "laplace3d_24": lambda: synth.laplace3d(24, shift=1e-3),
    "powerlaw_50k": lambda: synth.powerlaw_random(50000, 16.0, 2048, seed=11),
    "empty_rows": lambda: _with_empty_rows(12),
    "long_row": _one_long_row,
    "tiny": lambda: synth.CSR(np.array([0, 1, 3], np.int32), np.array([1, 0, 1], np.int32),
                              np.array([2.5, -1.0, 1 / 3]), 2, "tiny"),
    "all_empty": lambda: synth.CSR(np.zeros(6, np.int32), np.zeros(0, np.int32), np.zeros(0), 4, "empty"),
}


@pytest.mark.parametrize("name", list(MATS))
@pytest.mark.parametrize("upl", [1, 2, 4, gse.SCHEDULE_ROWS])
def test_spmv_levels_against_oracle(name, upl):
    A = MATS[name]()
    M = gse.GseMatrix.from_csr(A, attach=(64, 32))
    if upl == gse.SCHEDULE_ROWS:
        span = 0
        for rb in (128, 256):            # row blocks of the engine's and the SpMV's CTAs
            blocks = A.row_ptr[np.minimum(np.arange(0, A.n_rows + rb, rb), A.n_rows)].astype(np.int64)
            if A.n_rows:
                span = max(span, int(np.max((((blocks[1:] + 31) >> 5) << 5) - ((blocks[:-1] >> 5) << 5))))
        if span > 4096:                  # a row block too wide for the row schedule
            with pytest.raises(gse.GseError) as e:
                M.set_schedule(upl)
            assert e.value.code == gse.ERR_UNSUPPORTED
            return
    M.set_schedule(upl)
    x = synth.uniform_x(A.n_cols, seed=3)
    xd = torch.from_numpy(x).cuda()
    enc = oracle.encode(A.val)
    for k in (1, 2, 3):
        ak = oracle.decode(*enc, k)
        y = M.spmv(k, xd).cpu().numpy()
        check_spmv_rows(y, A, ak, x)
        # deterministic: a second run is bit-identical
        y2 = M.spmv(k, xd).cpu().numpy()
        assert np.array_equal(y.view(np.uint64), y2.view(np.uint64))
    y64 = M.spmv(gse.LEVEL_FP64, xd).cpu().numpy()
    check_spmv_rows(y64, A, A.val, x)
    if name != "extreme_range":          # FP32 cannot hold these values (inf / 0)
        y32 = M.spmv(gse.LEVEL_FP32, xd).cpu().numpy()
        check_spmv_rows(y32, A, A.val.astype(np.float32).astype(np.float64), x)
    M.free()


@pytest.mark.parametrize("seg,G", [((16, 16, 32), 32), ((16, 16, 16), 32), ((12, 16, 24), 32), ((16, 8, 8), 32),
                                   ((2, 16, 20), 32), ((16, 16, 20), 16), ((16, 16), 32), ((16,), 32)])
@pytest.mark.parametrize("upl", [1, 2, gse.SCHEDULE_ROWS])
def test_spmv_other_layouts_against_oracle(seg, G, upl):
    """Segment widths and group sizes other than the default 16/16/20 with groups
    of 32: the kernels read the widths from the matrix view (the default layout
    runs kernels with the widths compiled in)."""
    for A in (synth.powerlaw_random(20000, 16.0, 2048, seed=21), synth.poisson2d(40, 1.0 / 3.0)):
        M = gse.GseMatrix.from_csr(A, group_size=G, seg_bits=seg)
        try:
            M.set_schedule(upl)
        except gse.GseError as e:        # a row block too wide for the row schedule
            assert upl == gse.SCHEDULE_ROWS and e.code == gse.ERR_UNSUPPORTED
            M.free()
            continue
        x = synth.uniform_x(A.n_cols, seed=6)
        xd = torch.from_numpy(x).cuda()
        enc = oracle.encode(A.val, G, seg)
        for k in range(1, len(seg) + 1):
            check_spmv_rows(M.spmv(k, xd).cpu().numpy(), A, oracle.decode(*enc, k, G, seg), x)
        M.free()


def test_x_ones_integer_matrix_exact():
    """Sec. IV-A's x = 1 setting: 5-point Poisson at every level is exact."""
    A = synth.poisson2d(64)
    M = gse.GseMatrix.from_csr(A)
    ones = torch.ones(A.n_cols, dtype=torch.float64, device="cuda")
    deg = np.diff(A.row_ptr) - 1
    for k in (1, 2, 3):
        assert np.array_equal(M.spmv(k, ones).cpu().numpy(), 4.0 - deg)


@pytest.mark.parametrize("which", ["laplace3d_128", "powerlaw_1m"])
def test_full_size_sampled_rows(which):
    """The benchmark matrices at full size, in the launch configuration the
    benchmark times: 4000 sampled rows checked against the oracle."""
    A = synth.laplace3d(128) if which == "laplace3d_128" else synth.powerlaw_random(1_000_000, 16.0, 2048, seed=0)
    M = gse.GseMatrix.from_csr(A, attach=(64, 32))   # the schedule the benchmark runs (row statistics)
    x = synth.uniform_x(A.n_cols, seed=0)
    xd = torch.from_numpy(x).cuda()
    rng = np.random.default_rng(1)
    rows = np.unique(np.concatenate([rng.choice(A.n_rows, 4000, replace=False),
                                     [0, A.n_rows - 1, int(np.argmax(np.diff(A.row_ptr)))]]))
    enc = oracle.encode(A.val)
    for k in (1, 2, 3):
        ak = oracle.decode(*enc, k)
        check_spmv_rows(M.spmv(k, xd).cpu().numpy(), A, ak, x, rows=rows)
    check_spmv_rows(M.spmv(gse.LEVEL_FP64, xd).cpu().numpy(), A, A.val, x, rows=rows)
    M.free()


def test_autotune_keeps_results_within_tolerance():
    A = synth.powerlaw_random(30000, 16.0, 2048, seed=13)
    M = gse.GseMatrix.from_csr(A)
    M.autotune(2)
    x = synth.uniform_x(A.n_cols, seed=4)
    enc = oracle.encode(A.val)
    check_spmv_rows(M.spmv(2, torch.from_numpy(x).cuda()).cpu().numpy(), A, oracle.decode(*enc, 2), x)


def test_bad_level_rejected():
    A = synth.poisson2d(8)
    M = gse.GseMatrix.from_csr(A, seg_bits=(16, 16))
    x = torch.zeros(A.n_cols, dtype=torch.float64, device="cuda")
    for k in (0, 3, 64, 32):
        with pytest.raises(gse.GseError):
            M.spmv(k, x)
