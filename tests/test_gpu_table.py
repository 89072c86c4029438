"""The paper's global shared-exponent table format on the GPU vs the oracle
(Sec. III-B "Shared Exponents Extraction", Alg. 1, Alg. 2, Sec. III-C):
bit-exact table, indices and segments; bit-exact decode; SpMV within
1e-13 * sum_j |a_ij x_j| of the oracle's Dot2 sum at every level and schedule;
stepped CG on the table levels; the index kept in the head when the column
word has no spare bits (Sec. III-C); the sampled extraction (Sec. III-B)."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import check_spmv_rows

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2411_04686_gb300 as gse  # noqa: E402

SEG = (16, 16, 20)


def _extreme_range():
    rng = np.random.default_rng(14)
    n, m = 2000, 2000
    lens = rng.integers(1, 20, n)
    rp = np.zeros(n + 1, np.int64)
    np.cumsum(lens, out=rp[1:])
    col = np.concatenate([np.sort(rng.choice(m, L, replace=False)) for L in lens])
    val = rng.choice([-1.0, 1.0], rp[-1]) * 2.0 ** rng.uniform(-1022, 1015, rp[-1])
    return synth.CSR(rp.astype(np.int32), col.astype(np.int32), val, m, "extreme_range")


MATS = {
    "poisson32_third": lambda: synth.poisson2d(32, 1.0 / 3.0),
    "extreme_range": _extreme_range,
    "laplace3d_24": lambda: synth.laplace3d(24, shift=1e-3),
    "powerlaw_50k": lambda: synth.powerlaw_random(50000, 16.0, 2048, seed=11),
    "tiny": lambda: synth.CSR(np.array([0, 1, 3], np.int32), np.array([1, 0, 1], np.int32),
                              np.array([2.5, -1.0, 1 / 3]), 2, "tiny"),
}


@pytest.mark.parametrize("name", list(MATS))
@pytest.mark.parametrize("num_exp", [1, 2, 8, 64])
def test_table_encode_bit_exact(name, num_exp):
    A = MATS[name]()
    M = gse.GseMatrix.from_csr(A, num_exp=num_exp)
    table, idx = M.export_table()
    ref_table = oracle.table_build(A.val, num_exp)
    assert table.tolist() == ref_table.tolist()
    rh, r1, r2, ridx = oracle.table_encode(A.val, ref_table, SEG)
    assert np.array_equal(idx, ridx)
    head, t1, t2, _ = M.export()
    assert np.array_equal(head, rh) and np.array_equal(t1, r1) and np.array_equal(t2, r2)
    assert M.info().num_exp == len(table)
    for k in (1, 2, 3):
        dec = M.decode(k).cpu().numpy()
        ref = oracle.table_decode(rh, r1, r2, ridx, ref_table, k, SEG)
        assert np.array_equal(dec.view(np.uint64), ref.view(np.uint64)), k


@pytest.mark.parametrize("name", list(MATS))
@pytest.mark.parametrize("sched", [1, gse.SCHEDULE_ROWS])
@pytest.mark.parametrize("num_exp", [1, 8, 64])
def test_table_spmv_against_oracle(name, sched, num_exp):
    A = MATS[name]()
    M = gse.GseMatrix.from_csr(A, num_exp=num_exp, attach=(64,))
    try:
        M.set_schedule(sched)
    except gse.GseError as e:          # row blocks too wide for the row schedule
        assert e.code == gse.ERR_UNSUPPORTED and sched == gse.SCHEDULE_ROWS
        return
    x = synth.uniform_x(A.n_cols, seed=4)
    xd = torch.from_numpy(x).cuda()
    table, levels = oracle.table_levels(A.val, num_exp, SEG)
    for k in (1, 2, 3):
        y = M.spmv(k, xd).cpu().numpy()
        check_spmv_rows(y, A, levels[k - 1], x)
    # the FP64 baseline masks the exponent index out of the column words
    y64 = M.spmv(gse.LEVEL_FP64, xd).cpu().numpy()
    check_spmv_rows(y64, A, A.val, x)


@pytest.mark.parametrize("name,sched", [("laplace3d_128", gse.SCHEDULE_ROWS), ("powerlaw_1m", 1)])
def test_table_spmv_full_size_sampled(name, sched):
    A = synth.laplace3d(128) if name == "laplace3d_128" else synth.powerlaw_random(1_000_000, 16.0, 2048, seed=0)
    M = gse.GseMatrix.from_csr(A, num_exp=8)
    M.set_schedule(sched)
    x = synth.uniform_x(A.n_cols, seed=0)
    xd = torch.from_numpy(x).cuda()
    table, levels = oracle.table_levels(A.val, 8, SEG)
    rows = np.random.default_rng(1).choice(A.n_rows, 3000, replace=False)
    for k in (1, 2, 3):
        y = M.spmv(k, xd).cpu().numpy()
        check_spmv_rows(y, A, levels[k - 1], x, rows=rows)


def test_table_stepped_cg_against_oracle():
    A = synth.poisson2d(32, 1.0 / 3.0)
    M = gse.GseMatrix.from_csr(A, num_exp=8)
    b = synth.rhs_ones(A)
    x = torch.zeros(A.n_rows, dtype=torch.float64, device="cuda")
    info = M.cg(torch.from_numpy(b).cuda(), x, tol=1e-10, policy=gse.SCALED_CG)
    _, levels = oracle.table_levels(A.val, 8, SEG)
    ref = oracle.stepped_cg(A.row_ptr, A.col, levels, b, tol=1e-10, policy=oracle.SCALED_CG)
    assert info["status"] == gse.OK and info["rel_res_true"] < 1e-10
    assert info["k_final"] == ref["info"]["k_final"]
    assert abs(info["iters"] - ref["info"]["iters"]) <= 3
    assert np.max(np.abs(x.cpu().numpy() - ref["x"])) < 1e-8


def test_table_gmres_runs():
    A = synth.convdiff2d(32)
    M = gse.GseMatrix.from_csr(A, num_exp=8)
    b = synth.rhs_ones(A)
    x = torch.zeros(A.n_rows, dtype=torch.float64, device="cuda")
    info = M.gmres(torch.from_numpy(b).cuda(), x, tol=1e-10, policy=gse.SCALED_GMRES)
    assert info["status"] == gse.OK and info["rel_res_true"] < 1e-10


def _wide_matrix():
    # 40 distinct exponents -> 6 index bits -> columns must stay below 2^26 in the col word
    vals = 2.0 ** np.arange(-20, 20, dtype=np.float64) * np.where(np.arange(40) % 3, 1.0, -1.5)
    n_cols = (1 << 26) + 8
    cols = np.sort(np.random.default_rng(2).choice(n_cols, vals.size, replace=False)).astype(np.int32)
    cols[-1] = n_cols - 1
    return synth.CSR(np.array([0, 25, vals.size], np.int32), cols, vals, n_cols, "wide")


def test_table_index_without_spare_column_bits_goes_in_the_head():
    """Sec. III-C: when the column index has no spare bits for the exponent
    index, the value holds it.  Forcing the column word is refused; the default
    placement moves the index into the head and matches the oracle bit for bit."""
    A = _wide_matrix()
    with pytest.raises(gse.GseError) as e:
        gse.GseMatrix.from_csr(A, num_exp=64, index_place=gse.INDEX_COL)
    assert e.value.code == gse.ERR_UNSUPPORTED
    M = gse.GseMatrix.from_csr(A, num_exp=64)
    assert M.info().index_in_head == 1
    table = oracle.table_build(A.val, 64)
    rh, r1, r2 = oracle.table_encode_in_value(A.val, table, SEG)
    head, t1, t2, _ = M.export()
    assert np.array_equal(head, rh) and np.array_equal(t1, r1) and np.array_equal(t2, r2)
    x = synth.uniform_x(A.n_cols, seed=3)
    xd = torch.from_numpy(x).cuda()
    for k in (1, 2, 3):
        ref = oracle.table_decode_in_value(rh, r1, r2, table, k, SEG)
        check_spmv_rows(M.spmv(k, xd).cpu().numpy(), A, ref, x)
    del xd
    # with few entries the index fits in the column word
    assert gse.GseMatrix.from_csr(A, num_exp=2).info().index_in_head == 0


def test_table_rejects_bad_num_exp():
    A = synth.poisson2d(8)
    for ne in (-1, 65):
        with pytest.raises(gse.GseError) as e:
            gse.GseMatrix.from_csr(A, num_exp=ne)
        assert e.value.code == gse.ERR_INVALID


def test_batch_mixing_formats_and_schedules_equals_solo_bitwise():
    """One engine launch mixing per-group and table-format systems on both
    schedules (row and nonzero split) gives each system its solo result."""
    As = [s.build() for s in synth.batch_specs(9, seed=9, n_lo=300, n_hi=15000)]
    mats = []
    for i, A in enumerate(As):
        M = gse.GseMatrix.from_csr(A, num_exp=8 if i % 2 else 0)
        if i % 3 == 0:
            M.set_schedule(1)               # nonzero split in the engine
        mats.append(M)
    bs = [torch.from_numpy(synth.rhs_ones(A)).cuda() for A in As]
    xs = [torch.zeros(A.n_rows, dtype=torch.float64, device="cuda") for A in As]
    rc, infos = gse.batch_cg(mats, bs, xs)
    assert rc == gse.OK
    for M, A, b, xb, ib in zip(mats, As, bs, xs, infos):
        x1 = torch.zeros(A.n_rows, dtype=torch.float64, device="cuda")
        i1 = M.cg(b, x1)
        assert ib["status"] == gse.OK and ib["rel_res_true"] < 1e-10
        assert ib["iters"] == i1["iters"] and ib["switch_iter"] == i1["switch_iter"]
        assert torch.equal(xb, x1)


# ---- the exponent index kept in the head (GSE_INDEX_VALUE) -----------------------

@pytest.mark.parametrize("name", list(MATS))
@pytest.mark.parametrize("num_exp", [1, 2, 8, 64])
def test_table_in_value_bit_exact(name, num_exp):
    A = MATS[name]()
    M = gse.GseMatrix.from_csr(A, num_exp=num_exp, index_place=gse.INDEX_VALUE)
    table, idx = M.export_table()
    ref_table = oracle.table_build(A.val, num_exp)
    assert table.tolist() == ref_table.tolist()
    assert M.info().index_in_head == (1 if len(table) > 1 else 0)
    rh, r1, r2 = oracle.table_encode_in_value(A.val, ref_table, SEG)
    head, t1, t2, _ = M.export()
    assert np.array_equal(head, rh) and np.array_equal(t1, r1) and np.array_equal(t2, r2)
    assert np.array_equal(idx, oracle.table_encode(A.val, ref_table, SEG)[3])
    for k in (1, 2, 3):
        dec = M.decode(k).cpu().numpy()
        ref = oracle.table_decode_in_value(rh, r1, r2, ref_table, k, SEG)
        assert np.array_equal(dec.view(np.uint64), ref.view(np.uint64)), k


@pytest.mark.parametrize("name", list(MATS))
@pytest.mark.parametrize("sched", [1, gse.SCHEDULE_ROWS])
def test_table_in_value_spmv_against_oracle(name, sched):
    A = MATS[name]()
    M = gse.GseMatrix.from_csr(A, num_exp=8, index_place=gse.INDEX_VALUE, attach=(64,))
    try:
        M.set_schedule(sched)
    except gse.GseError as e:
        assert e.code == gse.ERR_UNSUPPORTED and sched == gse.SCHEDULE_ROWS
        return
    x = synth.uniform_x(A.n_cols, seed=5)
    xd = torch.from_numpy(x).cuda()
    _, levels = oracle.table_levels(A.val, 8, SEG, index_in_value=True)
    for k in (1, 2, 3):
        check_spmv_rows(M.spmv(k, xd).cpu().numpy(), A, levels[k - 1], x)
    check_spmv_rows(M.spmv(gse.LEVEL_FP64, xd).cpu().numpy(), A, A.val, x)


@pytest.mark.parametrize("name,sched", [("laplace3d_128", gse.SCHEDULE_ROWS), ("powerlaw_1m", 1)])
def test_table_in_value_full_size_sampled(name, sched):
    A = synth.laplace3d(128) if name == "laplace3d_128" else synth.powerlaw_random(1_000_000, 16.0, 2048, seed=0)
    M = gse.GseMatrix.from_csr(A, num_exp=8, index_place=gse.INDEX_VALUE)
    M.set_schedule(sched)
    x = synth.uniform_x(A.n_cols, seed=0)
    xd = torch.from_numpy(x).cuda()
    _, levels = oracle.table_levels(A.val, 8, SEG, index_in_value=True)
    rows = np.random.default_rng(2).choice(A.n_rows, 3000, replace=False)
    for k in (1, 2, 3):
        check_spmv_rows(M.spmv(k, xd).cpu().numpy(), A, levels[k - 1], x, rows=rows)


def test_table_in_value_stepped_cg_against_oracle():
    A = synth.poisson2d(32, 1.0 / 3.0)
    M = gse.GseMatrix.from_csr(A, num_exp=8, index_place=gse.INDEX_VALUE)
    b = synth.rhs_ones(A)
    x = torch.zeros(A.n_rows, dtype=torch.float64, device="cuda")
    info = M.cg(torch.from_numpy(b).cuda(), x, tol=1e-10, policy=gse.SCALED_CG)
    _, levels = oracle.table_levels(A.val, 8, SEG, index_in_value=True)
    ref = oracle.stepped_cg(A.row_ptr, A.col, levels, b, tol=1e-10, policy=oracle.SCALED_CG)
    assert info["status"] == gse.OK and info["rel_res_true"] < 1e-10
    assert info["k_final"] == ref["info"]["k_final"]
    assert abs(info["iters"] - ref["info"]["iters"]) <= 3
    assert np.max(np.abs(x.cpu().numpy() - ref["x"])) < 1e-8


def test_table_in_value_needs_a_magnitude_bit():
    # 40 entries take 6 index bits; a 7-bit head would keep no magnitude bit
    vals = _wide_matrix().val
    A = synth.CSR(np.array([0, vals.size], np.int32), np.arange(vals.size, dtype=np.int32), vals, 64, "narrow")
    with pytest.raises(gse.GseError) as e:
        gse.GseMatrix.from_csr(A, num_exp=64, index_place=gse.INDEX_VALUE, seg_bits=(7, 16, 20))
    assert e.value.code == gse.ERR_UNSUPPORTED
    M = gse.GseMatrix.from_csr(A, num_exp=64, index_place=gse.INDEX_VALUE, seg_bits=(8, 16, 20))
    table = oracle.table_build(A.val, 64)
    rh, _, _ = oracle.table_encode_in_value(A.val, table, (8, 16, 20))
    assert np.array_equal(M.export()[0], rh)


# ---- sampled exponent extraction (Sec. III-B) --------------------------------------

@pytest.mark.parametrize("name", list(MATS) + ["powerlaw_1m"])
@pytest.mark.parametrize("block_rows", [1, 16, 256])
def test_table_sampled_bit_exact(name, block_rows):
    A = synth.powerlaw_random(1_000_000, 16.0, 2048, seed=0) if name == "powerlaw_1m" else MATS[name]()
    rows = synth.sample_rows(A.n_rows, block_rows, seed=block_rows)
    M = gse.GseMatrix.from_csr(A, num_exp=8, sample_block_rows=block_rows, sample_rows=rows)
    table, idx = M.export_table()
    ref_table = oracle.table_build_sampled(A.row_ptr, A.val, 8, block_rows, rows)
    assert table.tolist() == ref_table.tolist()
    if block_rows == 1:
        assert table.tolist() == oracle.table_build(A.val, 8).tolist()
    rh, r1, r2, ridx = oracle.table_encode(A.val, ref_table, SEG)
    head, t1, t2, _ = M.export()
    assert np.array_equal(idx, ridx)
    assert np.array_equal(head, rh) and np.array_equal(t1, r1) and np.array_equal(t2, r2)
    if A.nnz < 100_000:
        x = synth.uniform_x(A.n_cols, seed=6)
        xd = torch.from_numpy(x).cuda()
        for k in (1, 2, 3):
            ref = oracle.table_decode(rh, r1, r2, ridx, ref_table, k, SEG)
            check_spmv_rows(M.spmv(k, xd).cpu().numpy(), A, ref, x)


def test_table_sampled_rejects_bad_rows():
    A = synth.poisson2d(8)                                  # 64 rows: 4 blocks of 16
    for rows in ([17, 16, 32, 48],                          # row 17 is not in block 0
                 [0, 16, 32, 64]):                          # row 64 is past the last row
        with pytest.raises(gse.GseError) as e:
            gse.GseMatrix.from_csr(A, num_exp=4, sample_block_rows=16, sample_rows=np.array(rows, np.int64))
        assert e.value.code == gse.ERR_INVALID
    with pytest.raises(ValueError):                         # one row per block
        gse.GseMatrix.from_csr(A, num_exp=4, sample_block_rows=16, sample_rows=np.array([0, 16], np.int64))
