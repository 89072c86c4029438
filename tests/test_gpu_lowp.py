"""FP16 and BF16 baselines (Sec. IV-C) on the GPU vs the oracle: bit-exact
storage (one round to nearest even from FP64, overflow kept as infinity and
counted), SpMV within 1e-13 * sum_j |a_ij x_j| on the widened values, CG on the
16-bit matrix, and FP16 overflow surfacing as a non-finite solve."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import check_spmv_rows

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2411_04686_gb300 as gse  # noqa: E402

KINDS = {gse.LEVEL_FP16: oracle.FP16, gse.LEVEL_BF16: oracle.BF16}


def _wide_range():
    """Values from FP16-subnormal to FP16-overflow magnitudes, both signs."""
    rng = np.random.default_rng(5)
    n, m = 3000, 2000
    lens = rng.integers(1, 12, n)
    rp = np.zeros(n + 1, np.int64)
    np.cumsum(lens, out=rp[1:])
    col = np.concatenate([np.sort(rng.choice(m, L, replace=False)) for L in lens])
    val = rng.choice([-1.0, 1.0], rp[-1]) * 10.0 ** rng.uniform(-9, 6, rp[-1])
    val[::97] = -0.0
    return synth.CSR(rp.astype(np.int32), col.astype(np.int32), val, m, "wide_range")


MATS = {
    "poisson32_third": lambda: synth.poisson2d(32, 1.0 / 3.0),
    "laplace3d_20": lambda: synth.laplace3d(20, shift=1e-3),
    "powerlaw_30k": lambda: synth.powerlaw_random(30000, 16.0, 2048, seed=3),
    "wide_range": _wide_range,
}


@pytest.mark.parametrize("name", list(MATS))
@pytest.mark.parametrize("level", [gse.LEVEL_FP16, gse.LEVEL_BF16])
def test_storage_bit_exact(name, level):
    A = MATS[name]()
    M = gse.GseMatrix.from_csr(A, attach=(level,))
    bits, ov = oracle.round16(A.val, KINDS[level])
    ref = oracle.widen16(bits, KINDS[level])
    dec = M.decode(level).cpu().numpy()
    assert np.array_equal(dec.view(np.uint64), ref.view(np.uint64))
    if level == gse.LEVEL_FP16:
        assert M.info().overflow16 == ov


@pytest.mark.parametrize("name", list(MATS))
@pytest.mark.parametrize("level", [gse.LEVEL_FP16, gse.LEVEL_BF16])
@pytest.mark.parametrize("sched", [1, gse.SCHEDULE_ROWS])
def test_spmv_against_oracle(name, level, sched):
    A = MATS[name]()
    M = gse.GseMatrix.from_csr(A, attach=(level,))
    try:
        M.set_schedule(sched)
    except gse.GseError as e:
        assert e.code == gse.ERR_UNSUPPORTED and sched == gse.SCHEDULE_ROWS
        return
    bits, ov = oracle.round16(A.val, KINDS[level])
    a = oracle.widen16(bits, KINDS[level])
    x = synth.uniform_x(A.n_cols, seed=2)
    y = M.spmv(level, torch.from_numpy(x).cuda()).cpu().numpy()
    if ov:                                   # rows that meet an infinity: the same non-finite result
        rows_inf = np.unique(np.repeat(np.arange(A.n_rows), np.diff(A.row_ptr))[~np.isfinite(a)])
        assert np.all(~np.isfinite(y[rows_inf]))
        keep = np.setdiff1d(np.arange(A.n_rows), rows_inf)
        check_spmv_rows(y, A, np.where(np.isfinite(a), a, 0.0), x, rows=keep)
    else:
        check_spmv_rows(y, A, a, x)


def test_fp32_subnormals_widen_exactly():
    vals = np.array([1e-40, -3e-42, 1.5e-45, 1.17e-38, 2.0, -0.0])
    A = synth.CSR(np.array([0, 2, 4, 6], np.int32), np.array([0, 1, 0, 1, 0, 1], np.int32), vals, 2, "sub32")
    M = gse.GseMatrix.from_csr(A, attach=(32,))
    dec = M.decode(gse.LEVEL_FP32).cpu().numpy()
    ref = vals.astype(np.float32).astype(np.float64)
    assert np.array_equal(dec.view(np.uint64), ref.view(np.uint64))


@pytest.mark.parametrize("level", [gse.LEVEL_FP16, gse.LEVEL_BF16])
def test_cg_on_16bit_values(level):
    A = synth.poisson2d(32, 1.0 / 3.0)
    M = gse.GseMatrix.from_csr(A, attach=(level,))
    b = synth.rhs_ones(A)
    x = torch.zeros(A.n_rows, dtype=torch.float64, device="cuda")
    info = M.cg(torch.from_numpy(b).cuda(), x, tol=1e-10, policy=gse.fp64_policy(gse.SCALED_CG, level))
    a = oracle.widen16(oracle.round16(A.val, KINDS[level])[0], KINDS[level])
    ref = oracle.cg(A.row_ptr, A.col, a, b, tol=1e-10)
    assert info["status"] == gse.OK
    assert abs(info["iters"] - ref["info"]["iters"]) <= 2
    assert np.max(np.abs(x.cpu().numpy() - ref["x"])) < 1e-8


def test_fp16_overflow_makes_the_solve_nonfinite():
    A = synth.laplace3d(10, shift=1e-3).scaled(2e4)      # diagonal 1.2e5 > 65504
    M = gse.GseMatrix.from_csr(A, attach=(gse.LEVEL_FP16, gse.LEVEL_BF16))
    assert M.info().overflow16 == A.n_rows
    b = torch.from_numpy(synth.rhs_ones(A)).cuda()
    x = torch.zeros(A.n_rows, dtype=torch.float64, device="cuda")
    info = M.cg(b, x, tol=1e-6, policy=gse.fp64_policy(gse.SCALED_CG, gse.LEVEL_FP16))
    assert info["status"] == gse.NONFINITE
    x.zero_()
    info = M.cg(b, x, tol=1e-6, policy=gse.fp64_policy(gse.SCALED_CG, gse.LEVEL_BF16))
    assert info["status"] == gse.OK                      # BF16 keeps FP32's range
