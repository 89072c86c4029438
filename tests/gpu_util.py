"""Helpers for the GPU parity tests (test infrastructure)."""
import numpy as np

import oracle
import synth


def sub_csr(A, rows):
    """CSR of the selected rows (same columns), for sampled oracle checks."""
    rows = np.asarray(rows, dtype=np.int64)
    lens = (A.row_ptr[rows + 1] - A.row_ptr[rows]).astype(np.int64)
    rp = np.zeros(rows.size + 1, np.int64)
    np.cumsum(lens, out=rp[1:])
    idx = np.concatenate([np.arange(A.row_ptr[r], A.row_ptr[r + 1]) for r in rows]) if rows.size else np.zeros(0, np.int64)
    return rp.astype(np.int32), idx


def check_spmv_rows(y_gpu, A, a_vals, x, rows=None, tol=1e-13):
    """|y_gpu_i - y_ref_i| <= tol * sum_j |a_ij x_j| + len_i * 2^-1074 (y_ref:
    the oracle's Dot2 on the same decoded values).  The second term is IEEE
    gradual underflow: a product or sum in the subnormal range carries an
    absolute error up to half the smallest subnormal, which no relative bound
    covers.  Empty rows must be exactly 0.  Returns the worst normalised error."""
    if rows is None:
        yref, yabs = oracle.spmv_dot2(A.row_ptr, A.col, a_vals, x)
        yg = y_gpu
        lens = np.diff(A.row_ptr)
    else:
        rp, idx = sub_csr(A, rows)
        yref, yabs = oracle.spmv_dot2(rp, A.col[idx], a_vals[idx], x)
        yg = y_gpu[rows]
        lens = np.diff(rp)
    err = np.abs(yg - yref)
    assert np.all(yg[lens == 0] == 0.0), "empty rows must give exactly 0"
    bad = err > tol * yabs + lens * 2.0 ** -1074
    assert not bad.any(), f"{bad.sum()} rows exceed {tol} * sum|a x|; worst {np.max(err / np.maximum(yabs, 1e-300))}"
    nz = yabs > 0
    return float(np.max(err[nz] / yabs[nz])) if nz.any() else 0.0
