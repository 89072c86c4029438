"""CPU oracle for GSE encoding, GSE-SpMV and the stepped CG/GMRES.

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's
CPU-baseline leg load this module; the product library never does.  The
arithmetic lives in ``gse_oracle.c`` (plain, single-threaded C written from the
paper); this file compiles it with gcc and marshals numpy arrays through
ctypes.  It shares no code with the CUDA path.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gse_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

OK, MAXITER, BREAKDOWN, NONFINITE = 0, 1, 2, 3
POLICY_NO_STAGNATION = 1
POLICY_FLOOR = 2


def build(force: bool = False) -> str:
    """Compiles the oracle into ``oracle/liboracle.so`` (gcc; OpenMP only
    spreads the rows of orc_gse_spmv_rows over threads for the timed CPU
    baselines, every other routine runs on one thread)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_I = ctypes.c_int
_D = ctypes.c_double


class Info(ctypes.Structure):
    _fields_ = [("status", _I), ("iters", _I), ("k_final", _I), ("switch_iter", _I * 3),
                ("rel_res_rec", _D), ("rel_res_true", _D)]

    def as_dict(self) -> dict:
        return {"status": self.status, "iters": self.iters, "k_final": self.k_final,
                "switch_iter": list(self.switch_iter), "rel_res_rec": self.rel_res_rec,
                "rel_res_true": self.rel_res_true}


class _Policy(ctypes.Structure):
    _fields_ = [("l", _I), ("t", _I), ("m", _I), ("rsd_limit", _D), ("ndec_limit", _I),
                ("reldec_limit", _D), ("max_iter", _I), ("restart", _I), ("k_start", _I),
                ("k_max", _I), ("flags", _I)]


@dataclass
class Policy:
    """Parameters of the precision-step policy (Sec. III-D, Sec. IV-D)."""
    l: int
    t: int
    m: int
    rsd_limit: float
    ndec_limit: int
    reldec_limit: float
    max_iter: int
    restart: int = 30
    k_start: int = 1
    k_max: int = 3
    flags: int = 0

    def c(self) -> _Policy:
        return _Policy(self.l, self.t, self.m, self.rsd_limit, self.ndec_limit, self.reldec_limit,
                       self.max_iter, self.restart, self.k_start, self.k_max, self.flags)


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        L.orc_encode.argtypes = [_I64, _P, _I, _P, _I, _P, _P, _P, _P]
        L.orc_decode.argtypes = [_I64, _P, _P, _P, _P, _I, _P, _I, _I, _P]
        L.orc_table_build.argtypes = [_I64, _P, _I, _P]
        L.orc_round16.argtypes = [_I64, _P, _I, _P, ctypes.POINTER(_I64)]
        L.orc_widen16.argtypes = [_I64, _P, _I, _P]
        L.orc_table_encode.argtypes = [_I64, _P, _P, _I, _P, _I, _P, _P, _P, _P]
        L.orc_table_decode.argtypes = [_I64, _P, _P, _P, _P, _P, _I, _P, _I, _I, _P]
        L.orc_table_build_sampled.argtypes = [_I64, _P, _P, _I, _I64, _P, _P]
        L.orc_table_encode_in_value.argtypes = [_I64, _P, _P, _I, _P, _I, _P, _P, _P]
        L.orc_table_decode_in_value.argtypes = [_I64, _P, _P, _P, _P, _I, _P, _I, _I, _P]
        L.orc_spmv.argtypes = [_I64, _P, _P, _P, _P, _P]
        L.orc_spmv.restype = None
        L.orc_gse_spmv.argtypes = [_I64, _P, _P, _P, _P, _P, _P, _I, _P, _I, _I, _P, _P]
        L.orc_gse_spmv_rows.argtypes = [_I64, _I64, _P, _P, _P, _P, _P, _P, _I, _P, _I, _I, _P, _P, _I]
        L.orc_spmv_dot2.argtypes = [_I64, _P, _P, _P, _P, _P, _P]
        L.orc_spmv_dot2.restype = None
        L.orc_cg.argtypes = [_I64, _P, _P, _P, _P, _P, _D, _I, ctypes.POINTER(Info), _P, _P, _P, _I]
        L.orc_gmres.argtypes = [_I64, _P, _P, _P, _P, _P, _D, _I, _I, ctypes.POINTER(Info), _P, _P]
        L.orc_step_metrics.argtypes = [_P, _I, _I, ctypes.POINTER(_D), ctypes.POINTER(_I),
                                       ctypes.POINTER(_D)]
        L.orc_step_decide.argtypes = [_D, _I, _D, _I, ctypes.POINTER(_Policy)]
        for f in (L.orc_stepped_cg, L.orc_stepped_gmres):
            f.argtypes = [_I64, _P, _P, _P, _P, _P, _D, ctypes.POINTER(_Policy),
                          ctypes.POINTER(Info), _P, _I]
        _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(_P)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _segs(seg_bits):
    s = list(seg_bits) + [0] * (3 - len(seg_bits))
    return np.array(s, dtype=np.int32), len(seg_bits)


def encode(val, group_size=32, seg_bits=(16, 16, 20)):
    """Returns (head u16, tail1 u16, tail2 u32, gexp i16) per Alg. 1 / Sec. III-B."""
    val = _c(val, np.float64)
    nnz = val.size
    sb, nseg = _segs(seg_bits)
    head = np.zeros(nnz, np.uint16)
    t1 = np.zeros(nnz, np.uint16)
    t2 = np.zeros(nnz, np.uint32)
    gexp = np.zeros((nnz + group_size - 1) // group_size, np.int16)
    rc = lib().orc_encode(nnz, _ptr(val), group_size, _ptr(sb), nseg, _ptr(head), _ptr(t1),
                          _ptr(t2), _ptr(gexp))
    if rc != 0:
        raise ValueError(f"orc_encode status {rc}")
    return head, t1, t2, gexp


def decode(head, tail1, tail2, gexp, k, group_size=32, seg_bits=(16, 16, 20)):
    head, tail1 = _c(head, np.uint16), _c(tail1, np.uint16)
    tail2, gexp = _c(tail2, np.uint32), _c(gexp, np.int16)
    sb, nseg = _segs(seg_bits)
    out = np.zeros(head.size, np.float64)
    rc = lib().orc_decode(head.size, _ptr(head), _ptr(tail1), _ptr(tail2), _ptr(gexp), group_size,
                          _ptr(sb), nseg, k, _ptr(out))
    if rc != 0:
        raise ValueError(f"orc_decode status {rc}")
    return out


def levels(val, group_size=32, seg_bits=(16, 16, 20)):
    """FP64 values of A_1 .. A_nseg decoded from the oracle's own encoding."""
    enc = encode(val, group_size, seg_bits)
    return [decode(*enc, k, group_size, seg_bits) for k in range(1, len(seg_bits) + 1)]


def table_build(val, num_exp):
    """The global shared-exponent table (Sec. III-B): int16 entries, each a
    most frequent exponent plus 1, with max(e) + 1 always present."""
    val = _c(val, np.float64)
    table = np.zeros(max(num_exp, 1), np.int16)
    n = lib().orc_table_build(val.size, _ptr(val), num_exp, _ptr(table))
    if n < 1:
        raise ValueError(f"orc_table_build status {n}")
    return table[:n].copy()


def table_encode(val, table, seg_bits=(16, 16, 20)):
    """Alg. 1 against the table: (head u16, tail1 u16, tail2 u32, idx u8)."""
    val = _c(val, np.float64)
    table = _c(table, np.int16)
    nnz = val.size
    sb, nseg = _segs(seg_bits)
    head = np.zeros(nnz, np.uint16)
    t1 = np.zeros(nnz, np.uint16)
    t2 = np.zeros(nnz, np.uint32)
    idx = np.zeros(nnz, np.uint8)
    rc = lib().orc_table_encode(nnz, _ptr(val), _ptr(table), table.size, _ptr(sb), nseg, _ptr(head), _ptr(t1),
                                _ptr(t2), _ptr(idx))
    if rc != 0:
        raise ValueError(f"orc_table_encode status {rc}")
    return head, t1, t2, idx


def table_decode(head, tail1, tail2, idx, table, k, seg_bits=(16, 16, 20)):
    head, tail1 = _c(head, np.uint16), _c(tail1, np.uint16)
    tail2, idx, table = _c(tail2, np.uint32), _c(idx, np.uint8), _c(table, np.int16)
    sb, nseg = _segs(seg_bits)
    out = np.zeros(head.size, np.float64)
    rc = lib().orc_table_decode(head.size, _ptr(head), _ptr(tail1), _ptr(tail2), _ptr(idx), _ptr(table), table.size,
                                _ptr(sb), nseg, k, _ptr(out))
    if rc != 0:
        raise ValueError(f"orc_table_decode status {rc}")
    return out


def table_build_sampled(row_ptr, val, num_exp, block_rows, sample_rows):
    """The table from the sampled extraction of Sec. III-B: the exponents of
    row sample_rows[b] stand for the block of block_rows rows b belongs to."""
    row_ptr, val = _c(row_ptr, np.int32), _c(val, np.float64)
    sample_rows = _c(sample_rows, np.int64)
    n_rows = row_ptr.size - 1
    if sample_rows.size != (n_rows + block_rows - 1) // block_rows:
        raise ValueError("one sample row per block")
    table = np.zeros(max(num_exp, 1), np.int16)
    n = lib().orc_table_build_sampled(n_rows, _ptr(row_ptr), _ptr(val), num_exp, block_rows, _ptr(sample_rows),
                                      _ptr(table))
    if n < 1:
        raise ValueError(f"orc_table_build_sampled status {n}")
    return table[:n].copy()


def table_encode_in_value(val, table, seg_bits=(16, 16, 20)):
    """The table format with the index in the top head bits (Sec. III-C's
    layout for column counts without spare bits): (head u16, tail1 u16, tail2 u32)."""
    val, table = _c(val, np.float64), _c(table, np.int16)
    nnz = val.size
    sb, nseg = _segs(seg_bits)
    head = np.zeros(nnz, np.uint16)
    t1 = np.zeros(nnz, np.uint16)
    t2 = np.zeros(nnz, np.uint32)
    rc = lib().orc_table_encode_in_value(nnz, _ptr(val), _ptr(table), table.size, _ptr(sb), nseg, _ptr(head),
                                         _ptr(t1), _ptr(t2))
    if rc != 0:
        raise ValueError(f"orc_table_encode_in_value status {rc}")
    return head, t1, t2


def table_decode_in_value(head, tail1, tail2, table, k, seg_bits=(16, 16, 20)):
    head, tail1 = _c(head, np.uint16), _c(tail1, np.uint16)
    tail2, table = _c(tail2, np.uint32), _c(table, np.int16)
    sb, nseg = _segs(seg_bits)
    out = np.zeros(head.size, np.float64)
    rc = lib().orc_table_decode_in_value(head.size, _ptr(head), _ptr(tail1), _ptr(tail2), _ptr(table), table.size,
                                         _ptr(sb), nseg, k, _ptr(out))
    if rc != 0:
        raise ValueError(f"orc_table_decode_in_value status {rc}")
    return out


def index_bits(n_table):
    """Bits an exponent index takes for a table of n_table entries."""
    return max(int(n_table) - 1, 0).bit_length()


def table_levels(val, num_exp, seg_bits=(16, 16, 20), table=None, index_in_value=False):
    """(table, [A_1 .. A_nseg values]) of the table format; the table is built
    from all values unless given; index_in_value selects the head layout."""
    if table is None:
        table = table_build(val, num_exp)
    if index_in_value:
        enc = table_encode_in_value(val, table, seg_bits)
        return table, [table_decode_in_value(*enc, table, k, seg_bits) for k in range(1, len(seg_bits) + 1)]
    enc = table_encode(val, table, seg_bits)
    return table, [table_decode(*enc, table, k, seg_bits) for k in range(1, len(seg_bits) + 1)]


FP16, BF16 = 16, 17


def round16(val, kind):
    """(bits uint16, n_overflow): FP16 (kind 16) or BF16 (kind 17) storage of
    the values, round to nearest even from FP64 (Sec. IV-C baselines)."""
    val = _c(val, np.float64)
    out = np.zeros(val.size, np.uint16)
    ov = _I64(0)
    rc = lib().orc_round16(val.size, _ptr(val), kind, _ptr(out), ctypes.byref(ov))
    if rc != 0:
        raise ValueError(f"orc_round16 status {rc}")
    return out, int(ov.value)


def widen16(bits, kind):
    bits = _c(bits, np.uint16)
    out = np.zeros(bits.size, np.float64)
    rc = lib().orc_widen16(bits.size, _ptr(bits), kind, _ptr(out))
    if rc != 0:
        raise ValueError(f"orc_widen16 status {rc}")
    return out


def spmv(row_ptr, col, a, x):
    row_ptr, col = _c(row_ptr, np.int32), _c(col, np.int32)
    a, x = _c(a, np.float64), _c(x, np.float64)
    n = row_ptr.size - 1
    y = np.zeros(n, np.float64)
    lib().orc_spmv(n, _ptr(row_ptr), _ptr(col), _ptr(a), _ptr(x), _ptr(y))
    return y


def gse_spmv(row_ptr, col, enc, k, x, group_size=32, seg_bits=(16, 16, 20)):
    row_ptr, col, x = _c(row_ptr, np.int32), _c(col, np.int32), _c(x, np.float64)
    head, t1, t2, gexp = (_c(enc[0], np.uint16), _c(enc[1], np.uint16), _c(enc[2], np.uint32),
                          _c(enc[3], np.int16))
    sb, nseg = _segs(seg_bits)
    n = row_ptr.size - 1
    y = np.zeros(n, np.float64)
    rc = lib().orc_gse_spmv(n, _ptr(row_ptr), _ptr(col), _ptr(head), _ptr(t1), _ptr(t2),
                            _ptr(gexp), group_size, _ptr(sb), nseg, k, _ptr(x), _ptr(y))
    if rc != 0:
        raise ValueError(f"orc_gse_spmv status {rc}")
    return y


def gse_spmv_rows(row_ptr, col, enc, k, x, r0, r1, threads=1, y=None, group_size=32, seg_bits=(16, 16, 20)):
    """gse_spmv over rows [r0, r1) only (y[r0:r1] written), on `threads` host
    threads; every row is summed as gse_spmv sums it."""
    row_ptr, col, x = _c(row_ptr, np.int32), _c(col, np.int32), _c(x, np.float64)
    head, t1, t2, gexp = (_c(enc[0], np.uint16), _c(enc[1], np.uint16), _c(enc[2], np.uint32),
                          _c(enc[3], np.int16))
    sb, nseg = _segs(seg_bits)
    if y is None:
        y = np.zeros(row_ptr.size - 1, np.float64)
    rc = lib().orc_gse_spmv_rows(int(r0), int(r1), _ptr(row_ptr), _ptr(col), _ptr(head), _ptr(t1), _ptr(t2),
                                 _ptr(gexp), group_size, _ptr(sb), nseg, k, _ptr(x), _ptr(y), int(threads))
    if rc != 0:
        raise ValueError(f"orc_gse_spmv_rows status {rc}")
    return y


def spmv_dot2(row_ptr, col, a, x):
    """Returns (y_ref, sum_j |a_ij x_j|) with the compensated Dot2 per row."""
    row_ptr, col = _c(row_ptr, np.int32), _c(col, np.int32)
    a, x = _c(a, np.float64), _c(x, np.float64)
    n = row_ptr.size - 1
    y = np.zeros(n, np.float64)
    ya = np.zeros(n, np.float64)
    lib().orc_spmv_dot2(n, _ptr(row_ptr), _ptr(col), _ptr(a), _ptr(x), _ptr(y), _ptr(ya))
    return y, ya


def cg(row_ptr, col, a, b, x0=None, tol=1e-10, max_iter=5000, trace_n=0):
    row_ptr, col = _c(row_ptr, np.int32), _c(col, np.int32)
    a, b = _c(a, np.float64), _c(b, np.float64)
    n = b.size
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64)
    info = Info()
    tr = [np.zeros((trace_n, n)) for _ in range(3)] if trace_n else [None] * 3
    lib().orc_cg(n, _ptr(row_ptr), _ptr(col), _ptr(a), _ptr(b), _ptr(x), tol, max_iter,
                 ctypes.byref(info), _ptr(tr[0]), _ptr(tr[1]), _ptr(tr[2]), trace_n)
    out = {"x": x, "info": info.as_dict()}
    if trace_n:
        out["r"], out["p"], out["xs"] = tr
    return out


def gmres(row_ptr, col, a, b, x0=None, tol=1e-10, restart=30, max_iter=15000, want_first_cycle=False):
    row_ptr, col = _c(row_ptr, np.int32), _c(col, np.int32)
    a, b = _c(a, np.float64), _c(b, np.float64)
    n = b.size
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64)
    info = Info()
    V = np.zeros((restart + 1, n)) if want_first_cycle else None
    H = np.zeros((restart + 1, restart)) if want_first_cycle else None
    lib().orc_gmres(n, _ptr(row_ptr), _ptr(col), _ptr(a), _ptr(b), _ptr(x), tol, restart, max_iter,
                    ctypes.byref(info), _ptr(V), _ptr(H))
    out = {"x": x, "info": info.as_dict()}
    if want_first_cycle:
        out["V"], out["H"] = V, H
    return out


def step_metrics(resid, t):
    """(RSD, nDec, relDec) of Eqs. 3-6 over the window ending at resid[-1]."""
    r = _c(resid, np.float64)
    rsd, nd, rd = _D(), _I(), _D()
    rc = lib().orc_step_metrics(_ptr(r), r.size, t, ctypes.byref(rsd), ctypes.byref(nd),
                                ctypes.byref(rd))
    if rc != 0:
        raise ValueError("window shorter than t + 1")
    return rsd.value, nd.value, rd.value


def step_decide(rsd, ndec, reldec, t, policy: Policy) -> int:
    p = policy.c()
    return lib().orc_step_decide(rsd, ndec, reldec, t, ctypes.byref(p))


def _stepped(fn, row_ptr, col, a_levels, b, x0, tol, policy: Policy, hist_cap):
    row_ptr, col, b = _c(row_ptr, np.int32), _c(col, np.int32), _c(b, np.float64)
    n = b.size
    lv = [_c(a, np.float64) for a in a_levels]
    arr = (_P * len(lv))(*[a.ctypes.data for a in lv])
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64)
    info = Info()
    hist = np.zeros(hist_cap) if hist_cap else None
    p = policy.c()
    fn(n, _ptr(row_ptr), _ptr(col), ctypes.cast(arr, _P), _ptr(b), _ptr(x), tol, ctypes.byref(p),
       ctypes.byref(info), _ptr(hist), hist_cap)
    out = {"x": x, "info": info.as_dict()}
    if hist_cap:
        out["hist"] = hist
    return out


def stepped_cg(row_ptr, col, a_levels, b, x0=None, tol=1e-10, policy: Policy | None = None,
               hist_cap=0):
    return _stepped(lib().orc_stepped_cg, row_ptr, col, a_levels, b, x0, tol, policy, hist_cap)


def stepped_gmres(row_ptr, col, a_levels, b, x0=None, tol=1e-10, policy: Policy | None = None,
                  hist_cap=0):
    return _stepped(lib().orc_stepped_gmres, row_ptr, col, a_levels, b, x0, tol, policy, hist_cap)


# Parameter presets.  PAPER_CG / PAPER_GMRES are the values printed in Sec. IV-D
# (l, t, m, RSD/nDec/relDec limits) with the caps of Sec. IV-A; SCALED keeps the
# paper's thresholds but shortens l/t/m (and nDec_limit in proportion to t) so
# that the stagnation checks can fire on systems that converge in hundreds of
# iterations.
PAPER_CG = Policy(l=3000, t=250, m=500, rsd_limit=0.50, ndec_limit=130, reldec_limit=0.45,
                  max_iter=5000)
PAPER_GMRES = Policy(l=9000, t=300, m=1500, rsd_limit=0.03, ndec_limit=80, reldec_limit=0.08,
                     max_iter=15000, restart=30)
SCALED_CG = Policy(l=50, t=25, m=10, rsd_limit=0.50, ndec_limit=13, reldec_limit=0.45,
                   max_iter=20000)
SCALED_GMRES = Policy(l=150, t=30, m=30, rsd_limit=0.03, ndec_limit=8, reldec_limit=0.08,
                      max_iter=20000, restart=30)
