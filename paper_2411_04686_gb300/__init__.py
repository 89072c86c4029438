"""Python binding of the GSE library (``libgse.so``, C ABI in ``include/gse.h``).

Argument marshalling only: every step of encode, SpMV and the solvers runs in
the library's CUDA kernels.  PyTorch provides device memory and the current
stream.  If the compiled library is missing the import of this module still
succeeds, but every call raises ``RuntimeError`` -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgse.so")

OK, MAXITER, BREAKDOWN, NONFINITE, TIMEOUT = 0, 1, 2, 3, 4
ERR_INVALID, ERR_NONFINITE, ERR_OOM, ERR_CUDA, ERR_UNSUPPORTED = -1, -2, -3, -4, -5
LEVEL_FP64, LEVEL_FP32, LEVEL_FP16, LEVEL_BF16 = 64, 32, 16, 17
POLICY_NO_STAGNATION, POLICY_FLOOR = 1, 2
SCHEDULE_ROWS = 8
INDEX_AUTO, INDEX_COL, INDEX_VALUE = 0, 1, 2

# every symbol include/gse.h declares
EXPORTS = ["gse_strerror", "gse_encode", "gse_attach_values", "gse_spmv", "gse_cg", "gse_cg_noalloc", "gse_gmres",
           "gse_batch_cg", "gse_engine_create", "gse_engine_submit", "gse_engine_run",
           "gse_engine_poll", "gse_engine_cancel", "gse_engine_destroy", "gse_export", "gse_decode",
           "gse_matrix_get_info", "gse_set_schedule", "gse_autotune", "gse_footprint",
           "gse_solve_footprint", "gse_free", "gse_encode_table", "gse_encode_table_ex", "gse_export_table",
           "gse_engine_launch", "gse_engine_wait", "gse_probe", "gse_test_timeout"]

_P = ctypes.c_void_p
_I = ctypes.c_int
_I64 = ctypes.c_int64
_D = ctypes.c_double


class GseError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        super().__init__(f"{what}: {strerror(code)} ({code})" if what else f"{strerror(code)} ({code})")


class CSR(ctypes.Structure):
    _fields_ = [("n_rows", _I64), ("n_cols", _I64), ("nnz", _I64), ("row_ptr", _P), ("col_idx", _P),
                ("val", _P), ("on_device", _I)]


class StepPolicy(ctypes.Structure):
    _fields_ = [("l", _I), ("t", _I), ("m", _I), ("rsd_limit", _D), ("ndec_limit", _I),
                ("reldec_limit", _D), ("max_iter", _I), ("restart", _I), ("k_start", _I),
                ("k_max", _I), ("flags", _I)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("status", _I), ("iters", _I), ("k_final", _I), ("switch_iter", _I * 3),
                ("rel_res_rec", _D), ("rel_res_true", _D), ("seconds", _D)]

    def as_dict(self) -> dict:
        return {"status": self.status, "iters": self.iters, "k_final": self.k_final,
                "switch_iter": list(self.switch_iter), "rel_res_rec": self.rel_res_rec,
                "rel_res_true": self.rel_res_true, "seconds": self.seconds}


class MatrixInfo(ctypes.Structure):
    _fields_ = [("n_rows", _I64), ("n_cols", _I64), ("nnz", _I64), ("n_groups", _I64),
                ("n_empty_rows", _I64), ("group_size", _I), ("n_seg", _I), ("seg_bits", _I * 3),
                ("max_row_len", _I), ("mean_row_len", _D), ("schedule", _I),
                ("bytes_level", _I64 * 3), ("num_exp", _I), ("overflow16", _I64),
                ("index_in_head", _I)]


_lib = None


def available() -> bool:
    return os.path.exists(LIB_PATH)


def lib():
    """Loads libgse.so (raises RuntimeError if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                           "(the GSE path has no CPU fallback)")
    L = ctypes.CDLL(LIB_PATH)
    L.gse_strerror.restype = ctypes.c_char_p
    L.gse_strerror.argtypes = [_I]
    L.gse_encode.argtypes = [ctypes.POINTER(CSR), _I, _P, _I, _P, ctypes.POINTER(_P)]
    L.gse_encode_table.argtypes = [ctypes.POINTER(CSR), _I, _P, _I, _P, ctypes.POINTER(_P)]
    L.gse_encode_table_ex.argtypes = [ctypes.POINTER(CSR), _I, _P, _I, _I, _I64, _P, _P, ctypes.POINTER(_P)]
    L.gse_export_table.argtypes = [_P, _P, _P, _P]
    L.gse_attach_values.argtypes = [_P, ctypes.POINTER(CSR), _I, _P]
    L.gse_spmv.argtypes = [_P, _I, _P, _P, _P]
    for f in (L.gse_cg, L.gse_cg_noalloc, L.gse_gmres):
        f.argtypes = [_P, _P, _P, _D, ctypes.POINTER(StepPolicy), ctypes.POINTER(SolveInfo), _P]
    L.gse_batch_cg.argtypes = [_I, _P, _P, _P, _D, ctypes.POINTER(StepPolicy), _P, _P]
    L.gse_engine_create.argtypes = [_I, _P, ctypes.POINTER(_P)]
    L.gse_engine_submit.argtypes = [_P, _P, _P, _P, _D, ctypes.POINTER(StepPolicy), ctypes.POINTER(_I)]
    L.gse_engine_run.argtypes = [_P, _I, _I, ctypes.POINTER(_I)]
    L.gse_engine_launch.argtypes = [_P, _I, _I]
    L.gse_engine_wait.argtypes = [_P, ctypes.POINTER(_I)]
    L.gse_engine_poll.argtypes = [_P, _P, _P, _I, ctypes.POINTER(_I)]
    L.gse_engine_cancel.argtypes = [_P, _I, ctypes.POINTER(SolveInfo)]
    L.gse_engine_destroy.argtypes = [_P]
    L.gse_engine_destroy.restype = None
    L.gse_export.argtypes = [_P, _P, _P, _P, _P]
    L.gse_decode.argtypes = [_P, _I, _P, _P]
    L.gse_matrix_get_info.argtypes = [_P, ctypes.POINTER(MatrixInfo)]
    L.gse_set_schedule.argtypes = [_P, _I]
    L.gse_autotune.argtypes = [_P, _I, _P]
    L.gse_footprint.argtypes = [_P]
    L.gse_footprint.restype = ctypes.c_size_t
    L.gse_solve_footprint.argtypes = [_P, _I, _I]
    L.gse_solve_footprint.restype = ctypes.c_size_t
    L.gse_free.argtypes = [_P]
    L.gse_free.restype = None
    L.gse_probe.argtypes = [_I, _I64, _P, _P, _P]
    L.gse_test_timeout.argtypes = [_P, _I]
    _lib = L
    return L


def strerror(code: int) -> str:
    try:
        return lib().gse_strerror(code).decode()
    except RuntimeError:
        return f"status {code}"


def _check(rc: int, what: str) -> int:
    if rc < 0:
        raise GseError(rc, what)
    return rc


def _stream_ptr(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dptr(t) -> ctypes.c_void_p:
    return ctypes.c_void_p(t.data_ptr())


@dataclass
class Policy:
    """Precision-step policy (Sec. III-D; the paper's values are in Sec. IV-D)."""
    l: int = 50
    t: int = 25
    m: int = 10
    rsd_limit: float = 0.50
    ndec_limit: int = 13
    reldec_limit: float = 0.45
    max_iter: int = 20000
    restart: int = 30
    k_start: int = 1
    k_max: int = 3
    flags: int = 0

    def c(self) -> StepPolicy:
        return StepPolicy(self.l, self.t, self.m, self.rsd_limit, self.ndec_limit, self.reldec_limit,
                          self.max_iter, self.restart, self.k_start, self.k_max, self.flags)


PAPER_CG = Policy(l=3000, t=250, m=500, rsd_limit=0.50, ndec_limit=130, reldec_limit=0.45, max_iter=5000)
PAPER_GMRES = Policy(l=9000, t=300, m=1500, rsd_limit=0.03, ndec_limit=80, reldec_limit=0.08,
                     max_iter=15000, restart=30)
SCALED_CG = Policy(l=50, t=25, m=10, rsd_limit=0.50, ndec_limit=13, reldec_limit=0.45, max_iter=20000)
SCALED_GMRES = Policy(l=150, t=30, m=30, rsd_limit=0.03, ndec_limit=8, reldec_limit=0.08,
                      max_iter=20000, restart=30)


def fp64_policy(p: Policy, bits: int = 64) -> Policy:
    """Same caps, plain CSR values (no stepping): bits = 64, 32, LEVEL_FP16 or
    LEVEL_BF16 selects the attached baseline values."""
    lv = {64: LEVEL_FP64, 32: LEVEL_FP32, LEVEL_FP16: LEVEL_FP16, LEVEL_BF16: LEVEL_BF16}[bits]
    return Policy(p.l, p.t, p.m, p.rsd_limit, p.ndec_limit, p.reldec_limit, p.max_iter, p.restart,
                  lv, lv, p.flags)


class GseMatrix:
    """An encoded matrix on the current CUDA device (owns a gse_handle)."""

    def __init__(self, row_ptr, col, val, n_cols=None, group_size=32, seg_bits=(16, 16, 20),
                 stream=None, attach=(), num_exp=0, index_place=INDEX_AUTO, sample_block_rows=0,
                 sample_rows=None):
        import torch
        L = lib()
        self._keep = []
        on_dev = isinstance(row_ptr, torch.Tensor) and row_ptr.is_cuda
        if on_dev:
            rp, cl, vl = (row_ptr.contiguous(), col.contiguous(), val.contiguous())
            self._keep += [rp, cl, vl]
            ptrs = (rp.data_ptr(), cl.data_ptr(), vl.data_ptr())
            n_rows, nnz = rp.numel() - 1, cl.numel()
        else:
            rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
            cl = np.ascontiguousarray(col, dtype=np.int32)
            vl = np.ascontiguousarray(val, dtype=np.float64)
            self._keep += [rp, cl, vl]
            ptrs = (rp.ctypes.data, cl.ctypes.data, vl.ctypes.data)
            n_rows, nnz = rp.size - 1, cl.size
        self.n_rows = n_rows
        self.n_cols = n_rows if n_cols is None else int(n_cols)
        self.nnz = nnz
        self.csr = CSR(n_rows, self.n_cols, nnz, ptrs[0], ptrs[1], ptrs[2], 1 if on_dev else 0)
        sb = (ctypes.c_int * 3)(*(list(seg_bits) + [0] * (3 - len(seg_bits))))
        h = ctypes.c_void_p()
        self.stream = _stream_ptr(stream)
        if num_exp:      # the paper's global exponent table (Sec. III-B)
            samp = None
            if sample_block_rows:        # sampled extraction: one row per block, drawn by the caller
                samp = np.ascontiguousarray(sample_rows, dtype=np.int64)
                if samp.size != (n_rows + sample_block_rows - 1) // sample_block_rows:
                    raise ValueError("sample_rows needs one row index per block of sample_block_rows rows")
            _check(L.gse_encode_table_ex(ctypes.byref(self.csr), num_exp, ctypes.cast(sb, _P), len(seg_bits),
                                         index_place, int(sample_block_rows),
                                         None if samp is None else samp.ctypes.data, self.stream, ctypes.byref(h)),
                   "gse_encode_table_ex")
        else:
            _check(L.gse_encode(ctypes.byref(self.csr), group_size, ctypes.cast(sb, _P), len(seg_bits),
                                self.stream, ctypes.byref(h)), "gse_encode")
        self.num_exp = num_exp
        self.h = h
        self.group_size = group_size
        self.seg_bits = tuple(seg_bits)
        for bits in attach:
            self.attach_values(bits)
        self._keep = [] if on_dev else self._keep   # host arrays may be needed by attach_values

    @classmethod
    def from_csr(cls, A, **kw):
        return cls(A.row_ptr, A.col, A.val, n_cols=A.n_cols, **kw)

    def attach_values(self, bits=64, val=None):
        L = lib()
        csr = self.csr
        if val is not None:
            v = np.ascontiguousarray(val, dtype=np.float64)
            self._keep.append(v)
            csr = CSR(self.csr.n_rows, self.csr.n_cols, self.csr.nnz, self.csr.row_ptr,
                      self.csr.col_idx, v.ctypes.data, 0)
        _check(L.gse_attach_values(self.h, ctypes.byref(csr), bits, self.stream), "gse_attach_values")

    def info(self) -> MatrixInfo:
        mi = MatrixInfo()
        _check(lib().gse_matrix_get_info(self.h, ctypes.byref(mi)), "gse_matrix_get_info")
        return mi

    def spmv(self, k, x, y=None, stream=None):
        import torch
        if y is None:
            y = torch.empty(self.n_rows, dtype=torch.float64, device=x.device)
        _check(lib().gse_spmv(self.h, k, _dptr(x), _dptr(y), _stream_ptr(stream)), "gse_spmv")
        return y

    def decode(self, k, stream=None):
        import torch
        out = torch.empty(max(self.nnz, 1), dtype=torch.float64, device="cuda")
        _check(lib().gse_decode(self.h, k, _dptr(out), _stream_ptr(stream)), "gse_decode")
        return out[: self.nnz]

    def export(self):
        head = np.zeros(self.nnz, np.uint16)
        t1 = np.zeros(self.nnz, np.uint16)
        t2 = np.zeros(self.nnz, np.uint32)
        gexp = np.zeros((self.nnz + self.group_size - 1) // self.group_size, np.int16)
        _check(lib().gse_export(self.h, head.ctypes.data, t1.ctypes.data, t2.ctypes.data,
                                None if self.num_exp else gexp.ctypes.data), "gse_export")
        return head, t1, t2, gexp

    def export_table(self):
        """(table int16, idx uint8) of a table-format handle."""
        table = np.zeros(64, np.int16)
        n = ctypes.c_int(0)
        idx = np.zeros(max(self.nnz, 1), np.uint8)
        _check(lib().gse_export_table(self.h, table.ctypes.data, ctypes.byref(n), idx.ctypes.data),
               "gse_export_table")
        return table[: n.value].copy(), idx[: self.nnz]

    def test_timeout(self, on: bool):
        """gse_test_timeout: the staged kernels of this handle issue no copy and
        their bounded waits run out at once (test hook)."""
        _check(lib().gse_test_timeout(self.h, 1 if on else 0), "gse_test_timeout")

    def set_schedule(self, upl: int):
        _check(lib().gse_set_schedule(self.h, upl), "gse_set_schedule")

    def autotune(self, k=1, stream=None):
        _check(lib().gse_autotune(self.h, k, _stream_ptr(stream)), "gse_autotune")

    def footprint(self) -> int:
        return int(lib().gse_footprint(self.h))

    def solve_footprint(self, method=0, restart=30) -> int:
        return int(lib().gse_solve_footprint(self.h, method, restart))

    def _solve(self, fn, b, x, tol, policy, stream):
        info = SolveInfo()
        pol = policy.c()
        rc = fn(self.h, _dptr(b), _dptr(x), tol, ctypes.byref(pol), ctypes.byref(info),
                _stream_ptr(stream))
        _check(rc, fn.__name__)
        return info.as_dict()

    def cg(self, b, x, tol=1e-10, policy: Policy = SCALED_CG, stream=None) -> dict:
        return self._solve(lib().gse_cg, b, x, tol, policy, stream)

    def gmres(self, b, x, tol=1e-10, policy: Policy = SCALED_GMRES, stream=None) -> dict:
        return self._solve(lib().gse_gmres, b, x, tol, policy, stream)

    def free(self):
        if getattr(self, "h", None):
            lib().gse_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


PROBE_DFMA_RATE, PROBE_DFMA_CHAINS, PROBE_DFMA_LATENCY, PROBE_GATHER_L1, PROBE_GATHER_L2 = 1, 2, 3, 4, 5


def probe(which: int, param: int = 0, table=None, stream=None):
    """gse_probe: (result, kernel ms) of one machine probe (include/gse.h)."""
    out = (ctypes.c_double * 2)()
    _check(lib().gse_probe(which, int(param), None if table is None else _dptr(table), out, _stream_ptr(stream)),
           "gse_probe")
    return out[0], out[1]


def batch_cg(mats, bs, xs, tol=1e-10, policy: Policy = SCALED_CG, stream=None):
    """Solves many systems concurrently (gse_batch_cg)."""
    n = len(mats)
    hs = (ctypes.c_void_p * n)(*[m.h.value for m in mats])
    bp = (ctypes.c_void_p * n)(*[b.data_ptr() for b in bs])
    xp = (ctypes.c_void_p * n)(*[x.data_ptr() for x in xs])
    infos = (SolveInfo * n)()
    pol = policy.c()
    rc = lib().gse_batch_cg(n, ctypes.cast(hs, _P), ctypes.cast(bp, _P), ctypes.cast(xp, _P), tol,
                            ctypes.byref(pol), ctypes.cast(infos, _P), _stream_ptr(stream))
    _check(rc, "gse_batch_cg")
    return rc, [i.as_dict() for i in infos]


class Engine:
    """Continuous-batching CG engine (gse_engine_*)."""

    def __init__(self, capacity: int, stream=None):
        self.e = ctypes.c_void_p()
        self.stream = _stream_ptr(stream)
        _check(lib().gse_engine_create(capacity, self.stream, ctypes.byref(self.e)), "gse_engine_create")
        self.capacity = capacity

    def submit(self, mat: GseMatrix, b, x, tol=1e-10, policy: Policy = SCALED_CG) -> int:
        slot = ctypes.c_int(-1)
        pol = policy.c()
        _check(lib().gse_engine_submit(self.e, mat.h, _dptr(b), _dptr(x), tol, ctypes.byref(pol),
                                       ctypes.byref(slot)), "gse_engine_submit")
        return slot.value

    def run(self, max_slots: int, batch: int = 8) -> int:
        n = ctypes.c_int(0)
        _check(lib().gse_engine_run(self.e, max_slots, batch, ctypes.byref(n)), "gse_engine_run")
        return n.value

    def launch(self, max_slots: int, batch: int = 8):
        """Queues max_slots iteration slots and returns at once (gse_engine_launch)."""
        _check(lib().gse_engine_launch(self.e, max_slots, batch), "gse_engine_launch")

    def wait(self) -> int:
        """Waits for the last launch; returns the systems still running."""
        n = ctypes.c_int(0)
        _check(lib().gse_engine_wait(self.e, ctypes.byref(n)), "gse_engine_wait")
        return n.value

    def poll(self):
        slots = (ctypes.c_int * self.capacity)()
        infos = (SolveInfo * self.capacity)()
        nd = ctypes.c_int(0)
        _check(lib().gse_engine_poll(self.e, ctypes.cast(slots, _P), ctypes.cast(infos, _P),
                                     self.capacity, ctypes.byref(nd)), "gse_engine_poll")
        return [(slots[i], infos[i].as_dict()) for i in range(nd.value)]

    def cancel(self, slot: int) -> dict:
        info = SolveInfo()
        _check(lib().gse_engine_cancel(self.e, slot, ctypes.byref(info)), "gse_engine_cancel")
        return info.as_dict()

    def close(self):
        if self.e:
            lib().gse_engine_destroy(self.e)
            self.e = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
