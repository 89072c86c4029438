"""gse_cg_noalloc, called through the C ABI, against gse_cg.

gse_cg_noalloc exists for callers that cannot allocate device memory after
their set-up (fixed memory budgets, allocators that forbid new allocations,
threads that must not let cudaMalloc/cudaFree synchronise the device).  It runs
the same CG kernels with all scratch in a fixed device array inside the
library, so its answer must match gse_cg's within the solver tolerance used by
the other tests, on consecutive calls (the array keeps the previous call's
contents).  This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2411_04686_gb300 as gse  # noqa: E402


def _call(fn, M, b, x, tol, pol):
    info = gse.SolveInfo()
    p = pol.c()
    rc = fn(M.h, ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(x.data_ptr()), tol, ctypes.byref(p),
            ctypes.byref(info), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return rc, info.as_dict()


@pytest.mark.parametrize("make", [lambda: synth.poisson2d(32, 1.0 / 3.0),
                                  lambda: synth.laplace3d(20, shift=1e-3),
                                  lambda: synth.laplace2d(256, 255, shift=1e-2, aniso=(1.0, 0.2))])
def test_noalloc_cg_matches_cg_on_consecutive_calls(make):
    L = gse.lib()
    A = make()
    M = gse.GseMatrix.from_csr(A, attach=(64,))
    b = torch.from_numpy(synth.rhs_ones(A)).cuda()
    for pol in (gse.SCALED_CG, gse.fp64_policy(gse.SCALED_CG)):
        x_ref = torch.zeros(A.n_rows, dtype=torch.float64, device="cuda")
        rc_ref, i_ref = _call(L.gse_cg, M, b, x_ref, 1e-10, pol)
        assert rc_ref == gse.OK
        for call in range(2):                 # the second call sees the first call's leftovers
            x = torch.zeros(A.n_rows, dtype=torch.float64, device="cuda")
            rc, info = _call(L.gse_cg_noalloc, M, b, x, 1e-10, pol)
            assert rc == gse.OK, info
            assert info["iters"] == i_ref["iters"] and info["k_final"] == i_ref["k_final"]
            assert info["switch_iter"] == i_ref["switch_iter"]
            assert info["rel_res_true"] < 1e-10
            assert np.max(np.abs(x.cpu().numpy() - x_ref.cpu().numpy())) < 1e-8
    M.free()


def test_noalloc_rejects_beyond_its_limit():
    L = gse.lib()
    A = synth.poisson2d(257)                   # 66049 rows > 65536
    M = gse.GseMatrix.from_csr(A)
    b = torch.from_numpy(synth.rhs_ones(A)).cuda()
    x = torch.zeros(A.n_rows, dtype=torch.float64, device="cuda")
    rc, _ = _call(L.gse_cg_noalloc, M, b, x, 1e-10, gse.SCALED_CG)
    assert rc == gse.ERR_UNSUPPORTED
    A = synth.poisson2d(16)
    M2 = gse.GseMatrix.from_csr(A)
    b = torch.from_numpy(synth.rhs_ones(A)).cuda()
    x = torch.zeros(A.n_rows, dtype=torch.float64, device="cuda")
    floor = gse.Policy(**{**gse.SCALED_CG.__dict__, "flags": gse.POLICY_FLOOR})
    rc, _ = _call(L.gse_cg_noalloc, M2, b, x, 1e-10, floor)
    assert rc == gse.ERR_UNSUPPORTED
