"""gse_cg_noalloc, called through the C ABI, against gse_cg.

gse_cg_noalloc exists for callers that cannot allocate device memory after
their set-up (fixed memory budgets, allocators that forbid new allocations,
threads that must not let cudaMalloc/cudaFree synchronise the device).  It runs
the same CG kernels with all scratch in a fixed device array inside the
library, so its answer equals gse_cg's bit for bit (solution, iteration
counts, switch iterations, and the true residual of a converged solve), on
consecutive calls (the array keeps the previous call's contents), on both SpMV
schedules, and on a handle that has never run a solve (nothing is allocated
lazily on the way).  This file is collected last on purpose."""
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


def _same(info, i_ref, x, x_ref):
    assert info["iters"] == i_ref["iters"] and info["k_final"] == i_ref["k_final"]
    assert info["switch_iter"] == i_ref["switch_iter"]
    assert info["rel_res_true"] < 1e-10 and info["rel_res_true"] == i_ref["rel_res_true"]
    assert torch.equal(x, x_ref)


@pytest.mark.parametrize("schedule", [0, 1])     # 0: automatic (lane-row here); 1: the nonzero split
@pytest.mark.parametrize("make", [lambda: synth.poisson2d(32, 1.0 / 3.0),
                                  lambda: synth.laplace3d(20, shift=1e-3),
                                  lambda: synth.laplace2d(256, 255, shift=1e-2, aniso=(1.0, 0.2))])
def test_noalloc_cg_matches_cg_on_consecutive_calls(make, schedule):
    L = gse.lib()
    A = make()
    M = gse.GseMatrix.from_csr(A, attach=(64,))
    M.set_schedule(schedule)
    b = torch.from_numpy(synth.rhs_ones(A)).cuda()
    for pol in (gse.SCALED_CG, gse.fp64_policy(gse.SCALED_CG)):
        x_ref = torch.zeros(A.n_rows, dtype=torch.float64, device="cuda")
        rc_ref, i_ref = _call(L.gse_cg, M, b, x_ref, 1e-10, pol)
        assert rc_ref == gse.OK
        for call in range(2):                 # the second call sees the first call's leftovers
            x = torch.zeros(A.n_rows, dtype=torch.float64, device="cuda")
            rc, info = _call(L.gse_cg_noalloc, M, b, x, 1e-10, pol)
            assert rc == gse.OK, info
            _same(info, i_ref, x, x_ref)
    M.free()


def test_noalloc_first_solve_on_a_fresh_handle_allocates_nothing():
    """A handle that has run no solve yet: gse_cg_noalloc leaves the device's
    free memory, torch's allocator and the handle's footprint unchanged, and
    its answer equals gse_cg's on another handle of the same matrix.  A first
    call on a third handle loads the kernels beforehand (the driver allocates
    kernel code on a kernel's first launch, which is not the solve's doing)."""
    L = gse.lib()
    A = synth.laplace3d(18, shift=1e-3).scaled(1.0 / 3.0)
    b = torch.from_numpy(synth.rhs_ones(A)).cuda()
    W = gse.GseMatrix.from_csr(A)
    xw = torch.zeros(A.n_rows, dtype=torch.float64, device="cuda")
    assert _call(L.gse_cg_noalloc, W, b, xw, 1e-10, gse.SCALED_CG)[0] == gse.OK
    M = gse.GseMatrix.from_csr(A)
    x = torch.zeros(A.n_rows, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    fp0, free0, torch0 = M.footprint(), torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
    rc, info = _call(L.gse_cg_noalloc, M, b, x, 1e-10, gse.SCALED_CG)
    assert rc == gse.OK, info
    assert M.footprint() == fp0
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_allocated() == torch0
    R = gse.GseMatrix.from_csr(A)
    x_ref = torch.zeros(A.n_rows, dtype=torch.float64, device="cuda")
    rc_ref, i_ref = _call(L.gse_cg, R, b, x_ref, 1e-10, gse.SCALED_CG)
    assert rc_ref == gse.OK
    _same(info, i_ref, x, x_ref)
    for h in (W, M, R):
        h.free()


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
