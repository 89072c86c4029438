"""GPU stepped CG / GMRES (Alg. 3, Sec. III-D) against the oracle: each solve
reports its iterations and true residual and its solution is compared with the
oracle's FP64 solve; batched and engine (served) solves equal solo solves."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2411_04686_gb300 as gse  # noqa: E402


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _solve(A, method="cg", policy=gse.SCALED_CG, tol=1e-10, attach=(64,)):
    M = gse.GseMatrix.from_csr(A, attach=attach)
    b = synth.rhs_ones(A)
    x = torch.zeros(A.n_rows, dtype=torch.float64, device="cuda")
    info = (M.cg if method == "cg" else M.gmres)(_dev(b), x, tol=tol, policy=policy)
    return M, b, x.cpu().numpy(), info


def test_fp64_cg_matches_oracle():
    A = synth.poisson2d(32)
    M, b, x, info = _solve(A, policy=gse.fp64_policy(gse.SCALED_CG))
    ref = oracle.cg(A.row_ptr, A.col, A.val, b, tol=1e-10)
    assert info["status"] == gse.OK
    assert abs(info["iters"] - ref["info"]["iters"]) <= 2
    assert info["rel_res_true"] < 1e-10
    assert np.max(np.abs(x - ref["x"])) < 1e-8


def test_stepped_cg_exact_head_stays_at_level1():
    A = synth.poisson2d(32)
    M, b, x, info = _solve(A)
    ref = oracle.stepped_cg(A.row_ptr, A.col, oracle.levels(A.val), b, tol=1e-10, policy=oracle.SCALED_CG)
    assert info["status"] == gse.OK and info["k_final"] == 1
    assert info["switch_iter"][1] == -1
    assert abs(info["iters"] - ref["info"]["iters"]) <= 2
    assert np.max(np.abs(x - 1.0)) < 1e-7


def test_stepped_cg_steps_on_non_dyadic_values():
    A = synth.poisson2d(32, 1.0 / 3.0)
    M, b, x, info = _solve(A)
    ref = oracle.stepped_cg(A.row_ptr, A.col, oracle.levels(A.val), b, tol=1e-10, policy=oracle.SCALED_CG)
    assert info["status"] == gse.OK and info["k_final"] == 3
    assert info["rel_res_true"] < 1e-10
    # same path as the oracle up to rounding: level switches within a few iterations
    for i in (1, 2):
        assert abs(info["switch_iter"][i] - ref["info"]["switch_iter"][i]) <= 3
    r = b - oracle.spmv(A.row_ptr, A.col, A.val, x)
    assert np.linalg.norm(r) / np.linalg.norm(b) < 2e-10
    assert np.max(np.abs(x - ref["x"])) < 1e-8


def test_floor_policy_steps_earlier_and_converges():
    A = synth.laplace3d(16, shift=1e-3)
    pol = gse.Policy(**{**gse.SCALED_CG.__dict__, "flags": gse.POLICY_FLOOR})
    M, b, x, info = _solve(A, policy=pol)
    assert info["status"] == gse.OK and info["k_final"] == 3 and info["rel_res_true"] < 1e-10
    M2, _, x2, info2 = _solve(A)
    assert info["switch_iter"][1] < info2["switch_iter"][1]
    ref = oracle.cg(A.row_ptr, A.col, A.val, b, tol=1e-12)
    assert np.max(np.abs(x - ref["x"])) < 1e-7


@pytest.mark.parametrize("scale", [1.0, 1.0 / 30.0])
def test_floor_policy_against_oracle(scale):
    """The floor trigger on the GPU steps at the oracle's iterations exactly:
    both compare the recurrence residual with eta_k ||x_j|| / ||b||, x_j the
    iterate after the iteration's update (reading R20)."""
    A = synth.laplace3d(16, shift=1e-3).scaled(scale)
    for flags in (gse.POLICY_FLOOR, gse.POLICY_FLOOR | gse.POLICY_NO_STAGNATION):
        pol = gse.Policy(**{**gse.SCALED_CG.__dict__, "flags": flags})
        M, b, x, info = _solve(A, policy=pol)
        opol = oracle.Policy(**{**oracle.SCALED_CG.__dict__, "flags": flags})
        ref = oracle.stepped_cg(A.row_ptr, A.col, oracle.levels(A.val), b, tol=1e-10, policy=opol)
        assert info["status"] == gse.OK and ref["info"]["status"] == oracle.OK
        assert info["k_final"] == ref["info"]["k_final"] == 3
        assert info["switch_iter"] == ref["info"]["switch_iter"], (flags, info, ref["info"])
        assert abs(info["iters"] - ref["info"]["iters"]) <= 2
        assert np.max(np.abs(x - ref["x"])) < 1e-8 / scale


def test_bounded_wait_timeout_is_reported_then_cleared():
    """A staged kernel's bounded barrier wait that runs out is reported as
    GSE_TIMEOUT by the solve, and the next solve on the same handle is clean.
    The handle's test flag makes its staged kernels issue no copy, so every
    wait runs out with nothing in flight (no fault, no hang).  The table
    format with its index in the head, on the row schedule, runs the staged row
    kernel in the CG engine."""
    A = synth.poisson2d(32, 1.0 / 3.0)
    M = gse.GseMatrix.from_csr(A, num_exp=8, index_place=gse.INDEX_VALUE)
    M.set_schedule(gse.SCHEDULE_ROWS)
    b = _dev(synth.rhs_ones(A))
    short = gse.Policy(**{**gse.SCALED_CG.__dict__, "max_iter": 12})
    M.test_timeout(True)
    x = torch.zeros(A.n_rows, dtype=torch.float64, device="cuda")
    info = M.cg(b, x, policy=short)
    assert info["status"] == gse.TIMEOUT, info
    M.test_timeout(False)
    x = torch.zeros(A.n_rows, dtype=torch.float64, device="cuda")
    info = M.cg(b, x, tol=1e-10, policy=gse.SCALED_CG)
    table, levels = oracle.table_levels(A.val, 8, (16, 16, 20), index_in_value=True)
    ref = oracle.stepped_cg(A.row_ptr, A.col, levels, synth.rhs_ones(A), tol=1e-10, policy=oracle.SCALED_CG)
    assert info["status"] == gse.OK and info["rel_res_true"] < 1e-10
    for i in (1, 2):
        assert abs(info["switch_iter"][i] - ref["info"]["switch_iter"][i]) <= 3
    assert np.max(np.abs(x.cpu().numpy() - ref["x"])) < 1e-8
    M.free()


def test_cg_zero_rhs_and_nonfinite():
    A = synth.poisson2d(8)
    M = gse.GseMatrix.from_csr(A)
    x = torch.ones(A.n_rows, dtype=torch.float64, device="cuda")
    info = M.cg(torch.zeros(A.n_rows, dtype=torch.float64, device="cuda"), x)
    assert info["status"] == gse.OK and torch.all(x == 0)
    b = torch.ones(A.n_rows, dtype=torch.float64, device="cuda")
    b[3] = float("nan")
    x.zero_()
    info = M.cg(b, x)
    assert info["status"] == gse.NONFINITE


def test_stepped_gmres_against_oracle():
    A = synth.convdiff2d(32, peclet=10.0).scaled(1.0 / 3.0)
    M, b, x, info = _solve(A, method="gmres", policy=gse.SCALED_GMRES)
    ref = oracle.stepped_gmres(A.row_ptr, A.col, oracle.levels(A.val), b, tol=1e-10,
                               policy=oracle.SCALED_GMRES)
    assert info["status"] == gse.OK and info["k_final"] == 3 and info["rel_res_true"] < 1e-10
    assert abs(info["iters"] - ref["info"]["iters"]) <= 0.1 * ref["info"]["iters"] + 5
    assert np.max(np.abs(x - ref["x"])) < 1e-7


def test_fp64_gmres_matches_oracle():
    A = synth.convdiff2d(40, peclet=10.0)
    M, b, x, info = _solve(A, method="gmres", policy=gse.fp64_policy(gse.SCALED_GMRES))
    ref = oracle.gmres(A.row_ptr, A.col, A.val, b, tol=1e-10)
    assert info["status"] == gse.OK and info["rel_res_true"] < 1e-10
    assert abs(info["iters"] - ref["info"]["iters"]) <= 3
    assert np.max(np.abs(x - ref["x"])) < 1e-8


def _systems(count, seed):
    specs = synth.batch_specs(count, seed=seed, n_lo=200, n_hi=20000)
    return [s.build() for s in specs]


def test_batch_equals_solo_bitwise():
    As = _systems(12, 5)
    mats = [gse.GseMatrix.from_csr(A) for A in As]
    bs = [_dev(synth.rhs_ones(A)) for A in As]
    xs = [torch.zeros(A.n_rows, dtype=torch.float64, device="cuda") for A in As]
    rc, infos = gse.batch_cg(mats, bs, xs)
    assert rc == gse.OK
    for M, A, b, xb, ib in zip(mats, As, bs, xs, infos):
        x1 = torch.zeros(A.n_rows, dtype=torch.float64, device="cuda")
        i1 = M.cg(b, x1)
        assert ib["status"] == gse.OK and ib["rel_res_true"] < 1e-10
        assert ib["iters"] == i1["iters"] and ib["switch_iter"] == i1["switch_iter"]
        assert torch.equal(xb, x1)


def test_engine_continuous_batching_matches_solo():
    As = _systems(10, 6)
    mats = [gse.GseMatrix.from_csr(A) for A in As]
    bs = [_dev(synth.rhs_ones(A)) for A in As]
    eng = gse.Engine(4)
    xs = {}
    pending = list(range(len(As)))
    slot_of = {}
    results = {}
    while pending or slot_of:
        while pending and len(slot_of) < 4:
            i = pending.pop(0)
            xs[i] = torch.zeros(As[i].n_rows, dtype=torch.float64, device="cuda")
            s = eng.submit(mats[i], bs[i], xs[i])
            slot_of[s] = i
        eng.run(7, batch=4)      # few slots per call: systems join mid-flight
        for s, info in eng.poll():
            results[slot_of.pop(s)] = info
    eng.close()
    for i, A in enumerate(As):
        x1 = torch.zeros(A.n_rows, dtype=torch.float64, device="cuda")
        i1 = mats[i].cg(bs[i], x1)
        assert results[i]["status"] == gse.OK
        assert results[i]["iters"] == i1["iters"]
        assert torch.equal(xs[i], x1)


def test_engine_launch_wait_overlaps_encoding_and_matches_solo():
    """gse_engine_launch returns before the slots run; matrices encoded while a
    launch is in flight join at the next step and every result equals its solo
    solve bit for bit."""
    As = _systems(10, 7)
    bs = [_dev(synth.rhs_ones(A)) for A in As]
    eng = gse.Engine(4)
    xs, mats, slot_of, results = {}, {}, {}, {}
    pending, ready = list(range(len(As))), []
    launched = False
    while pending or slot_of or ready:
        # encode while the previous launch runs
        while pending and len(slot_of) + len(ready) < 4:
            i = pending.pop(0)
            mats[i] = gse.GseMatrix.from_csr(As[i])
            xs[i] = torch.zeros(As[i].n_rows, dtype=torch.float64, device="cuda")
            ready.append(i)
        if launched:
            eng.wait()
        for s, info in eng.poll():
            results[slot_of.pop(s)] = info
        for i in ready:
            slot_of[eng.submit(mats[i], bs[i], xs[i])] = i
        ready = []
        launched = bool(slot_of)
        if launched:
            eng.launch(7, batch=4)
    eng.close()
    for i, A in enumerate(As):
        x1 = torch.zeros(A.n_rows, dtype=torch.float64, device="cuda")
        i1 = mats[i].cg(bs[i], x1)
        assert results[i]["status"] == gse.OK
        assert results[i]["iters"] == i1["iters"]
        assert torch.equal(xs[i], x1)


@pytest.mark.parametrize("sched", [1, gse.SCHEDULE_ROWS])
def test_stepped_cg_on_each_engine_schedule(sched):
    """The engine's SpMV phase runs either schedule; both reach the same answer."""
    A = synth.laplace3d(12, shift=1e-2).scaled(1.0 / 3.0)
    M = gse.GseMatrix.from_csr(A)
    M.set_schedule(sched)
    b = torch.from_numpy(synth.rhs_ones(A)).cuda()
    x = torch.zeros(A.n_rows, dtype=torch.float64, device="cuda")
    info = M.cg(b, x, tol=1e-10, policy=gse.SCALED_CG)
    ref = oracle.stepped_cg(A.row_ptr, A.col, oracle.levels(A.val), synth.rhs_ones(A), tol=1e-10,
                            policy=oracle.SCALED_CG)
    assert info["status"] == gse.OK and info["k_final"] == 3 and info["rel_res_true"] < 1e-10
    assert abs(info["iters"] - ref["info"]["iters"]) <= 3
    assert np.max(np.abs(x.cpu().numpy() - ref["x"])) < 1e-8


def _arrow_spd(n=3000, dense=4, seed=3):
    """Symmetric, strictly diagonally dominant (so SPD) matrix: a tridiagonal band
    plus `dense` full rows and columns, values not dyadic.  Its dense rows span
    whole 256-nonzero chunks with no row end."""
    rng = np.random.default_rng(seed)
    rows, cols, vals = [], [], []
    for i in range(n - 1):
        v = -1.0 / 3.0 - 0.1 * rng.random()
        rows += [i, i + 1]; cols += [i + 1, i]; vals += [v, v]
    for k in range(dense):
        w = (rng.random(n) - 0.5) * 0.02 / 3.0
        for j in range(dense, n):
            rows += [k, j]; cols += [j, k]; vals += [w[j], w[j]]
    off = {}
    for r, c, v in zip(rows, cols, vals):
        off[(r, c)] = off.get((r, c), 0.0) + v
    rsum = np.zeros(n)
    for (r, c), v in off.items():
        rsum[r] += abs(v)
    for i in range(n):
        off[(i, i)] = rsum[i] + 0.05 + 0.01 * rng.random()
    keys = sorted(off)
    r = np.array([k[0] for k in keys], dtype=np.int64)
    row_ptr = np.zeros(n + 1, dtype=np.int32)
    np.add.at(row_ptr, r + 1, 1)
    row_ptr = np.cumsum(row_ptr).astype(np.int32)
    col = np.array([k[1] for k in keys], dtype=np.int32)
    val = np.array([off[k] for k in keys])
    return synth.CSR(row_ptr, col, val, n, "arrow")


def test_stepped_cg_nonzero_split_with_dense_rows():
    """Rows longer than a chunk (chunks with no row end) through the engine's
    nonzero-split SpMV phase with its p.Ap epilogue, against the oracle."""
    A = _arrow_spd()
    assert np.diff(A.row_ptr).max() > 2 * 256
    M = gse.GseMatrix.from_csr(A)
    M.set_schedule(1)
    b = synth.rhs_ones(A)
    x = torch.zeros(A.n_rows, dtype=torch.float64, device="cuda")
    info = M.cg(_dev(b), x, tol=1e-10, policy=gse.SCALED_CG)
    ref = oracle.stepped_cg(A.row_ptr, A.col, oracle.levels(A.val), b, tol=1e-10, policy=oracle.SCALED_CG)
    assert info["status"] == gse.OK and info["rel_res_true"] < 1e-10
    assert info["k_final"] == ref["info"]["k_final"]
    assert abs(info["iters"] - ref["info"]["iters"]) <= 3
    assert np.max(np.abs(x.cpu().numpy() - ref["x"])) < 1e-8
    # the standalone SpMV on the same matrix at every level, row by row
    xv = synth.uniform_x(A.n_cols, seed=5)
    enc = oracle.encode(A.val)
    for k in (1, 2, 3):
        y = M.spmv(k, _dev(xv)).cpu().numpy()
        yref, yabs = oracle.spmv_dot2(A.row_ptr, A.col, oracle.decode(*enc, k), xv)
        assert np.all(np.abs(y - yref) <= 1e-13 * yabs), k


def test_server_mixed_stream_equals_solo():
    """Served solves (continuous batching, admission by a memory budget that
    lets only a few systems in at once) give the solo results bit for bit."""
    from paper_2411_04686_gb300 import serve
    As = _systems(9, 8)
    pool = [(A, synth.rhs_ones(A)) for A in As]
    budget = 3 * max(serve.estimate_footprint(A.n_rows, A.nnz) for A in As)
    srv = serve.Server(lambda i: pool[i], capacity=8, mem_budget=budget, slots_per_step=5)
    for i, A in enumerate(As):
        srv.submit(serve.Request(i, 0.0, A.n_rows, A.nnz, payload=i))
    xs = {}
    orig = srv.place

    def place(A, b):
        M, bd, x = orig(A, b)
        xs[id(A)] = x
        return M, bd, x

    srv.place = place
    peak = 0
    while srv.queue or srv.active:
        srv.step()
        peak = max(peak, len(srv.active))
        assert srv.used <= budget             # admission never exceeds the memory budget
    srv.close()
    assert 1 < peak < len(As) and len(srv.done) == len(As)
    for c in srv.done:
        A, b = pool[c.rid]
        M = gse.GseMatrix.from_csr(A)
        x1 = torch.zeros(A.n_rows, dtype=torch.float64, device="cuda")
        i1 = M.cg(_dev(b), x1)
        assert c.info["status"] == gse.OK and c.info["iters"] == i1["iters"]
        assert torch.equal(xs[id(A)], x1)
