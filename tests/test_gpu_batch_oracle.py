"""Batched and served stepped CG pinned to the oracle.

A mix of SPD systems drawn like the batched workload (2D and 3D Laplacians,
random per-axis anisotropy in [0.01, 1], diagonal shift log-uniform in
[1e-4, 1e-1], sizes up to 2e4 rows) is solved three ways on the GPU: in one
gse_batch_cg call, through the engine with systems joining while others run,
and through serve.Server under a memory budget.  Every result is compared with
oracle.stepped_cg on the same matrix and right-hand side (the stepped CG of
Alg. 3 with the readings of Sec. III-D), and with its solo GPU solve, bit for
bit: each result is the same alone and in the mix.

The solution check is a bound, not a fixed tolerance: both solves reach a
true relative residual below 1e-10, so ||x - x_ref||_2 <= (||r|| + ||r_ref||)
/ lambda_min(A) < 2e-10 ||b|| / lambda_min(A), and for these Dirichlet
Laplacians lambda_min = shift + sum_a 4 eps_a sin^2(pi / (2 (N_a + 1))).
"""
import math

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2411_04686_gb300 as gse  # noqa: E402

SPECS = synth.batch_specs(10, seed=21, n_lo=1000, n_hi=20000)


def _lambda_min(spec):
    return spec.shift + sum(4.0 * e * math.sin(math.pi / (2.0 * (N + 1))) ** 2 for e, N in zip(spec.aniso, spec.dims))


@pytest.fixture(scope="module")
def mix():
    out = []
    for spec in SPECS:
        A = spec.build()
        b = synth.rhs_ones(A)
        ref = oracle.stepped_cg(A.row_ptr, A.col, oracle.levels(A.val), b, tol=1e-10, policy=oracle.SCALED_CG)
        bound = 2e-10 * float(np.linalg.norm(b)) / _lambda_min(spec)
        out.append((spec, A, b, ref, bound))
    return out


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _check_against_oracle(info, x, ref, bound, what):
    ri = ref["info"]
    assert info["status"] == gse.OK and ri["status"] == oracle.OK, (what, info, ri)
    assert info["k_final"] == ri["k_final"] == 3, (what, info, ri)
    for i in (1, 2):
        assert abs(info["switch_iter"][i] - ri["switch_iter"][i]) <= 3, (what, info, ri)
    assert abs(info["iters"] - ri["iters"]) <= 2, (what, info, ri)
    assert info["rel_res_true"] < 1e-10 and ri["rel_res_true"] < 1e-10, (what, info, ri)
    err = float(np.max(np.abs(x - ref["x"])))
    assert err <= bound, (what, err, bound)


def _solo(A, b):
    M = gse.GseMatrix.from_csr(A)
    x = torch.zeros(A.n_rows, dtype=torch.float64, device="cuda")
    info = M.cg(_dev(b), x)
    M.free()
    return info, x


def test_mix_is_varied():
    """The draw covers both dimensions, strong anisotropy and small shifts."""
    dims = {s.dim for s in SPECS}
    assert dims == {2, 3}
    assert min(min(s.aniso) for s in SPECS) < 0.1 and min(s.shift for s in SPECS) < 1e-3
    assert max(s.n for s in SPECS) > 10000 and min(s.n for s in SPECS) < 3000


def test_batch_cg_against_oracle(mix):
    mats = [gse.GseMatrix.from_csr(A) for _, A, _, _, _ in mix]
    bs = [_dev(b) for _, _, b, _, _ in mix]
    xs = [torch.zeros(A.n_rows, dtype=torch.float64, device="cuda") for _, A, _, _, _ in mix]
    rc, infos = gse.batch_cg(mats, bs, xs)
    assert rc == gse.OK
    for (spec, A, b, ref, bound), x, info in zip(mix, xs, infos):
        _check_against_oracle(info, x.cpu().numpy(), ref, bound, ("batch", spec))
        i1, x1 = _solo(A, b)
        assert info["iters"] == i1["iters"] and info["switch_iter"] == i1["switch_iter"]
        assert torch.equal(x, x1)
    for M in mats:
        M.free()


def test_batch_cg_floor_policy_against_oracle(mix):
    """The batch under the scaled policy plus the perturbation-floor trigger
    (reading R20; its decision is taken per system in the x-update phase)
    steps at the oracle's iterations, system by system, and equals each
    system's solo solve bit for bit."""
    pol = gse.Policy(**{**gse.SCALED_CG.__dict__, "flags": gse.POLICY_FLOOR})
    opol = oracle.Policy(**{**oracle.SCALED_CG.__dict__, "flags": oracle.POLICY_FLOOR})
    mats = [gse.GseMatrix.from_csr(A) for _, A, _, _, _ in mix]
    bs = [_dev(b) for _, _, b, _, _ in mix]
    xs = [torch.zeros(A.n_rows, dtype=torch.float64, device="cuda") for _, A, _, _, _ in mix]
    rc, infos = gse.batch_cg(mats, bs, xs, policy=pol)
    assert rc == gse.OK
    for (spec, A, b, _, bound), M, x, info in zip(mix, mats, xs, infos):
        ref = oracle.stepped_cg(A.row_ptr, A.col, oracle.levels(A.val), b, tol=1e-10, policy=opol)
        ri = ref["info"]
        assert info["status"] == gse.OK and ri["status"] == oracle.OK, (spec, info, ri)
        assert info["k_final"] == ri["k_final"] == 3, (spec, info, ri)
        assert info["switch_iter"] == ri["switch_iter"], (spec, info, ri)
        assert abs(info["iters"] - ri["iters"]) <= 2, (spec, info, ri)
        assert info["rel_res_true"] < 1e-10 and ri["rel_res_true"] < 1e-10
        assert float(np.max(np.abs(x.cpu().numpy() - ref["x"]))) <= bound
        x1 = torch.zeros(A.n_rows, dtype=torch.float64, device="cuda")
        i1 = M.cg(_dev(b), x1, policy=pol)
        assert info["iters"] == i1["iters"] and info["switch_iter"] == i1["switch_iter"]
        assert torch.equal(x, x1)
    for M in mats:
        M.free()


def test_engine_staggered_against_oracle(mix):
    """Systems join the engine while others are mid-solve (capacity 3, few
    slots per step) and each finishes where the oracle does."""
    mats = [gse.GseMatrix.from_csr(A) for _, A, _, _, _ in mix]
    bs = [_dev(b) for _, _, b, _, _ in mix]
    eng = gse.Engine(3)
    xs, slot_of, results = {}, {}, {}
    pending = list(range(len(mix)))
    while pending or slot_of:
        while pending and len(slot_of) < 3:
            i = pending.pop(0)
            xs[i] = torch.zeros(mix[i][1].n_rows, dtype=torch.float64, device="cuda")
            slot_of[eng.submit(mats[i], bs[i], xs[i])] = i
        eng.run(11, batch=4)
        for s, info in eng.poll():
            results[slot_of.pop(s)] = info
    eng.close()
    for i, (spec, A, b, ref, bound) in enumerate(mix):
        _check_against_oracle(results[i], xs[i].cpu().numpy(), ref, bound, ("engine", spec))
        i1, x1 = _solo(A, b)
        assert results[i]["iters"] == i1["iters"] and torch.equal(xs[i], x1)
    for M in mats:
        M.free()


def test_server_against_oracle(mix):
    """Served solves under a memory budget that admits only a few systems at
    a time: every completion matches the oracle and its solo solve."""
    from paper_2411_04686_gb300 import serve
    pool = [(A, b) for _, A, b, _, _ in mix]
    budget = 3 * max(serve.estimate_footprint(A.n_rows, A.nnz) for A, _ in pool)
    srv = serve.Server(lambda i: pool[i], capacity=8, mem_budget=budget, slots_per_step=7)
    for i, (A, _) in enumerate(pool):
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
        assert srv.used <= budget
    srv.close()
    assert 1 < peak < len(pool) and len(srv.done) == len(pool)
    for c in srv.done:
        spec, A, b, ref, bound = mix[c.rid]
        x = xs[id(A)]
        _check_against_oracle(c.info, x.cpu().numpy(), ref, bound, ("served", spec))
        i1, x1 = _solo(A, b)
        assert c.info["iters"] == i1["iters"] and torch.equal(x, x1)
