"""Pins for the oracle's FP64 CG / GMRES(30) and the stepped solvers (Alg. 3,
Sec. III-D): textbook invariants, dense LU solves and the CG error bound."""
import numpy as np
import pytest

import oracle
import synth


def _solve_dense(A):
    return np.linalg.solve(A.dense(), synth.rhs_ones(A))


def test_cg_invariants_on_spd():
    A = synth.laplace2d(14, 13, shift=0.05, aniso=(1.0, 0.3))
    b = synth.rhs_ones(A)
    T = 12
    out = oracle.cg(A.row_ptr, A.col, A.val, b, tol=1e-300, max_iter=T - 1, trace_n=T)
    D = A.dense()
    R, Pm, X = out["r"], out["p"], out["xs"]
    xs = np.linalg.solve(D, b)
    for i in range(T - 1):
        for j in range(i):
            # residuals mutually orthogonal, directions A-conjugate
            assert abs(R[i] @ R[j]) <= 1e-9 * np.linalg.norm(R[i]) * np.linalg.norm(R[j])
            assert abs(Pm[i] @ D @ Pm[j]) <= 1e-9 * np.sqrt((Pm[i] @ D @ Pm[i]) * (Pm[j] @ D @ Pm[j]))
    errA = [np.sqrt((xs - X[i]) @ D @ (xs - X[i])) for i in range(T)]
    assert all(errA[i + 1] <= errA[i] * (1 + 1e-12) for i in range(T - 1))
    # textbook bound ||e_j||_A <= 2 ((sqrt(k)-1)/(sqrt(k)+1))^j ||e_0||_A
    ev = np.linalg.eigvalsh(D)
    rho = (np.sqrt(ev[-1] / ev[0]) - 1) / (np.sqrt(ev[-1] / ev[0]) + 1)
    assert all(errA[j] <= 2 * rho ** j * errA[0] * (1 + 1e-10) for j in range(T))


def test_cg_solution_and_iteration_count():
    A = synth.poisson2d(32)
    b = synth.rhs_ones(A)
    out = oracle.cg(A.row_ptr, A.col, A.val, b, tol=1e-10, max_iter=5000)
    info = out["info"]
    assert info["status"] == oracle.OK and info["rel_res_true"] < 1e-9
    assert np.max(np.abs(out["x"] - 1.0)) < 1e-7
    # kappa(5-point Poisson 32x32) = cot^2(pi/(2*33)) ~ 441; the A-norm bound
    # caps CG at sqrt(kappa)/2 * ln(2/tol) ~ 250 iterations (b = A*1 is smooth,
    # so it needs far fewer)
    kappa = 1 / np.tan(np.pi / 66) ** 2
    assert 10 < info["iters"] <= int(np.sqrt(kappa) / 2 * np.log(2 / 1e-10)) + 10


def test_gmres_invariants_and_dense_solve():
    rng = np.random.default_rng(5)
    A = synth.convdiff2d(7, peclet=50.0)
    D = A.dense()
    b = rng.uniform(-1, 1, A.n_rows)
    m = 10
    out = oracle.gmres(A.row_ptr, A.col, A.val, b, tol=1e-12, restart=m, max_iter=2000,
                       want_first_cycle=True)
    V, H = out["V"], out["H"]
    assert np.linalg.norm(V @ V.T - np.eye(m + 1)) < 1e-12                   # orthonormal basis
    assert np.linalg.norm(D @ V[:m].T - V.T @ H) < 1e-12 * np.linalg.norm(D)  # Arnoldi relation
    assert out["info"]["status"] == oracle.OK
    assert np.allclose(out["x"], np.linalg.solve(D, b), rtol=0, atol=1e-9)


def test_gmres_full_restart_finite_termination():
    """With restart >= n GMRES reaches the solution in at most n steps."""
    rng = np.random.default_rng(6)
    n = 12
    D = rng.normal(size=(n, n)) + n * np.eye(n)
    rows, cols = np.nonzero(D)
    rp = np.zeros(n + 1, np.int32)
    np.cumsum(np.bincount(rows, minlength=n), out=rp[1:])
    b = rng.normal(size=n)
    out = oracle.gmres(rp, cols.astype(np.int32), D[rows, cols], b, tol=1e-13, restart=n, max_iter=n)
    assert out["info"]["iters"] <= n
    assert np.allclose(out["x"], np.linalg.solve(D, b), atol=1e-11)


def test_gmres_residual_nonincreasing_within_cycles():
    A = synth.convdiff2d(16, peclet=10.0)
    b = synth.rhs_ones(A)
    lv = oracle.levels(A.val)
    pol = oracle.Policy(l=10 ** 9, t=30, m=30, rsd_limit=0.03, ndec_limit=8, reldec_limit=0.08,
                        max_iter=3000, restart=30, k_start=3, k_max=3)
    out = oracle.stepped_gmres(A.row_ptr, A.col, lv, b, tol=1e-10, policy=pol, hist_cap=3000)
    h = out["hist"][: out["info"]["iters"]]
    for c in range(0, h.size, 30):
        seg = h[c:c + 30]
        assert np.all(np.diff(seg) <= 1e-15)


def test_stepped_cg_exact_head_never_steps():
    """5-point Poisson with values 4 and -1 is exact in the head (A_1 = A), so
    the stepped CG finishes at level 1 with the same answer as FP64 CG."""
    A = synth.poisson2d(32)
    b = synth.rhs_ones(A)
    lv = oracle.levels(A.val)
    assert np.array_equal(lv[0], A.val)
    out = oracle.stepped_cg(A.row_ptr, A.col, lv, b, tol=1e-10, policy=oracle.SCALED_CG)
    i = out["info"]
    assert i["status"] == oracle.OK and i["k_final"] == 1 and i["switch_iter"][1] == -1
    ref = oracle.cg(A.row_ptr, A.col, A.val, b, tol=1e-10)
    assert i["iters"] == ref["info"]["iters"]
    assert np.array_equal(out["x"], ref["x"])


def test_stepped_cg_steps_to_level3_on_non_dyadic_values():
    A = synth.poisson2d(32, scale=1.0 / 3.0)
    b = synth.rhs_ones(A)
    lv = oracle.levels(A.val)
    assert not np.array_equal(lv[0], A.val)
    out = oracle.stepped_cg(A.row_ptr, A.col, lv, b, tol=1e-10, policy=oracle.SCALED_CG, hist_cap=5000)
    i = out["info"]
    assert i["status"] == oracle.OK and i["k_final"] == 3
    assert 0 < i["switch_iter"][1] < i["switch_iter"][2]
    assert i["rel_res_true"] < 1e-10
    # the true FP64 residual agrees (A_3 differs from A by < 2^-50 relative)
    r = b - oracle.spmv(A.row_ptr, A.col, A.val, out["x"])
    assert np.linalg.norm(r) / np.linalg.norm(b) < 2e-10
    assert np.max(np.abs(out["x"] - 1.0)) < 1e-6


def test_stepped_cg_level1_floor():
    """Without stepping, CG on A_1 converges to A_1^-1 b: its true residual
    stalls near ||(A - A_1) x|| / ||b||, far above 1e-10 (Sec. III-D's reason
    to raise the precision)."""
    A = synth.laplace3d(10, shift=1e-3)
    b = synth.rhs_ones(A)
    lv = oracle.levels(A.val)
    out = oracle.cg(A.row_ptr, A.col, lv[0], b, tol=1e-12, max_iter=5000)
    r = b - oracle.spmv(A.row_ptr, A.col, A.val, out["x"])
    floor = np.linalg.norm(oracle.spmv(A.row_ptr, A.col, A.val - lv[0], out["x"])) / np.linalg.norm(b)
    assert np.linalg.norm(r) / np.linalg.norm(b) == pytest.approx(floor, rel=1e-2)
    assert floor > 1e-8


def test_stepped_gmres_reaches_tol_at_level3():
    A = synth.convdiff2d(24, peclet=10.0).scaled(1.0 / 3.0)
    b = synth.rhs_ones(A)
    lv = oracle.levels(A.val)
    out = oracle.stepped_gmres(A.row_ptr, A.col, lv, b, tol=1e-10, policy=oracle.SCALED_GMRES)
    i = out["info"]
    assert i["status"] == oracle.OK and i["k_final"] == 3 and i["rel_res_true"] < 1e-10
    ref = oracle.gmres(A.row_ptr, A.col, A.val, b, tol=1e-10)
    assert np.allclose(out["x"], ref["x"], atol=1e-7)


def test_zero_rhs():
    A = synth.poisson2d(4)
    b = np.zeros(A.n_rows)
    lv = oracle.levels(A.val)
    for f in (oracle.stepped_cg, oracle.stepped_gmres):
        out = f(A.row_ptr, A.col, lv, b, x0=np.ones(A.n_rows), tol=1e-10, policy=oracle.SCALED_CG)
        assert out["info"]["status"] == oracle.OK and np.all(out["x"] == 0)


def _floor_policy(flags):
    return oracle.Policy(**{**oracle.SCALED_CG.__dict__, "flags": flags})


def test_floor_trigger_fires_where_the_residual_meets_the_floor():
    """The perturbation-floor trigger (beyond the paper): level k is left at the
    first iteration j with ||r_j|| / ||b|| <= eta_k ||x_j|| / ||b||, eta_k the
    infinity norm of A_3 - A_k.  Checked against the plain CG on A_1 (which
    runs the stepped solver's level-1 arithmetic) and scipy's matrix norm."""
    sp = pytest.importorskip("scipy.sparse")
    # scaled so that no value is exact at level 1 (diagonal and off-diagonal
    # errors have opposite signs) and ||x|| is about 30 ||b||
    A = synth.laplace3d(10, shift=1e-3).scaled(1.0 / 30.0)
    b = synth.rhs_ones(A)
    lv = oracle.levels(A.val)
    pol = _floor_policy(oracle.POLICY_FLOOR | oracle.POLICY_NO_STAGNATION)
    out = oracle.stepped_cg(A.row_ptr, A.col, lv, b, tol=1e-10, policy=pol)
    i = out["info"]
    assert i["status"] == oracle.OK and i["k_final"] == 3 and i["rel_res_true"] < 1e-10
    js = i["switch_iter"][1]
    assert js > 0
    eta = sp.linalg.norm(sp.csr_matrix((lv[2] - lv[0], A.col, A.row_ptr), shape=(A.n_rows, A.n_cols)), np.inf)
    assert eta > 0
    tr = oracle.cg(A.row_ptr, A.col, lv[0], b, tol=1e-30, max_iter=js, trace_n=js + 1)
    nb = np.linalg.norm(b)
    res = np.linalg.norm(tr["r"], axis=1) / nb
    flo = eta * np.linalg.norm(tr["xs"], axis=1) / nb
    assert np.linalg.norm(tr["xs"][js]) > 10 * nb
    assert np.all(res[1:js] > flo[1:js])
    assert res[js] <= flo[js]
    # without the trigger (and without stagnation checks) level 1 runs on
    no = oracle.stepped_cg(A.row_ptr, A.col, lv, b, tol=1e-10, policy=_floor_policy(oracle.POLICY_NO_STAGNATION))
    assert no["info"]["switch_iter"][1] > js


def test_floor_trigger_is_silent_when_the_head_is_exact():
    # values 4 and -1 are exact at level 1: eta = 0, so the trigger never fires
    A = synth.poisson2d(32)
    b = synth.rhs_ones(A)
    lv = oracle.levels(A.val)
    a = oracle.stepped_cg(A.row_ptr, A.col, lv, b, tol=1e-10, policy=_floor_policy(oracle.POLICY_FLOOR))
    c = oracle.stepped_cg(A.row_ptr, A.col, lv, b, tol=1e-10, policy=oracle.SCALED_CG)
    assert a["info"] == c["info"] and np.array_equal(a["x"], c["x"])


def test_reported_true_residual_is_recomputed_from_x():
    """info.rel_res_true is ||b - A x|| / ||b|| for the returned x (dense
    product in numpy), not the recurrence's estimate."""
    A = synth.convdiff2d(12, peclet=10.0)
    D = A.dense()
    b = synth.rhs_ones(A)
    nb = np.linalg.norm(b)
    for out in (oracle.cg(A.row_ptr, A.col, A.val, b, tol=1e-8, max_iter=7),
                oracle.gmres(A.row_ptr, A.col, A.val, b, tol=1e-8, restart=5, max_iter=12)):
        assert out["info"]["status"] == oracle.MAXITER
        assert out["info"]["rel_res_true"] == pytest.approx(np.linalg.norm(b - D @ out["x"]) / nb, rel=1e-10)
    lv = oracle.levels(A.val)
    pol = oracle.Policy(l=10 ** 9, t=5, m=5, rsd_limit=0.5, ndec_limit=0, reldec_limit=0.45, max_iter=9)
    for f in (oracle.stepped_cg, oracle.stepped_gmres):
        out = f(A.row_ptr, A.col, lv, b, tol=1e-8, policy=pol)
        r = b - oracle.spmv(A.row_ptr, A.col, lv[2], out["x"])       # measured with A_kmax
        assert out["info"]["rel_res_true"] == pytest.approx(np.linalg.norm(r) / nb, rel=1e-10)


def _always_step(l, t, m, restart, max_iter):
    # rsd >= 0 > rsd_limit and ndec < ndec_limit always hold: Condition 1
    # fires at every check, so the step iterations follow from l, t, m alone
    return oracle.Policy(l=l, t=t, m=m, rsd_limit=-1.0, ndec_limit=10 ** 6, reldec_limit=0.45,
                         max_iter=max_iter, restart=restart)


def test_stepped_cg_check_schedule():
    """Checks fall at j >= l with j mod m = 0 once t + 1 residuals have been
    recorded since the last level change; each check raises k by one level.
    l = 20, m = 10, t = 12: the first check (j = 20, 20 entries) steps to
    k = 2 and clears the history; j = 30 has 10 entries, too few; j = 40 has 20
    and steps to k = 3."""
    A = synth.poisson2d(32)
    b = synth.rhs_ones(A)
    lv = oracle.levels(A.val)
    out = oracle.stepped_cg(A.row_ptr, A.col, lv, b, tol=1e-300, policy=_always_step(20, 12, 10, 30, 60),
                            hist_cap=100)
    i = out["info"]
    assert i["status"] == oracle.MAXITER and i["iters"] == 60 and i["k_final"] == 3
    assert i["switch_iter"] == [0, 20, 40]
    # the same policy starting at k = 2 steps once, at the first check
    p2 = oracle.Policy(**{**_always_step(20, 12, 10, 30, 60).__dict__, "k_start": 2})
    i2 = oracle.stepped_cg(A.row_ptr, A.col, lv, b, tol=1e-300, policy=p2)["info"]
    assert i2["switch_iter"] == [-1, 0, 20]


def test_stepped_gmres_check_schedule():
    """GMRES changes level only at a cycle end, and only when the cycle crossed
    a multiple of m at or after l.  restart 30, l = m = 20, t = 5: cycle 1
    (j = 30) crossed 20 and steps to k = 2; cycle 2 (j = 60) crossed 40 and 60
    and steps to k = 3."""
    A = synth.convdiff2d(24, peclet=10.0)
    b = synth.rhs_ones(A)
    lv = oracle.levels(A.val)
    out = oracle.stepped_gmres(A.row_ptr, A.col, lv, b, tol=1e-300, policy=_always_step(20, 5, 20, 30, 90),
                               hist_cap=100)
    i = out["info"]
    assert i["status"] == oracle.MAXITER and i["iters"] == 90 and i["k_final"] == 3
    assert i["switch_iter"] == [0, 30, 60]
    # m = 45: cycle 1 (j = 30) crosses no multiple of 45, cycle 2 (j = 60)
    # crosses 45, cycle 3 (j = 90) crosses 90
    i45 = oracle.stepped_gmres(A.row_ptr, A.col, lv, b, tol=1e-300,
                               policy=_always_step(20, 5, 45, 30, 90))["info"]
    assert i45["switch_iter"] == [0, 60, 90]


def test_plain_solvers_zero_rhs_give_zero():
    """b = 0: the solution of a nonsingular system is x = 0, whatever x0."""
    A = synth.poisson2d(6)
    b = np.zeros(A.n_rows)
    for out in (oracle.cg(A.row_ptr, A.col, A.val, b, x0=np.ones(A.n_rows)),
                oracle.gmres(A.row_ptr, A.col, A.val, b, x0=np.ones(A.n_rows))):
        assert out["info"]["status"] == oracle.OK and out["info"]["iters"] == 0
        assert np.all(out["x"] == 0)


def test_cg_breakdown_on_a_negative_definite_matrix():
    """p.Ap <= 0 ends plain CG with BREAKDOWN before any update (-A is
    negative definite, so p_0.A p_0 < 0)."""
    A = synth.poisson2d(6)
    b = synth.rhs_ones(A)
    out = oracle.cg(A.row_ptr, A.col, -A.val, b, max_iter=50)
    assert out["info"]["status"] == oracle.BREAKDOWN and out["info"]["iters"] == 0
    assert np.all(out["x"] == 0)


def test_breakdown_below_kmax_steps_a_level():
    """Reading of the stepped solvers: a breakdown at k < k_max raises the
    level (the truncated operator may have lost definiteness), at k_max it is
    reported.  The levels are given directly: A_1 = 0 breaks both CG
    (p.Ap = 0) and GMRES (a zero Hessenberg column) at once, A_1 = -A breaks
    CG; A_2 = A_3 = A then solve the system from level 2 on."""
    A = synth.poisson2d(8)
    b = synth.rhs_ones(A)
    pol = oracle.Policy(l=10 ** 9, t=5, m=5, rsd_limit=0.5, ndec_limit=0, reldec_limit=0.45, max_iter=500)
    runs = [(oracle.stepped_cg, 0.0 * A.val), (oracle.stepped_cg, -A.val), (oracle.stepped_gmres, 0.0 * A.val)]
    for f, a1 in runs:
        out = f(A.row_ptr, A.col, [a1, A.val, A.val], b, tol=1e-10, policy=pol)
        i = out["info"]
        assert i["status"] == oracle.OK and i["switch_iter"][:2] == [0, 0], (f.__name__, i)
        assert i["rel_res_true"] < 1e-10
        assert np.max(np.abs(out["x"] - 1.0)) < 1e-8
        # at k_max the same breakdown is reported
        bad = f(A.row_ptr, A.col, [a1, a1, a1], b, tol=1e-10, policy=pol)["info"]
        assert bad["status"] == oracle.BREAKDOWN and bad["k_final"] == 3


def test_ok_only_below_tol_in_the_true_residual():
    """At k_max a recurrence residual below tol is not enough: the true
    residual decides, and the recurrence restarts from it otherwise.  With a
    tolerance below the attainable accuracy (1e-18) the recurrence residual
    keeps falling but the true one cannot, so the solve must not report OK."""
    A = synth.poisson2d(16)
    b = synth.rhs_ones(A)
    lv = oracle.levels(A.val)
    pol = oracle.Policy(l=10 ** 9, t=5, m=5, rsd_limit=0.5, ndec_limit=0, reldec_limit=0.45, max_iter=400,
                        k_start=3)
    for f in (oracle.stepped_cg, oracle.stepped_gmres):
        out = f(A.row_ptr, A.col, lv, b, tol=1e-18, policy=pol, hist_cap=400)
        i = out["info"]
        assert i["status"] == oracle.MAXITER and i["iters"] == 400, (f.__name__, i)
        assert 1e-18 < i["rel_res_true"] < 1e-13
        assert np.min(out["hist"]) < 1e-18       # the recurrence went below tol


def test_stepped_gmres_history_is_the_least_squares_residual():
    """The history the stepped GMRES monitors is |g_(i+1)| / ||b||, one entry
    per inner iteration: it ends at the reported recurrence residual and, in a
    run without level changes, equals the plain GMRES residual sequence."""
    A = synth.convdiff2d(12, peclet=10.0)
    b = synth.rhs_ones(A)
    lv = oracle.levels(A.val)
    pol = oracle.Policy(l=10 ** 9, t=5, m=5, rsd_limit=0.5, ndec_limit=0, reldec_limit=0.45, max_iter=45,
                        restart=15, k_start=3)
    out = oracle.stepped_gmres(A.row_ptr, A.col, lv, b, tol=1e-14, policy=pol, hist_cap=100)
    i = out["info"]
    h = out["hist"]
    assert i["iters"] == 45 and np.all(h[:45] > 0) and np.all(h[45:] == 0)
    assert h[44] == i["rel_res_rec"]
    for c in (15, 30, 45):                    # the plain GMRES stopped after c iterations
        ref = oracle.gmres(A.row_ptr, A.col, lv[2], b, tol=1e-14, restart=15, max_iter=c)
        assert ref["info"]["rel_res_rec"] == h[c - 1]
