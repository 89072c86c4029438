"""GPU encoder vs the oracle: bit-exact segments, group exponents and decoded
values (Sec. III-B, Alg. 1, Fig. 3; decode per Alg. 2)."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2411_04686_gb300 as gse  # noqa: E402


def _random_csr(n, m, mean, seed, empty_frac=0.0, lo=-12, hi=12):
    rng = np.random.default_rng(seed)
    lens = rng.poisson(mean, n)
    lens[rng.random(n) < empty_frac] = 0
    lens = np.minimum(lens, m)
    rp = np.zeros(n + 1, np.int64)
    np.cumsum(lens, out=rp[1:])
    col = np.concatenate([np.sort(rng.choice(m, L, replace=False)) for L in lens]) if rp[-1] else np.zeros(0, np.int64)
    val = rng.choice([-1.0, 1.0], rp[-1]) * 2.0 ** rng.uniform(lo, hi, rp[-1])
    val[rng.random(rp[-1]) < 0.02] = 0.0
    if rp[-1] > 3:
        val[1] = 5e-324          # a subnormal
        val[2] = -0.0
    return synth.CSR(rp.astype(np.int32), col.astype(np.int32), val, m, "random")


def _extreme_csr():
    """Values over the whole normal range (E_g up to 2047) with DBL_MAX, the
    smallest normal exponents, a subnormal and -0.0 among them."""
    A = _random_csr(2000, 1500, 8.0, 5, lo=-1020, hi=1020)
    A.val[3] = np.finfo(np.float64).max
    A.val[4] = 2.0 ** -1022
    A.val[5] = -2.0 ** -1021
    return A


CASES = [
    ("poisson32", lambda: synth.poisson2d(32)),
    ("extreme", _extreme_csr),
    ("poisson32_third", lambda: synth.poisson2d(32, 1.0 / 3.0)),
    ("random_ragged", lambda: _random_csr(3001, 2500, 9.0, 1, empty_frac=0.1)),
    ("powerlaw", lambda: synth.powerlaw_random(20000, 16.0, 2048, seed=2)),
    ("tiny", lambda: _random_csr(3, 5, 2.0, 3)),
]
SEGS = [(16, 16, 20), (16, 16, 32), (16, 16, 16), (12, 16, 24), (16, 8, 8), (16,), (16, 16), (2, 16, 20)]


@pytest.mark.parametrize("name,make", CASES)
@pytest.mark.parametrize("G", [32, 16, 8])
def test_encode_bit_exact(name, make, G):
    A = make()
    for seg in SEGS if G == 32 else [(16, 16, 20)]:
        M = gse.GseMatrix.from_csr(A, group_size=G, seg_bits=seg)
        got = M.export()
        ref = oracle.encode(A.val, G, seg)
        for a, b, what in zip(got, ref, ("head", "tail1", "tail2", "gexp")):
            assert np.array_equal(a.astype(np.int64), b.astype(np.int64)), (name, G, seg, what)
        for k in range(1, len(seg) + 1):
            d = M.decode(k).cpu().numpy()
            dr = oracle.decode(*ref, k, G, seg)
            assert np.array_equal(d.view(np.uint64), dr.view(np.uint64)), (name, G, seg, k)
        M.free()


def test_encode_from_device_arrays():
    A = synth.powerlaw_random(5000, 8.0, 500, seed=4)
    dev = [torch.from_numpy(a).cuda() for a in (A.row_ptr, A.col, A.val)]
    M = gse.GseMatrix(*dev, n_cols=A.n_cols)
    ref = oracle.encode(A.val)
    for a, b in zip(M.export(), ref):
        assert np.array_equal(a.astype(np.int64), b.astype(np.int64))


def test_encode_rejects_bad_input():
    A = synth.poisson2d(4)
    bad = A.val.copy()
    bad[5] = np.inf
    with pytest.raises(gse.GseError) as e:
        gse.GseMatrix(A.row_ptr, A.col, bad, n_cols=A.n_cols)
    assert e.value.code == gse.ERR_NONFINITE
    bad = A.val.copy()
    bad[0] = np.nan
    with pytest.raises(gse.GseError):
        gse.GseMatrix(A.row_ptr, A.col, bad, n_cols=A.n_cols)
    col = A.col.copy()
    col[3] = A.n_cols           # out of range
    with pytest.raises(gse.GseError) as e:
        gse.GseMatrix(A.row_ptr, col, A.val, n_cols=A.n_cols)
    assert e.value.code == gse.ERR_INVALID
    rp = A.row_ptr.copy()
    rp[3], rp[4] = rp[4], rp[3]  # not monotone
    with pytest.raises(gse.GseError):
        gse.GseMatrix(rp, A.col, A.val, n_cols=A.n_cols)
    with pytest.raises(gse.GseError) as e:
        gse.GseMatrix(A.row_ptr, A.col, A.val, n_cols=A.n_cols, seg_bits=(16, 16, 21))
    assert e.value.code == gse.ERR_UNSUPPORTED


def test_full_size_128cube_sampled_groups():
    """At the benchmark size: the encoding of sampled groups matches the oracle."""
    A = synth.laplace3d(128)
    M = gse.GseMatrix.from_csr(A)
    head, t1, t2, gexp = M.export()
    rng = np.random.default_rng(0)
    groups = rng.choice(gexp.size, 2000, replace=False)
    idx = (groups[:, None] * 32 + np.arange(32)).ravel()
    idx = idx[idx < A.nnz]
    ref = oracle.encode(A.val[idx.reshape(-1, 32)].ravel() if idx.size % 32 == 0 else A.val[idx])
    assert np.array_equal(head[idx], ref[0]) and np.array_equal(t1[idx], ref[1]) and np.array_equal(t2[idx], ref[2])
    assert np.array_equal(gexp[groups], ref[3])
