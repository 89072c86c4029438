"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module only builds CSR matrices and vectors (numpy, host memory).  It holds
none of the method's arithmetic: no encoding, no SpMV, no solver step.  Every
matrix is CSR with int32 row pointers and column indices, columns sorted within
each row, rows in row-major grid order, FP64 values.

The shapes stand in for the paper's SuiteSparse workloads (Sec. IV-A), which are
not available here: 2D/3D finite-difference Laplacians (SPD, for CG), a
convection-diffusion operator (nonsymmetric, for GMRES) and a random matrix with
power-law row lengths and values spread over many binades.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class CSR:
    row_ptr: np.ndarray   # int32[n_rows + 1]
    col: np.ndarray       # int32[nnz]
    val: np.ndarray       # float64[nnz]
    n_cols: int
    name: str = ""

    @property
    def n_rows(self) -> int:
        return self.row_ptr.size - 1

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def dense(self) -> np.ndarray:
        """Dense copy for tiny matrices (tests only)."""
        d = np.zeros((self.n_rows, self.n_cols))
        rows = np.repeat(np.arange(self.n_rows), np.diff(self.row_ptr))
        np.add.at(d, (rows, self.col), self.val)
        return d

    def scaled(self, s: float) -> "CSR":
        return CSR(self.row_ptr, self.col, self.val * s, self.n_cols, self.name + f"*{s:g}")


def _from_stencil(cols: np.ndarray, vals: np.ndarray, valid: np.ndarray, n: int, name: str) -> CSR:
    """cols/vals/valid are (n, s) with the stencil entries of each row in
    increasing column order."""
    counts = valid.sum(axis=1)
    row_ptr = np.zeros(n + 1, np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    if row_ptr[-1] >= 2**31:
        raise ValueError("nnz must stay below 2^31")
    return CSR(row_ptr.astype(np.int32), cols[valid].astype(np.int32), vals[valid].astype(np.float64),
               n, name)


def poisson2d(N: int, scale: float = 1.0) -> CSR:
    """2D 5-point Poisson on an N x N grid, Dirichlet boundary: 4 on the
    diagonal, -1 off it (times `scale`).  n = N^2, nnz = 5N^2 - 4N."""
    n = N * N
    i = np.arange(n)
    gx, gy = i % N, i // N
    offs = [(-N, gy > 0), (-1, gx > 0), (0, np.ones(n, bool)), (1, gx < N - 1), (N, gy < N - 1)]
    cols = np.stack([i + o for o, _ in offs], axis=1)
    valid = np.stack([m for _, m in offs], axis=1)
    vals = np.stack([np.full(n, 4.0 if o == 0 else -1.0) for o, _ in offs], axis=1) * scale
    return _from_stencil(cols, vals, valid, n, f"poisson2d_{N}")


def laplace3d(N: int, shift: float = 0.0, aniso=(1.0, 1.0, 1.0), dims=None) -> CSR:
    """3D 7-point Laplacian on an N^3 (or dims) grid, Dirichlet boundary:
    diagonal 2*(ex+ey+ez) + shift, off-diagonal -e_axis.
    For N = 128: n = 2,097,152, nnz = 14,581,760."""
    nx, ny, nz = dims if dims is not None else (N, N, N)
    n = nx * ny * nz
    i = np.arange(n, dtype=np.int64)
    gx, gy, gz = i % nx, (i // nx) % ny, i // (nx * ny)
    ex, ey, ez = aniso
    diag = 2.0 * (ex + ey + ez) + shift
    offs = [(-nx * ny, gz > 0, -ez), (-nx, gy > 0, -ey), (-1, gx > 0, -ex), (0, None, diag),
            (1, gx < nx - 1, -ex), (nx, gy < ny - 1, -ey), (nx * ny, gz < nz - 1, -ez)]
    cols = np.empty((n, 7), np.int64)
    valid = np.empty((n, 7), bool)
    vals = np.empty((n, 7), np.float64)
    for s, (o, m, v) in enumerate(offs):
        cols[:, s] = i + o
        valid[:, s] = True if m is None else m
        vals[:, s] = v
    return _from_stencil(cols, vals, valid, n, f"laplace3d_{nx}x{ny}x{nz}")


def laplace2d(nx: int, ny: int, shift: float = 0.0, aniso=(1.0, 1.0)) -> CSR:
    """2D 5-point anisotropic Laplacian: diagonal 2*(ex+ey) + shift."""
    n = nx * ny
    i = np.arange(n, dtype=np.int64)
    gx, gy = i % nx, i // nx
    ex, ey = aniso
    diag = 2.0 * (ex + ey) + shift
    offs = [(-nx, gy > 0, -ey), (-1, gx > 0, -ex), (0, None, diag), (1, gx < nx - 1, -ex),
            (nx, gy < ny - 1, -ey)]
    cols = np.stack([i + o for o, _, _ in offs], axis=1)
    valid = np.stack([np.ones(n, bool) if m is None else m for _, m, _ in offs], axis=1)
    vals = np.stack([np.full(n, v) for _, _, v in offs], axis=1)
    return _from_stencil(cols, vals, valid, n, f"laplace2d_{nx}x{ny}")


def convdiff2d(N: int, peclet: float = 10.0) -> CSR:
    """-Laplace(u) + beta . grad(u) on the unit square, h = 1/(N+1),
    beta = (peclet, peclet), first-order upwind, scaled by h^2, Dirichlet:
    centre 4 + h(bx+by), west -1 - h bx, south -1 - h by, east = north = -1.
    Nonsymmetric.  For N = 1024: nnz = 5,238,784."""
    n = N * N
    h = 1.0 / (N + 1)
    bx = by = peclet
    i = np.arange(n, dtype=np.int64)
    gx, gy = i % N, i // N
    offs = [(-N, gy > 0, -1.0 - h * by), (-1, gx > 0, -1.0 - h * bx), (0, None, 4.0 + h * (bx + by)),
            (1, gx < N - 1, -1.0), (N, gy < N - 1, -1.0)]
    cols = np.stack([i + o for o, _, _ in offs], axis=1)
    valid = np.stack([np.ones(n, bool) if m is None else m for _, m, _ in offs], axis=1)
    vals = np.stack([np.full(n, v) for _, _, v in offs], axis=1)
    return _from_stencil(cols, vals, valid, n, f"convdiff2d_{N}_pe{peclet:g}")


def _powerlaw_alpha(mean: float, lmax: int) -> float:
    L = np.arange(1, lmax + 1, dtype=np.float64)
    lo, hi = 0.5, 4.0
    for _ in range(200):
        a = 0.5 * (lo + hi)
        w = L ** (-a)
        m = (L * w).sum() / w.sum()
        if m > mean:
            lo = a
        else:
            hi = a
    return 0.5 * (lo + hi)


def powerlaw_random(n: int = 1_000_000, mean: float = 16.0, lmax: int = 2048, seed: int = 0,
                    mag_lo: float = -3.0, mag_hi: float = 3.0, n_cols: int | None = None) -> CSR:
    """Random nonsymmetric matrix: row lengths from a discrete power law
    p(L) ~ L^-alpha on [1, lmax] with alpha set (by bisection) so that the mean
    is `mean`, one row forced to length lmax; columns uniform without
    replacement, sorted; values with a random sign and magnitude
    10^U(mag_lo, mag_hi)."""
    rng = np.random.default_rng(seed)
    n_cols = n if n_cols is None else n_cols
    lmax = min(lmax, n_cols)
    alpha = _powerlaw_alpha(mean, lmax)
    L = np.arange(1, lmax + 1, dtype=np.float64)
    p = L ** (-alpha)
    cdf = np.cumsum(p / p.sum())
    lens = np.searchsorted(cdf, rng.random(n), side="right") + 1
    lens = np.minimum(lens, lmax)
    lens[rng.integers(0, n)] = lmax
    row_ptr = np.zeros(n + 1, np.int64)
    np.cumsum(lens, out=row_ptr[1:])
    nnz = int(row_ptr[-1])
    rows = np.repeat(np.arange(n, dtype=np.int64), lens)
    cols = rng.integers(0, n_cols, size=nnz, dtype=np.int64)
    # resample duplicates within a row until every row's columns are distinct
    for _ in range(100):
        key = rows * n_cols + cols
        order = np.argsort(key, kind="stable")
        key = key[order]
        cols = cols[order]
        dup = np.zeros(nnz, bool)
        dup[1:] = key[1:] == key[:-1]
        if not dup.any():
            break
        cols[dup] = rng.integers(0, n_cols, size=int(dup.sum()), dtype=np.int64)
    else:
        raise RuntimeError("could not draw distinct columns")
    sign = np.where(rng.random(nnz) < 0.5, -1.0, 1.0)
    val = sign * 10.0 ** rng.uniform(mag_lo, mag_hi, size=nnz)
    return CSR(row_ptr.astype(np.int32), cols.astype(np.int32), val, n_cols,
               f"powerlaw_{n}_mean{mean:g}")


def uniform_x(n: int, seed: int = 0) -> np.ndarray:
    """x ~ U[-1, 1], FP64."""
    return np.random.default_rng(seed).uniform(-1.0, 1.0, size=n)


def sample_rows(n_rows: int, block_rows: int, seed: int = 0) -> np.ndarray:
    """One uniformly drawn row index per block of block_rows consecutive rows
    (the last block may be shorter): the random choice of the sampled exponent
    extraction, drawn here so that every consumer sees the same rows."""
    rng = np.random.default_rng(seed)
    first = np.arange(0, n_rows, block_rows, dtype=np.int64)
    size = np.minimum(block_rows, n_rows - first)
    return first + rng.integers(0, size, dtype=np.int64)


def rhs_ones(A: CSR) -> np.ndarray:
    """b = A * ones (row sums), accumulated left to right in FP64."""
    rows = np.repeat(np.arange(A.n_rows), np.diff(A.row_ptr))
    return np.bincount(rows, weights=A.val, minlength=A.n_rows)


@dataclass
class SystemSpec:
    dim: int
    dims: tuple
    aniso: tuple
    shift: float

    @property
    def n(self) -> int:
        return int(np.prod(self.dims))

    def build(self) -> CSR:
        if self.dim == 2:
            return laplace2d(self.dims[0], self.dims[1], self.shift, self.aniso)
        return laplace3d(0, self.shift, self.aniso, dims=self.dims)


def batch_specs(count: int = 512, seed: int = 0, n_lo: float = 1e3, n_hi: float = 2.56e5) -> list:
    """SPD systems of uneven size: n log-uniform in [n_lo, n_hi]; 2D or 3D with
    probability 1/2; grid side round(n^(1/d)); anisotropy per axis U[0.01, 1];
    diagonal shift log-uniform in [1e-4, 1e-1]."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        n = float(np.exp(rng.uniform(np.log(n_lo), np.log(n_hi))))
        d = 2 if rng.random() < 0.5 else 3
        side = max(2, int(round(n ** (1.0 / d))))
        aniso = tuple(float(v) for v in rng.uniform(0.01, 1.0, size=d))
        shift = float(np.exp(rng.uniform(np.log(1e-4), np.log(1e-1))))
        out.append(SystemSpec(d, (side,) * d, aniso, shift))
    return out


def shard_specs(specs: list, rank: int, world: int) -> list:
    """The systems one of `world` replicas solves (round robin)."""
    return specs[rank::world]
