"""Seeded synthetic total-least-squares problems.

This module only builds inputs. It holds none of the solver's arithmetic and is the one
module that both the CUDA path's tests/bench and the CPU oracle's tests draw inputs from.

Problem families (all from the model problems of Sec. 4 of Oktay & Carson, arXiv 2305.19028):

* ``dense_problem`` -- the Bjorck-type matrix of Sec. 4.3, A = Y [diag(D); 0] Z^T, here with
  Y, Z single random Householder reflectors (so the SVD of A is known exactly: singular values
  D, right singular vectors the columns of Z), D log-spaced from 1 down to ``d_lo``,
  x_true ~ N(0, I) and b = A x_true + e with e ~ N(0, noise^2 I).  ``haar=True`` uses
  Haar-random orthogonal Y, Z instead (stress variant, as with the random orthogonal matrices
  of Sec. 4.3).
* ``csr_problem`` -- a sparse A with a fixed number of uniform random columns per row plus a
  unit diagonal block, N(0,1) values, each column multiplied by 10^U(-2,0).
* ``batch_problem`` -- one member of the uneven batch: n ~ U{32..512}, m = n * U{4..20},
  D log-spaced in [10^-U(1,4), 1].

Random draws use numpy ``Generator(PCG64(seed))`` in a fixed order (sizes, D range, y, z,
x_true, e) so every consumer sees identical inputs for a seed.
"""
from __future__ import annotations

import dataclasses
import numpy as np

__all__ = ["DenseProblem", "CsrProblem", "log_spaced_d", "dense_problem", "csr_problem",
           "batch_problem", "csr_to_dense", "delta_matrix_problem", "van_huffel_problem",
           "random_matrix_problem", "bjorck_problem"]


@dataclasses.dataclass
class DenseProblem:
    A: np.ndarray          # (m, n) float64, row-major (C order)
    b: np.ndarray          # (m,) float64
    x_true: np.ndarray     # (n,) float64, the noise-free solution used to build b
    D: np.ndarray | None   # (n,) singular values of A when known by construction, else None
    y: np.ndarray | None   # unit Householder vector of Y (m,), when Y is a single reflector
    z: np.ndarray | None   # unit Householder vector of Z (n,), when Z is a single reflector
    seed: int

    @property
    def m(self) -> int:
        return self.A.shape[0]

    @property
    def n(self) -> int:
        return self.A.shape[1]


@dataclasses.dataclass
class CsrProblem:
    m: int
    n: int
    row_ptr: np.ndarray    # (m+1,) int64
    col_idx: np.ndarray    # (nnz,) int32, sorted within each row, no duplicates
    val: np.ndarray        # (nnz,) float64
    b: np.ndarray          # (m,) float64
    x_true: np.ndarray     # (n,) float64
    seed: int

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])


def log_spaced_d(n: int, d_lo: float) -> np.ndarray:
    """D_i = 10^(log10(d_lo) * (i-1)/(n-1)), i = 1..n: descending from 1 to d_lo."""
    if n == 1:
        return np.ones(1)
    return 10.0 ** (np.log10(d_lo) * np.arange(n) / (n - 1))


def _reflect_rows(M: np.ndarray, y: np.ndarray) -> np.ndarray:
    # (I - 2 y y^T) M for unit y, in O(mn)
    return M - 2.0 * np.outer(y, y @ M)


def _reflect_cols(M: np.ndarray, z: np.ndarray) -> np.ndarray:
    # M (I - 2 z z^T)^T = M (I - 2 z z^T) for unit z
    return M - 2.0 * np.outer(M @ z, z)


def _haar_orthogonal(rng: np.random.Generator, k: int, cols: int) -> np.ndarray:
    G = rng.standard_normal((k, cols))
    Q, Rq = np.linalg.qr(G)
    return Q * np.sign(np.diag(Rq))


def dense_problem(m: int, n: int, d_lo: float = 1e-2, noise: float = 1e-6, seed: int = 0,
                  haar: bool = False) -> DenseProblem:
    """A = Y [diag(D); 0] Z^T, b = A x_true + e (see module docstring)."""
    if not (m >= n >= 1):
        raise ValueError("need m >= n >= 1")
    rng = np.random.Generator(np.random.PCG64(seed))
    D = log_spaced_d(n, d_lo)
    M = np.zeros((m, n))
    M[np.arange(n), np.arange(n)] = D
    if haar:
        Y1 = _haar_orthogonal(rng, m, n)        # only the first n columns of Y matter
        Z = _haar_orthogonal(rng, n, n)
        A = (Y1 * D) @ Z.T
        y = z = None
    else:
        y = rng.standard_normal(m)
        y /= np.linalg.norm(y)
        z = rng.standard_normal(n)
        z /= np.linalg.norm(z)
        A = _reflect_cols(_reflect_rows(M, y), z)
    x_true = rng.standard_normal(n)
    e = noise * rng.standard_normal(m)
    A = np.ascontiguousarray(A)
    b = A @ x_true + e
    return DenseProblem(A=A, b=b, x_true=x_true, D=D, y=y, z=z, seed=seed)


def batch_problem(i: int, noise: float = 1e-6) -> DenseProblem:
    """Member i of the uneven batch: seed 1000+i, n ~ U{32..512}, m = n*U{4..20},
    D log-spaced in [10^-U(1,4), 1]."""
    seed = 1000 + i
    rng = np.random.Generator(np.random.PCG64(seed))
    n = int(rng.integers(32, 513))
    ratio = int(rng.integers(4, 21))
    d_lo = 10.0 ** (-rng.uniform(1.0, 4.0))
    return dense_problem(n * ratio, n, d_lo=d_lo, noise=noise, seed=seed)


def selector_problem(seed: int) -> DenseProblem:
    """A problem of the selector network's training / evaluation distribution (seeds 10000.. for
    training, 100000.. held out): n ~ U{32..512}, m = n*U{4..12}, D log-spaced in
    [10^-U(1,6), 1], noise std 10^-U(3,7) (so that sigma_{n+1} / sigma'_n, which the second
    constraint of Sec. 3.1 depends on, varies over several orders of magnitude)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n = int(rng.integers(32, 513))
    ratio = int(rng.integers(4, 13))
    d_lo = 10.0 ** (-rng.uniform(1.0, 6.0))
    noise = 10.0 ** (-rng.uniform(3.0, 7.0))
    return dense_problem(n * ratio, n, d_lo=d_lo, noise=noise, seed=seed)


def selector_problem_wide(seed: int):
    """A problem of the selector configuration's wider distribution (seeds 200000.. for training,
    300000.. held out): dense or sparse with equal probability, n ~ U{64..2048},
    m = n*U{4..12}, noise std 10^-U(3,7). Dense: D log-spaced in [10^-U(1,6), 1]. Sparse (as
    csr_problem): 12 entries per row plus the unit diagonal block, column scales
    10^U(-U(1,6), 0)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    sparse = bool(rng.uniform() < 0.5)
    n = int(rng.integers(64, 2049))
    ratio = int(rng.integers(4, 13))
    lo = float(rng.uniform(1.0, 6.0))
    noise = 10.0 ** (-rng.uniform(3.0, 7.0))
    if sparse:
        return csr_problem(n * ratio, n, nnz_per_row=12, noise=noise, seed=seed, col_scale_lo=-lo)
    return dense_problem(n * ratio, n, d_lo=10.0 ** (-lo), noise=noise, seed=seed)


def csr_problem(m: int, n: int, nnz_per_row: int = 12, noise: float = 1e-3, seed: int = 0,
                col_scale_lo: float = -2.0) -> CsrProblem:
    """Sparse A: nnz_per_row distinct uniform columns per row, N(0,1) values, A[i,i] += 1 for
    i < n, every column scaled by 10^U(col_scale_lo, 0); b = A x_true + N(0, noise^2)."""
    if not (m >= n >= 1) or nnz_per_row > n:
        raise ValueError("need m >= n >= nnz_per_row >= 1")
    rng = np.random.Generator(np.random.PCG64(seed))
    scales = 10.0 ** rng.uniform(col_scale_lo, 0.0, size=n)
    # distinct columns per row: argpartition of uniform keys is O(n) per row, so sample with
    # rejection instead (nnz_per_row << n): draw, sort, resample duplicates.
    cols = rng.integers(0, n, size=(m, nnz_per_row))
    cols.sort(axis=1)
    for _ in range(64):
        dup = np.zeros(cols.shape, dtype=bool)
        dup[:, 1:] = cols[:, 1:] == cols[:, :-1]
        rows = np.nonzero(dup.any(axis=1))[0]
        if rows.size == 0:
            break
        fresh = rng.integers(0, n, size=(rows.size, nnz_per_row))
        cols[rows] = np.where(dup[rows], fresh, cols[rows])
        cols[rows] = np.sort(cols[rows], axis=1)
    else:
        raise RuntimeError("could not draw distinct columns")
    vals = rng.standard_normal((m, nnz_per_row))
    # unit diagonal block: A[i, i] += 1 for i < n (merged with an existing entry if present)
    diag_rows = np.arange(n)
    has = cols[diag_rows] == diag_rows[:, None]
    hit = has.any(axis=1)
    vals[diag_rows[hit], np.argmax(has[hit], axis=1)] += 1.0
    miss = diag_rows[~hit]
    row_cols = [cols[i] for i in range(m)]
    row_vals = [vals[i] for i in range(m)]
    for i in miss:
        c = np.append(cols[i], i)
        v = np.append(vals[i], 1.0)
        o = np.argsort(c, kind="stable")
        row_cols[i] = c[o]
        row_vals[i] = v[o]
    counts = np.fromiter((len(c) for c in row_cols), dtype=np.int64, count=m)
    row_ptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    col_idx = np.concatenate(row_cols).astype(np.int32)
    val = np.concatenate(row_vals) * scales[col_idx]
    x_true = rng.standard_normal(n)
    e = noise * rng.standard_normal(m)
    # b = A x_true + e, row by row from the CSR arrays
    prod = val * x_true[col_idx]
    b = np.add.reduceat(prod, row_ptr[:-1]) + e
    return CsrProblem(m=m, n=n, row_ptr=row_ptr, col_idx=col_idx, val=val, b=b,
                      x_true=x_true, seed=seed)


def csr_to_dense(p: CsrProblem) -> np.ndarray:
    A = np.zeros((p.m, p.n))
    rows = np.repeat(np.arange(p.m), np.diff(p.row_ptr))
    np.add.at(A, (rows, p.col_idx), p.val)
    return A


def delta_matrix_problem(delta: float = 1e-2, eps: float = 1e-1, seed: int = 1) -> DenseProblem:
    """The 9x4 'delta matrix' of Sec. 4.2 with b = ones, perturbed as (A + E) x = b + e with
    E = eps * Ebar .* A and e = eps * ebar .* b, Ebar, ebar ~ U(-1, 1) elementwise."""
    A = np.zeros((9, 4))
    A[0, 0] = delta
    A[2, 1] = delta
    A[6, 2] = 1.0
    A[8, 3] = 1.0
    b = np.ones(9)
    rng = np.random.Generator(np.random.PCG64(seed))
    Ebar = rng.uniform(-1.0, 1.0, size=A.shape)
    ebar = rng.uniform(-1.0, 1.0, size=9)
    return DenseProblem(A=A + eps * Ebar * A, b=b + eps * ebar * b, x_true=np.ones(4),
                        D=None, y=None, z=None, seed=seed)


def van_huffel_problem(n: int = 100, eps: float = 1e-6, seed: int = 1) -> DenseProblem:
    """The n x (n-2) matrix of Sec. 4.5: n-1 on the diagonal of the top (n-2)x(n-2) block, -1
    everywhere else; b = (-1, ..., -1, n-1, -1); perturbed by eps * U(0,1) entries."""
    A = -np.ones((n, n - 2))
    A[np.arange(n - 2), np.arange(n - 2)] = n - 1.0
    b = -np.ones(n)
    b[n - 2] = n - 1.0
    rng = np.random.Generator(np.random.PCG64(seed))
    E = eps * rng.uniform(0.0, 1.0, size=A.shape)
    e = eps * rng.uniform(0.0, 1.0, size=n)
    return DenseProblem(A=np.ascontiguousarray(A + E), b=b + e, x_true=np.zeros(n - 2),
                        D=None, y=None, z=None, seed=seed)


def random_matrix_problem(m: int = 100, n: int = 60, eps: float = 1e-6, seed: int = 0) -> DenseProblem:
    """Sec. 4.1: A ~ U(0,1)^{m x n}, b = ones, perturbed as (A + E) x = b + e with
    E = eps * U(0,1)^{m x n}, e = eps * U(0,1)^m."""
    rng = np.random.Generator(np.random.PCG64(seed))
    A = rng.uniform(0.0, 1.0, size=(m, n))
    E = eps * rng.uniform(0.0, 1.0, size=(m, n))
    e = eps * rng.uniform(0.0, 1.0, size=m)
    return DenseProblem(A=np.ascontiguousarray(A + E), b=np.ones(m) + e, x_true=np.zeros(n),
                        D=None, y=None, z=None, seed=seed)


def bjorck_problem(m: int = 30, n: int = 15, eps: float = 0.05, seed: int = 1) -> DenseProblem:
    """Sec. 4.3: A = Y [D; 0] Z^T with Haar-random orthogonal Y, Z, D = diag(1, 2^-1, ...,
    2^-(n-1)), b = A x with x = (1, 1/2, ..., 1/n), perturbed by E = eps * U(0,1)^{m x n},
    e = eps * U(0,1)^m."""
    rng = np.random.Generator(np.random.PCG64(seed))
    D = 2.0 ** -np.arange(n)
    Y1 = _haar_orthogonal(rng, m, n)
    Z = _haar_orthogonal(rng, n, n)
    A = (Y1 * D) @ Z.T
    x = 1.0 / np.arange(1, n + 1)
    b = A @ x
    E = eps * rng.uniform(0.0, 1.0, size=(m, n))
    e = eps * rng.uniform(0.0, 1.0, size=m)
    return DenseProblem(A=np.ascontiguousarray(A + E), b=b + e, x_true=x, D=None, y=None,
                        z=None, seed=seed)
