"""The seeded input recipes (the module both the oracle and the GPU path draw from) against
their stated definitions: shapes, ranges, structure and determinism. No method arithmetic."""
from __future__ import annotations

import numpy as np

from paper_2305_19028_gb300 import synth


def test_dense_problems_are_deterministic_per_seed():
    a = synth.dense_problem(300, 30, d_lo=1e-3, noise=1e-4, seed=5)
    b = synth.dense_problem(300, 30, d_lo=1e-3, noise=1e-4, seed=5)
    c = synth.dense_problem(300, 30, d_lo=1e-3, noise=1e-4, seed=6)
    assert np.array_equal(a.A, b.A) and np.array_equal(a.b, b.b)
    assert not np.array_equal(a.A, c.A)
    # D log-spaced from 1 down to d_lo; b = A x_true + e with e of the stated size
    assert np.allclose(a.D, np.logspace(0.0, -3.0, 30), rtol=1e-12)
    e = a.b - a.A @ a.x_true
    assert 0.5e-4 < np.std(e) < 2e-4


def test_batch_members_follow_the_uneven_recipe():
    # member i: seed 1000 + i, n ~ U{32..512}, m = n * U{4..20}, D in [10^-U(1,4), 1]
    ns, ratios = [], []
    for i in range(64):
        p = synth.batch_problem(i)
        m, n = p.A.shape
        assert 32 <= n <= 512 and m % n == 0 and 4 <= m // n <= 20
        assert p.seed == 1000 + i
        assert np.isclose(p.D[0], 1.0) and 1e-4 * (1 - 1e-12) <= p.D[-1] <= 1e-1 * (1 + 1e-12)
        ns.append(n)
        ratios.append(m // n)
    # uneven: the sizes spread over the range
    assert max(ns) - min(ns) > 240 and max(ratios) - min(ratios) >= 10


def test_selector_problems_follow_their_recipe():
    for seed in range(10000, 10032):
        p = synth.selector_problem(seed)
        m, n = p.A.shape
        assert 32 <= n <= 512 and m % n == 0 and 4 <= m // n <= 12
        assert 1e-6 * (1 - 1e-12) <= p.D[-1] <= 1e-1 * (1 + 1e-12)


def test_csr_problem_structure():
    # nnz_per_row distinct columns per row, a unit diagonal added to the first n rows (merged
    # when the column is already drawn), column scales in [10^-2, 1], b = A x_true + e
    m, n = 3000, 200
    p = synth.csr_problem(m, n, nnz_per_row=12, noise=1e-3, seed=4)
    assert p.row_ptr[0] == 0 and p.row_ptr[-1] == p.col_idx.size == p.val.size
    counts = np.diff(p.row_ptr)
    assert np.all(counts[n:] == 12) and np.all((counts[:n] == 12) | (counts[:n] == 13))
    for i in range(m):
        c = p.col_idx[p.row_ptr[i]:p.row_ptr[i + 1]]
        assert np.all(np.diff(c) > 0) and c[0] >= 0 and c[-1] < n
        if i < n:
            assert i in c
    A = synth.csr_to_dense(p)
    e = p.b - A @ p.x_true
    assert 0.5e-3 < np.std(e) < 2e-3
    # each column is its N(0,1) values (plus the unit diagonal) times one scale in [1e-2, 1]
    colmax = np.abs(A).max(axis=0)
    assert np.all(colmax > 0) and np.all(colmax < 10.0)
    q = synth.csr_problem(m, n, nnz_per_row=12, noise=1e-3, seed=4)
    assert np.array_equal(p.col_idx, q.col_idx) and np.array_equal(p.val, q.val)
