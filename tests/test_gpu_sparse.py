"""GPU parity of the CSR path (A stored by rows and by columns on the device) against the FP64
oracle on the dense expansion of the same seeded problems, and at the full 200000 x 4000 size
against the oracle run on the CSR matrix itself, plus the TLS invariants there."""
from __future__ import annotations

import numpy as np
import pytest
import scipy.linalg as sla

import oracle.rqi_pcgtls as O
from paper_2305_19028_gb300 import synth, tls

pytestmark = pytest.mark.gpu

U32, U64 = 2.0 ** -24, 2.0 ** -53


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    tls.load()


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def _ctx(p, u_f="bf16", u="fp32", **opt):
    ctx = tls.tls_create_csr(p.m, p.n, p.row_ptr, p.col_idx, p.val, p.b)
    tls.tls_factor(ctx, u_f, tls.tls_default_options(u=u, **opt))
    return ctx


@pytest.mark.parametrize("m,n,u_f,u", [(3000, 300, "bf16", "fp32"), (2000, 257, "fp16", "fp32"),
                                       (1500, 200, "fp64", "fp64"), (640, 64, "fp32", "fp32")])
def test_sparse_solve_matches_oracle(m, n, u_f, u):
    p = synth.csr_problem(m, n, nnz_per_row=12, noise=1e-3, seed=2)
    A = synth.csr_to_dense(p)
    ctx = _ctx(p, u_f, u)
    try:
        x, sigma, info = tls.tls_solve(ctx, tol=0.0, max_rqi=12)
    finally:
        tls.tls_destroy(ctx)
    xo, so, _ = O.rqi_pcgtls(A, p.b, tol=0.0, max_rqi=12)
    assert abs(sigma - so) <= 1e-10 * so, (sigma, so, info)
    assert _rel(x, xo) <= 1e-8, info


def test_sparse_residual_block_matches_oracle():
    p = synth.csr_problem(2500, 300, nnz_per_row=12, noise=1e-3, seed=5)
    A = synth.csr_to_dense(p)
    x = p.x_true + 1e-3 * np.random.default_rng(1).standard_normal(p.n)
    ctx = tls.tls_create_csr(p.m, p.n, p.row_ptr, p.col_idx, p.val, p.b)
    try:
        f, sc = tls.tls_residual(ctx, x)
    finally:
        tls.tls_destroy(ctx)
    r, s2, fo, go, psio = O.residual_block(A, p.b, x)
    fscale = p.m * U64 * (np.abs(A).T @ (np.abs(A) @ np.abs(x) + np.abs(p.b))).max()
    assert np.max(np.abs(f - fo)) <= 8 * fscale
    assert abs(sc["sigma2"] - s2) <= 1e-10 * s2
    assert abs(sc["psi"] - psio) <= 1e-6 * psio + 8 * fscale


def test_sparse_column_index_with_long_and_empty_rows():
    """The device-built column index on rows of 0 to 150 entries (several 32-entry chunks per
    row; empty rows): the A^T products of the FP64 residual block and the column norms match
    the dense expansion."""
    rng = np.random.default_rng(11)
    m, n = 3000, 150
    lens = rng.integers(0, 13, size=m)
    lens[rng.choice(m, 40, replace=False)] = rng.integers(33, n + 1, size=40)
    lens[:n] = np.maximum(lens[:n], 1)
    rows = [np.sort(rng.choice(n, k, replace=False)) for k in lens]
    for i in range(n):                        # every column has an entry (diagonal)
        if i not in rows[i]:
            rows[i] = np.sort(np.append(rows[i][1:], i))
    rp = np.zeros(m + 1, dtype=np.int64)
    np.cumsum([len(r) for r in rows], out=rp[1:])
    ci = np.concatenate(rows).astype(np.int32)
    va = rng.standard_normal(ci.size)
    A = np.zeros((m, n))
    for i in range(m):
        A[i, rows[i]] = va[rp[i]:rp[i + 1]]
    b = A @ rng.standard_normal(n) + 1e-3 * rng.standard_normal(m)
    x = rng.standard_normal(n)
    ctx = tls.tls_create_csr(m, n, rp, ci, va, b)
    try:
        f, sc = tls.tls_residual(ctx, x)
        tls.tls_factor(ctx, "fp64", tls.tls_default_options(u="fp64"))
        _, d, _ = tls.tls_export_factor(ctx)
    finally:
        tls.tls_destroy(ctx)
    r, s2, fo, go, psio = O.residual_block(A, b, x)
    fscale = m * U64 * (np.abs(A).T @ (np.abs(A) @ np.abs(x) + np.abs(b))).max()
    assert np.max(np.abs(f - fo)) <= 8 * fscale
    d_ref = np.linalg.norm(A, axis=0)
    assert np.max(np.abs(d - d_ref) / d_ref) <= m * U64


@pytest.mark.parametrize("u_f", ["bf16", "fp16"])
def test_sparse_gram_matches_definition(u_f):
    p = synth.csr_problem(2000, 150, nnz_per_row=12, noise=1e-3, seed=7)
    A = synth.csr_to_dense(p)
    ctx = _ctx(p, u_f, "fp32")
    try:
        R, d, H = tls.tls_export_factor(ctx)
    finally:
        tls.tls_destroy(ctx)
    d_ref = np.linalg.norm(A, axis=0)
    assert np.max(np.abs(d - d_ref) / d_ref) <= p.m * U32
    As = A.astype(np.float32) * (1.0 / d).astype(np.float32)
    if u_f == "fp16":
        As = As.astype(np.float16).astype(np.float64)
    else:
        mant, ex = np.frexp(As.astype(np.float64))
        As = np.ldexp(np.rint(mant * 256.0) / 256.0, ex)
    bound = p.m * U32 * (np.abs(As).T @ np.abs(As))
    assert np.all(np.abs(H - As.T @ As) <= bound)
    assert np.allclose(H, H.T, rtol=0, atol=0)


def test_sparse_full_size_matches_oracle_and_invariants():
    # the 200000 x 4000 CSR workload (12 nnz per row plus a unit diagonal block, column scales
    # 10^U(-2,0), noise 1e-3) with u_f = BF16, in the launch configuration the benchmark times:
    # against the FP64 oracle on the same CSR matrix (its Cholesky factor of A^T A and the
    # normal-equation LS start; only products with A and A^T), sigma rel <= 1e-10 and
    # x rel <= 1e-8; then the TLS conditions at the returned (x, sigma) with exact sparse
    # products on the host: f = -A^T r - sigma^2 x = 0 and g = -b^T r + sigma^2 = 0 (Eq. (2)),
    # and the Rayleigh-quotient identity of Alg. 2
    sp = pytest.importorskip("scipy.sparse")
    p = synth.csr_problem(200000, 4000, nnz_per_row=12, noise=1e-3, seed=0)
    ctx = _ctx(p, "bf16", "fp32")
    try:
        x, sigma, info = tls.tls_solve(ctx, tol=1e-16, max_rqi=12)
    finally:
        tls.tls_destroy(ctx)
    A = sp.csr_matrix((p.val, p.col_idx, p.row_ptr), shape=(p.m, p.n))
    R = O.r_factor_cholesky(A)
    x0 = sla.solve_triangular(R, sla.solve_triangular(R, A.T @ p.b, trans="T"))
    xo, so, _ = O.rqi_pcgtls(A, p.b, R=R, x0=x0, tol=0.0, max_rqi=12)
    assert abs(sigma - so) <= 1e-10 * so, (sigma, so, info)
    assert np.linalg.norm(x - xo) <= 1e-8 * np.linalg.norm(xo), info
    r = p.b - A @ x
    s2 = sigma * sigma
    nA = np.sqrt((p.val ** 2).sum())
    f = -(A.T @ r) - s2 * x
    assert np.linalg.norm(f) / (nA ** 2 * np.linalg.norm(x) + nA * np.linalg.norm(p.b)) < 1e-13
    assert abs(-(p.b @ r) + s2) / (p.b @ p.b) < 1e-13
    assert abs((r @ r) / (1 + x @ x) - s2) <= 1e-12 * s2
    assert info["stop_reason"] in (tls.STOP_PSI_UP, tls.STOP_TOL)
