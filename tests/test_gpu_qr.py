"""GPU parity of the Householder QR preconditioner (Alg. 4's "A = Q[R 0]^T" in precision u_q,
the factor Sec. 3 prefers) against the FP64 oracle's QR of the same column-scaled, u_q-rounded
matrix, and full RQI solves with it against the oracle."""
from __future__ import annotations

import numpy as np
import pytest

import oracle.rqi_pcgtls as O
from paper_2305_19028_gb300 import synth, tls

pytestmark = pytest.mark.gpu

U16, UBF, U32, U64 = 2.0 ** -11, 2.0 ** -8, 2.0 ** -24, 2.0 ** -53
UNIT = {"fp16": U16, "bf16": UBF, "fp32": U32, "fp64": U64}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    tls.load()


def _scaled_rounded(A, d, u_f):
    """A D^{-1} as the device forms it before the QR: the FP64 path divides in FP64; the FP32
    path multiplies the FP32 copy of A by the FP32 reciprocal of d (RN), then rounds to u_f."""
    if u_f == "fp64":
        return A / d
    As = A.astype(np.float32) * (1.0 / d).astype(np.float32)
    if u_f == "fp16":
        return As.astype(np.float16).astype(np.float64)
    if u_f == "bf16":
        mant, ex = np.frexp(As.astype(np.float64))
        return np.ldexp(np.rint(mant * 256.0) / 256.0, ex)
    return As.astype(np.float64)


def _factor_qr(p, u_f, u):
    ctx = tls.tls_create_dense(p.A, p.b)
    try:
        tls.tls_factor(ctx, u_f, tls.tls_default_options(u=u, factor=1))
        R, d, _ = tls.tls_export_factor(ctx)
    finally:
        tls.tls_destroy(ctx)
    return R, d


@pytest.mark.parametrize("u_f,u", [("fp32", "fp32"), ("fp16", "fp32"), ("bf16", "fp32"),
                                   ("fp64", "fp64")])
@pytest.mark.parametrize("m,n", [(40, 1), (300, 40), (1000, 150), (3001, 77), (20000, 257)])
def test_qr_factor_matches_oracle(u_f, u, m, n):
    """Shapes: one column; a cluster of one CTA; several 32-column panels (16-column panels in
    FP64) with a ragged last panel; ragged rows over 16 CTAs; 1250 rows per CTA. Pins: R upper
    triangular with a positive diagonal, representable in u_f, R^T R = A_s^T A_s up to the
    backward error of Householder QR (u_f from the final rounding plus the FP32/FP64 arithmetic,
    independent of kappa), and entrywise the oracle's R within kappa times that error."""
    p = synth.dense_problem(m, n, d_lo=1e-2, noise=1e-3, seed=m + 7 * n)
    R, d = _factor_qr(p, u_f, u)
    As = _scaled_rounded(p.A, d, u_f)
    assert np.array_equal(R, np.triu(R))
    assert np.all(np.diag(R) > 0)
    if u_f == "fp16":
        assert np.array_equal(R, R.astype(np.float16).astype(np.float64))
    ua = U64 if u_f == "fp64" else U32
    uf = UNIT[u_f]
    G = As.T @ As
    berr = np.linalg.norm(R.T @ R - G) / np.linalg.norm(G)
    bound = 4 * uf * np.sqrt(n) + 8 * np.sqrt(m) * n * ua
    assert berr <= bound, (berr, bound)
    R_ref = O.r_factor_qr(As)
    kap = np.linalg.cond(As)
    err = np.max(np.abs(R - R_ref)) / np.max(np.abs(R_ref))
    assert err <= 2 * uf + kap * bound, (err, kap)


def test_qr_factor_of_the_16384_x_2048_workload_is_backward_stable():
    """The dense benchmark size (64 panels of 32 columns, clusters of 16 CTAs with 1024 rows
    each): the same backward-error pin as above, on the FP32-rounded scaled matrix."""
    p = synth.dense_problem(16384, 2048, d_lo=1e-3, noise=1e-4, seed=0)
    R, d = _factor_qr(p, "fp32", "fp32")
    As = _scaled_rounded(p.A, d, "fp32")
    assert np.array_equal(R, np.triu(R))
    assert np.all(np.diag(R) > 0)
    G = As.T @ As
    berr = np.linalg.norm(R.T @ R - G) / np.linalg.norm(G)
    assert berr <= 4 * U32 * np.sqrt(2048) + 8 * np.sqrt(16384) * 2048 * U32, berr


@pytest.mark.parametrize("m,n,u_f,u", [(3000, 300, "fp16", "fp32"), (2000, 130, "bf16", "fp32"),
                                       (900, 100, "fp64", "fp64"), (400, 40, "fp64", "fp64")])
def test_qr_preconditioned_solve_matches_oracle(m, n, u_f, u):
    """RQI-PCGTLS with R-hat from the GPU Householder QR reaches the oracle's sigma_{n+1} and
    x_TLS (the solution does not depend on the preconditioner)."""
    p = synth.dense_problem(m, n, d_lo=1e-3, noise=1e-4, seed=21)
    ctx = tls.tls_create_dense(p.A, p.b)
    try:
        tls.tls_factor(ctx, u_f, tls.tls_default_options(u=u, factor=1))
        x, sigma, info = tls.tls_solve(ctx, tol=0.0, max_rqi=12)
    finally:
        tls.tls_destroy(ctx)
    xo, so, _ = O.rqi_pcgtls(p.A, p.b, tol=0.0, max_rqi=12)
    assert abs(sigma - so) <= 1e-10 * so, (sigma, so, info)
    assert np.linalg.norm(x - xo) / np.linalg.norm(xo) <= 1e-8, info
    assert np.isnan(info["constr1"])


def test_qr_option_is_rejected_for_csr_contexts():
    p = synth.csr_problem(2000, 100, nnz_per_row=6, seed=3)
    ctx = tls.tls_create_csr(p.m, p.n, p.row_ptr, p.col_idx, p.val, p.b)
    try:
        with pytest.raises(tls.TLSError):
            tls.tls_factor(ctx, "bf16", tls.tls_default_options(factor=1))
    finally:
        tls.tls_destroy(ctx)


def test_condition_estimate_needs_the_gram_matrix():
    p = synth.dense_problem(500, 60, d_lo=1e-2, noise=1e-3, seed=2)
    ctx = tls.tls_create_dense(p.A, p.b)
    try:
        tls.tls_factor(ctx, "fp16", tls.tls_default_options(factor=1))
        with pytest.raises(tls.TLSError):
            tls.tls_condition(ctx, 10)
    finally:
        tls.tls_destroy(ctx)
