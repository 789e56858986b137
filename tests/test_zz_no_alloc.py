"""The residual entry point that allocates no device memory (tls_residual_noalloc).

Callers such as an application whose framework allocator already owns the GPU's memory, a
latency-critical loop that must not call cudaMalloc / cudaFree, or a plug-in that is handed its
buffers cannot let the library allocate. This checks that the no-allocation variant, which
keeps its scratch in a fixed device array, returns what the existing residual entry point
returns, and what the FP64 oracle's residual block (Alg. 2, Eq. (2), Eq. (4)) returns, on two
calls in a row (the second reuses the scratch the first left behind). The cases cover a padded
leading dimension, few rows (some CTAs of the pass get no rows) and n at the entry point's
limit (every per-thread column slot in use).
Collected last on purpose, so a failure here does not hide the other GPU tests.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle.rqi_pcgtls as O
from paper_2305_19028_gb300 import synth, tls

pytestmark = pytest.mark.gpu

U64 = 2.0 ** -53

CASES = [
    # (m, n, lda)
    (3000, 700, 700),
    (10, 7, 8),          # 3 CTAs of 4 rows, padded rows
    (257, 200, 256),     # padded lda, ragged last CTA
    (4200, 4096, 4096),  # n at TLS_NOALLOC_MAX_N
    (4097, 4096, 4104),  # n at the limit with a padded lda
]


def _tols(A, b, x):
    m = A.shape[0]
    fscale = m * U64 * (np.abs(A).T @ (np.abs(A) @ np.abs(x) + np.abs(b))).max()
    gscale = 8 * m * U64 * (np.abs(b) @ (np.abs(A) @ np.abs(x) + np.abs(b)))
    return fscale, gscale


def _check(fh, sh, f_ref, s2, g, psi, rr, br, fscale, gscale):
    # FP64 sums in another order (the same bounds as the residual parity test)
    assert np.max(np.abs(fh - f_ref)) <= 8 * fscale
    assert abs(sh[0] - s2) <= 1e-10 * s2
    assert abs(sh[1] - g) <= gscale
    assert abs(sh[2] - psi) <= 1e-6 * psi + 8 * fscale
    assert abs(sh[3] - rr) <= 1e-10 * rr
    assert abs(sh[4] - br) <= gscale


@pytest.mark.parametrize("m,n,lda", CASES)
def test_noalloc_residual_matches_existing_entry_point_and_oracle_twice(m, n, lda):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    tls.load()
    p = synth.dense_problem(m, n, d_lo=1e-2, noise=1e-3, seed=21 + n)
    rng = np.random.default_rng(5)
    xs = [p.x_true + 1e-3 * rng.standard_normal(n), p.x_true - 2e-3 * rng.standard_normal(n)]

    # references: the existing residual entry point and the FP64 oracle
    ctx = tls.tls_create_dense(p.A, p.b)
    try:
        refs = [tls.tls_residual(ctx, x) for x in xs]
    finally:
        tls.tls_destroy(ctx)

    dev = torch.device("cuda", 0)
    Ap = np.zeros((m, lda))
    Ap[:, :n] = p.A
    Ap[:, n:] = np.nan               # padding must never be read
    A = torch.from_numpy(Ap).to(dev)[:, :n]
    assert A.stride() == (lda, 1)
    b = torch.from_numpy(p.b).to(dev)
    f = torch.empty(n, dtype=torch.float64, device=dev)
    scal = torch.empty(5, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()
    for x, (f_ref, sc_ref) in zip(xs, refs):
        xd = torch.from_numpy(x).to(dev)
        f.fill_(float("nan"))
        scal.fill_(float("nan"))
        tls.tls_residual_noalloc(A, b, xd, f, scal, stream=stream.cuda_stream)
        stream.synchronize()
        fh = f.cpu().numpy()
        sh = scal.cpu().numpy()
        fscale, gscale = _tols(p.A, p.b, x)
        _check(fh, sh, f_ref, sc_ref["sigma2"], sc_ref["g"], sc_ref["psi"], sc_ref["rr"],
               sc_ref["br"], fscale, gscale)
        r, s2, fo, go, psio = O.residual_block(p.A, p.b, x)
        _check(fh, sh, fo, s2, go, psio, float(r @ r), float(p.b @ r), fscale, gscale)


def test_noalloc_rejects_n_above_its_limit():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dev = torch.device("cuda", 0)
    n = 4097
    A = torch.zeros((n, n), dtype=torch.float64, device=dev)
    v = torch.zeros(n, dtype=torch.float64, device=dev)
    scal = torch.zeros(5, dtype=torch.float64, device=dev)
    with pytest.raises(tls.TLSError) as e:
        tls.tls_residual_noalloc(A, v, v, v, scal)
    assert e.value.status == 1


def test_noalloc_binding_rejects_mismatched_tensors():
    # wrong dtype, a transposed A and short vectors are refused before any kernel runs
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dev = torch.device("cuda", 0)
    m, n = 64, 16
    A = torch.zeros((m, n), dtype=torch.float64, device=dev)
    b = torch.zeros(m, dtype=torch.float64, device=dev)
    x = torch.zeros(n, dtype=torch.float64, device=dev)
    f = torch.zeros(n, dtype=torch.float64, device=dev)
    scal = torch.zeros(5, dtype=torch.float64, device=dev)
    bad_calls = [
        (A.float(), b, x, f, scal),
        (torch.zeros((n, m), dtype=torch.float64, device=dev).t(), b, x, f, scal),
        (A, b[:-1], x, f, scal),
        (A, b, x[:-1], f, scal),
        (A, b, x, f[:-1], scal),
        (A, b, x, f, scal[:4]),
    ]
    for args in bad_calls:
        with pytest.raises(tls.TLSError) as e:
            tls.tls_residual_noalloc(*args)
        assert e.value.status == 1
