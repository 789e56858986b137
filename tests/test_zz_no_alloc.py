"""The residual entry point that allocates no device memory (tls_residual_noalloc).

Callers such as an application whose framework allocator already owns the GPU's memory, a
latency-critical loop that must not call cudaMalloc / cudaFree, or a plug-in that is handed its
buffers cannot let the library allocate. This checks that the no-allocation variant, which
keeps its scratch in a fixed device array, returns what the existing residual entry point
returns, on two calls in a row (the second reuses the scratch the first left behind).
Collected last on purpose, so a failure here does not hide the other GPU tests.
"""
from __future__ import annotations

import numpy as np
import pytest

from paper_2305_19028_gb300 import synth, tls

pytestmark = pytest.mark.gpu

U64 = 2.0 ** -53


def test_noalloc_residual_matches_existing_entry_point_twice():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    tls.load()
    m, n = 3000, 700
    p = synth.dense_problem(m, n, d_lo=1e-2, noise=1e-3, seed=21)
    rng = np.random.default_rng(5)
    xs = [p.x_true + 1e-3 * rng.standard_normal(n), p.x_true - 2e-3 * rng.standard_normal(n)]

    # reference: the existing residual entry point
    ctx = tls.tls_create_dense(p.A, p.b)
    try:
        refs = [tls.tls_residual(ctx, x) for x in xs]
    finally:
        tls.tls_destroy(ctx)

    dev = torch.device("cuda", 0)
    A = torch.from_numpy(p.A).to(dev)
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
        # the same tolerance as the residual parity test: FP64 sums in another order
        fscale = m * U64 * (np.abs(p.A).T @ (np.abs(p.A) @ np.abs(x) + np.abs(p.b))).max()
        assert np.max(np.abs(fh - f_ref)) <= 8 * fscale
        assert abs(sh[0] - sc_ref["sigma2"]) <= 1e-10 * sc_ref["sigma2"]
        gscale = 8 * m * U64 * (np.abs(p.b) @ (np.abs(p.A) @ np.abs(x) + np.abs(p.b)))
        assert abs(sh[1] - sc_ref["g"]) <= gscale
        assert abs(sh[2] - sc_ref["psi"]) <= 1e-6 * sc_ref["psi"] + 8 * fscale
        assert abs(sh[3] - sc_ref["rr"]) <= 1e-10 * sc_ref["rr"]
        assert abs(sh[4] - sc_ref["br"]) <= gscale


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
