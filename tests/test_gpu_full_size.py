"""Parity at the benchmark sizes, in the launch configuration the benchmark times: the dense
16384 x 2048 problem (u_f FP16, u FP32, u_r FP64, tolerance 1e-16, at most 12 RQI steps) against
the FP64 oracle on the whole problem, and the packed batch of 512 uneven problems against the
oracle on a sample of its members (the oracle on all 512 takes minutes on the host)."""
from __future__ import annotations

import numpy as np
import pytest

import oracle.rqi_pcgtls as O
from paper_2305_19028_gb300 import synth, tls

pytestmark = pytest.mark.gpu

SIGMA_TOL, X_TOL = 1e-10, 1e-8


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    tls.load()


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def test_dense_16384x2048_matches_oracle():
    p = synth.dense_problem(16384, 2048, d_lo=1e-3, noise=1e-4, seed=0)
    ctx = tls.tls_create_dense(p.A, p.b)
    try:
        tls.tls_factor(ctx, "fp16", tls.tls_default_options(u="fp32"))
        # the benchmark's path: the inner solves in one launch each, every reduction in a fixed
        # order, so a second solve on the same factor repeats the first bit for bit
        x, sigma, info = tls.tls_solve(ctx, tol=1e-16, max_rqi=12)
        x2, sigma2, info2 = tls.tls_solve(ctx, tol=1e-16, max_rqi=12)
        # the multi-launch path (fixed-order reductions) repeats itself bit for bit
        tls.tls_set_pcg_fused(ctx, 2)
        x3, sigma3, info3 = tls.tls_solve(ctx, tol=1e-16, max_rqi=12)
        x4, sigma4, _ = tls.tls_solve(ctx, tol=1e-16, max_rqi=12)
    finally:
        tls.tls_destroy(ctx)
    xo, so, _ = O.rqi_pcgtls(p.A, p.b, tol=0.0, max_rqi=12)
    for xx, ss, ii in ((x, sigma, info), (x2, sigma2, info2), (x3, sigma3, info3)):
        assert abs(ss - so) <= SIGMA_TOL * so, (ss, so, ii)
        assert _rel(xx, xo) <= X_TOL, ii
    assert sigma2 == sigma and np.array_equal(x, x2)
    assert sigma4 == sigma3 and np.array_equal(x3, x4)
    assert info["u_f_used"] == tls.TLS_FP16 and info["pass_variant"][0] >= 0


def test_batch_512_sampled_members_match_oracle():
    probs = [synth.batch_problem(i) for i in range(512)]
    with tls.Batch([(p.A, p.b) for p in probs]) as bt:
        bt.factor("fp16", u="fp32")
        xs, sig, infos, per = bt.solve(tol=1e-16, max_rqi=12)
    assert per == [0] * 512
    sizes = [p.A.size for p in probs]
    sample = sorted({0, 1, 97, 255, 384, 511, int(np.argmax(sizes)), int(np.argmin(sizes))})
    for i in sample:
        p = probs[i]
        xo, so, _ = O.rqi_pcgtls(p.A, p.b, tol=0.0, max_rqi=12)
        assert abs(sig[i] - so) <= SIGMA_TOL * so, (i, p.A.shape, sig[i], so, infos[i])
        assert _rel(xs[i], xo) <= X_TOL, (i, p.A.shape, infos[i])
    # every member: sigma is the smallest singular value's estimate, so it is positive and
    # bounded by ||b|| / sqrt(1 + ||x||^2) (the TLS objective at x is at most that of x = 0)
    for i, p in enumerate(probs):
        assert 0.0 < sig[i] <= np.linalg.norm(p.b) * (1 + 1e-12), i
