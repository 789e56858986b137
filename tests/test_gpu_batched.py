"""Batched solves: independent problems of uneven sizes driven concurrently (each context on
its own stream), every result compared with the FP64 oracle run on the same seeded problem."""
from __future__ import annotations

import numpy as np
import pytest

import oracle.rqi_pcgtls as O
from paper_2305_19028_gb300 import synth, tls

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    tls.load()


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def test_concurrent_batch_matches_oracle():
    probs = [synth.batch_problem(i) for i in range(6)]
    ctxs = [tls.tls_create_dense(p.A, p.b) for p in probs]
    try:
        opt = tls.tls_default_options(u="fp32")
        per = tls.tls_factor_batched(ctxs, "fp16", opt)
        assert per == [0] * len(ctxs)
        xs, sig, infos, per, st = tls.tls_solve_batched(ctxs, tol=0.0, max_rqi=12)
        assert st == 0 and per == [0] * len(ctxs)
        for p, x, s, info in zip(probs, xs, sig, infos):
            xo, so, _ = O.rqi_pcgtls(p.A, p.b, tol=0.0, max_rqi=12)
            assert abs(s - so) <= 1e-10 * so, (p.A.shape, s, so, info)
            assert _rel(x, xo) <= 1e-8, (p.A.shape, info)
            # an FP16 factor of a problem with kappa(A D^-1)^2 u_f >> 1 is outside the Cholesky
            # constraint of Sec. 3.1; the solve falls back to a higher-precision factor
            assert info["fallbacks"] == 0 or info["u_f_used"] >= tls.PREC["fp32"]
    finally:
        for c in ctxs:
            tls.tls_destroy(c)


def test_batched_reports_per_problem_status():
    good = synth.dense_problem(120, 12, seed=3)
    ctxs = [tls.tls_create_dense(good.A, good.b), tls.tls_create_dense(good.A, good.b)]
    try:
        tls.tls_factor(ctxs[0], "fp32", tls.tls_default_options(u="fp32"))
        # the second context is never factored: a state error for it alone
        xs, sig, infos, per, st = tls.tls_solve_batched(ctxs, tol=0.0, max_rqi=8)
        assert per[0] == 0 and per[1] == tls.STATUS.index("TLS_ERR_STATE")
        assert st == tls.STATUS.index("TLS_ERR_STATE")
        xo, so, _ = O.rqi_pcgtls(good.A, good.b, tol=0.0, max_rqi=8)
        assert abs(sig[0] - so) <= 1e-10 * so
    finally:
        for c in ctxs:
            tls.tls_destroy(c)
