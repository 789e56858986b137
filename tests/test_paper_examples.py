"""The examples of Sec. 4 as a regression suite: Example 1 (random 100 x 60), Example 2 (the
delta matrix, 9 x 4), Example 3 (Bjorck 30 x 15), Example 5 (Van Huffel, 100 x 98), rebuilt by
`synth` with the sizes, value distributions and perturbations the paper states (the MATLAB random
streams themselves cannot be reproduced, so iteration counts are compared qualitatively; Example
4's construction is garbled in the text and is not rebuilt).

GPU: the plain FP64 method and the mixed form (u_f = FP16, u = FP32) reach the TLS solution of
each example (the SVD of [A, b], Sec. 1) to the same limiting accuracy (Sec. 4.1-4.5), and on
Example 5 the mixed form needs at least as many RQI steps as the plain one (Sec. 4.5).
CPU: the Sec. 4.3 observation that a half-precision PCGTLS working precision limits the accuracy
of x, reproduced with the FP64 oracle whose inner solves are rounded to FP16 step by step, next to
the same run with FP32 inner solves.
"""
from __future__ import annotations

import numpy as np
import pytest
import scipy.linalg as sla

import oracle.rqi_pcgtls as O
from paper_2305_19028_gb300 import synth
from tests._pins import U64, kappa_tls, tls_by_svd

EXAMPLES = {
    "random_100x60": lambda: synth.random_matrix_problem(seed=0),
    "delta_9x4": lambda: synth.delta_matrix_problem(seed=1),
    "bjorck_30x15": lambda: synth.bjorck_problem(seed=1),
    "van_huffel_100": lambda: synth.van_huffel_problem(seed=1),
}


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def _x_tol(p, s_ref):
    # x_TLS is sensitive in proportion to kappa_TLS (Sec. 1): FP64 rounding of the data and of a
    # backward-stable solve moves it by about kappa_TLS u relative
    return max(1e-8, 1e4 * U64 * kappa_tls(p.A, s_ref) * (1.0 + np.linalg.norm(p.b)))


# ------------------------------------------------------------------------------------------
# CPU: Sec. 4.3, u_p = half
# ------------------------------------------------------------------------------------------
def _pcgtls_rounded(dtype):
    """Alg. 3 (A-explicit operator) with every vector result rounded to `dtype` (the working
    precision u_p of Alg. 4), in the oracle's step order."""
    def rnd(v):
        return np.asarray(v, dtype=np.float64).astype(dtype).astype(np.float64)

    def pcgtls(A, R, sigma2, f, l, mode="A", cg_tol=None, cg_max=None):
        Rl = rnd(R)
        s = rnd(sla.solve_triangular(Rl, rnd(f), trans="T", lower=False))
        p = s.copy()
        w = np.zeros_like(s)
        eta = float(rnd(s @ s))
        it = 0
        for _ in range(l + 1):
            q = rnd(sla.solve_triangular(Rl, p, lower=False))
            t = rnd(A @ q)
            delta = float(rnd(t @ t - sigma2 * (q @ q)))
            if delta <= 0.0:
                return w, it, delta < 0.0
            alpha = eta / delta
            w = rnd(w + alpha * q)
            v = rnd(sla.solve_triangular(Rl, rnd(A.T @ t - sigma2 * q), trans="T", lower=False))
            s = rnd(s - alpha * v)
            eta_new = float(rnd(s @ s))
            if eta_new == 0.0:
                break
            p = rnd(s + (eta_new / eta) * p)
            eta = eta_new
            it += 1
        return w, it, False

    return pcgtls


@pytest.mark.parametrize("seed", [1, 5, 7])
def test_half_precision_pcgtls_limits_the_accuracy_of_x(monkeypatch, seed):
    # Sec. 4.3 (Example 3, u_p = half): x stalls near the half-precision level, while the same
    # iteration with single-precision inner solves reaches the FP64 solution. Seeds whose draw
    # leaves a clear gap sigma_{n+1} < sigma'_n (ratio <= 0.91); with eps = 0.05 some draws put
    # sigma_{n+1} within 2 % of sigma'_n, where RQI from the LS start can reach another
    # singular pair at any precision.
    p = synth.bjorck_problem(seed=seed)
    s_ref, x_ref = tls_by_svd(p.A, p.b)
    errs = {}
    for name, dt in (("fp16", np.float16), ("fp32", np.float32)):
        monkeypatch.setattr(O, "pcgtls", _pcgtls_rounded(dt))
        x, s, _ = O.rqi_pcgtls(p.A, p.b, tol=0.0, max_rqi=15)
        errs[name] = _rel(x, x_ref)
    monkeypatch.undo()
    assert errs["fp16"] > 1e-7, errs
    assert errs["fp32"] < 1e-4 * errs["fp16"], errs


# ------------------------------------------------------------------------------------------
# GPU: the examples solved by the library
# ------------------------------------------------------------------------------------------
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    from paper_2305_19028_gb300 import tls
    tls.load()
    return tls


def _solve(tls, p, u_f, u):
    ctx = tls.tls_create_dense(p.A, p.b)
    try:
        tls.tls_factor(ctx, u_f, tls.tls_default_options(u=u))
        return tls.tls_solve(ctx, tol=0.0, max_rqi=30)
    finally:
        tls.tls_destroy(ctx)


@pytest.mark.gpu
@pytest.mark.parametrize("name", list(EXAMPLES))
@pytest.mark.parametrize("u_f,u", [("fp64", "fp64"), ("fp16", "fp32")])
def test_example_reaches_the_tls_solution(name, u_f, u):
    tls = _gpu()
    p = EXAMPLES[name]()
    s_ref, x_ref = tls_by_svd(p.A, p.b)
    x, sigma, info = _solve(tls, p, u_f, u)
    assert abs(sigma - s_ref) <= 1e-10 * s_ref, (name, sigma, s_ref, info)
    assert _rel(x, x_ref) <= _x_tol(p, s_ref), (name, _rel(x, x_ref), info)


@pytest.mark.gpu
@pytest.mark.parametrize("name", list(EXAMPLES))
def test_mixed_and_plain_reach_the_same_limiting_accuracy(name):
    # Sec. 4.1-4.5: the mixed form may need more RQI steps, but ends where the plain one does
    tls = _gpu()
    p = EXAMPLES[name]()
    xp, sp, ip = _solve(tls, p, "fp64", "fp64")
    xm, sm, im = _solve(tls, p, "fp16", "fp32")
    s_ref, x_ref = tls_by_svd(p.A, p.b)
    tol = _x_tol(p, s_ref)
    assert abs(sm - sp) <= 1e-10 * sp
    assert _rel(xm, xp) <= tol, (name, ip, im)


@pytest.mark.gpu
def test_mixed_needs_at_least_the_plain_steps_on_example_5():
    # Sec. 4.5 (Van Huffel, n = 100): the mixed-precision solve takes more RQI steps than the
    # uniform one with the same preconditioner type
    tls = _gpu()
    p = EXAMPLES["van_huffel_100"]()
    _, _, ip = _solve(tls, p, "fp64", "fp64")
    _, _, im = _solve(tls, p, "fp16", "fp32")
    assert im["rqi_steps"] >= ip["rqi_steps"], (ip, im)


@pytest.mark.gpu
def test_half_precision_working_precision_is_refused():
    # Sec. 4.3: u_p = half limits the attainable accuracy; the library accepts FP32 and FP64 only
    tls = _gpu()
    p = EXAMPLES["bjorck_30x15"]()
    ctx = tls.tls_create_dense(p.A, p.b)
    try:
        with pytest.raises(tls.TLSError) as e:
            tls.tls_factor(ctx, "fp16", tls.tls_default_options(u="fp16"))
        assert e.value.status == 1
    finally:
        tls.tls_destroy(ctx)
