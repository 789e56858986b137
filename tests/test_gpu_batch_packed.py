"""Packed batch (tls_batch_*): many dense problems of uneven sizes solved in lock step, every
phase one launch for the whole batch. Each problem is compared with the FP64 oracle run on the
same seeded input, with the tolerances of the single-problem parity tests."""
from __future__ import annotations

import ctypes as C

import numpy as np
import pytest

import oracle.rqi_pcgtls as O
from paper_2305_19028_gb300 import synth, tls

pytestmark = pytest.mark.gpu

U16, UBF, U32, U64 = 2.0 ** -11, 2.0 ** -8, 2.0 ** -24, 2.0 ** -53


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    tls.load()


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def _mixed_problems():
    # members of the uneven batch (n ~ U{32..512}, m = n U{4..20}) plus edge shapes: one
    # column, a square problem, the largest n, rows not a multiple of any tile
    probs = [synth.batch_problem(i) for i in range(6)]
    probs.append(synth.dense_problem(37, 1, d_lo=1e-1, noise=1e-3, seed=11))
    probs.append(synth.dense_problem(70, 70, d_lo=1e-1, noise=1e-3, seed=12))
    probs.append(synth.dense_problem(2053, 512, d_lo=1e-2, noise=1e-4, seed=13))
    probs.append(synth.dense_problem(333, 33, d_lo=1e-3, noise=1e-4, seed=14))
    return probs


def _check_against_oracle(probs, xs, sig, infos):
    for p, x, s, info in zip(probs, xs, sig, infos):
        xo, so, _ = O.rqi_pcgtls(p.A, p.b, tol=0.0, max_rqi=12)
        m, n = p.A.shape
        atol = 64 * U64 * (np.linalg.norm(p.A) + np.linalg.norm(p.b)) if m == n else 0.0
        assert abs(s - so) <= 1e-10 * so + atol, (p.A.shape, s, so, info)
        if m > n:
            assert _rel(x, xo) <= 1e-8, (p.A.shape, info)


@pytest.mark.parametrize("u_f", ["fp16", "bf16"])
def test_packed_batch_matches_oracle(u_f):
    probs = _mixed_problems()
    with tls.Batch([(p.A, p.b) for p in probs]) as bt:
        bt.factor(u_f, u="fp32")
        xs, sig, infos, per = bt.solve(tol=0.0, max_rqi=12)
    assert per == [0] * len(probs)
    _check_against_oracle(probs, xs, sig, infos)


def test_packed_batch_plain_fp64_matches_oracle():
    probs = _mixed_problems()[:5]
    with tls.Batch([(p.A, p.b) for p in probs]) as bt:
        bt.factor("fp64", u="fp64")
        xs, sig, infos, per = bt.solve(tol=0.0, max_rqi=12)
    assert all(i["u_f_used"] == tls.PREC["fp64"] and i["fallbacks"] == 0 for i in infos)
    _check_against_oracle(probs, xs, sig, infos)


def _rounded_scaled(A, d, u_f):
    if u_f == "fp64":
        return A / d
    As = A.astype(np.float32) * (1.0 / d).astype(np.float32)
    if u_f == "fp16":
        return As.astype(np.float16).astype(np.float64)
    if u_f == "bf16":
        mant, ex = np.frexp(As.astype(np.float64))
        return np.ldexp(np.rint(mant * 256.0) / 256.0, ex)
    return As.astype(np.float64)


@pytest.mark.parametrize("u_f,u", [("fp16", "fp32"), ("bf16", "fp32"), ("fp32", "fp32"),
                                   ("fp64", "fp64")])
def test_packed_factor_matches_definitions(u_f, u):
    # per problem: d_j = ||a_j||, H = A_s^T A_s of the u_f-rounded scaled matrix (FP32
    # accumulation), R_H upper triangular in u_f with R_H^T R_H = H + s I up to rounding
    probs = [synth.dense_problem(300, 64, d_lo=1e-2, noise=1e-3, seed=3),
             synth.dense_problem(777, 130, d_lo=1e-2, noise=1e-3, seed=4),
             synth.dense_problem(97, 5, d_lo=1e-1, noise=1e-3, seed=5)]
    with tls.Batch([(p.A, p.b) for p in probs]) as bt:
        bt.factor(u_f, u=u, shift_first=0)
        for i, p in enumerate(probs):
            R, d, H = bt.export_factor(i)
            m, n = p.A.shape
            d_ref = np.linalg.norm(p.A, axis=0)
            assert np.max(np.abs(d - d_ref) / d_ref) <= 1e-13
            As = _rounded_scaled(p.A, d, u_f)
            H_ref = As.T @ As
            bound = (m * U32 if u_f != "fp64" else m * U64) * (np.abs(As).T @ np.abs(As))
            assert np.all(np.abs(H - H_ref) <= 2 * bound + 1e-30)
            assert np.array_equal(R, np.triu(R))
            if u_f == "fp16":
                assert np.array_equal(R, R.astype(np.float16).astype(np.float64))
            ufac = {"fp16": U16, "bf16": UBF, "fp32": U32, "fp64": U64}[u_f]
            berr = np.linalg.norm(R.T @ R - H) / np.linalg.norm(H)
            assert berr <= 4 * ufac * np.sqrt(n) + (n * U32 if u_f != "fp64" else 0)


def test_packed_zero_column_breaks_down_then_shifts():
    p = synth.dense_problem(200, 30, d_lo=1e-1, noise=1e-3, seed=2)
    A = p.A.copy()
    A[:, 7] = 0.0
    good = synth.dense_problem(150, 20, d_lo=1e-1, noise=1e-3, seed=6)
    with tls.Batch([(A, p.b), (good.A, good.b)]) as bt:
        bt.factor("fp16", u="fp32", shift_first=0, fallback=0)
        xs, sig, infos, per = bt.solve(tol=0.0, max_rqi=3)
    assert infos[0]["shifts"] >= 1 and infos[0]["fail_pivot"] == 7 and infos[0]["shift"] > 0
    assert infos[1]["shifts"] == 0 and infos[1]["shift"] == 0.0


def test_packed_batch_validation():
    p = synth.dense_problem(600, 513, seed=1)
    with pytest.raises(tls.TLSError):
        tls.Batch([(p.A, p.b)])                 # n above the packed-batch limit
    q = synth.dense_problem(50, 5, seed=1)
    with tls.Batch([(q.A, q.b)]) as bt:
        with pytest.raises(tls.TLSError):
            bt.solve()                          # before factor: state error


def test_graph_replay_equals_eager_launches():
    # the solve is captured once as a CUDA graph and replayed; with profiling on the same
    # launches run eagerly with a synchronisation per RQI step. Every kernel is deterministic,
    # so all three runs give bit-identical results.
    probs = _mixed_problems()[:6]
    with tls.Batch([(p.A, p.b) for p in probs]) as bt:
        bt.factor("fp16", u="fp32", fallback=0)
        x1, s1, i1, _ = bt.solve(tol=0.0, max_rqi=12)
        x2, s2, i2, _ = bt.solve(tol=0.0, max_rqi=12)
        bt.profile(True)
        x3, s3, i3, _ = bt.solve(tol=0.0, max_rqi=12)
        prof = bt.profile_get()
    assert np.array_equal(s1, s2) and np.array_equal(s1, s3)
    for a, b, c in zip(x1, x2, x3):
        assert np.array_equal(a, b) and np.array_equal(a, c)
    assert [i["rqi_steps"] for i in i1] == [i["rqi_steps"] for i in i3]
    assert prof["pcg_pass2"][0] > 0 and prof["resid_pass"][0] > 0


def _batch_raw(arrays, on_device):
    """tls_batch_create_dense through the C ABI with each A's own row stride."""
    lib = tls.load()
    k = len(arrays)
    ms = (C.c_int64 * k)(*[A.shape[0] for A, _, _ in arrays])
    ns = (C.c_int64 * k)(*[A.shape[1] for A, _, _ in arrays])
    ld = (C.c_int64 * k)(*[ld_ for _, _, ld_ in arrays])
    ptr = (lambda t: t.data_ptr()) if on_device else (lambda a: a.ctypes.data)
    ap = (C.c_void_p * k)(*[ptr(A) for A, _, _ in arrays])
    bp = (C.c_void_p * k)(*[ptr(b) for _, b, _ in arrays])
    h = C.c_void_p()
    st = lib.tls_batch_create_dense(C.byref(h), k, ms, ns, ap, ld, bp, int(on_device), None)
    assert st == 0
    bt = tls.Batch.__new__(tls.Batch)
    bt.h, bt.k = h, k
    bt.shapes = [tuple(A.shape) for A, _, _ in arrays]
    return bt


def test_strided_inputs_host_and_device_give_identical_results():
    """Row strides wider than n on the host and on the device (the rows are copied whole and
    placed by one kernel): bit-identical to the contiguous batch."""
    torch = pytest.importorskip("torch")
    probs = _mixed_problems()
    with tls.Batch([(p.A, p.b) for p in probs]) as bt:
        bt.factor("fp16", u="fp32")
        x0, s0, _, _ = bt.solve(tol=0.0, max_rqi=12)
    wide = []
    for j, p in enumerate(probs):
        m, n = p.A.shape
        W = np.full((m, n + 3 + j % 5), np.nan)
        W[:, :n] = p.A
        wide.append((W, p.b))
    host = [(W[:, :p.A.shape[1]], b, W.shape[1]) for (W, b), p in zip(wide, probs)]
    dev = []
    for (W, b), p in zip(wide, probs):
        Wd = torch.from_numpy(W).cuda()
        dev.append((Wd[:, :p.A.shape[1]], torch.from_numpy(b).cuda(), W.shape[1]))
    for arrays, on_device in ((host, False), (dev, True)):
        bt = _batch_raw(arrays, on_device)
        try:
            bt.factor("fp16", u="fp32")
            x1, s1, _, _ = bt.solve(tol=0.0, max_rqi=12)
        finally:
            bt.close()
        assert np.array_equal(s0, s1)
        for a, b in zip(x0, x1):
            assert np.array_equal(a, b)
