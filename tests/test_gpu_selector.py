"""Selector network: the library's forward / backward / Adam kernels against the FP64 oracle of
the network, training on the GPU, the features the batch computes, and the gain of the trained
network over the method without it."""
from __future__ import annotations

import ctypes as C

import numpy as np
import pytest

import oracle.mlp as M
import oracle.rqi_pcgtls as O
from paper_2305_19028_gb300 import selector, synth, tls

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    t.cuda.set_device(0)
    tls.load()
    return t


def _data(n, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    P = rng.normal(0.0, 0.25, size=M.N_PARAMS).astype(np.float32)
    X = rng.normal(size=(n, 16)).astype(np.float32)
    y = rng.integers(0, 3, size=n).astype(np.int32)
    t = rng.normal(size=n).astype(np.float32)
    mask = (rng.uniform(size=n) < 0.7).astype(np.float32)
    return P, X, y, t, mask


def test_forward_matches_oracle(torch):
    P, X, *_ = _data(77, 1)
    out = selector.Trainer(P).forward(torch.tensor(X, device="cuda")).cpu().numpy()
    ref, _ = M.forward(P.astype(np.float64), X.astype(np.float64), fp16=True)
    # FP16-rounded weights on both sides; FP32 accumulation of <= 64-term sums on the device
    assert np.max(np.abs(out - ref)) <= 2e-5 * (1.0 + np.max(np.abs(ref)))


@pytest.mark.parametrize("use_idx", [False, True])
def test_gradient_matches_oracle(torch, use_idx):
    P, X, y, t, mask = _data(150, 2)
    lam = 0.3
    tr = selector.Trainer(P)
    Xd = torch.tensor(X, device="cuda")
    yd = torch.tensor(y, device="cuda")
    td = torch.tensor(t, device="cuda")
    md = torch.tensor(mask, device="cuda")
    if use_idx:
        idx = np.random.Generator(np.random.PCG64(5)).permutation(150)[:97].astype(np.int32)
        tr.grad(Xd, yd, td, md, idx=torch.tensor(idx, device="cuda"), lam=lam)
        sel = idx
    else:
        tr.grad(Xd, yd, td, md, lam=lam)
        sel = np.arange(150)
    g = tr.g.cpu().numpy()
    L = float(tr.loss.item())
    Lr, gr = M.loss_and_grad(P.astype(np.float64), X[sel].astype(np.float64), y[sel], t[sel],
                             mask[sel], lam, fp16=True)
    assert L == pytest.approx(Lr, rel=1e-5)
    assert np.linalg.norm(g - gr) <= 1e-5 * np.linalg.norm(gr)
    assert np.max(np.abs(g - gr)) <= 1e-5 * np.max(np.abs(gr))


def test_adam_step_matches_definition(torch):
    P, X, y, t, mask = _data(64, 3)
    tr = selector.Trainer(P)
    Xd, yd, td, md = (torch.tensor(a, device="cuda") for a in (X, y, t, mask))
    m = np.zeros_like(P, dtype=np.float64)
    v = np.zeros_like(P, dtype=np.float64)
    p = P.astype(np.float64)
    for step in range(1, 4):
        tr.grad(Xd, yd, td, md, lam=0.2)
        g = tr.g.cpu().numpy().astype(np.float64)
        tr.step(1e-2)
        # Adam (Kingma & Ba 2015) with bias correction
        m = 0.9 * m + 0.1 * g
        v = 0.999 * v + 0.001 * g * g
        p = p - 1e-2 * (m / (1 - 0.9 ** step)) / (np.sqrt(v / (1 - 0.999 ** step)) + 1e-8)
        # continue from the device parameters so that rounding does not accumulate
        assert np.max(np.abs(tr.params() - p)) <= 1e-5 * (1 + np.max(np.abs(p)))
        p = tr.params().astype(np.float64)


def test_training_learns_a_separable_rule(torch):
    # labels from a known rule of two features; the GPU-trained network must recover it
    rng = np.random.Generator(np.random.PCG64(9))
    F = rng.normal(size=(3000, 16)).astype(np.float32)
    y = np.where(F[:, 0] + 0.5 * F[:, 3] > 0.6, 2, np.where(F[:, 0] - F[:, 5] < -0.8, 1, 0))
    t = (0.5 * F[:, 1] - 2.0).astype(np.float32)
    params, mean, scale, hist = selector.train(F[:2500], y[:2500].astype(np.int32), t[:2500],
                                               np.ones(2500, np.float32), epochs=150, lr=3e-3)
    assert hist[-1] < 0.5 * hist[0]
    out = selector.predict(params, mean, scale, F[2500:])
    acc = (out[:, :3].argmax(axis=1) == y[2500:]).mean()
    assert acc >= 0.93
    assert np.sqrt(np.mean((out[:, 3] - t[2500:]) ** 2)) <= 0.3


def test_batch_features_match_definitions(torch):
    probs = [synth.dense_problem(400, 40, d_lo=1e-3, noise=1e-5, seed=21),
             synth.dense_problem(999, 130, d_lo=1e-1, noise=1e-4, seed=22)]
    with tls.Batch([(p.A, p.b) for p in probs]) as bt:
        bt.factor("fp16", u="fp32")
        F = bt.features()
        for i, p in enumerate(probs):
            R, d, _ = bt.export_factor(i)
            m, n = p.A.shape
            assert F[i, 0] == pytest.approx(np.log10(m), abs=1e-6)
            assert F[i, 1] == pytest.approx(np.log10(n), abs=1e-6)
            dn = np.linalg.norm(p.A, axis=0)
            assert F[i, 3] == pytest.approx(np.log10(dn.max() / dn.min()), abs=1e-5)
            assert F[i, 5] == pytest.approx(np.log10(np.linalg.norm(p.b) / np.linalg.norm(p.A)),
                                            abs=1e-5)
            r = np.diag(R)
            assert F[i, 6] == pytest.approx(np.log10(r.max() / r.min()), abs=1e-5)
            Winv = np.linalg.inv(R)
            assert F[i, 10] == pytest.approx(np.log10(np.linalg.norm(Winv)), abs=1e-3)
            # power iteration approaches ||W||_2 from below
            w2 = np.linalg.norm(Winv, 2)
            assert np.log10(w2) - 0.1 <= F[i, 11] <= np.log10(w2) + 1e-4


def test_trained_selector_gains_over_fp16_first(torch):
    model = selector.load_model()
    if model is None:
        pytest.skip("no trained selector model in the package")
    params, mean, scale = model
    probs = [synth.selector_problem(100000 + i) for i in range(160)]
    ref = [O.rqi_pcgtls(p.A, p.b, tol=0.0, max_rqi=12)[:2] for p in probs]

    def run(auto):
        import time
        with tls.Batch([(p.A, p.b) for p in probs]) as bt:
            if auto:
                bt.set_selector(params, mean, scale)
            t0 = time.perf_counter()
            bt.factor("auto" if auto else "fp16", u="fp32")
            xs, sig, infos, per = bt.solve(tol=0.0, max_rqi=12)
            torch.cuda.synchronize()
            return time.perf_counter() - t0, xs, sig, infos

    run(False)   # warm-up (autotuning of the pass tiles)
    t_base, xb, sb, ib = run(False)
    t_sel, xa, sa, ia = run(True)
    ok_b = ok_a = 0
    for (xo, so), x1, s1, x2, s2 in zip(ref, xb, sb, xa, sa):
        ok_b += abs(s1 - so) <= 1e-10 * so and np.linalg.norm(x1 - xo) <= 1e-8 * np.linalg.norm(xo)
        ok_a += abs(s2 - so) <= 1e-10 * so and np.linalg.norm(x2 - xo) <= 1e-8 * np.linalg.norm(xo)
    fb_b = sum(i["fallbacks"] for i in ib)
    fb_a = sum(i["fallbacks"] for i in ia)
    print(f"fp16-first {t_base * 1e3:.1f} ms, {fb_b} fallbacks, {ok_b} accurate; "
          f"selector {t_sel * 1e3:.1f} ms, {fb_a} fallbacks, {ok_a} accurate")
    assert ok_a >= ok_b
    assert fb_a < fb_b
    assert t_sel < t_base


def test_single_context_features_match_batch(torch):
    # the single-problem feature kernels compute the batch's 16 features (the same network
    # serves both paths); the factors differ only in the order of rounding of the inverse
    probs = [synth.dense_problem(400, 40, d_lo=1e-3, noise=1e-5, seed=21),
             synth.dense_problem(999, 130, d_lo=1e-1, noise=1e-4, seed=22),
             synth.selector_problem(100007)]
    with tls.Batch([(p.A, p.b) for p in probs]) as bt:
        bt.factor("fp16", u="fp32")
        Fb = bt.features()
    for i, p in enumerate(probs):
        ctx = tls.tls_create_dense(p.A, p.b)
        try:
            tls.tls_factor(ctx, "fp16", tls.tls_default_options(u="fp32"))
            F = tls.tls_features(ctx)
        finally:
            tls.tls_destroy(ctx)
        np.testing.assert_allclose(F, Fb[i], rtol=0, atol=2e-3)


def test_single_context_auto_factor(torch):
    # TLS_AUTO = factor at FP16, features, network, refactor at its pick: the solve must equal a
    # solve from a plain factor at the precision it ended with (cg_fixed = 1 leaves the network's
    # tolerance unused); accuracy over many problems is the gain test's and the evaluation's
    model = selector.load_model()
    if model is None:
        pytest.skip("no trained selector model in the package")
    params, mean, scale = model
    names = {0: "fp16", 1: "bf16", 2: "fp32", 3: "fp64"}
    opt = tls.tls_default_options(u="fp32", fallback=0)
    picked = set()
    for seed in (100001, 100002, 100003, 100011):
        p = synth.selector_problem(seed)
        ctx = tls.tls_create_dense(p.A, p.b)
        try:
            tls.tls_set_selector(ctx, params, mean, scale)
            tls.tls_factor(ctx, "auto", opt)
            x, s, info = tls.tls_solve(ctx, tol=0.0, max_rqi=12)
        finally:
            tls.tls_destroy(ctx)
        uf = info["u_f_used"]
        picked.add(uf)
        ctx = tls.tls_create_dense(p.A, p.b)
        try:
            tls.tls_factor(ctx, names[uf], opt)
            x2, s2, _ = tls.tls_solve(ctx, tol=0.0, max_rqi=12)
        finally:
            tls.tls_destroy(ctx)
        assert s == s2
        np.testing.assert_array_equal(x, x2)
    assert picked <= {0, 1, 2, 3}
