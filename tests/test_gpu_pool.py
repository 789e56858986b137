"""The block cache (tls_pool_*): cached blocks are reused across contexts, the statistics add
up, and no result depends on what a buffer held before -- every path is run once on blocks
filled with 0xFF bytes (NaN in every FP32 / FP64 word) and once on blocks filled with zeros,
and the results must be bit-identical."""
from __future__ import annotations

import numpy as np
import pytest

from paper_2305_19028_gb300 import selector, synth, tls

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    tls.load()
    yield
    tls.tls_pool_poison(None)
    tls.tls_pool_enable(True)


def _dense(p, u_f, u, tol=0.0, max_rqi=10):
    ctx = tls.tls_create_dense(p.A, p.b)
    try:
        tls.tls_factor(ctx, u_f, tls.tls_default_options(u=u))
        x, s, info = tls.tls_solve(ctx, tol=tol, max_rqi=max_rqi)
    finally:
        tls.tls_destroy(ctx)
    return x, s, info["rqi_steps"], info["cg_iters"]


def _sparse(p, u_f):
    ctx = tls.tls_create_csr(p.m, p.n, p.row_ptr, p.col_idx, p.val, p.b)
    try:
        tls.tls_factor(ctx, u_f, tls.tls_default_options(u="fp32"))
        x, s, info = tls.tls_solve(ctx, tol=0.0, max_rqi=10)
    finally:
        tls.tls_destroy(ctx)
    return x, s, info["rqi_steps"], info["cg_iters"]


def _batch(probs, u_f, model=None):
    with tls.Batch([(p.A, p.b) for p in probs]) as bt:
        if model is not None:
            bt.set_selector(*model)
        bt.factor(u_f, u="fp32")
        xs, sig, infos, per = bt.solve(tol=0.0, max_rqi=10)
        F = bt.features()
    return xs, sig, [i["rqi_steps"] for i in infos], per, F


def _run_all():
    out = []
    out.append(_dense(synth.dense_problem(400, 40, d_lo=1e-2, noise=1e-6, seed=1), "fp64", "fp64"))
    out.append(_dense(synth.dense_problem(230, 7, d_lo=1e-2, noise=1e-4, seed=2), "fp16", "fp32"))
    out.append(_dense(synth.dense_problem(3000, 300, d_lo=1e-3, noise=1e-4, seed=3), "fp16", "fp32"))
    out.append(_dense(synth.dense_problem(2500, 457, d_lo=1e-2, noise=1e-4, seed=4), "bf16", "fp64"))
    out.append(_sparse(synth.csr_problem(3000, 250, nnz_per_row=12, noise=1e-3, seed=5), "bf16"))
    probs = [synth.batch_problem(i) for i in range(12)]
    out.append(_batch(probs, "fp16"))
    out.append(_batch(probs, "auto", selector.load_model()))
    return out


def _same(a, b):
    if isinstance(a, (tuple, list)):
        assert len(a) == len(b)
        for u, v in zip(a, b):
            _same(u, v)
    elif isinstance(a, np.ndarray):
        assert a.shape == b.shape and a.tobytes() == b.tobytes()
    else:
        assert a == b or (a != a and b != b)


def test_results_do_not_depend_on_previous_buffer_contents():
    res = {}
    for byte in (0xFF, 0x00):
        tls.tls_pool_trim()           # every block below is newly allocated and filled
        tls.tls_pool_poison(byte)
        try:
            res[byte] = _run_all()
        finally:
            tls.tls_pool_poison(None)
    for r in res[0xFF]:
        assert np.all(np.isfinite(np.asarray(r[1])))
    _same(res[0xFF], res[0x00])


def test_cache_reuses_blocks_and_trims():
    tls.tls_pool_enable(True)
    tls.tls_pool_trim()
    p = synth.dense_problem(2000, 200, d_lo=1e-2, noise=1e-4, seed=7)
    r1 = _dense(p, "fp16", "fp32")
    st1 = tls.tls_pool_stats()
    assert st1["cached_device"] > p.A.nbytes and st1["cached_host"] > 0
    r2 = _dense(p, "fp16", "fp32")               # served from the cache: nothing new
    st2 = tls.tls_pool_stats()
    assert st2["cached_device"] == st1["cached_device"]
    assert st2["cached_host"] == st1["cached_host"]
    _same(r1, r2)
    ctx = tls.tls_create_dense(p.A, p.b)
    live = tls.tls_pool_stats()
    assert live["live_device"] >= p.A.nbytes
    assert live["cached_device"] < st1["cached_device"]
    tls.tls_destroy(ctx)
    freed = tls.tls_pool_trim()
    assert freed >= st1["cached_device"]
    st3 = tls.tls_pool_stats()
    assert st3["cached_device"] == 0 and st3["cached_host"] == 0


def test_pool_off_frees_and_gives_the_same_results():
    p = synth.dense_problem(1500, 120, d_lo=1e-2, noise=1e-4, seed=8)
    tls.tls_pool_enable(True)
    r_on = _dense(p, "fp16", "fp32")
    tls.tls_pool_enable(False)
    try:
        assert tls.tls_pool_stats()["cached_device"] == 0
        r_off = _dense(p, "fp16", "fp32")
        assert tls.tls_pool_stats()["cached_device"] == 0
    finally:
        tls.tls_pool_enable(True)
    _same(r_on, r_off)


def test_caller_allocator_blocks_go_back_to_it():
    torch = pytest.importorskip("torch")
    p = synth.dense_problem(800, 60, d_lo=1e-2, noise=1e-4, seed=9)
    ref = _dense(p, "fp16", "fp32")
    tls.tls_pool_trim()
    before = torch.cuda.memory_allocated()
    ctx = tls.tls_create_dense(p.A, p.b)         # from the cache
    tls.use_torch_allocator(True)
    try:
        ctx2 = tls.tls_create_dense(p.A, p.b)    # from torch
        assert torch.cuda.memory_allocated() > before
        tls.tls_factor(ctx2, "fp16", tls.tls_default_options(u="fp32"))
        x, s, info = tls.tls_solve(ctx2, tol=0.0, max_rqi=10)
    finally:
        tls.use_torch_allocator(False)
    tls.tls_destroy(ctx2)                        # back to torch although the hook is unset
    assert torch.cuda.memory_allocated() == before
    tls.tls_destroy(ctx)
    _same(ref, (x, s, info["rqi_steps"], info["cg_iters"]))
