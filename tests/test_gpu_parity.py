"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on identical seeded
inputs. Tolerances follow from the arithmetic of each step (stated per test)."""
from __future__ import annotations

import numpy as np
import pytest
import scipy.linalg as sla

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


class Ctx:
    def __init__(self, A, b, u_f="fp16", u="fp32", fused=0, **opt):
        self.ctx = tls.tls_create_dense(A, b)
        if fused:
            tls.tls_set_pcg_fused(self.ctx, fused)
        self.opt = tls.tls_default_options(u=u, **opt)
        tls.tls_factor(self.ctx, u_f, self.opt)

    def __enter__(self):
        return self.ctx

    def __exit__(self, *a):
        tls.tls_destroy(self.ctx)


# ------------------------------------------------------------------------------------------
# residual block (FP64): Alg. 2 lines r_k..g_k, Eq. (2), Eq. (4)
# ------------------------------------------------------------------------------------------
@pytest.mark.parametrize("m,n", [(64, 1), (200, 37), (1000, 130), (3000, 700)])
def test_residual_block_matches_oracle(m, n):
    p = synth.dense_problem(m, n, d_lo=1e-2, noise=1e-3, seed=m + n)
    x = p.x_true + 1e-3 * np.random.default_rng(0).standard_normal(n)
    ctx = tls.tls_create_dense(p.A, p.b)
    try:
        f, sc = tls.tls_residual(ctx, x)
    finally:
        tls.tls_destroy(ctx)
    r, s2, fo, go, psio = O.residual_block(p.A, p.b, x)
    # FP64 dot products in a different order: error ~ n u (|A||x| + |b|) per entry of r
    scale_r = n * U64 * (np.abs(p.A) @ np.abs(x) + np.abs(p.b)).max()
    assert abs(sc["rr"] - r @ r) <= 4 * scale_r * np.linalg.norm(r) * np.sqrt(m) + 1e-300
    assert abs(sc["sigma2"] - s2) <= 1e-10 * s2
    fscale = m * U64 * (np.abs(p.A).T @ (np.abs(p.A) @ np.abs(x) + np.abs(p.b))).max()
    assert np.max(np.abs(f - fo)) <= 8 * fscale
    assert abs(sc["g"] - go) <= 8 * m * U64 * (np.abs(p.b) @ (np.abs(p.A) @ np.abs(x) + np.abs(p.b)))
    assert abs(sc["psi"] - psio) <= 1e-6 * psio + 8 * fscale


U_DF = 2.0 ** -48     # the double-FP32 residual: A and x carried as FP32 pairs to 2^-48


@pytest.mark.parametrize("m,n", [(64, 1), (3001, 40), (1000, 700), (5003, 2100), (4500, 4100),
                                 (8100, 7900)])
def test_double_fp32_residual_matches_oracle(m, n):
    """The residual pass in double-FP32 arithmetic (FP32 working precision: A as A32 + Alo,
    products by TwoProd, sums in FP32 pairs, r_i as a pair, ||r||^2 and b^T r in FP64) against
    the FP64 oracle and against the FP64 pass on the same data. Error model: A and x carried to
    2^-48, each product's dropped low-low term 2^-48, pair sums of a few dozen terms: the
    entries of r within about 64 * 2^-48 of (|A||x| + |b|) plus the FP64 reductions' n u. Shapes
    cover the tile sizes (4, 2 and 1 rows: n_pad up to 2048, 4096, 8192) and ragged row
    blocks; above n_pad = 4096 no FP64 pass exists to compare with."""
    p = synth.dense_problem(m, n, d_lo=1e-2, noise=1e-3, seed=m + 3 * n)
    x = p.x_true + 1e-3 * np.random.default_rng(1).standard_normal(n)
    npad = -(-n // 64) * 64
    with Ctx(p.A, p.b, u_f="fp32", u="fp32") as ctx:
        f, sc = tls.tls_residual(ctx, x)
        x1, s1, info = tls.tls_solve(ctx, tol=0.0, max_rqi=1)
        assert info["pass_variant"][0] == 4
        if npad <= 4096:
            assert tls.load().tls_set_pass_variant(ctx, 3, 0) == 0    # the FP64 pass
            f64, sc64 = tls.tls_residual(ctx, x)
        else:
            assert tls.load().tls_set_pass_variant(ctx, 3, 0) == 1
            f64, sc64 = f, sc
    r, s2, fo, go, psio = O.residual_block(p.A, p.b, x)
    u = 64 * U_DF + n * U64
    ax = np.abs(p.A) @ np.abs(x) + np.abs(p.b)
    scale_r = u * ax.max()
    fscale = (64 * U_DF + m * U64) * (np.abs(p.A).T @ ax).max()
    for ff, ss in ((f, sc), (f64, sc64)):
        assert abs(ss["rr"] - r @ r) <= 4 * scale_r * np.linalg.norm(r) * np.sqrt(m) + 1e-300
        assert abs(ss["sigma2"] - s2) <= 1e-10 * s2
        assert np.max(np.abs(ff - fo)) <= 8 * fscale
        assert abs(ss["g"] - go) <= 8 * (64 * U_DF + m * U64) * (np.abs(p.b) @ ax)
        assert abs(ss["psi"] - psio) <= 1e-6 * psio + 8 * fscale
    assert np.max(np.abs(f - f64)) <= 16 * fscale


# ------------------------------------------------------------------------------------------
# factor: column scaling, Gram of the u_f-rounded scaled matrix, Cholesky, R_H in u_f (Sec. 3.1)
# ------------------------------------------------------------------------------------------
def _rounded_scaled(A, d, u_f):
    """A_s as the device forms it: FP64 path A / d; FP32 path fl32(fl32(A) * fl32(1/d)) rounded
    (to nearest even) to u_f."""
    if u_f == "fp64":
        return A / d
    As = A.astype(np.float32) * (1.0 / d).astype(np.float32)     # FP32 product, RN
    if u_f == "fp16":
        return As.astype(np.float16).astype(np.float64)
    if u_f == "bf16":
        # round-to-nearest-even to 8 significant bits
        mant, ex = np.frexp(As.astype(np.float64))
        return np.ldexp(np.rint(mant * 256.0) / 256.0, ex)
    return As.astype(np.float64)


@pytest.mark.parametrize("m,n", [(800, 130), (5000, 2100)])
def test_factor_chain_matches_one_launch_per_step(m, n):
    """The FP32 factor's block steps in one persistent launch give the same factor, bit for bit,
    as one launch per block step (the same arithmetic in the same order)."""
    p = synth.dense_problem(m, n, d_lo=1e-2, noise=1e-3, seed=5)
    out = []
    for chain in (1, 2, 0):
        ctx = tls.tls_create_dense(p.A, p.b)
        try:
            tls.tls_set_factor_chain(ctx, chain)
            tls.tls_factor(ctx, "fp16", tls.tls_default_options(u="fp32"))
            out.append(tls.tls_export_factor(ctx))
        finally:
            tls.tls_destroy(ctx)
    for chained in out[:2]:
        for a_, b_ in zip(chained, out[2]):
            assert np.array_equal(np.asarray(a_), np.asarray(b_))


@pytest.mark.parametrize("u_f", ["fp16", "bf16"])
def test_tensor_core_trailing_updates_match_definitions(u_f):
    """n = 2500 (n_pad = 2560): the first block steps, whose trailing matrices are too large for
    the persistent chain, update on the tensor cores with the panel rows rounded to u_f (FP32
    accumulation); the factor meets the same backward-error bound as the FP32 CUDA-core updates
    (R_H^T R_H = H up to 4 u_f sqrt(n) + n u_32 of ||H||), is upper triangular and representable
    in u_f, and its solve still reaches the oracle's answer."""
    m, n = 3000, 2500
    p = synth.dense_problem(m, n, d_lo=1e-2, noise=1e-3, seed=9)
    ufac = {"fp16": U16, "bf16": UBF}[u_f]
    res = {}
    for tcu in (1, 0):
        ctx = tls.tls_create_dense(p.A, p.b)
        try:
            tls.tls_set_factor_tc(ctx, tcu)
            tls.tls_factor(ctx, u_f, tls.tls_default_options(u="fp32"))
            R, d, H = tls.tls_export_factor(ctx)
            x, sigma, info = tls.tls_solve(ctx, tol=0.0, max_rqi=12)
        finally:
            tls.tls_destroy(ctx)
        res[tcu] = (R, H, x, sigma)
    xo, so, _ = O.rqi_pcgtls(p.A, p.b, tol=0.0, max_rqi=12)
    for tcu, (R, H, x, sigma) in res.items():
        assert np.array_equal(R, np.triu(R))
        if u_f == "fp16":
            assert np.array_equal(R, R.astype(np.float16).astype(np.float64))
        berr = np.linalg.norm(R.T @ R - H) / np.linalg.norm(H)
        assert berr <= 4 * ufac * np.sqrt(n) + n * U32, (tcu, berr)
        assert abs(sigma - so) <= 1e-10 * so, (tcu, sigma, so)
        assert _rel(x, xo) <= 1e-8, tcu
    # the same Gram matrix enters both factors
    assert np.array_equal(res[0][1], res[1][1])


@pytest.mark.parametrize("u_f,u", [("fp16", "fp32"), ("bf16", "fp32"), ("fp32", "fp32"),
                                   ("fp64", "fp64")])
@pytest.mark.parametrize("m,n", [(300, 64), (777, 130)])
def test_factor_matches_definitions(u_f, u, m, n):
    p = synth.dense_problem(m, n, d_lo=1e-2, noise=1e-3, seed=3)
    with Ctx(p.A, p.b, u_f=u_f, u=u) as ctx:
        R, d, H = tls.tls_export_factor(ctx)
    # column norms: FP32 accumulation (u = fp32) or FP64
    d_ref = np.linalg.norm(p.A, axis=0)
    assert np.max(np.abs(d - d_ref) / d_ref) <= (m * U32 if u == "fp32" else 1e-13)
    As = _rounded_scaled(p.A, d, u_f)
    H_ref = As.T @ As
    bound = (m * U32 if u_f != "fp64" else m * U64) * (np.abs(As).T @ np.abs(As))
    assert np.all(np.abs(H - H_ref) <= 2 * bound + 1e-30)
    # R_H upper triangular, representable in u_f, and a Cholesky factor of H up to rounding
    assert np.allclose(R, np.triu(R), atol=0)
    if u_f == "fp16":
        assert np.array_equal(R, R.astype(np.float16).astype(np.float64))
    ufac = {"fp16": U16, "bf16": UBF, "fp32": U32, "fp64": U64}[u_f]
    berr = np.linalg.norm(R.T @ R - H) / np.linalg.norm(H)
    assert berr <= 4 * ufac * np.sqrt(n) + (n * U32 if u_f != "fp64" else 0)


def test_working_copy_is_fp32_round_to_nearest():
    # the FP32 copy of A is formed with integer instructions; it must equal IEEE RN exactly,
    # including signed zeros, subnormal FP32 results and ties
    p = synth.dense_problem(300, 70, d_lo=1e-2, noise=1e-3, seed=4)
    A = p.A.copy()
    A[0, :8] = [0.0, -0.0, 1e-40, -3e-39, 1.0 + 2.0 ** -24, 1.0 + 3 * 2.0 ** -24, 2.0 ** -149,
                -(1.0 + 2.0 ** -23 + 2.0 ** -24)]
    with Ctx(A, p.b, u_f="fp16", u="fp32") as ctx:
        A32 = tls.tls_export_working_copy(ctx)
    ref = A.astype(np.float32)
    assert np.array_equal(A32.view(np.uint32), ref.view(np.uint32))


# ------------------------------------------------------------------------------------------
# preconditioner products and PCGTLS (Alg. 3) against the oracle with the same R
# ------------------------------------------------------------------------------------------
@pytest.mark.parametrize("u_f,u", [("fp16", "fp32"), ("fp64", "fp64")])
def test_precond_matches_oracle(u_f, u):
    p = synth.dense_problem(500, 150, d_lo=1e-2, noise=1e-3, seed=5)
    y = np.random.default_rng(1).standard_normal(150)
    with Ctx(p.A, p.b, u_f=u_f, u=u) as ctx:
        RH, d, _ = tls.tls_export_factor(ctx)
        s0, uu = tls.tls_precond(ctx, y)
    R = RH * d[None, :]
    s_ref = sla.solve_triangular(R, y, trans="T", lower=False)
    u_ref = sla.solve_triangular(R, s_ref, lower=False)
    kap = np.linalg.cond(RH)
    tol = (20 * kap * 150 * U32) if u == "fp32" else (20 * kap * 150 * U64)
    assert _rel(s0, s_ref) <= tol
    assert _rel(uu, u_ref) <= 2 * tol * kap


@pytest.mark.parametrize("u_f,u,m,n", [("fp16", "fp32", 500, 150), ("fp16", "fp32", 3000, 2100),
                                       ("fp64", "fp64", 500, 150), ("bf16", "fp32", 900, 1)])
def test_triangular_solves_match_oracle_and_inverse_products(u_f, u, m, n):
    """Alg. 3's R^{-T} and R^{-1} by blocked substitution on the factor (tls_precond_trsv)
    against scipy's triangular solves with the same R = R_H D, and against the products with
    the explicit inverse that the solve uses (tls_precond). Shapes: one block, 33 blocks with a
    ragged last one, FP64, a single column."""
    p = synth.dense_problem(m, n, d_lo=1e-2, noise=1e-3, seed=7)
    y = np.random.default_rng(3).standard_normal(n)
    with Ctx(p.A, p.b, u_f=u_f, u=u) as ctx:
        RH, d, _ = tls.tls_export_factor(ctx)
        st, ut = tls.tls_precond_trsv(ctx, y)
        sw, uw = tls.tls_precond(ctx, y)
    R = RH * d[None, :]
    s_ref = sla.solve_triangular(R, y, trans="T", lower=False)
    u_ref = sla.solve_triangular(R, s_ref, lower=False)
    kap = np.linalg.cond(RH)
    uu = U32 if u == "fp32" else U64
    tol = 20 * kap * n * uu
    assert _rel(st, s_ref) <= tol
    assert _rel(ut, u_ref) <= 2 * tol * kap
    assert _rel(st, sw) <= 2 * tol
    assert _rel(ut, uw) <= 4 * tol * kap


@pytest.mark.parametrize("u_f,u,fused", [("fp16", "fp32", 1), ("fp16", "fp32", 2),
                                         ("fp64", "fp64", 0)])
@pytest.mark.parametrize("modeA", [1, 0])
def test_pcgtls_matches_oracle(u_f, u, fused, modeA):
    """Both FP32 forms of the A-explicit solve (one persistent launch per solve, fused = 1; a
    pass launch and a step-tail launch per step, fused = 2) and Alg. 3 as printed (mode R)."""
    m, n = 900, 200
    p = synth.dense_problem(m, n, d_lo=1e-2, noise=1e-3, seed=6)
    rng = np.random.default_rng(2)
    f0 = rng.standard_normal(n)
    f1 = rng.standard_normal(n)
    sigma2 = 0.3 * p.D[-1] ** 2
    steps = 4
    with Ctx(p.A, p.b, u_f=u_f, u=u, mode_A=modeA, fused=fused) as ctx:
        RH, d, _ = tls.tls_export_factor(ctx)
        w0, w1, it, bad = tls.tls_pcgtls(ctx, sigma2, f0, f1, steps=steps)
        w0s, _, it1, _ = tls.tls_pcgtls(ctx, sigma2, f0, None, steps=steps)
    R = RH * d[None, :]
    mode = "A" if modeA else "R"
    r0, i0, _ = O.pcgtls(p.A, R, sigma2, f0, steps - 1, mode=mode)
    r1, i1, _ = O.pcgtls(p.A, R, sigma2, f1, steps - 1, mode=mode)
    assert it == [steps, steps] and bad == [0, 0] and it1[0] == steps
    kap = np.linalg.cond(RH)
    tol = (50 * kap * n * U32) if u == "fp32" else (50 * kap * n * U64)
    assert _rel(w0, r0) <= tol
    assert _rel(w1, r1) <= tol
    # the paired solve and the single solve share nothing but the pass over A
    assert _rel(w0s, w0) <= tol


def _precond_residual(A, R, sigma2, f, w):
    # ||R^{-T}(f - (A^T A - sigma^2 I) w)|| in FP64: what Alg. 3's ||s_j|| stands for
    r = f - (A.T @ (A @ w) - sigma2 * w)
    return float(np.linalg.norm(sla.solve_triangular(R, r, trans="T", lower=False)))


@pytest.mark.parametrize("u_f,u,tol,fused", [("fp16", "fp32", 1e-4, 1), ("fp16", "fp32", 1e-4, 2),
                                             ("bf16", "fp32", 1e-3, 1), ("fp64", "fp64", 1e-9, 0)])
def test_pcgtls_tolerance_mode_matches_oracle(u_f, u, tol, fused):
    """PCGTLS with a relative tolerance on ||s_j|| (cg_fixed = 0, the mode the selector's
    tolerance output uses) against the oracle's cg_tol mode on the same factor: the stop step
    agrees to within one step (the FP32 recurrence crosses the threshold at its own rounding),
    the GPU iterate meets the tolerance, and it equals the oracle's iterate of the same step
    count element by element at the bound of the fixed-step parity test."""
    m, n = 900, 200
    p = synth.dense_problem(m, n, d_lo=1e-2, noise=1e-3, seed=16)
    rng = np.random.default_rng(8)
    f0 = rng.standard_normal(n)
    f1 = rng.standard_normal(n)
    sigma2 = 0.3 * p.D[-1] ** 2
    cap = 60
    with Ctx(p.A, p.b, u_f=u_f, u=u, cg_fixed=0, cg_tol=tol, cg_max=cap, fused=fused) as ctx:
        RH, d, _ = tls.tls_export_factor(ctx)
        w0, w1, it, bad = tls.tls_pcgtls(ctx, sigma2, f0, f1, steps=cap, cg_tol=tol)
    R = RH * d[None, :]
    kap = np.linalg.cond(RH)
    ueps = U32 if u == "fp32" else U64
    assert bad == [0, 0]
    for f, w, i_gpu in ((f0, w0, it[0]), (f1, w1, it[1])):
        wo, i_or, bad_o = O.pcgtls(p.A, R, sigma2, f, 0, cg_tol=tol, cg_max=cap)
        assert not bad_o and 1 <= i_gpu < cap
        assert abs(i_gpu - i_or) <= 1, (i_gpu, i_or)
        s0 = float(np.linalg.norm(sla.solve_triangular(R, f, trans="T", lower=False)))
        # the GPU stopped once its ||s_j|| met the tolerance: the true preconditioned residual
        # of its iterate is within the recurrence drift (a few kappa n u) of tol ||s_0||
        assert _precond_residual(p.A, R, sigma2, f, w) <= (tol + 50 * kap * n * ueps) * s0
        # element-wise against the oracle's iterate after the same number of steps
        w_same, _, _ = O.pcgtls(p.A, R, sigma2, f, i_gpu - 1)
        assert _rel(w, w_same) <= 50 * kap * n * ueps


@pytest.mark.parametrize("m,n,u_f,u,cg_tol", [(1000, 130, "fp16", "fp32", 1e-3),
                                              (2500, 300, "bf16", "fp32", 1e-2),
                                              (400, 40, "fp64", "fp64", 1e-6),
                                              (4096, 512, "fp16", "fp32", 1e-4)])
def test_solve_tolerance_mode_matches_oracle(m, n, u_f, u, cg_tol):
    """Full RQI-PCGTLS with the inner solves to a relative tolerance (cg_fixed = 0) against the
    oracle's RQI-PCGTLS in its cg_tol mode: sigma rel <= 1e-10, x rel <= 1e-8."""
    p = synth.dense_problem(m, n, d_lo=1e-3, noise=1e-4, seed=5)
    with Ctx(p.A, p.b, u_f=u_f, u=u, cg_fixed=0, cg_tol=cg_tol, cg_max=40) as ctx:
        x, sigma, info = tls.tls_solve(ctx, tol=0.0, max_rqi=15)
    xo, so, io = O.rqi_pcgtls(p.A, p.b, tol=0.0, max_rqi=15, cg_tol=cg_tol, cg_max=40)
    assert abs(sigma - so) <= 1e-10 * so, (sigma, so, info)
    assert _rel(x, xo) <= 1e-8, info
    assert info["stop_reason"] in (tls.STOP_PSI_UP, tls.STOP_TOL)
    # the inner solves ran to the tolerance, not the fixed k+1 schedule
    fixed = sum(2 * (k + 1) for k in range(1, info["rqi_steps"]))
    assert info["cg_iters"] != fixed or info["rqi_steps"] <= 2


FUSED_SHAPES = [
    # (m, n): n_pad 64 and 704 (8 rows per tile held in shared memory, 4 in registers), 2048
    # (4 rows), 2112 (two float4 groups per thread), 4160 (three groups); m leaves CTAs without
    # rows (m < 152) or gives ragged last tiles
    (100, 40), (3001, 700), (9000, 2048), (5003, 2100), (4500, 4100),
]


@pytest.mark.parametrize("load", [3, 4, 5, 6, 7])
@pytest.mark.parametrize("m,n", FUSED_SHAPES)
def test_one_launch_pcgtls_matches_multi_launch_and_oracle(m, n, load):
    """The one-launch PCGTLS solve (every step's pass over A, reductions and the product with
    (R^T R)^{-1} in one cooperative launch) against the multi-launch path and the oracle with
    the same factor, for every ring geometry, tile loading and tile holding the kernel has; and
    that it is the path that ran."""
    p = synth.dense_problem(m, n, d_lo=1e-2, noise=1e-3, seed=17)
    rng = np.random.default_rng(9)
    f0, f1 = rng.standard_normal(n), rng.standard_normal(n)
    sigma2 = 0.3 * p.D[-1] ** 2
    steps = 6
    out = {}
    for fused in (load, 2):
        with Ctx(p.A, p.b, u_f="fp16", u="fp32", fused=fused) as ctx:
            RH, d, _ = tls.tls_export_factor(ctx)
            tls.tls_profile_enable(ctx, True)
            out[fused] = tls.tls_pcgtls(ctx, sigma2, f0, f1, steps=steps)
            prof = tls.tls_profile_get(ctx)
            tls.tls_profile_enable(ctx, False)
        launched = prof["pcg_solve2"][0]
        assert (launched == 1) if fused != 2 else (launched == 0), prof
    R = RH * d[None, :]
    kap = np.linalg.cond(RH)
    tol = 50 * kap * n * U32
    for f, k in ((f0, 0), (f1, 1)):
        wo, _, _ = O.pcgtls(p.A, R, sigma2, f, steps - 1)
        w_one, w_multi = out[load][k], out[2][k]
        assert _rel(w_one, wo) <= tol
        assert _rel(w_one, w_multi) <= tol
    assert out[load][2] == [steps, steps] and out[load][3] == [0, 0]


def test_one_launch_atomic_form_matches_fixed_order_form():
    """The one-launch solve with A^T t summed by float atomics (reproducible = 0, one grid
    barrier less per step) against the fixed-order form and the oracle; the fixed-order form
    repeats itself bit for bit."""
    m, n = 9000, 2048
    p = synth.dense_problem(m, n, d_lo=1e-2, noise=1e-3, seed=17)
    rng = np.random.default_rng(9)
    f0, f1 = rng.standard_normal(n), rng.standard_normal(n)
    sigma2 = 0.3 * p.D[-1] ** 2
    steps = 6
    out = {}
    for rep in (1, 0):
        with Ctx(p.A, p.b, u_f="fp16", u="fp32", fused=1, reproducible=rep) as ctx:
            RH, d, _ = tls.tls_export_factor(ctx)
            out[rep] = tls.tls_pcgtls(ctx, sigma2, f0, f1, steps=steps)
            if rep:
                again = tls.tls_pcgtls(ctx, sigma2, f0, f1, steps=steps)
                assert all(np.array_equal(a_, b_) for a_, b_ in zip(out[rep][:2], again[:2]))
    R = RH * d[None, :]
    tol = 50 * np.linalg.cond(RH) * n * U32
    for f, k in ((f0, 0), (f1, 1)):
        wo, _, _ = O.pcgtls(p.A, R, sigma2, f, steps - 1)
        assert _rel(out[0][k], wo) <= tol and _rel(out[1][k], wo) <= tol
        assert _rel(out[0][k], out[1][k]) <= tol


@pytest.mark.parametrize("fused", [1, 2])
def test_solve_paths_match_oracle(fused):
    p = synth.dense_problem(6000, 1000, d_lo=1e-3, noise=1e-4, seed=2)
    with Ctx(p.A, p.b, u_f="fp16", u="fp32", fused=fused) as ctx:
        x, sigma, info = tls.tls_solve(ctx, tol=0.0, max_rqi=12)
    xo, so, _ = O.rqi_pcgtls(p.A, p.b, tol=0.0, max_rqi=12)
    assert abs(sigma - so) <= 1e-10 * so, (sigma, so, info)
    assert _rel(x, xo) <= 1e-8, info


def test_pcgtls_flags_indefinite_shift():
    p = synth.dense_problem(300, 40, d_lo=1e-1, noise=1e-3, seed=7)
    with Ctx(p.A, p.b, u_f="fp32", u="fp32") as ctx:
        _, _, it, bad = tls.tls_pcgtls(ctx, 4.0 * p.D[0] ** 2, np.ones(40), None, steps=5)
    assert bad[0] == 1 and it[0] < 5


# ------------------------------------------------------------------------------------------
# full RQI-PCGTLS solves: sigma rel err <= 1e-10, x rel err <= 1e-8 vs the FP64 oracle
# ------------------------------------------------------------------------------------------
CASES = [
    # (m, n, d_lo, noise, u_f, u)
    (400, 40, 1e-2, 1e-6, "fp64", "fp64"),     # the all-FP64 400 x 40 workload
    (400, 40, 1e-2, 1e-6, "fp16", "fp32"),
    (64, 1, 1e-1, 1e-3, "fp16", "fp32"),
    (97, 97, 1e-1, 1e-3, "fp64", "fp64"),      # square
    (400, 40, 1e-2, 1e-6, "fp64", "fp64"),     # the one-CTA solve (n <= 64, FP64)
    (230, 7, 1e-3, 1e-5, "fp64", "fp64"),      # the one-CTA solve, ragged
    (64, 64, 1e-1, 1e-3, "fp64", "fp64"),      # the one-CTA solve, square
    (1000, 130, 1e-3, 1e-4, "fp16", "fp32"),   # ragged n
    (1000, 130, 1e-3, 1e-4, "bf16", "fp32"),
    (2500, 300, 1e-3, 1e-4, "fp16", "fp32"),
    (4096, 512, 1e-3, 1e-4, "fp16", "fp32"),
    (4096, 512, 1e-3, 1e-4, "fp64", "fp64"),
]


@pytest.mark.parametrize("m,n,dlo,noise,u_f,u", CASES)
def test_solve_matches_oracle(m, n, dlo, noise, u_f, u):
    p = synth.dense_problem(m, n, d_lo=dlo, noise=noise, seed=0)
    with Ctx(p.A, p.b, u_f=u_f, u=u) as ctx:
        x, sigma, info = tls.tls_solve(ctx, tol=0.0, max_rqi=12)
    xo, so, io = O.rqi_pcgtls(p.A, p.b, tol=0.0, max_rqi=12)
    # relative 1e-10; for m = n, sigma_{n+1} = 0 exactly and both sides carry only rounding of
    # size u ||[A, b]|| (Weyl), so the bar there is absolute
    atol = 64 * U64 * (np.linalg.norm(p.A) + np.linalg.norm(p.b)) if m == n else 0.0
    assert abs(sigma - so) <= 1e-10 * so + atol, (sigma, so, info)
    assert _rel(x, xo) <= 1e-8, info
    assert info["stop_reason"] in (tls.STOP_PSI_UP, tls.STOP_TOL, tls.STOP_MAX_RQI)


SMALL_CASES = [
    # (m, n, d_lo, noise): dense FP64 problems solved in one launch
    (400, 40, 1e-2, 1e-6),     # the all-FP64 400 x 40 workload (cluster of 16 CTAs)
    (230, 7, 1e-3, 1e-5),      # ragged: 230 rows over 8 CTAs
    (64, 64, 1e-1, 1e-3),      # square, 64 rows: cluster of 4
    (24, 20, 1e-2, 1e-4),      # too few rows for a cluster: one CTA (path 2 refuses)
    (2000, 64, 1e-3, 1e-4),    # 125 rows per CTA, n at the limit; too large for one CTA
]


@pytest.mark.parametrize("m,n,dlo,noise", SMALL_CASES)
@pytest.mark.parametrize("path", [2, 1, 3])
def test_small_paths_match_oracle(path, m, n, dlo, noise):
    """The one-launch solves (on a thread-block cluster, path 2; in one CTA, path 1) and the
    multi-kernel path (3) on the same problems, each against the oracle."""
    p = synth.dense_problem(m, n, d_lo=dlo, noise=noise, seed=4)
    xo, so, _ = O.rqi_pcgtls(p.A, p.b, tol=0.0, max_rqi=12)
    ctx = tls.tls_create_dense(p.A, p.b)
    try:
        assert tls.load().tls_set_small_path(ctx, path) == 0
        tls.tls_factor(ctx, "fp64", tls.tls_default_options(u="fp64"))
        if path == 2 and m // 2 < 16:
            with pytest.raises(tls.TLSError):
                tls.tls_solve(ctx, tol=0.0, max_rqi=12)
            return
        x, sigma, info = tls.tls_solve(ctx, tol=0.0, max_rqi=12)
    finally:
        tls.tls_destroy(ctx)
    one_cta_fits = m * n <= 20000
    if path == 2:
        assert info["pass_variant"][0] == -2 and info["pass_variant"][1] >= 2, info
    elif path == 1 and one_cta_fits:
        assert info["pass_variant"] == [-1, 1], info
    else:
        assert info["pass_variant"][0] >= 0, info
    atol = 64 * U64 * (np.linalg.norm(p.A) + np.linalg.norm(p.b)) if m == n else 0.0
    assert abs(sigma - so) <= 1e-10 * so + atol, (sigma, so, info)
    assert _rel(x, xo) <= 1e-8, info


def test_small_path_argument_checked():
    p = synth.dense_problem(50, 5, seed=1)
    ctx = tls.tls_create_dense(p.A, p.b)
    try:
        assert tls.load().tls_set_small_path(ctx, 4) == 1     # TLS_ERR_ARG
        assert tls.load().tls_set_small_path(ctx, -1) == 1
    finally:
        tls.tls_destroy(ctx)


def test_refactor_with_another_working_precision():
    # the column norms and the FP32 copy of A are computed once per context: a context factored
    # first for u = FP64 (no FP32 copy yet) and then for u = FP32 still solves correctly, and so
    # does a repeat of the first
    p = synth.dense_problem(2500, 300, d_lo=1e-3, noise=1e-4, seed=3)
    xo, so, _ = O.rqi_pcgtls(p.A, p.b, tol=0.0, max_rqi=12)
    ctx = tls.tls_create_dense(p.A, p.b)
    try:
        for u_f, u in (("fp64", "fp64"), ("fp16", "fp32"), ("fp64", "fp64"), ("bf16", "fp32")):
            tls.tls_factor(ctx, u_f, tls.tls_default_options(u=u))
            x, sigma, info = tls.tls_solve(ctx, tol=0.0, max_rqi=12)
            assert abs(sigma - so) <= 1e-10 * so, (u_f, u, info)
            assert _rel(x, xo) <= 1e-8, (u_f, u, info)
    finally:
        tls.tls_destroy(ctx)


def test_solve_before_factor_is_a_state_error():
    p = synth.dense_problem(50, 5, seed=1)
    ctx = tls.tls_create_dense(p.A, p.b)
    try:
        with pytest.raises(tls.TLSError) as e:
            tls.tls_solve(ctx)
        assert e.value.status == 4
    finally:
        tls.tls_destroy(ctx)


def test_solve_to_device_memory_matches_oracle():
    """tls_solve_device writes all n entries of x into a torch CUDA tensor (NaN before the
    solve), and that x is the oracle's; a tensor of another length is refused before the call.
    The problem is one of the host-output cases above."""
    import torch
    p = synth.dense_problem(1000, 130, d_lo=1e-3, noise=1e-4, seed=0)
    xo, so, _ = O.rqi_pcgtls(p.A, p.b, tol=0.0, max_rqi=12)
    with Ctx(p.A, p.b, u_f="fp16", u="fp32") as ctx:
        xd = torch.full((130,), float("nan"), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()   # the fill runs on torch's stream, the solve on the context's
        sigma, info = tls.tls_solve_device(ctx, xd, tol=0.0, max_rqi=12)
        with pytest.raises(tls.TLSError, match="130 entries"):
            tls.tls_solve_device(ctx, torch.zeros(131, dtype=torch.float64, device="cuda"))
    x = xd.cpu().numpy()
    assert np.all(np.isfinite(x))
    assert abs(sigma - so) <= 1e-10 * so, (sigma, so, info)
    assert _rel(x, xo) <= 1e-8, info


@pytest.mark.parametrize("shift_first", [0, 1])
def test_zero_column_breaks_down_then_shifts(shift_first):
    # A zero column makes H singular: the pivot at that column is 0. Started unshifted, the
    # factor breaks down there (reported pivot 7) and takes the shift rung before it succeeds;
    # started from the diagonal perturbation 2 u_f it succeeds at once.
    p = synth.dense_problem(200, 30, d_lo=1e-1, noise=1e-3, seed=2)
    A = p.A.copy()
    A[:, 7] = 0.0
    ctx = tls.tls_create_dense(A, p.b)
    try:
        tls.tls_factor(ctx, "fp16", tls.tls_default_options(shift_first=shift_first, fallback=0))
        x, s, info = tls.tls_solve(ctx, tol=0.0, max_rqi=3)
        assert info["shift"] > 0
        if shift_first:
            assert info["shifts"] == 0 and info["shift"] == pytest.approx(2 * U16)
        else:
            assert info["shifts"] >= 1 and info["fail_pivot"] == 7
    finally:
        tls.tls_destroy(ctx)


@pytest.mark.parametrize("u_f", ["fp16", "bf16"])
@pytest.mark.parametrize("m,n", [(512, 128), (1000, 130), (2100, 300), (1536, 576)])
def test_tensor_core_gram_matches_cuda_core_gram(u_f, m, n):
    # tcgen05 Gram (FP32 accumulation in TMEM) vs the CUDA-core kernel on the same rounded
    # inputs: both are FP32 sums of exact FP16/BF16 products, so they agree to m u_32 |A|^T|A|.
    # Shapes cover ragged n (n not a multiple of the 128-row tile) and m not a multiple of 64.
    p = synth.dense_problem(m, n, d_lo=1e-2, noise=1e-3, seed=9)
    with Ctx(p.A, p.b, u_f=u_f, u="fp32") as ctx:
        _, d, H_tc = tls.tls_export_factor(ctx)
    with Ctx(p.A, p.b, u_f=u_f, u="fp32", gram_simt=1) as ctx:
        _, d2, H_simt = tls.tls_export_factor(ctx)
    assert np.array_equal(d, d2)
    As = _rounded_scaled(p.A, d, u_f)
    bound = m * U32 * (np.abs(As).T @ np.abs(As))
    assert np.all(np.abs(H_tc - H_simt) <= 2 * bound)
    assert np.all(np.abs(H_tc - As.T @ As) <= bound)
    assert np.allclose(H_tc, H_tc.T, rtol=0, atol=0)


# ------------------------------------------------------------------------------------------
# Sec. 3.1 constraint estimates on the GPU vs the oracle's exact SVD values and the paper's
# printed bounds (Examples 1, 2, 3, 5)
# ------------------------------------------------------------------------------------------
from tests.conftest import read_golden  # noqa: E402

_EXAMPLES_GPU = {
    "random_100x60": lambda: synth.random_matrix_problem(seed=0),
    "delta_9x4": lambda: synth.delta_matrix_problem(seed=1),
    "bjorck_30x15": lambda: synth.bjorck_problem(seed=1),
    "van_huffel_100": lambda: synth.van_huffel_problem(seed=1),
}


@pytest.mark.parametrize("row", read_golden("paper_constraint_bounds.txt"), ids=lambda r: r[0])
def test_condition_estimates(row):
    name, c1_paper, c2_paper = row[0], float(row[1]), float(row[2])
    p = _EXAMPLES_GPU[name]()
    with Ctx(p.A, p.b, u_f="fp64", u="fp64") as ctx:
        tls.tls_solve(ctx, tol=0.0, max_rqi=12)
        est = tls.tls_condition(ctx, iters=60)
    c = O.constraints(p.A, p.b)
    # power iterations approach the extreme singular values from inside: kappa from below
    assert 0.5 <= est["kappa"] / c["kappa"] <= 1.0 + 1e-6
    # with an FP64 factor, ||R^{-1}||_F = ||A^+||_F up to rounding
    assert est["kappa_F"] == pytest.approx(c["kappa_F"], rel=1e-8)
    assert est["sigma_n1"] == pytest.approx(c["sigma_n1"], rel=1e-8)
    assert c["constr1"] * (1 - 1e-9) <= est["constr1"] <= 2.0 * c["constr1"]
    f2 = 25.0 if name == "bjorck_30x15" else 2.5
    assert c1_paper / 2.5 <= est["constr1"] <= c1_paper * 2.5
    assert c2_paper / f2 <= est["constr2"] <= c2_paper * f2


def test_condition_estimate_generator_problem():
    # A = Y [diag(D); 0] Z^T: sigma'_1 = 1 and sigma'_n = d_lo exactly
    p = synth.dense_problem(3000, 200, d_lo=1e-3, noise=1e-4, seed=3)
    with Ctx(p.A, p.b, u_f="fp64", u="fp64") as ctx:
        est = tls.tls_condition(ctx, iters=200)
    assert est["sigma1"] == pytest.approx(1.0, rel=5e-3)
    assert est["sigma_n"] == pytest.approx(1e-3, rel=5e-3)
    assert est["norm_F"] == pytest.approx(np.linalg.norm(p.D), rel=1e-12)


@pytest.mark.parametrize("variant", [0, 1, 2, 3])
@pytest.mark.parametrize("m,n", [(3001, 700), (4099, 2048)])
def test_pass_variants_match_oracle(variant, m, n):
    # every kernel the autotuner can pick for the passes over A (register, bulk-copy staged with
    # 256 / 512 threads, pipelined register) against the oracle: the FP64 residual block and a
    # paired PCGTLS solve; ragged row counts
    p = synth.dense_problem(m, n, d_lo=1e-2, noise=1e-3, seed=9)
    rng = np.random.default_rng(4)
    x = p.x_true + 1e-3 * rng.standard_normal(n)
    f0, f1 = rng.standard_normal(n), rng.standard_normal(n)
    sigma2 = 0.3 * p.D[-1] ** 2
    with Ctx(p.A, p.b, u_f="fp16", u="fp32") as ctx:
        if tls.load().tls_set_pass_variant(ctx, variant, variant) != 0:
            pytest.skip("the staged kernel does not fit this n")
        f, sc = tls.tls_residual(ctx, x)
        RH, d, _ = tls.tls_export_factor(ctx)
        w0, w1, it, bad = tls.tls_pcgtls(ctx, sigma2, f0, f1, steps=4)
    r, s2, fo, go, psio = O.residual_block(p.A, p.b, x)
    assert abs(sc["sigma2"] - s2) <= 1e-10 * s2
    fscale = m * U64 * (np.abs(p.A).T @ (np.abs(p.A) @ np.abs(x) + np.abs(p.b))).max()
    assert np.max(np.abs(f - fo)) <= 8 * fscale
    R = RH * d[None, :]
    r0, _, _ = O.pcgtls(p.A, R, sigma2, f0, 3)
    r1, _, _ = O.pcgtls(p.A, R, sigma2, f1, 3)
    tol = 50 * np.linalg.cond(RH) * n * U32
    assert it == [4, 4] and bad == [0, 0]
    assert _rel(w0, r0) <= tol and _rel(w1, r1) <= tol


# ------------------------------------------------------------------------------------------
# fallback triggers: the constraint guard of Sec. 3.1 (Eq. (9)) at factor time, and a stalled or
# indefinite PCGTLS solve during RQI (the precision fallback before max_rqi)
# ------------------------------------------------------------------------------------------
def test_constraint_guard_escalates_a_factor_that_violates_constraint_2():
    # Haar-random Y, Z with kappa(A) = 1e3: column scaling leaves kappa_F(A D^{-1}) near
    # kappa_F(A), so 1 / (sqrt(n) ||R_H^{-1}||_F) falls below u_fp16 and the guard refactors
    p = synth.dense_problem(2000, 200, d_lo=1e-3, noise=1e-4, seed=3, haar=True)
    xo, so, _ = O.rqi_pcgtls(p.A, p.b, tol=0.0, max_rqi=12)
    with Ctx(p.A, p.b, u_f="fp16", u="fp32", constr_guard=1.0) as ctx:
        x, sigma, info = tls.tls_solve(ctx, tol=0.0, max_rqi=12)
    assert info["escalations"] >= 1 and info["u_f_used"] >= tls.TLS_FP32, info
    assert info["fallback_trigger"] == tls.TRIGGER_CONSTRAINT, info
    assert info["constr2_scaled"] < U16
    assert abs(sigma - so) <= 1e-10 * so and _rel(x, xo) <= 1e-8, info


def test_constraint_guard_keeps_a_factor_that_meets_constraint_2():
    # the same size with a single reflector Z: the column scaling equilibrates A, the scaled
    # constraint 2 is above u_fp16 and the FP16 factor stays
    p = synth.dense_problem(2000, 200, d_lo=1e-3, noise=1e-4, seed=3)
    xo, so, _ = O.rqi_pcgtls(p.A, p.b, tol=0.0, max_rqi=12)
    with Ctx(p.A, p.b, u_f="fp16", u="fp32", constr_guard=1.0) as ctx:
        x, sigma, info = tls.tls_solve(ctx, tol=0.0, max_rqi=12)
    assert info["escalations"] == 0 and info["u_f_used"] == tls.TLS_FP16, info
    assert info["constr2_scaled"] > U16
    assert info["fallback_trigger"] == tls.TRIGGER_NONE and info["fallbacks"] == 0
    assert abs(sigma - so) <= 1e-10 * so and _rel(x, xo) <= 1e-8, info


@pytest.mark.parametrize("stall", [1, 0])
def test_stalled_inner_solve_falls_back_before_max_rqi(stall):
    # kappa(A) = 1e4 with Haar Y, Z (noise 1e-6: sigma_{n+1} / sigma'_n = 0.03, a well-posed
    # TLS problem): the FP16 factor leaves PCGTLS with k + 1 steps making no progress (the
    # preconditioned residual grows). With stall_fallback the solve refactors in FP32 at the
    # first stalled pair of solves (trigger STALL or NOT_SPD); without it only after max_rqi
    # steps. Both end at the oracle's answer.
    p = synth.dense_problem(2000, 200, d_lo=1e-4, noise=1e-6, seed=3, haar=True)
    xo, so, _ = O.rqi_pcgtls(p.A, p.b, tol=0.0, max_rqi=12)
    with Ctx(p.A, p.b, u_f="fp16", u="fp32", stall_fallback=stall) as ctx:
        x, sigma, info = tls.tls_solve(ctx, tol=0.0, max_rqi=12)
    assert info["fallbacks"] >= 1 and info["u_f_used"] >= tls.TLS_FP32, info
    if stall:
        assert info["fallback_trigger"] in (tls.TRIGGER_STALL, tls.TRIGGER_NOT_SPD), info
    else:
        assert info["fallback_trigger"] == tls.TRIGGER_MAX_RQI, info
    assert abs(sigma - so) <= 1e-10 * so and _rel(x, xo) <= 1e-8, info


def test_info_reports_the_papers_constraints():
    # Example 1 of Sec. 4 (U(0,1) 100 x 60): tls_info.constr1 / constr2 (Eq. (5), Eq. (9) with
    # the solve's sigma) against the oracle's exact-SVD values
    p = synth.random_matrix_problem(seed=0)
    with Ctx(p.A, p.b, u_f="fp64", u="fp64", constraint_iters=60) as ctx:
        _, sigma, info = tls.tls_solve(ctx, tol=0.0, max_rqi=12)
    c = O.constraints(p.A, p.b)
    assert c["constr1"] * (1 - 1e-9) <= info["constr1"] <= 2.0 * c["constr1"]
    assert info["constr2"] == pytest.approx(c["constr2"], rel=0.5)
    with Ctx(p.A, p.b, u_f="fp64", u="fp64") as ctx:
        _, _, info0 = tls.tls_solve(ctx, tol=0.0, max_rqi=12)
    assert np.isnan(info0["constr1"]) and np.isnan(info0["constr2"])


# ------------------------------------------------------------------------------------------
# Alg. 3 as printed (mode R: the operator I - sigma^2 R^{-T} R^{-1}, no pass over A) as a full
# solve, and the hybrid that starts in that form and switches to the operator with A
# ------------------------------------------------------------------------------------------
@pytest.mark.parametrize("m,n,u", [(1000, 130, "fp64"), (3000, 300, "fp32"), (400, 40, "fp64")])
def test_mode_R_solve_matches_oracle_mode_R(m, n, u):
    # with an FP64 factor, R^T R = A^T A to rounding, and the printed form converges like the
    # operator with A (Sec. 2): against the oracle's mode R run and the closed form
    p = synth.dense_problem(m, n, d_lo=1e-2, noise=1e-5, seed=11)
    with Ctx(p.A, p.b, u_f="fp64", u=u, mode_A=0) as ctx:
        x, sigma, info = tls.tls_solve(ctx, tol=0.0, max_rqi=15)
    xo, so, _ = O.rqi_pcgtls(p.A, p.b, tol=0.0, max_rqi=15, mode="R")
    assert abs(sigma - so) <= 1e-10 * so, (sigma, so, info)
    assert _rel(x, xo) <= 1e-8, info
    assert info["mode_switch_k"] == -1


@pytest.mark.parametrize("u_f", ["fp16", "bf16"])
def test_hybrid_solve_matches_oracle(u_f):
    # u_f = FP16 / BF16: the printed form alone stalls short of the solution (its operator is
    # R^T R, off by about u_f), the hybrid switches to the operator with A and converges
    p = synth.dense_problem(4096, 512, d_lo=1e-3, noise=1e-4, seed=2)
    with Ctx(p.A, p.b, u_f=u_f, u="fp32", mode_A=2) as ctx:
        x, sigma, info = tls.tls_solve(ctx, tol=0.0, max_rqi=20)
    xo, so, _ = O.rqi_pcgtls(p.A, p.b, tol=0.0, max_rqi=20)
    assert abs(sigma - so) <= 1e-10 * so, (sigma, so, info)
    assert _rel(x, xo) <= 1e-8, info
    assert info["mode_switch_k"] >= 2, info


def test_mode_argument_checked():
    p = synth.dense_problem(100, 10, seed=1)
    ctx = tls.tls_create_dense(p.A, p.b)
    try:
        with pytest.raises(tls.TLSError) as e:
            tls.tls_factor(ctx, "fp16", tls.tls_default_options(mode_A=3))
        assert e.value.status == 1
    finally:
        tls.tls_destroy(ctx)
