"""Pins of the FP64 oracle against references that do not use its code.

Each pin follows a statement of Oktay & Carson, arXiv 2305.19028:
* the SVD definition of sigma_{n+1} and x_TLS (Sec. 1),
* the augmented eigenproblem Eq. (1) (closed form via the secular equation, invariants),
* Eq. (2) (f = g = 0 at the solution) and the Rayleigh-quotient identity of Alg. 2,
* special cases (zero noise: sigma_{n+1} = 0 and [E, r] = 0, Sec. 1; n = 1: a 2x2 eigenproblem),
* printed values (Table 2 unit roundoffs, the constraint bounds of Sec. 4, a hand example).
A planted-mistake test at the end checks that these pins catch plausible slips in the oracle.
"""
from __future__ import annotations

import math

import numpy as np
import pytest
import scipy.linalg as sla

import oracle.rqi_pcgtls as O
from paper_2305_19028_gb300 import synth
from tests._pins import U64, kappa_tls, tls_by_secular, tls_by_svd, weyl_sigma_tol
from tests.conftest import read_golden


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


# ------------------------------------------------------------------------------------------
# generator sanity: the SVD of A is known by construction
# ------------------------------------------------------------------------------------------
@pytest.mark.parametrize("m,n", [(30, 7), (64, 64), (200, 33)])
def test_generator_singular_values_are_D(m, n):
    p = synth.dense_problem(m, n, d_lo=1e-3, noise=1e-5, seed=3)
    sv = np.linalg.svd(p.A, compute_uv=False)
    assert np.allclose(sv, p.D, rtol=1e-13, atol=1e-15)
    # right singular vectors are the columns of Z = I - 2 z z^T
    Z = np.eye(n) - 2 * np.outer(p.z, p.z)
    AZ = p.A @ Z
    assert np.allclose(np.linalg.norm(AZ, axis=0), p.D, rtol=1e-12)


# ------------------------------------------------------------------------------------------
# SVD pin on small problems (Sec. 1: x_TLS = -v(1:n, n+1)/v(n+1, n+1))
# ------------------------------------------------------------------------------------------
SMALL = [
    (8, 1, 1e-1, 1e-3, 0),
    (9, 9, 1e-1, 1e-3, 1),      # square
    (40, 17, 1e-2, 1e-4, 2),
    (120, 64, 1e-2, 1e-5, 3),
    (400, 40, 1e-2, 1e-6, 0),   # the 400 x 40 all-FP64 workload
]


@pytest.mark.parametrize("m,n,dlo,noise,seed", SMALL)
@pytest.mark.parametrize("mode", ["A", "R"])
def test_oracle_matches_svd(m, n, dlo, noise, seed, mode):
    p = synth.dense_problem(m, n, d_lo=dlo, noise=noise, seed=seed)
    x, sigma, info = O.rqi_pcgtls(p.A, p.b, tol=0.0, max_rqi=10, mode=mode)
    s_ref, x_ref = tls_by_svd(p.A, p.b)
    # both sides carry FP64 rounding of size ~u ||[A b]|| in sigma (Weyl)
    assert abs(sigma - s_ref) <= weyl_sigma_tol(p.A, p.b) + 1e-13 * s_ref
    kt = kappa_tls(p.A, s_ref)
    assert _rel(x, x_ref) <= max(1e-12, 1e3 * U64 * kt * (1 + np.linalg.norm(p.b)))
    assert info.stop_reason in (O.STOP_PSI_UP, O.STOP_TOL, O.STOP_MAX_RQI)


# ------------------------------------------------------------------------------------------
# secular-equation pin on larger generator problems (closed form, no SVD)
# ------------------------------------------------------------------------------------------
@pytest.mark.parametrize("m,n,dlo,noise", [(400, 40, 1e-2, 1e-6), (2048, 256, 1e-3, 1e-4),
                                           (3000, 500, 1e-3, 1e-4)])
def test_oracle_matches_secular_equation(m, n, dlo, noise):
    p = synth.dense_problem(m, n, d_lo=dlo, noise=noise, seed=0)
    s_ref, x_ref, _ = tls_by_secular(p)
    x, sigma, info = O.rqi_pcgtls(p.A, p.b, tol=0.0, max_rqi=10)
    assert abs(sigma - s_ref) <= weyl_sigma_tol(p.A, p.b) + 1e-13 * s_ref
    kt = p.D[0] / (p.D[-1] - s_ref)
    assert _rel(x, x_ref) <= max(1e-12, 1e3 * U64 * kt * (1 + np.linalg.norm(p.b)))


def test_secular_pin_agrees_with_svd():
    # the two independent references agree with each other
    p = synth.dense_problem(150, 30, d_lo=1e-2, noise=1e-3, seed=5)
    s1, x1, _ = tls_by_secular(p)
    s2, x2 = tls_by_svd(p.A, p.b)
    assert abs(s1 - s2) <= weyl_sigma_tol(p.A, p.b)
    assert _rel(x1, x2) < 1e-10


# ------------------------------------------------------------------------------------------
# invariants at the returned (x, sigma), in extended precision
# ------------------------------------------------------------------------------------------
def test_invariants_at_solution():
    p = synth.dense_problem(1500, 120, d_lo=1e-3, noise=1e-4, seed=7)
    x, sigma, _ = O.rqi_pcgtls(p.A, p.b, tol=0.0, max_rqi=10)
    L = np.longdouble
    A, b, xl, s2 = p.A.astype(L), p.b.astype(L), x.astype(L), L(sigma) ** 2
    r = b - A @ xl
    nA = np.linalg.norm(p.A, 2)
    # Eq. (2): f = -A^T r - sigma^2 x = 0  <=>  (A^T A - sigma^2 I) x = A^T b
    f = -(A.T @ r) - s2 * xl
    assert float(np.linalg.norm(f)) / (nA ** 2 * np.linalg.norm(x) + nA * np.linalg.norm(p.b)) < 1e-13
    # Eq. (2): g = -b^T r + sigma^2 = 0
    assert abs(float(-(b @ r) + s2)) / (np.linalg.norm(p.b) ** 2) < 1e-13
    # Rayleigh quotient identity of Alg. 2: sigma^2 = |r|^2 / (1 + |x|^2)
    assert abs(float((r @ r) / (1 + xl @ xl) - s2)) <= 1e-12 * float(s2)
    # interlacing / uniqueness condition (Sec. 3): sigma_{n+1} < sigma'_n
    assert sigma < np.linalg.svd(p.A, compute_uv=False)[-1]


# ------------------------------------------------------------------------------------------
# special cases
# ------------------------------------------------------------------------------------------
def test_zero_noise_gives_exact_fit():
    # Sec. 1: if sigma_{n+1} = 0 then [E, r] = 0 and x_TLS solves A x = b
    p = synth.dense_problem(200, 20, d_lo=1e-2, noise=0.0, seed=11)
    x, sigma, _ = O.rqi_pcgtls(p.A, p.b, tol=0.0, max_rqi=10)
    assert sigma <= 1e-13 * (np.linalg.norm(p.A) + np.linalg.norm(p.b))
    assert _rel(x, p.x_true) < 1e-11


def test_n_equals_one_closed_form():
    # n = 1: Eq. (1) is the 2x2 eigenproblem [[a.a, a.b], [b.a, b.b]]; sigma_2^2 is its smaller
    # eigenvalue (a quadratic), and x = -v_1 / v_2 for its eigenvector.
    rng = np.random.default_rng(4)
    a = rng.standard_normal(50)
    b = 0.7 * a + 0.05 * rng.standard_normal(50)
    aa, ab, bb = a @ a, a @ b, b @ b
    lam = 0.5 * (aa + bb) - math.sqrt(0.25 * (aa - bb) ** 2 + ab * ab)
    x_ref = ab / (aa - lam)         # first row: (aa - lam) x = ab
    x, sigma, _ = O.rqi_pcgtls(a[:, None], b, tol=0.0, max_rqi=10)
    assert abs(sigma ** 2 - lam) <= 1e-12 * lam
    assert abs(x[0] - x_ref) <= 1e-12 * abs(x_ref)


def test_hand_computed_residual_step():
    vals = {k: float(v) for k, v in read_golden("residual_hand_example.txt")}
    A = np.array([[2.0, 0.0], [0.0, 1.0], [0.0, 0.0]])
    b = np.ones(3)
    r, sigma2, f, g, psi = O.residual_block(A, b, np.array([0.5, 1.0]))
    assert np.allclose(r, [0, 0, 1], atol=0)
    assert sigma2 == pytest.approx(vals["sigma2"], rel=1e-15)
    assert f[0] == pytest.approx(vals["f0"], rel=1e-15)
    assert f[1] == pytest.approx(vals["f1"], rel=1e-15)
    assert g == pytest.approx(vals["g"], rel=1e-15)
    assert psi == pytest.approx(vals["psi"], rel=1e-15)


# ------------------------------------------------------------------------------------------
# Alg. 3 against a direct solve of the shifted system
# ------------------------------------------------------------------------------------------
@pytest.mark.parametrize("mode", ["A", "R"])
def test_pcgtls_converges_to_direct_solution(mode):
    p = synth.dense_problem(300, 50, d_lo=1e-2, noise=1e-3, seed=2)
    R = O.r_factor_qr(p.A)
    s_n = p.D[-1]
    sigma2 = 0.5 * s_n ** 2
    f = np.random.default_rng(1).standard_normal(50)
    w_ref = np.linalg.solve(p.A.T @ p.A - sigma2 * np.eye(50), f)
    # preconditioned spectrum lies in [1 - sigma^2/sigma'_n^2, 1] = [0.5, 1]: fast convergence
    w, it, bad = O.pcgtls(p.A, R, sigma2, f, l=40)
    assert not bad
    assert _rel(w, w_ref) < 1e-11
    # l-step semantics: j = 0..l runs l + 1 steps
    _, it3, _ = O.pcgtls(p.A, R, sigma2, f, l=3)
    assert it3 == 4


def test_pcgtls_modes_agree_for_exact_R():
    # Sec. 2: with R^T R = A^T A, Alg. 3 as printed and the A-explicit operator coincide
    p = synth.dense_problem(200, 30, d_lo=1e-2, noise=1e-3, seed=8)
    R = O.r_factor_cholesky(p.A)
    f = np.random.default_rng(2).standard_normal(30)
    s2 = 0.3 * p.D[-1] ** 2
    wa, _, _ = O.pcgtls(p.A, R, s2, f, l=5, mode="A")
    wr, _, _ = O.pcgtls(p.A, R, s2, f, l=5, mode="R")
    assert _rel(wa, wr) < 1e-10


def test_pcgtls_flags_indefinite_shift():
    # Sec. 3: A^T A - sigma^2 I must be SPD; a shift above sigma'_n^2 breaks it
    p = synth.dense_problem(100, 10, d_lo=1e-1, noise=1e-3, seed=9)
    R = O.r_factor_qr(p.A)
    f = np.ones(10)
    _, _, bad = O.pcgtls(p.A, R, 4.0 * p.D[0] ** 2, f, l=5)
    assert bad


def test_r_factors_agree():
    # Sec. 3: the R of Householder QR equals the Cholesky factor of A^T A (full rank)
    p = synth.dense_problem(80, 20, d_lo=1e-1, noise=1e-3, seed=6)
    Rq = O.r_factor_qr(p.A)
    Rc = O.r_factor_cholesky(p.A)
    assert np.allclose(Rq, np.triu(Rq))
    assert np.all(np.diag(Rq) > 0)
    assert np.allclose(Rq, Rc, rtol=1e-10, atol=1e-12)


def test_ls_solution_matches_lstsq():
    p = synth.dense_problem(90, 25, d_lo=1e-2, noise=1e-2, seed=12)
    x = O.ls_solution(p.A, p.b)
    x_ref = np.linalg.lstsq(p.A, p.b, rcond=None)[0]
    assert _rel(x, x_ref) < 1e-12


# ------------------------------------------------------------------------------------------
# Alg. 3 with a relative tolerance on ||s_j|| (the inexact-solve option, Sec. 3): the stop
# test and the accuracy it implies, from an independent recomputation of the residual
# ------------------------------------------------------------------------------------------
def _precond_residual(A, R, sigma2, f, w):
    """||R^{-T}(f - (A^T A - sigma^2 I) w)||: the s_j that Alg. 3 carries is R^{-T} times the
    residual of its iterate w_j (exact arithmetic), recomputed here from w alone."""
    r = f - (A.T @ (A @ w) - sigma2 * w)
    return float(np.linalg.norm(sla.solve_triangular(R, r, trans="T", lower=False)))


@pytest.mark.parametrize("tol", [1e-3, 1e-8])
@pytest.mark.parametrize("mode", ["A", "R"])
def test_pcgtls_tolerance_mode_stops_at_the_relative_residual(tol, mode):
    p = synth.dense_problem(400, 60, d_lo=1e-2, noise=1e-3, seed=13)
    R = O.r_factor_qr(p.A)
    sigma2 = 0.5 * p.D[-1] ** 2        # preconditioned spectrum in [0.5, 1]
    f = np.random.default_rng(3).standard_normal(60)
    s0 = float(np.linalg.norm(sla.solve_triangular(R, f, trans="T", lower=False)))
    w, it, bad = O.pcgtls(p.A, R, sigma2, f, l=0, mode=mode, cg_tol=tol, cg_max=200)
    assert not bad and 1 <= it < 200
    # the returned iterate meets the tolerance (up to the rounding of the recomputation) ...
    assert _precond_residual(p.A, R, sigma2, f, w) <= tol * s0 * (1 + 1e-6) + 1e-12 * s0
    # ... and the one before it does not (the loop stops at the first step that meets it)
    w_prev, it_prev, _ = O.pcgtls(p.A, R, sigma2, f, l=0, mode=mode, cg_tol=tol, cg_max=it - 1)
    assert it_prev == it - 1
    assert _precond_residual(p.A, R, sigma2, f, w_prev) > tol * s0 * (1 - 1e-6)
    # accuracy implied by the tolerance: ||R (w - w*)|| <= ||s|| / lambda_min(C) with the
    # preconditioned matrix C = I - sigma^2 R^{-T} R^{-1}, lambda_min = 1 - sigma^2/sigma'_n^2
    w_ref = np.linalg.solve(p.A.T @ p.A - sigma2 * np.eye(60), f)
    lam = 1.0 - sigma2 / p.D[-1] ** 2
    assert np.linalg.norm(R @ (w - w_ref)) <= tol * s0 / lam * (1 + 1e-6) + 1e-10 * s0


def test_pcgtls_tolerance_mode_caps_at_cg_max():
    p = synth.dense_problem(400, 60, d_lo=1e-3, noise=1e-3, seed=14)
    R = O.r_factor_cholesky(p.A[:, :]) * (1.0 + 1e-3)   # an inexact factor: slow convergence
    f = np.ones(60)
    _, it, bad = O.pcgtls(p.A, R, 0.1 * p.D[-1] ** 2, f, l=0, cg_tol=1e-30, cg_max=7)
    assert it == 7 and not bad


# ------------------------------------------------------------------------------------------
# the psi stop rule of Sec. 3 (strict) and its >= variant of Sec. 4.2, on a prescribed psi
# sequence: the rule decides from the psi values alone
# ------------------------------------------------------------------------------------------
@pytest.mark.parametrize("ge,stop_k,best_k", [(True, 3, 2), (False, 5, 4)])
def test_psi_rule_on_prescribed_sequence(monkeypatch, ge, stop_k, best_k):
    seq = [5.0, 4.0, 4.0, 3.0, 3.5, 1.0, 0.5]
    real = O.residual_block
    calls = []

    def fake(A, b, x):
        r, s2, f, g, _ = real(A, b, x)
        calls.append(1)
        return r, s2, f, g, seq[len(calls) - 1]

    monkeypatch.setattr(O, "residual_block", fake)
    p = synth.dense_problem(60, 5, d_lo=1e-1, noise=1e-3, seed=2)
    _, _, info = O.rqi_pcgtls(p.A, p.b, tol=0.0, max_rqi=20, psi_rule_ge=ge)
    # Sec. 4.2 stops on psi_{k+1} >= psi_k: at the repeated 4.0 (k = 3), keeping k = 2;
    # Sec. 3 stops on psi_{k+1} > psi_k: at 3.5 (k = 5), keeping the last non-increasing k = 4
    assert info.stop_reason == O.STOP_PSI_UP
    assert info.rqi_steps == stop_k and info.best_k == best_k
    assert info.psi == seq[:stop_k]


def test_psi_rule_ge_never_runs_longer_than_the_strict_rule():
    for seed in range(4):
        p = synth.dense_problem(300, 30, d_lo=1e-2, noise=1e-4, seed=seed)
        _, s_ge, i_ge = O.rqi_pcgtls(p.A, p.b, tol=0.0, max_rqi=15, psi_rule_ge=True)
        _, s_gt, i_gt = O.rqi_pcgtls(p.A, p.b, tol=0.0, max_rqi=15, psi_rule_ge=False)
        assert i_ge.rqi_steps <= i_gt.rqi_steps
        # both end at the TLS solution (the secular-equation closed form)
        s_ref, _, _ = tls_by_secular(p)
        assert abs(s_ge - s_ref) <= weyl_sigma_tol(p.A, p.b) + 1e-13 * s_ref


# ------------------------------------------------------------------------------------------
# the column-scaled Gram matrix and the Cholesky success bounds (Sec. 3.1)
# ------------------------------------------------------------------------------------------
@pytest.mark.parametrize("m,n", [(50, 8), (300, 40)])
def test_scaled_gram_is_the_gram_of_the_equilibrated_columns(m, n):
    rng = np.random.default_rng(m)
    A = rng.standard_normal((m, n)) * 10.0 ** rng.uniform(-3, 2, size=n)
    H, d = O.scaled_gram(A)
    # D holds the column norms; H has a unit diagonal and is symmetric
    assert np.allclose(d, np.linalg.norm(A, axis=0), rtol=1e-14)
    assert np.allclose(np.diag(H), 1.0, rtol=0, atol=1e-14)
    assert np.array_equal(H, H.T)
    # its eigenvalues are the squared singular values of A D^{-1} (an SVD, not a Gram)
    sv = np.linalg.svd(A / np.linalg.norm(A, axis=0), compute_uv=False)
    assert np.allclose(np.sort(np.linalg.eigvalsh(H)), np.sort(sv ** 2), rtol=1e-10, atol=1e-14)


def _two_column_matrix(theta, c1, c2, m=6):
    """Columns c1 e_1 and c2 (cos(theta) e_1 + sin(theta) e_2): the scaled Gram matrix is
    [[1, cos theta], [cos theta, 1]], so lambda_min(H) = 1 - cos(theta) in closed form."""
    A = np.zeros((m, 2))
    A[0, 0] = c1
    A[0, 1] = c2 * math.cos(theta)
    A[1, 1] = c2 * math.sin(theta)
    return A


@pytest.mark.parametrize("theta", [0.3, 1.0, math.pi / 2])
def test_cholesky_bounds_on_known_spectrum(theta):
    A = _two_column_matrix(theta, 3.0, 0.02)
    b = np.array([1.0, -2.0, 0.5, 0.25, 0.0, 1.0])
    c = O.constraints(A, b)
    lam = 1.0 - math.cos(theta)
    n = 2
    # scaled-Cholesky success bound of Sec. 3.1 at the closed-form lambda_min(H)
    assert c["chol_scaled"] == pytest.approx(lam / ((2 * lam + n) * (n + 1)), rel=1e-12)
    # Wilkinson's bound 1/(20 n^{3/2} kappa(A)^2) with kappa from the closed-form 2x2 Gram
    G = np.array([[9.0, 3.0 * 0.02 * math.cos(theta)], [3.0 * 0.02 * math.cos(theta), 4e-4]])
    ev = np.linalg.eigvalsh(G)
    kappa = math.sqrt(ev[-1] / ev[0])
    assert c["kappa"] == pytest.approx(kappa, rel=1e-9)
    assert c["chol_wilkinson"] == pytest.approx(1.0 / (20 * n ** 1.5 * kappa ** 2), rel=1e-9)
    # orthogonal columns (theta = pi/2): H = I, the bound is 1/((2 + n)(n + 1)) whatever the norms
    if theta == math.pi / 2:
        assert c["chol_scaled"] == pytest.approx(1.0 / 12.0, rel=1e-12)
        assert c["kappa"] == pytest.approx(3.0 / 0.02, rel=1e-12)


def test_van_huffel_scaled_gram_closed_form():
    # unperturbed Sec. 4.5 matrix (n x (n-2)): A^T A = n^2 I - n J, diagonal n^2 - n, so
    # H = (n I - J) / (n - 1) with eigenvalues n / (n - 1) (multiplicity n - 3) and
    # (n - (n - 2)) / (n - 1) = 2 / (n - 1)
    n = 40
    p = synth.van_huffel_problem(n=n, eps=0.0)
    H, _ = O.scaled_gram(p.A)
    ev = np.linalg.eigvalsh(H)
    assert ev[0] == pytest.approx(2.0 / (n - 1), rel=1e-12)
    assert np.allclose(ev[1:], n / (n - 1), rtol=1e-12)
    c = O.constraints(p.A, p.b)
    lam = 2.0 / (n - 1)
    assert c["chol_scaled"] == pytest.approx(lam / ((2 * lam + (n - 2)) * (n - 1)), rel=1e-12)


# ------------------------------------------------------------------------------------------
# printed values of the paper
# ------------------------------------------------------------------------------------------
def test_table2_unit_roundoffs():
    rows = {k: float(v) for k, v in read_golden("table2_unit_roundoff.txt")}
    for name, dt in (("fp16", np.float16), ("fp32", np.float32), ("fp64", np.float64)):
        u = float(np.finfo(dt).eps) / 2
        assert u == pytest.approx(rows[name], rel=5e-3)
    assert 2.0 ** -113 == pytest.approx(rows["fp128"], rel=5e-3)


_EXAMPLES = {
    "random_100x60": lambda: synth.random_matrix_problem(seed=0),
    "delta_9x4": lambda: synth.delta_matrix_problem(seed=1),
    "bjorck_30x15": lambda: synth.bjorck_problem(seed=1),
    "van_huffel_100": lambda: synth.van_huffel_problem(seed=1),
}


@pytest.mark.parametrize("row", read_golden("paper_constraint_bounds.txt"), ids=lambda r: r[0])
def test_constraint_bounds_order_of_magnitude(row):
    name, c1, c2 = row[0], float(row[1]), float(row[2])
    p = _EXAMPLES[name]()
    c = O.constraints(p.A, p.b)
    assert c1 / 2.5 <= c["constr1"] <= c1 * 2.5
    # constr2 of the Bjorck example depends strongly on the random draw (sigma_{n+1}/sigma'_n is
    # close to 1), so only its order of magnitude is pinned there
    f2 = 25.0 if name == "bjorck_30x15" else 2.5
    assert c2 / f2 <= c["constr2"] <= c2 * f2


def test_van_huffel_condition_closed_form():
    # A^T A = n^2 I - n J for the unperturbed Sec. 4.5 matrix, so kappa(A) = sqrt(n / 2)
    p = synth.van_huffel_problem(n=100, eps=0.0)
    c = O.constraints(p.A, p.b)
    assert c["kappa"] == pytest.approx(math.sqrt(50.0), rel=1e-12)


# ------------------------------------------------------------------------------------------
# planted mistakes: each must be caught by at least one of the pins above
# ------------------------------------------------------------------------------------------
_ORIG_RESIDUAL = O.residual_block


def _mut_f_sign(A, b, x):
    r, s2, f, g, psi = _ORIG_RESIDUAL(A, b, x)
    return r, s2, f + 2 * s2 * x, g, psi


def _mut_g_sign(A, b, x):
    r, s2, f, g, psi = _ORIG_RESIDUAL(A, b, x)
    return r, s2, f, g + 2 * (b @ r), psi


def _mut_rq(A, b, x):
    r = b - A @ x
    s2 = (r @ r) / (x @ x)                      # dropped the +1 of the Rayleigh quotient
    f = -(A.T @ r) - s2 * x
    g = -(b @ r) + s2
    return r, s2, f, g, math.sqrt((f @ f + g * g) / (x @ x + 1))


def _mut_delta(A, R, sigma2, st, mode="A"):
    # dropped the shift term of delta_j
    p = st["p"]
    q = sla.solve_triangular(R, p, lower=False)
    t = A @ q
    delta = float(t @ t)
    alpha = st["eta"] / delta
    v = sla.solve_triangular(R, A.T @ t - sigma2 * q, trans="T", lower=False)
    s = st["s"] - alpha * v
    eta = float(s @ s)
    return {"w": st["w"] + alpha * q, "s": s, "p": s + eta / st["eta"] * p, "eta": eta}, delta


def _mut_transposed_solve(A, R, sigma2, st, mode="A"):
    # R^{-1} where Alg. 3 applies R^{-T}
    p = st["p"]
    q = sla.solve_triangular(R, p, lower=False)
    t = A @ q
    delta = float(t @ t - sigma2 * (q @ q))
    alpha = st["eta"] / delta
    v = sla.solve_triangular(R, A.T @ t - sigma2 * q, lower=False)
    s = st["s"] - alpha * v
    eta = float(s @ s)
    return {"w": st["w"] + alpha * q, "s": s, "p": s + eta / st["eta"] * p, "eta": eta}, delta


def _pins_pass() -> bool:
    try:
        test_oracle_matches_secular_equation(400, 40, 1e-2, 1e-6)
        test_oracle_matches_secular_equation(2048, 256, 1e-3, 1e-4)
        test_pcgtls_converges_to_direct_solution("A")
        test_n_equals_one_closed_form()
        test_hand_computed_residual_step()
    except AssertionError:
        return False
    return True


@pytest.mark.parametrize("target,mutant", [
    ("residual_block", _mut_f_sign), ("residual_block", _mut_g_sign),
    ("residual_block", _mut_rq), ("pcgtls_step", _mut_delta),
    ("pcgtls_step", _mut_transposed_solve)])
def test_planted_mistakes_are_caught(monkeypatch, target, mutant):
    assert _pins_pass()
    monkeypatch.setattr(O, target, mutant)
    assert not _pins_pass(), f"planted mistake in {target} went unnoticed"


# ------------------------------------------------------------------------------------------
# selector network oracle: backpropagation pinned by central finite differences
# ------------------------------------------------------------------------------------------
def test_mlp_oracle_gradient_matches_finite_differences():
    import oracle.mlp as M
    rng = np.random.Generator(np.random.PCG64(7))
    P = rng.normal(0.0, 0.3, size=M.N_PARAMS)
    X = rng.normal(size=(6, M.N_IN))
    y = rng.integers(0, 3, size=6)
    t = rng.normal(size=6)
    mask = np.array([1.0, 0.0, 1.0, 1.0, 0.0, 1.0])
    lam = 0.7
    _, g = M.loss_and_grad(P, X, y, t, mask, lam)
    assert g.shape == (M.N_PARAMS,)
    h = 1e-6
    for k in rng.choice(M.N_PARAMS, size=300, replace=False):
        e = np.zeros(M.N_PARAMS)
        e[k] = h
        fd = (M.loss_and_grad(P + e, X, y, t, mask, lam)[0] -
              M.loss_and_grad(P - e, X, y, t, mask, lam)[0]) / (2 * h)
        assert abs(fd - g[k]) <= 1e-7 + 1e-5 * abs(fd), (k, fd, g[k])


def test_mlp_oracle_special_cases():
    import oracle.mlp as M
    # zero weights: uniform softmax, loss log 3 plus the regression term on out[3] = 0
    P = np.zeros(M.N_PARAMS)
    X = np.ones((4, M.N_IN))
    y = np.array([0, 1, 2, 0])
    t = np.array([1.0, -2.0, 0.5, 0.0])
    L, g = M.loss_and_grad(P, X, y, t, np.ones(4), 0.5)
    assert L == pytest.approx(np.log(3.0) + 0.5 * np.mean(t ** 2), rel=1e-14)
    # the bias gradient of the logits is the mean of (softmax - one-hot): (1/3 - freq)
    b3 = g[-4:]
    assert b3[:3] == pytest.approx([1 / 3 - 2 / 4, 1 / 3 - 1 / 4, 1 / 3 - 1 / 4], abs=1e-15)
    assert b3[3] == pytest.approx(2 * 0.5 * np.mean(0.0 - t), abs=1e-15)
    # FP16 storage: the forward pass equals the FP64 pass on the rounded weights
    rng = np.random.Generator(np.random.PCG64(3))
    P = rng.normal(0.0, 0.5, size=M.N_PARAMS)
    Ph = P.astype(np.float32).astype(np.float16).astype(np.float64)
    assert np.array_equal(M.forward(P, X, fp16=True)[0], M.forward(Ph, X)[0])


def test_oracle_on_sparse_input_matches_dense_input():
    # the oracle only applies A and A^T: a scipy CSR matrix with the Cholesky R and the
    # normal-equation start gives the dense QR run's result (same exact-arithmetic method)
    sp = pytest.importorskip("scipy.sparse")
    p = synth.csr_problem(3000, 200, nnz_per_row=12, noise=1e-3, seed=0)
    A = sp.csr_matrix((p.val, p.col_idx, p.row_ptr), shape=(p.m, p.n))
    R = O.r_factor_cholesky(A)
    x0 = sla.solve_triangular(R, sla.solve_triangular(R, A.T @ p.b, trans="T"))
    x1, s1, _ = O.rqi_pcgtls(A, p.b, R=R, x0=x0, tol=0.0, max_rqi=12)
    x2, s2, _ = O.rqi_pcgtls(A.toarray(), p.b, tol=0.0, max_rqi=12)
    assert abs(s1 - s2) <= 1e-12 * s2
    assert np.linalg.norm(x1 - x2) <= 1e-10 * np.linalg.norm(x2)


# planted mistakes in the parts pinned above: each must fail one of those pins
_ORIG_SCALED_GRAM = O.scaled_gram
_ORIG_CONSTRAINTS = O.constraints
_ORIG_PCGTLS = O.pcgtls
_ORIG_RQI = O.rqi_pcgtls


def _mut_one_sided_scaling(A):
    G = A.T @ A
    d = np.sqrt(np.diag(G))
    return G / d[:, None] ** 2, d                  # D^{-2} G instead of D^{-1} G D^{-1}


def _mut_lambda_max(A, b, n_plus_1_sigma=None):
    c = _ORIG_CONSTRAINTS(A, b, n_plus_1_sigma)
    n = A.shape[1]
    H, _ = O.scaled_gram(A)
    lam = np.linalg.eigvalsh(H)[-1]                # largest instead of smallest eigenvalue
    c["chol_scaled"] = lam / ((2.0 * lam + n) * (n + 1))
    return c


def _mut_tol_on_eta(A, R, sigma2, f, l, mode="A", cg_tol=None, cg_max=None):
    # compares eta = ||s||^2 with tol * ||s_0|| (a dropped square root)
    return _ORIG_PCGTLS(A, R, sigma2, f, l, mode, None if cg_tol is None else cg_tol ** 2,
                        cg_max)


def _mut_ge_as_gt(*a, **k):
    k["psi_rule_ge"] = False
    return _ORIG_RQI(*a, **k)


def _new_pins_pass(monkeypatch_fixture=None) -> bool:
    try:
        test_scaled_gram_is_the_gram_of_the_equilibrated_columns(50, 8)
        test_cholesky_bounds_on_known_spectrum(0.3)
        test_van_huffel_scaled_gram_closed_form()
        test_pcgtls_tolerance_mode_stops_at_the_relative_residual(1e-3, "A")
    except AssertionError:
        return False
    return True


@pytest.mark.parametrize("target,mutant", [
    ("scaled_gram", _mut_one_sided_scaling), ("constraints", _mut_lambda_max),
    ("pcgtls", _mut_tol_on_eta)])
def test_planted_mistakes_in_scaling_bounds_and_tolerance_are_caught(monkeypatch, target, mutant):
    assert _new_pins_pass()
    monkeypatch.setattr(O, target, mutant)
    assert not _new_pins_pass(), f"planted mistake in {target} went unnoticed"


def test_planted_psi_rule_mistake_is_caught(monkeypatch):
    # a >= rule that behaves like > must fail the prescribed-sequence pin
    seq = [5.0, 4.0, 4.0, 3.0, 3.5, 1.0, 0.5]
    real = O.residual_block
    calls = []

    def fake(A, b, x):
        r, s2, f, g, _ = real(A, b, x)
        calls.append(1)
        return r, s2, f, g, seq[len(calls) - 1]

    monkeypatch.setattr(O, "residual_block", fake)
    p = synth.dense_problem(60, 5, d_lo=1e-1, noise=1e-3, seed=2)
    _, _, info = _mut_ge_as_gt(p.A, p.b, tol=0.0, max_rqi=20, psi_rule_ge=True)
    assert (info.rqi_steps, info.best_k) != (3, 2)
