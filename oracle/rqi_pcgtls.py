"""Plain FP64 CPU oracle for RQI-PCGTLS (Oktay & Carson, arXiv 2305.19028).

TEST INFRASTRUCTURE ONLY. It is imported by ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py``; the library's solve path never imports it and
shares no code with it (it uses numpy/scipy only).

Everything here runs in IEEE double precision and follows the paper's algorithms step by step
in the paper's order and notation:

* Alg. 2 (RQI for TLS, Sec. 2) / Alg. 4 (RQI-PCGTLS-MP, Sec. 3) with every precision set to
  double: the outer Rayleigh quotient iteration.
* Alg. 3 (l-step PCGTLS, Sec. 2): the inner preconditioned CG for (A^T A - sigma^2 I) w = f.
* Eq. (4): the normalised residual psi_k and the stop rule psi_{k+1} > psi_k (Sec. 3).
* Sec. 1: the LS start x_LS = R^{-1} Q_1^T b from a Householder QR of A.
* Sec. 3: the preconditioner R from Householder QR of A (the paper's default) or the Cholesky
  factor of A^T A (the alternative the paper discusses), and the column-scaled Gram matrix
  H = D^{-1} fl(A^T A) D^{-1} with D = sqrt(diag(A^T A)).
* Sec. 3.1: the two constraints on the factorisation precision, Eq. (5) and Eq. (9), and the
  scaled-Cholesky success bound, evaluated from their definitions with an exact SVD.

Readings of the paper taken here, where it is silent, garbled or ambiguous:

* PCGTLS operator, "mode A" (default): delta_j = ||A q_j||^2 - sigma^2 ||q_j||^2 and
  s_{j+1} = s_j - alpha_j R^{-T}(A^T A q_j - sigma^2 q_j). Alg. 3 as printed ("mode R") uses
  ||p_j||^2 and p_j for those two terms, which is the same when R^T R = A^T A exactly.
* Alg. 3's loop "j = 0..l" runs l+1 steps; RQI step k uses l = k (k+1 steps, Alg. 4). An
  optional relative tolerance on ||s_j|| / ||s_0|| stops earlier. delta_j <= 0 stops the loop
  and flags loss of positive definiteness.
* Alg. 2 line "f_k = -A^T r_k - sigma_k^2 x" uses x = x_k.
* Stop at the first of: psi_k <= tol * (||A||_F^2 + ||b||^2) for k >= 2; psi_k > psi_{k-1}
  (or >= when ``psi_rule_ge``); k > max_rqi. The iterate with the smallest psi is returned with
  sigma = sqrt(sigma_k^2) of that iterate. The tolerance test starts at k = 2: psi_1 is taken at
  the inverse-iteration start x_1 (Alg. 2, before the loop), whose error is only first order in
  psi_1, so a small psi_1 (a small sigma_{n+1}) does not make x_1 accurate.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import scipy.linalg as sla

__all__ = ["OracleInfo", "r_factor_qr", "r_factor_cholesky", "ls_solution", "scaled_gram",
           "pcgtls_init", "pcgtls_step", "pcgtls", "rqi_pcgtls", "residual_block", "constraints",
           "STOP_TOL", "STOP_PSI_UP",
           "STOP_MAX_RQI"]

STOP_TOL = 1        # psi_k <= tol * scale
STOP_PSI_UP = 2     # psi_k > psi_{k-1}  (Sec. 3, after Eq. (4))
STOP_MAX_RQI = 3    # k reached max_rqi


# --------------------------------------------------------------------------------------------
# Preconditioner R (Sec. 3)
# --------------------------------------------------------------------------------------------
def r_factor_qr(A: np.ndarray) -> np.ndarray:
    """R of the Householder QR A = Q [R; 0] (Alg. 4, step 'Compute A = Q[R 0]^T'), in FP64,
    with the signs normalised so that diag(R) > 0 (then R is the Cholesky factor of A^T A,
    Sec. 3)."""
    R = np.linalg.qr(A, mode="r")
    s = np.sign(np.diag(R))
    s[s == 0] = 1.0
    return np.triu(R * s[:, None])


def _is_sparse(A) -> bool:
    return hasattr(A, "tocsr")


def r_factor_cholesky(A) -> np.ndarray:
    """Upper-triangular Cholesky factor of A^T A (the alternative preconditioner, Sec. 3).
    A may be dense or a scipy sparse matrix (A^T A is then formed sparse and factored dense)."""
    G = A.T @ A
    if _is_sparse(G):
        G = G.toarray()
    return np.linalg.cholesky(G).T


def scaled_gram(A: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """H = D^{-1} (A^T A) D^{-1} with D = diag(sqrt(diag(A^T A))) (two-sided diagonal scaling,
    Sec. 3.1). Returns (H, d) with d the diagonal of D."""
    G = A.T @ A
    d = np.sqrt(np.diag(G))
    return G / np.outer(d, d), d


def ls_solution(A: np.ndarray, b: np.ndarray) -> np.ndarray:
    """x_LS = R^{-1} Q_1^T b from the Householder QR of A (Sec. 1)."""
    Q1, R = np.linalg.qr(A, mode="reduced")
    return sla.solve_triangular(R, Q1.T @ b, lower=False)


# --------------------------------------------------------------------------------------------
# Alg. 3: l-step PCGTLS
# --------------------------------------------------------------------------------------------
def pcgtls_init(R: np.ndarray, f: np.ndarray) -> dict:
    """Alg. 3 initialisation: w_0 = 0, p_0 = s_0 = R^{-T} f, eta_0 = ||s_0||^2."""
    s = sla.solve_triangular(R, f, trans="T", lower=False)
    return {"w": np.zeros(R.shape[0]), "s": s, "p": s.copy(), "eta": float(s @ s)}


def pcgtls_step(A: np.ndarray | None, R: np.ndarray, sigma2: float, st: dict,
                mode: str = "A") -> tuple[dict, float]:
    """One pass j of the Alg. 3 loop. Returns (new state, delta_j); when delta_j <= 0 the
    state is returned unchanged (the loop ends there)."""
    p, s, w, eta = st["p"], st["s"], st["w"], st["eta"]
    q = sla.solve_triangular(R, p, lower=False)                 # q_j = R^{-1} p_j
    if mode == "A":
        t = A @ q
        delta = float(t @ t - sigma2 * (q @ q))                 # ||A q_j||^2 - sigma^2 ||q_j||^2
    else:
        delta = float(p @ p - sigma2 * (q @ q))                 # ||p_j||^2 - sigma^2 ||q_j||^2
    if delta <= 0.0:
        return st, delta
    alpha = eta / delta                                          # alpha_j = eta_j / delta_j
    w = w + alpha * q                                            # w_{j+1} = w_j + alpha_j q_j
    if mode == "A":
        v = sla.solve_triangular(R, A.T @ t - sigma2 * q, trans="T", lower=False)
    else:
        v = p - sigma2 * sla.solve_triangular(R, q, trans="T", lower=False)
    s = s - alpha * v                                            # s_{j+1}
    eta_new = float(s @ s)                                       # eta_{j+1} = ||s_{j+1}||^2
    beta = eta_new / eta                                         # beta_j = eta_{j+1} / eta_j
    p = s + beta * p                                             # p_{j+1} = s_{j+1} + beta_j p_j
    return {"w": w, "s": s, "p": p, "eta": eta_new}, delta


def pcgtls(A: np.ndarray | None, R: np.ndarray, sigma2: float, f: np.ndarray, l: int,
           mode: str = "A", cg_tol: float | None = None, cg_max: int | None = None):
    """Approximately solve (A^T A - sigma2 I) w = f by Alg. 3, preconditioned with R.

    mode "A": the operator applies A (see module docstring); mode "R": Alg. 3 as printed.
    Runs j = 0..l (l+1 steps) unless ``cg_tol`` is given, in which case it runs until
    ||s_{j+1}|| <= cg_tol * ||s_0|| or ``cg_max`` steps.
    Returns (w, iterations, not_spd).
    """
    st = pcgtls_init(R, f)
    eta0 = st["eta"]
    steps = (l + 1) if cg_tol is None else (cg_max if cg_max is not None else 10 * R.shape[0])
    it = 0
    not_spd = False
    for _ in range(steps):
        if st["eta"] == 0.0:
            break
        st, delta = pcgtls_step(A, R, sigma2, st, mode)
        if delta <= 0.0:                                         # Alg. 3: "while delta_j != 0"
            not_spd = delta < 0.0
            break
        it += 1
        if cg_tol is not None and math.sqrt(st["eta"]) <= cg_tol * math.sqrt(eta0):
            break
    return st["w"], it, not_spd


# --------------------------------------------------------------------------------------------
# Alg. 2 / Alg. 4: RQI for TLS
# --------------------------------------------------------------------------------------------
def residual_block(A: np.ndarray, b: np.ndarray, x: np.ndarray):
    """One RQI residual step (Alg. 2 lines 'r_k' .. 'g_k', Eq. (2), Eq. (4)):
    r = b - A x, sigma2 = r^T r / (1 + x^T x), f = -A^T r - sigma2 x, g = -b^T r + sigma2,
    psi = sqrt((||f||^2 + g^2) / (||x||^2 + 1)). Returns (r, sigma2, f, g, psi)."""
    r = b - A @ x
    xx = x @ x
    sigma2 = (r @ r) / (1.0 + xx)
    f = -(A.T @ r) - sigma2 * x
    g = -(b @ r) + sigma2
    psi = math.sqrt((f @ f + g * g) / (xx + 1.0))
    return r, sigma2, f, g, psi


@dataclasses.dataclass
class OracleInfo:
    stop_reason: int
    rqi_steps: int               # RQI loop iterations whose residual was evaluated
    cg_iters: int                # total PCGTLS steps over both solves of every RQI step
    not_spd: bool
    psi: list                    # psi_k for k = 1, 2, ...
    sigma2: list                 # sigma_k^2 for k = 1, 2, ...
    best_k: int                  # index (1-based) of the returned iterate


def rqi_pcgtls(A: np.ndarray, b: np.ndarray, R: np.ndarray | None = None,
               x0: np.ndarray | None = None, tol: float = 1e-12, max_rqi: int = 10,
               mode: str = "A", cg_tol: float | None = None, cg_max: int | None = None,
               psi_rule_ge: bool = False):
    """RQI-PCGTLS in FP64 (Alg. 2 with the solves of Alg. 3, i.e. Alg. 4 at u = u_p = u_q =
    double). Returns (x, sigma, info). A may be a scipy sparse matrix: the method only applies
    A and A^T to vectors (then R and x0 must be given)."""
    sparse = _is_sparse(A)
    if sparse:
        A = A.tocsr().astype(np.float64)
        if R is None or x0 is None:
            raise ValueError("a sparse A needs R and x0")
    else:
        A = np.asarray(A, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    if R is None:
        R = r_factor_qr(A)
    # lines 1-5: LS start, one inverse-iteration step
    x = ls_solution(A, b) if x0 is None else np.array(x0, dtype=np.float64)
    r0 = b - A @ x
    sigma2_0 = (r0 @ r0) / (1.0 + x @ x)
    u0 = sla.solve_triangular(R, sla.solve_triangular(R, x, trans="T", lower=False),
                              lower=False)                       # A^T A u_0 = x_0 via R^T R
    x = x + sigma2_0 * u0
    scale = float((A.multiply(A).sum() if sparse else np.sum(A * A)) + b @ b)
    best = None
    psis, sig2s = [], []
    prev_psi = math.inf
    cg_total = 0
    not_spd = False
    stop = STOP_MAX_RQI
    k = 0
    while True:
        k += 1
        r, sigma2, f, g, psi = residual_block(A, b, x)
        psis.append(psi)
        sig2s.append(sigma2)
        increased = (psi >= prev_psi) if psi_rule_ge else (psi > prev_psi)
        if increased:
            stop = STOP_PSI_UP
            break
        best = (k, x.copy(), sigma2)
        if k >= 2 and psi <= tol * scale:
            stop = STOP_TOL
            break
        if k > max_rqi:
            stop = STOP_MAX_RQI
            break
        prev_psi = psi
        # solve (A^T A - sigma_k^2 I) w_k = -f_k
        w, it1, bad1 = pcgtls(A, R, sigma2, -f, k, mode, cg_tol, cg_max)
        z = x + w
        beta = (z @ f - g) / (z @ x + 1.0)
        # solve (A^T A - sigma_k^2 I) u_k = x_k
        u, it2, bad2 = pcgtls(A, R, sigma2, x, k, mode, cg_tol, cg_max)
        cg_total += it1 + it2
        not_spd = not_spd or bad1 or bad2
        x = z + beta * u
    bk, bx, bs2 = best
    info = OracleInfo(stop_reason=stop, rqi_steps=k, cg_iters=cg_total, not_spd=not_spd,
                      psi=psis, sigma2=sig2s, best_k=bk)
    return bx, math.sqrt(max(bs2, 0.0)), info


# --------------------------------------------------------------------------------------------
# Sec. 3.1: constraints on the factorisation precision
# --------------------------------------------------------------------------------------------
def constraints(A: np.ndarray, b: np.ndarray, n_plus_1_sigma: float | None = None) -> dict:
    """Evaluate, from an exact SVD, the heuristic constraints of Sec. 3.1:
    constr1 = kappa(A)^{-1} (Eq. (5)); constr2 = kappa_F(A)^{-1} (1 - sigma_{n+1}^2/sigma'_n^2)
    (Eq. (9)); the scaled-Cholesky success bound lambda_min(H)/((2 lambda_min(H) + n)(n+1));
    and Wilkinson's 1/(20 n^{3/2} kappa(A)^2)."""
    n = A.shape[1]
    sv = np.linalg.svd(A, compute_uv=False)
    if n_plus_1_sigma is None:
        n_plus_1_sigma = np.linalg.svd(np.column_stack([A, b]), compute_uv=False)[-1]
    kappa = sv[0] / sv[-1]
    kappa_f = math.sqrt(np.sum(sv ** 2)) * math.sqrt(np.sum(sv ** -2.0))
    H, _ = scaled_gram(A)
    lam = np.linalg.eigvalsh(H)[0]
    return {
        "kappa": kappa,
        "kappa_F": kappa_f,
        "sigma_n1": n_plus_1_sigma,
        "sigma_n_prime": sv[-1],
        "constr1": 1.0 / kappa,
        "constr2": (1.0 - n_plus_1_sigma ** 2 / sv[-1] ** 2) / kappa_f,
        "chol_scaled": lam / ((2.0 * lam + n) * (n + 1)),
        "chol_wilkinson": 1.0 / (20.0 * n ** 1.5 * kappa ** 2),
    }
