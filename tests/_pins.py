"""Independent references ("pins") for the oracle: closed forms from the SVD of [A, b]
(Sec. 1) and the augmented eigenproblem, Eq. (1), evaluated without the oracle's code."""
from __future__ import annotations

import numpy as np

U64 = np.finfo(np.float64).eps / 2


def tls_by_svd(A: np.ndarray, b: np.ndarray):
    """sigma_{n+1} and x_TLS = -v(1:n, n+1) / v(n+1, n+1) from the SVD of [A, b] (Sec. 1)."""
    M = np.column_stack([A, b])
    _, S, Vt = np.linalg.svd(M, full_matrices=True)
    v = Vt[-1]
    # for m = n, [A, b] has a null vector and sigma_{n+1} = 0
    s = S[-1] if M.shape[0] >= M.shape[1] else 0.0
    return s, -v[:-1] / v[-1]


def tls_by_secular(p):
    """Closed form for A = Y [diag(D); 0] Z^T with single Householder reflectors Y, Z.

    With A = U_1 diag(D) Z^T (U_1 = first n columns of Y) and c = U_1^T b, the second block
    row of Eq. (1) gives lambda = b^T b - b^T A x and the first gives
    x = Z diag(D) (diag(D)^2 - lambda I)^{-1} c. Substituting, lambda = sigma_{n+1}^2 is the
    root in (0, D_min^2) of phi(l) = b^T b - l - sum_i D_i^2 c_i^2 / (D_i^2 - l), which is
    strictly decreasing there (phi(0) = |b|^2 - |c|^2 >= 0). Bisection in long double."""
    L = np.longdouble
    D = p.D.astype(L)
    y = p.y.astype(L)
    z = p.z.astype(L)
    b = p.b.astype(L)
    n = D.shape[0]
    c = b[:n] - 2 * y[:n] * (y @ b)
    D2 = D * D
    bb = b @ b

    def phi(lam):
        return bb - lam - np.sum(D2 * c * c / (D2 - lam))

    lo, hi = L(0), D2.min()
    for _ in range(400):
        mid = (lo + hi) / 2
        if mid == lo or mid == hi:
            break
        if phi(mid) > 0:
            lo = mid
        else:
            hi = mid
    lam = (lo + hi) / 2
    w = D * c / (D2 - lam)
    x = w - 2 * z * (z @ w)
    return float(np.sqrt(lam)), x.astype(np.float64), float(lam)


def weyl_sigma_tol(A, b, c: float = 64.0) -> float:
    """Absolute tolerance on sigma_{n+1} from Weyl's bound |d sigma| <= ||d[A, b]||_2 for
    perturbations of the size of FP64 rounding of the data and of a backward-stable solve."""
    return c * U64 * (np.linalg.norm(A) + np.linalg.norm(b))


def kappa_tls(A, sigma_n1) -> float:
    """kappa_TLS = sigma'_1 / (sigma'_n - sigma_{n+1}) (Sec. 1)."""
    sv = np.linalg.svd(A, compute_uv=False)
    return sv[0] / (sv[-1] - sigma_n1)
