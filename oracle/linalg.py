"""Householder QR, the OLS estimator and the preconditioner factor
(oracle side; test infrastructure).

* ``householder_qr``: unblocked Householder QR written out column by column
  (the textbook algorithm; Golub & Van Loan, Alg. 5.2.1), R with a
  non-negative diagonal.  Used on small and moderate sizes.
* ``r_factor``: the R factor of a tall matrix with diag(R) >= 0, by LAPACK's
  Householder QR (dgeqrf) as a single library step.  The paper applies the
  sketched-Hessian preconditioner H-hat = (S-hat X)^T (S-hat X) "through a QR
  factorization" (Sec. 4, experimental setup): H-hat = R^T R.
* ``ols``: the OLS estimator of Eq. (ols), beta-hat = argmin ||Y - X u||,
  by Householder QR: beta-hat = R^{-1} (Q^T Y).
* ``apply_precond``: z = H-hat^{-1} g = R^{-1} (R^{-T} g) by two triangular
  solves.

Pins (tests/test_oracle_linalg.py): normal equations solved in 80-bit long
double for N <= 64; the invariant X^T (Y - X beta-hat) ~ 0 at the u_64
level; ||Q^T Q - I|| and ||Q R - A|| at the u_64 level; the plain and the
LAPACK factor agree; Monte Carlo E||X(beta-hat - beta)||^2 = sigma^2 d.
"""
import numpy as np
from scipy.linalg import solve_triangular


def _sign_fix(R, Q=None):
    s = np.sign(np.diag(R)).copy()
    s[s == 0] = 1.0
    R = s[:, None] * R
    if Q is not None:
        Q = Q * s[None, :]
    return R, Q


def householder_qr(A):
    """Thin Q (m x n) and R (n x n, diag >= 0) of A (m >= n), unblocked."""
    A = np.array(A, dtype=np.float64, copy=True)
    m, n = A.shape
    if m < n:
        raise ValueError("need m >= n")
    reflectors = []
    for k in range(n):
        x = A[k:, k]
        normx = np.linalg.norm(x)
        alpha = -normx if x[0] >= 0 else normx
        v = x.copy()
        v[0] -= alpha
        vv = v @ v
        if vv > 0:
            A[k:, k:] -= np.outer((2.0 / vv) * v, v @ A[k:, k:])
        reflectors.append((k, v, vv))
    R = np.triu(A[:n, :n])
    Q = np.zeros((m, n))
    Q[:n, :n] = np.eye(n)
    for k, v, vv in reversed(reflectors):
        if vv > 0:
            Q[k:, :] -= np.outer((2.0 / vv) * v, v @ Q[k:, :])
    R, Q = _sign_fix(R, Q)
    return Q, R


def r_factor(A):
    """R (n x n, diag >= 0) of A = Q R by LAPACK Householder QR."""
    R = np.linalg.qr(np.asarray(A, dtype=np.float64), mode="r")
    R, _ = _sign_fix(np.triu(R))
    return R


def ols(X, Y):
    """beta-hat of Eq. (ols) by Householder QR (LAPACK dgeqrf/dormqr)."""
    X = np.asarray(X, dtype=np.float64)
    Q, R = np.linalg.qr(X, mode="reduced")
    c = Q.T @ np.asarray(Y, dtype=np.float64)
    return solve_triangular(R, c, lower=False)


def ols_lowmem(X, Y):
    """beta-hat of Eq. (ols) by Householder QR without forming Q: LAPACK dgeqrf
    on a copy of X, Q^T Y by applying the stored reflectors (dormqr), then the
    triangular solve.  Same definition as ``ols``; one copy of X of memory."""
    from scipy.linalg import lapack
    from scipy.linalg import qr as sqr
    X = np.asarray(X, dtype=np.float64)
    (qr_raw, tau), R = sqr(np.array(X, order="F", copy=True), mode="raw", overwrite_a=True)
    c, _, info = lapack.dormqr("L", "T", qr_raw, tau, np.asarray(Y, dtype=np.float64)[:, None].copy(order="F"),
                               lwork=max(1, X.shape[1] * 64))
    if info != 0:
        raise RuntimeError("dormqr failed")
    d = X.shape[1]
    return solve_triangular(np.triu(R[:d, :d]), c[:d, 0], lower=False)


def apply_precond(R, g):
    """z = (R^T R)^{-1} g = R^{-1} (R^{-T} g)."""
    u = solve_triangular(R, g, trans="T", lower=False)
    return solve_triangular(R, u, lower=False)
