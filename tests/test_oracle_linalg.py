"""Pins for the oracle's Householder QR and OLS estimator (Eq. ols)."""
import numpy as np
import pytest

from oracle.linalg import apply_precond, householder_qr, ols, ols_lowmem, r_factor
from paper_2607_25272_b300.inputs import gaussian_problem, svd_problem

U64 = np.finfo(np.float64).eps / 2


def _normal_equations_longdouble(X, Y):
    """Brute force: Gauss-Jordan on X^T X beta = X^T Y in 80-bit arithmetic."""
    Xl = X.astype(np.longdouble)
    Yl = Y.astype(np.longdouble)
    n = X.shape[1]
    A = np.zeros((n, n + 1), dtype=np.longdouble)
    for i in range(n):
        for j in range(n):
            A[i, j] = np.sum(Xl[:, i] * Xl[:, j])
        A[i, n] = np.sum(Xl[:, i] * Yl)
    for c in range(n):
        piv = c + int(np.argmax(np.abs(A[c:, c])))
        A[[c, piv]] = A[[piv, c]]
        A[c] = A[c] / A[c, c]
        for r in range(n):
            if r != c:
                A[r] = A[r] - A[r, c] * A[c]
    return A[:, n].astype(np.float64)


@pytest.mark.parametrize("N,d", [(8, 1), (12, 3), (40, 5), (64, 8)])
def test_ols_matches_long_double_normal_equations(N, d):
    X, Y, _ = gaussian_problem(N, d, 0.5, seed=N * 10 + d)
    b_ref = _normal_equations_longdouble(X, Y)
    b = ols(X, Y)
    kappa = np.linalg.cond(X)
    assert np.allclose(b, b_ref, rtol=0, atol=50 * U64 * kappa**2 * np.abs(b_ref).max() + 1e-14)
    Q, R = householder_qr(X)
    b2 = np.linalg.solve(R, Q.T @ Y)
    assert np.allclose(b2, b_ref, rtol=0, atol=50 * U64 * kappa**2 * np.abs(b_ref).max() + 1e-14)


@pytest.mark.parametrize("N,d", [(200, 7), (1000, 31), (333, 50)])
def test_householder_orthogonality_and_reconstruction(N, d):
    X, _, _ = gaussian_problem(N, d, 1.0, seed=d)
    Q, R = householder_qr(X)
    assert np.linalg.norm(Q.T @ Q - np.eye(d)) < 20 * d * U64 * np.sqrt(N)
    assert np.linalg.norm(Q @ R - X) < 20 * d * U64 * np.sqrt(N) * np.linalg.norm(X)
    assert np.all(np.diag(R) >= 0) and np.allclose(R, np.triu(R))
    # the plain and the LAPACK factors agree (R is unique with diag >= 0)
    assert np.allclose(r_factor(X), R, rtol=0, atol=1e-12 * np.linalg.norm(R))


def test_normal_equation_invariant_ill_conditioned():
    X, Y, _ = svd_problem(4000, 40, 1e6, 0.1, seed=3)
    b = ols(X, Y)
    r = Y - X @ b
    g = X.T @ r
    assert np.linalg.norm(g) <= 100 * U64 * np.linalg.norm(X, "fro") * np.linalg.norm(r) * np.sqrt(4000)


def test_ols_matches_svd_least_squares():
    X, Y, _ = svd_problem(2000, 20, 1e4, 0.3, seed=9)
    b = ols(X, Y)
    b_svd = np.linalg.lstsq(X, Y, rcond=None)[0]
    assert np.linalg.norm(X @ (b - b_svd)) <= 1e-11 * np.linalg.norm(X @ b)


def test_ols_prediction_error_is_sigma2_d():
    # E||X(beta-hat - beta)||^2 = sigma^2 d (Sec. 4: the OLS target sigma^2 d)
    N, d, sigma = 300, 6, 0.7
    vals = []
    for s in range(300):
        X, Y, beta = gaussian_problem(N, d, sigma, seed=10_000 + s)
        e = X @ (ols(X, Y) - beta)
        vals.append(e @ e)
    vals = np.array(vals)
    se = vals.std() / np.sqrt(len(vals))
    assert abs(vals.mean() - sigma**2 * d) < 3.5 * se


def test_apply_precond_is_inverse_gram():
    rng = np.random.default_rng(1)
    A = rng.standard_normal((50, 9))
    R = r_factor(A)
    g = rng.standard_normal(9)
    z = apply_precond(R, g)
    assert np.allclose((A.T @ A) @ z, g, atol=1e-12 * np.linalg.norm(g) * np.linalg.cond(A) ** 2)


def test_ols_lowmem_matches_ols():
    X, Y, _ = svd_problem(3000, 30, 1e5, 0.3, seed=13)
    b1, b2 = ols(X, Y), ols_lowmem(X, Y)
    assert np.linalg.norm(X @ (b1 - b2)) <= 1e-11 * np.linalg.norm(X @ b1)
