"""Pins for the oracle's nested SRHT (Sec. 2.1, Sec. 2.2)."""
import numpy as np
import pytest

from oracle.philox import TAG_P, feistel_permute, rademacher_signs
from oracle.srht import (fwht_rows, hat_order, nested_order, nested_sketches,
                         padded_rows, srht_row, srht_transform,
                         sylvester_matrix)
from paper_2607_25272_b300.inputs import gaussian_problem


@pytest.mark.parametrize("n", [1, 2, 4, 8, 64, 1024])
def test_fwht_equals_explicit_sylvester(n):
    rng = np.random.default_rng(n)
    M = rng.standard_normal((n, 3))
    H = sylvester_matrix(n)
    assert np.allclose(fwht_rows(M.copy()), H @ M, rtol=0, atol=1e-13 * np.abs(M).sum())


@pytest.mark.parametrize("n", [1, 2, 4, 16, 512])
def test_sylvester_matrix_and_fwht_match_scipy_hadamard(n):
    """The oracle's normalised Sylvester matrix equals scipy's Hadamard matrix
    (Sylvester's construction) divided by sqrt(n), entry for entry, and the
    fast transform applies that library matrix."""
    from scipy.linalg import hadamard
    Hs = hadamard(n).astype(np.float64) / np.sqrt(n)
    assert np.array_equal(sylvester_matrix(n), Hs)
    M = np.random.default_rng(n + 1).standard_normal((n, 4))
    assert np.allclose(fwht_rows(M.copy()), Hs @ M, rtol=0, atol=1e-13 * np.abs(M).sum())


def test_sylvester_orthogonal_involution():
    H = sylvester_matrix(256)
    assert np.allclose(H @ H, np.eye(256), atol=1e-13)
    # the recursive structure H_2n = [[H, H], [H, -H]] / sqrt 2
    h = sylvester_matrix(128) * np.sqrt(128)
    big = np.block([[h, h], [h, -h]]) / np.sqrt(256)
    assert np.allclose(big, H, atol=1e-15)
    x = np.random.default_rng(0).standard_normal((256, 2))
    y = fwht_rows(fwht_rows(x.copy()))
    assert np.allclose(y, x, atol=1e-13)
    assert np.allclose(np.linalg.norm(fwht_rows(x.copy()), axis=0), np.linalg.norm(x, axis=0))


def test_padded_rows():
    assert [padded_rows(n) for n in (1, 2, 3, 4, 5, 20000, 1 << 20)] == [1, 2, 4, 4, 8, 32768, 1 << 20]


@pytest.mark.parametrize("N,d", [(1000, 7), (4096, 5), (37, 3)])
def test_transform_rows_match_defining_sum(N, d):
    X, Y, _ = gaussian_problem(N, d, 1.0, seed=N)
    ZX, ZY = srht_transform(X, Y, seed=21)
    n_pad = padded_rows(N)
    for j in (0, 1, n_pad // 2, n_pad - 1, 5 % n_pad):
        zx, zy = srht_row(X, Y, 21, j)
        scale = np.abs(X).sum() / np.sqrt(n_pad)
        assert np.allclose(ZX[j], zx, rtol=0, atol=1e-13 * scale)
        assert np.isclose(ZY[j], zy, rtol=0, atol=1e-13 * np.abs(Y).sum())


def test_transform_is_orthogonal_on_padded_data():
    # Z = H D P X' with H, D, P orthogonal: Z^T Z = X^T X, Z^T Z_Y = X^T Y.
    X, Y, _ = gaussian_problem(3000, 6, 1.0, seed=2)
    ZX, ZY = srht_transform(X, Y, seed=4)
    assert np.allclose(ZX.T @ ZX, X.T @ X, rtol=1e-12, atol=1e-9)
    assert np.allclose(ZX.T @ ZY, X.T @ Y, rtol=1e-12, atol=1e-9)


def test_transform_uses_signs_and_permutation():
    # H D P X' for a unit vector e_k is column P^{-1}(k) of H times its sign
    N = 64
    k = 9
    X = np.zeros((N, 1))
    X[k, 0] = 1.0
    ZX, _ = srht_transform(X, np.zeros(N), seed=3)
    perm = feistel_permute(np.arange(N), 6, TAG_P, seed=3)
    j = int(np.nonzero(perm == k)[0][0])
    signs = rademacher_signs(N, seed=3)
    expect = sylvester_matrix(N)[:, j] * signs[j]
    assert np.allclose(ZX[:, 0], expect, atol=1e-15)


def test_full_sampling_special_case():
    # m = N' keeps every row: S = sqrt(N'/N') H D P is orthogonal.
    X, Y, _ = gaussian_problem(512, 4, 1.0, seed=8)
    ZX, ZY = srht_transform(X, Y, seed=1)
    stages, A_hat = nested_sketches(ZX, ZY, [512], 512, seed=1)
    A, b = stages[0]
    assert np.allclose(A.T @ A, X.T @ X, rtol=1e-12)
    assert np.allclose(A_hat.T @ A_hat, X.T @ X, rtol=1e-12)


def test_sketch_is_unbiased_in_expectation():
    # E[S^T S] = I for S = sqrt(N'/m)(H D P)_{I,:}: average (S x)^T (S y) over
    # seeds equals x^T y (pins the sqrt(N'/m) scale and the sampling).
    rng = np.random.default_rng(5)
    N, m = 256, 32
    X = rng.standard_normal((N, 2))
    est = []
    for s in range(600):
        ZX, ZY = srht_transform(X, np.zeros(N), seed=1000 + s)
        stages, _ = nested_sketches(ZX, ZY, [m], m, seed=1000 + s)
        A = stages[0][0]
        est.append(A.T @ A)
    est = np.array(est)
    mean = est.mean(axis=0)
    se = est.std(axis=0) / np.sqrt(len(est))
    truth = X.T @ X
    assert np.all(np.abs(mean - truth) < 5 * se + 1e-12)


def test_nested_sets_are_nested_and_distinct():
    n_pad = 1 << 12
    pi = nested_order(n_pad, 2048, seed=6)
    assert len(np.unique(pi)) == 2048 and pi.max() < n_pad
    hat = hat_order(n_pad, 300, seed=6)
    assert len(np.unique(hat)) == 300
    # the independent sample is not the prefix of pi
    assert not np.array_equal(np.sort(hat), np.sort(pi[:300]))


def test_embedding_distortion_shrinks_with_m():
    # Lemma 2.2 qualitatively: ||U^T S^T S U - I|| decreases as m grows.
    rng = np.random.default_rng(2)
    N, d = 4096, 8
    U, _ = np.linalg.qr(rng.standard_normal((N, d)))
    ZU, Zy = srht_transform(U, np.zeros(N), seed=17)
    ms = [64, 256, 1024, 2048]
    stages, _ = nested_sketches(ZU, Zy, ms, 64, seed=17)
    eps = [np.linalg.norm(A.T @ A - np.eye(d), 2) for A, _ in stages]
    assert eps[0] > eps[-1]
    assert eps[-1] < 0.5


def test_sketch_and_solve_prediction_efficiency():
    """The prediction-efficiency lemma the paper quotes for SRHT sketch-and-
    solve estimators (Dobriban and Liu; appendix, proof of the iteration
    bounds): E||X(beta~ - beta)||^2 / E||X(beta-hat - beta)||^2 -> (1 - gamma) /
    (xi - gamma) with gamma = d/N, xi = m/N, i.e. (N - d)/(m - d) = 4.2 here.
    Monte Carlo over 60 noise draws and sketch seeds on a design with
    heavy-tailed leverage (rows scaled by |t_3| before orthonormalising), where
    sampling rows without the transform is far less efficient; the OLS level
    itself is sigma^2 d."""
    from paper_2607_25272_b300.inputs import svd_problem
    N, d, m, sigma, T = 4096, 64, 1024, 1.0, 60
    X, _, beta = svd_problem(N, d, 1e2, sigma, seed=7, leverage_df=3)
    rng = np.random.default_rng(1)
    e_sketch = e_rows = e_ols = 0.0
    for t in range(T):
        Y = X @ beta + sigma * rng.standard_normal(N)
        ZX, ZY = srht_transform(X, Y, seed=100 + t)
        (A, b), = nested_sketches(ZX, ZY, [m], 2 * d, seed=100 + t)[0]
        b_sketch = np.linalg.lstsq(A, b, rcond=None)[0]
        b_ols = np.linalg.lstsq(X, Y, rcond=None)[0]
        rows = rng.choice(N, m, replace=False)
        b_rows = np.linalg.lstsq(X[rows], Y[rows], rcond=None)[0]
        e_sketch += np.sum((X @ (b_sketch - beta)) ** 2)
        e_rows += np.sum((X @ (b_rows - beta)) ** 2)
        e_ols += np.sum((X @ (b_ols - beta)) ** 2)
    predicted = (N - d) / (m - d)
    assert abs(e_sketch / e_ols / predicted - 1) < 0.12
    assert e_rows / e_ols > 1.3 * predicted        # the transform is what spreads the leverage
    assert abs(e_ols / T / (sigma ** 2 * d) - 1) < 0.1
