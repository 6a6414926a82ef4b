"""The seeded input recipes (inputs.py): each family has the structure the
workloads state (singular values, condition number, orthonormal factors,
leverage, column scales, noise level), is a pure function of its seed, and
the device recipe's closed-form OLS estimator (used by the bench lines of
the large workloads) is the least-squares solution.  All on the CPU; the
device recipe runs on torch's CPU device here."""
import numpy as np
import pytest

from paper_2607_25272_b300 import inputs as I


def _geometric(d, kappa):
    return kappa ** (-np.arange(d) / max(d - 1, 1))


def test_orthonormal_basis_is_orthonormal_to_1e13():
    G = np.random.default_rng(0).standard_normal((20000, 50))
    U = I.orthonormal_basis(G)
    assert np.abs(U.T @ U - np.eye(50)).max() <= 1e-13
    # the same column space as G
    coef, *_ = np.linalg.lstsq(U, G, rcond=None)
    assert np.abs(U @ coef - G).max() <= 1e-10 * np.abs(G).max()


@pytest.mark.parametrize("kappa,df", [(1e4, None), (1e6, None), (1e8, 3)])
def test_svd_problem_has_the_stated_spectrum(kappa, df):
    N, d = 6000, 24
    X, Y, beta = I.svd_problem(N, d, kappa, 0.1, seed=5, leverage_df=df)
    sv = np.linalg.svd(X, compute_uv=False)
    # LAPACK's SVD finds sigma_min to about eps kappa relative
    tol = 100 * np.finfo(float).eps * kappa
    assert np.allclose(sv, _geometric(d, kappa), rtol=tol, atol=0)
    assert abs(sv[0] / sv[-1] / kappa - 1) <= tol


def test_leverage_option_gives_heavy_tailed_leverage():
    N, d = 20000, 10
    X0, _, _ = I.svd_problem(N, d, 1e2, 0.1, seed=2)
    X3, _, _ = I.svd_problem(N, d, 1e2, 0.1, seed=2, leverage_df=3)

    def leverage(X):
        Q, _ = np.linalg.qr(X)
        return (Q ** 2).sum(1)

    l0, l3 = leverage(X0), leverage(X3)
    assert abs(l0.sum() - d) < 1e-8 and abs(l3.sum() - d) < 1e-8   # trace of the hat matrix
    # Gaussian rows: max leverage a few times the mean d/N; t(3)-scaled rows: far larger
    assert l0.max() < 10 * d / N
    assert l3.max() > 50 * d / N


def test_response_and_noise_level():
    N, d, sigma = 200000, 8, 0.3
    for X, Y, beta in (I.gaussian_problem(N, d, sigma, seed=4),
                       I.svd_problem(N, d, 1e3, sigma, seed=4),
                       I.paper_problem(N, d, 1e3, sigma ** 2, seed=4)):
        r = Y - X @ beta
        assert abs(r.std() / sigma - 1) < 0.01
        assert abs(r.mean()) < 5 * sigma / np.sqrt(N)


def test_paper_and_scaled_column_recipes():
    N, d = 50000, 12
    X, _, _ = I.paper_problem(N, d, 1e4, 1e-8, seed=3)
    norms = np.linalg.norm(X, axis=0) / np.sqrt(N)
    assert np.allclose(norms, _geometric(d, 1e4), rtol=0.03)
    X, _, _ = I.scaled_columns_problem(N, d, 1e-3, 1e3, 1.0, seed=3)
    scales = np.linalg.norm(X, axis=0) / np.sqrt(N)
    assert np.all(scales > 1e-3 * 0.95) and np.all(scales < 1e3 * 1.05)


@pytest.mark.parametrize("gen,args", [(I.gaussian_problem, (3000, 7, 0.5)),
                                      (I.svd_problem, (3000, 7, 1e5, 0.5)),
                                      (I.paper_problem, (3000, 7, 1e5, 0.25)),
                                      (I.scaled_columns_problem, (3000, 7, 1e-2, 1e2, 0.5))])
def test_generators_are_pure_functions_of_the_seed(gen, args):
    a = gen(*args, seed=11)
    b = gen(*args, seed=11)
    c = gen(*args, seed=12)
    for u, v in zip(a, b):
        assert np.array_equal(u, v)
    assert not np.array_equal(a[0], c[0])


@pytest.mark.parametrize("df", [None, 3])
def test_device_recipe_closed_form_ols_on_the_cpu(df):
    """svd_problem_device on torch's CPU device: X has the stated spectrum, and
    V diag(1/s) (U^T Y) from its returned factors is the least-squares
    solution (the property the bench lines of the large workloads use)."""
    torch = pytest.importorskip("torch")
    N, d, kappa = 8000, 16, 1e6
    X, Y, beta, uty, s, V = I.svd_problem_device(N, d, kappa, 0.5, seed=3, leverage_df=df,
                                                 device="cpu")
    Xn, Yn = X.numpy(), Y.numpy()
    sv = np.linalg.svd(Xn, compute_uv=False)
    assert np.allclose(sv, _geometric(d, kappa), rtol=100 * np.finfo(float).eps * kappa, atol=0)
    b_closed = (V @ (uty / s)).numpy()
    b_ls, *_ = np.linalg.lstsq(Xn, Yn, rcond=None)
    err = np.linalg.norm(Xn @ (b_closed - b_ls)) / np.linalg.norm(Xn @ b_ls)
    assert err <= 100 * np.finfo(float).eps * kappa    # both sides to LAPACK's eps kappa
    assert torch.equal(X, I.svd_problem_device(N, d, kappa, 0.5, seed=3, leverage_df=df,
                                               device="cpu")[0])
