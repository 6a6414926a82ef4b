"""Pins for the oracle's CountSketch variant (SPCG-CS, Sec. 4.3) and the
tuned schedule of Sec. 4.3."""
import numpy as np
import pytest

from oracle import countsketch as CS
from oracle.linalg import ols
from oracle.metrics import rel_pred_error
from oracle.spcg import default_schedule, tuned_schedule
from paper_2607_25272_b300.inputs import gaussian_problem, svd_problem


def test_scatter_equals_explicit_matrix():
    rng = np.random.default_rng(0)
    X = rng.standard_normal((300, 4))
    h, s = CS.stage_hash(300, 64, seed=3)
    S = CS.explicit_matrix(h, s, 64)
    assert np.allclose(CS.countsketch_apply(X, h, s, 64), S @ X, atol=1e-13)
    # one nonzero of modulus one per column
    assert np.all((S != 0).sum(0) == 1) and np.all(np.abs(S[S != 0]) == 1)


def test_folding_equals_hash_mod_m():
    rng = np.random.default_rng(1)
    X = rng.standard_normal((500, 3))
    h, s = CS.stage_hash(500, 128, seed=9)
    top = CS.countsketch_apply(X, h, s, 128)
    for m in (64, 16, 1):
        direct = CS.countsketch_apply(X, h % m, s, m)
        assert np.allclose(CS.fold(top, m), direct, atol=1e-13)


def test_hashes_uniform_and_independent_of_tags():
    h, s = CS.stage_hash(1 << 16, 256, seed=5)
    counts = np.bincount(h, minlength=256)
    from scipy import stats
    assert stats.chisquare(counts).pvalue > 1e-6
    assert abs(s.mean()) < 6 / np.sqrt(s.size)
    hh, _ = CS.hat_hash(1 << 16, 300, seed=5)
    assert hh.min() >= 0 and hh.max() < 300
    assert stats.chisquare(np.bincount(hh, minlength=300)).pvalue > 1e-6


def test_countsketch_unbiased():
    rng = np.random.default_rng(2)
    N, m = 200, 16
    X = rng.standard_normal((N, 2))
    est = []
    for seed in range(800):
        h, s = CS.stage_hash(N, m, seed)
        A = CS.countsketch_apply(X, h, s, m)
        est.append(A.T @ A)
    est = np.array(est)
    se = est.std(0) / np.sqrt(len(est))
    assert np.all(np.abs(est.mean(0) - X.T @ X) < 5 * se + 1e-12)


@pytest.mark.parametrize("tol", [1e-6, 1e-10])
def test_spcg_cs_reaches_ols(tol):
    for seed, (X, Y, _) in enumerate([gaussian_problem(20000, 50, 1.0, seed=1),
                                      svd_problem(16384, 40, 1e6, 0.1, seed=2)]):
        out = CS.spcg_cs(X, Y, seed + 1, default_schedule(*X.shape), tol=tol)
        assert out["converged"]
        assert rel_pred_error(X, out["beta"], ols(X, Y)) <= tol


def test_tuned_schedule_matches_paper_setting():
    s = tuned_schedule(1 << 22, 64)
    assert s["m"] == [1 << k for k in range(10, 17)] + [1 << 20]
    assert s["a"] == [4] * 8 and s["r"] == 384
    s = tuned_schedule(20000, 50)   # small problems keep the structure below N'/4
    assert all(a < b for a, b in zip(s["m"], s["m"][1:])) and s["m"][-1] <= 32768 // 4
