"""Parity of the batched persistent solver with the FP64 oracle.

Each problem is FP32-valued; the oracle solves the same values promoted to
FP64 (Householder OLS), and every batched solution must meet the stopping
rule's target, 1e-6 relative prediction error."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.linalg import ols
from oracle.metrics import rel_pred_error
from paper_2607_25272_b300 import spcg as S
from paper_2607_25272_b300.inputs import scaled_columns_problem

pytestmark = pytest.mark.gpu


def make_batch(n, seed, nmin=12, nmax=14, lo=1e-3, hi=1e3):
    rng = np.random.default_rng(seed)
    probs = []
    for i in range(n):
        N = int(rng.integers(2 ** nmin, 2 ** nmax + 1))
        d = int(rng.integers(16, 257))
        X, Y, _ = scaled_columns_problem(N, d, lo, hi, 1.0, seed=seed * 1000 + i)
        probs.append((X.astype(np.float32), Y.astype(np.float32)))
    return probs


def to_device(probs):
    Xs, Ys = [], []
    for X, Y in probs:
        N, d = X.shape
        ld = (d + 3) // 4 * 4
        Xd = torch.zeros((N, ld), dtype=torch.float32, device="cuda")
        Xd[:, :d] = torch.from_numpy(X).cuda()
        Xs.append(Xd[:, :d])
        Ys.append(torch.from_numpy(Y).cuda())
    return Xs, Ys


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    S.lib()


def test_batched_solves_match_oracle_twice():
    probs = make_batch(24, seed=5)
    Xs, Ys = to_device(probs)
    B = S.Batch(Xs, Ys)
    for rep in range(2):       # the second solve replays the captured graph
        rc, st, it, ms = B.solve(7, 1e-6)
        assert rc == S.SPCG_OK and all(v == 0 for v in st)
        for (X, Y), beta in zip(probs, B.betas):
            X64, Y64 = X.astype(np.float64), Y.astype(np.float64)
            assert rel_pred_error(X64, beta.cpu().numpy(), ols(X64, Y64)) <= 1e-6
    B.close()


def test_batched_autotuner_and_tiles_keep_results():
    probs = make_batch(12, seed=9)
    Xs, Ys = to_device(probs)
    B = S.Batch(Xs, Ys)
    chosen = B.autotune(3, 1e-6)
    assert all(c in (0, 4096, 8192, 16384) for c in chosen)
    B.set_tiles([1024, 2048, 4096, 16384])
    rc, st, _, _ = B.solve(3, 1e-6)
    assert rc == S.SPCG_OK
    for (X, Y), beta in zip(probs, B.betas):
        X64, Y64 = X.astype(np.float64), Y.astype(np.float64)
        assert rel_pred_error(X64, beta.cpu().numpy(), ols(X64, Y64)) <= 1e-6
    B.close()


def test_batched_rejects_bad_problem():
    X = torch.zeros((100, 300), dtype=torch.float32, device="cuda")   # d > 256
    Y = torch.zeros(100, dtype=torch.float32, device="cuda")
    with pytest.raises(S.SpcgError) as e:
        S.Batch([X], [Y])
    assert e.value.status == S.SPCG_E_INVALID_ARG


def test_batched_every_row_width():
    """Rows per warp follow d: 32, 16, 8, 4, 2 or 1 rows share a warp for d up
    to 8, 16, 32, 64, 128 and 256; widths at and just past each boundary,
    every problem against the oracle's OLS at 1e-6."""
    widths = [3, 8, 9, 16, 17, 32, 33, 64, 65, 128, 129, 256]
    rng = np.random.default_rng(77)
    probs = []
    for i, d in enumerate(widths):
        N = int(rng.integers(4096, 9000))
        X, Y, _ = scaled_columns_problem(N, d, 1e-2, 1e2, 1.0, seed=7700 + i)
        probs.append((X.astype(np.float32), Y.astype(np.float32)))
    Xs, Ys = to_device(probs)
    B = S.Batch(Xs, Ys)
    rc, st, it, ms = B.solve(13, 1e-6)
    assert rc == S.SPCG_OK and all(v == 0 for v in st)
    for (X, Y), beta in zip(probs, B.betas):
        X64, Y64 = X.astype(np.float64), Y.astype(np.float64)
        assert rel_pred_error(X64, beta.cpu().numpy(), ols(X64, Y64)) <= 1e-6, X.shape
    B.close()


def test_one_call_batched_solve():
    """spcg_solve_batched: create, solve and destroy in one call, same answers."""
    probs = make_batch(6, seed=31)
    Xs, Ys = to_device(probs)
    betas, st, it, rc = S.spcg_solve_batched(Xs, Ys, 5, 1e-6)
    assert rc == S.SPCG_OK and all(v == 0 for v in st)
    for (X, Y), beta in zip(probs, betas):
        X64, Y64 = X.astype(np.float64), Y.astype(np.float64)
        assert rel_pred_error(X64, beta.cpu().numpy(), ols(X64, Y64)) <= 1e-6
