"""The residual-mode pass g = A^T (b - A x) (the true gradient of the Stage II
stopping rule, Sec. 2.2) through spcg_resid_apply_typed, against FP64 on the
host, for FP64 rows and for the double-FP32 pair the mixed path trusts.

Bounds are stated against the magnitude M = |A|^T (|b| + |A| |x|):
* FP64: every product and sum rounds once per term, |dg| <= gamma_n M with
  n = d + 5 + (rows per consumer lane) + partial sums; 2^-40 M is far above
  that for these sizes and far below any indexing mistake;
* pair: TwoProd/TwoSum keep products and sums exact but for terms near
  2^-48 relative; 2^-40 M again.
The cancellation case takes x ~ 1e8 and b = A x + noise, as at the OLS
solution of an ill-conditioned problem, where |A| |x| exceeds |b - A x| by
about eight orders of magnitude.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2607_25272_b300 import spcg as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    S.lib()


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _case(m, d, seed, cancel):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((m, d)) * np.exp(rng.uniform(-2, 2, size=d))[None, :]
    if cancel:
        x = rng.standard_normal(d) * 1e8
        b = A @ x + rng.standard_normal(m)
    else:
        x = rng.standard_normal(d)
        b = rng.standard_normal(m)
    return A, b, x


CASES = [(1, 1, False), (1000, 33, False), (4097, 256, True), (100003, 50, False),
         (20000, 500, True), (513, 1000, False), (60000, 1000, True), (3001, 257, True)]


@pytest.mark.parametrize("m,d,cancel", CASES)
def test_resid_fp64(m, d, cancel):
    A, b, x = _case(m, d, 11 * m + d, cancel)
    ld = (d + 1) // 2 * 2
    Ad = torch.zeros((m, ld), dtype=torch.float64, device="cuda")
    Ad[:, :d] = cuda(A)
    s = S.Solver(cuda(np.random.default_rng(0).standard_normal((d + 2, d))), cuda(np.zeros(d + 2)))
    g = s.resid_apply(Ad[:, :d], cuda(b), cuda(x)).cpu().numpy()
    s.close()
    ref = A.T @ (b - A @ x)
    mag = np.abs(A).T @ (np.abs(b) + np.abs(A) @ np.abs(x))
    assert np.all(np.abs(g - ref) <= 2.0 ** -40 * mag + 1e-300)


@pytest.mark.parametrize("m,d,cancel", CASES)
def test_resid_pair(m, d, cancel):
    A, b, x = _case(m, d, 13 * m + d, cancel)
    Ah = A.astype(np.float32)
    Al = (A - Ah.astype(np.float64)).astype(np.float32)
    ld = (d + 3) // 4 * 4
    buf = torch.zeros(2 * m * ld, dtype=torch.float32, device="cuda")
    v = buf.view(2, m, ld)
    v[0, :, :d] = cuda(Ah)
    v[1, :, :d] = cuda(Al)
    s = S.Solver(cuda(np.random.default_rng(0).standard_normal((d + 2, d))), cuda(np.zeros(d + 2)))
    g = s.resid_apply(buf, cuda(b), cuda(x), dtype=3, m=m, lda=ld).cpu().numpy()
    s.close()
    Ap = Ah.astype(np.float64) + Al.astype(np.float64)
    ref = Ap.T @ (b - Ap @ x)
    mag = np.abs(Ap).T @ (np.abs(b) + np.abs(Ap) @ np.abs(x))
    assert np.all(np.abs(g - ref) <= 2.0 ** -40 * mag + 1e-300)


def test_pair_gradient_meets_the_stopping_metric_at_kappa_1e8():
    """The double-FP32 true gradient at the OLS solution of a kappa = 1e8
    problem, measured where the stopping rule measures it: in the R^{-T}
    metric, against (tol/2) ||R beta|| with tol = 1e-6.  A magnitude-relative
    bound cannot see an error that this metric amplifies by ||D R^{-1}||, so
    this is the check that the pair arithmetic really is double-FP32 (a
    single lost error term leaves it near FP32 accuracy, five orders of
    magnitude worse).  Reference: the gradient in 80-bit extended precision."""
    from scipy.linalg import solve_triangular
    from paper_2607_25272_b300.inputs import svd_problem
    N, d = 65536, 200
    X, Y, _ = svd_problem(N, d, 1e8, 1.0, seed=4, leverage_df=3)
    Q, R = np.linalg.qr(X)
    bo = np.linalg.solve(R, Q.T @ Y)
    del Q
    XL = X.astype(np.longdouble)
    g_exact = (XL.T @ (Y.astype(np.longdouble) - XL @ bo.astype(np.longdouble))).astype(np.float64)
    del XL
    thr = 5e-7 * np.linalg.norm(R @ bo)

    def metric(g):
        return np.linalg.norm(solve_triangular(R.T, g - g_exact, lower=True))

    Xd, Yd, bd = cuda(X), cuda(Y), cuda(bo)
    s = S.Solver(Xd, Yd)
    g64 = s.resid_apply(Xd, Yd, bd).cpu().numpy()
    ld = (d + 3) // 4 * 4
    buf = torch.zeros(2 * N * ld, dtype=torch.float32, device="cuda")
    v = buf.view(2, N, ld)
    v[0, :, :d] = Xd.float()
    v[1, :, :d] = (Xd - v[0, :, :d].double()).float()
    gdf = s.resid_apply(buf, Yd, bd, dtype=3, m=N, lda=ld).cpu().numpy()
    s.close()
    assert metric(g64) <= thr / 100
    assert metric(gdf) <= thr / 4
