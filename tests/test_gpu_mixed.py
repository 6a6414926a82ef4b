"""Parity of the mixed-precision path (SPCG_PREC_MIXED) with the FP64 oracle.

Stage I reads a BF16 copy of the sketched rows with FP32 accumulation; Stage
II iterates on an FP32 copy of X with compensated accumulation and confirms
every stop on an FP64 true gradient.  Tolerances:

* FP32 operand: t_i = a_i . p is an FP32 dot product of d terms (plus a
  five-level shuffle tree), |dt_i| <= gamma32_{d+5} sum_c |a_ic p_c|; the
  compensated accumulation of w_j = sum_i a_ij t_i returns the sum with
  error <= 2 u32 |w_j| + gamma32_m^2 sum_i |a_ij t_i|;
* BF16 operand: the same dot, and a plain FP32 accumulation of at most m
  terms, |dw_j| <= (gamma32_{d+5} + gamma32_m) (|A|^T (|A| |p|))_j;
* the solve: the target of the stopping rule, 1e-6 relative prediction error
  against the oracle's OLS estimator (the FP64 true gradient decides).
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import linalg as OL
from oracle import srht as OR
from oracle import spcg as OS
from oracle.metrics import rel_pred_error
from paper_2607_25272_b300 import spcg as S
from paper_2607_25272_b300.inputs import gaussian_problem, scaled_columns_problem, svd_problem

pytestmark = pytest.mark.gpu
U32 = 2.0 ** -24


def g32(n):
    return n * U32 / (1 - n * U32)


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    S.lib()


def mixed_opts():
    o = S.Opts()
    o.precision = S.PREC_MIXED
    return o


@pytest.mark.parametrize("m,d", [(1, 1), (1000, 33), (4097, 256), (3001, 257), (100003, 50),
                                 (20000, 500), (513, 1000), (20011, 1000)])
def test_fp32_pass_parity(m, d):
    rng = np.random.default_rng(m + 3 * d)
    A32 = rng.standard_normal((m, d)).astype(np.float32)
    p = rng.standard_normal(d)
    ld = (d + 3) // 4 * 4
    Ad = torch.zeros((m, ld), dtype=torch.float32, device="cuda")
    Ad[:, :d] = cuda(A32)
    s = S.Solver(cuda(rng.standard_normal((d + 2, d))), cuda(np.zeros(d + 2)))
    w = s.gram_apply_typed(Ad[:, :d], cuda(p)).cpu().numpy()
    s.close()
    A = A32.astype(np.float64)
    p32 = p.astype(np.float32).astype(np.float64)
    ref = A.T @ (A @ p32)
    mag = np.abs(A).T @ (np.abs(A) @ np.abs(p32))
    bound = g32(d + 5) * mag + 2 * U32 * np.abs(ref) + g32(m) ** 2 * mag + 1e-300
    assert np.all(np.abs(w - ref) <= bound)


@pytest.mark.parametrize("m,d", [(1, 1), (1000, 33), (4097, 256), (100003, 50), (20000, 500),
                                 (3001, 1000), (513, 777)])
def test_bf16_pass_parity(m, d):
    rng = np.random.default_rng(m + 5 * d)
    At = torch.from_numpy(rng.standard_normal((m, d))).to(torch.bfloat16)
    p = rng.standard_normal(d)
    ld = (d + 7) // 8 * 8
    Ad = torch.zeros((m, ld), dtype=torch.bfloat16, device="cuda")
    Ad[:, :d] = At.cuda()
    s = S.Solver(cuda(rng.standard_normal((d + 2, d))), cuda(np.zeros(d + 2)))
    w = s.gram_apply_typed(Ad[:, :d], cuda(p)).cpu().numpy()
    s.close()
    A = At.to(torch.float64).numpy()
    p32 = p.astype(np.float32).astype(np.float64)
    ref = A.T @ (A @ p32)
    bound = (g32(d + 5) + g32(m)) * (np.abs(A).T @ (np.abs(A) @ np.abs(p32))) + 1e-300
    assert np.all(np.abs(w - ref) <= bound)


def test_mixed_prefix_rows_are_bf16_of_the_transform():
    N, d, seed = 20000, 50, 1
    X, Y, _ = gaussian_problem(N, d, 1.0, seed=seed)
    s = S.Solver(cuda(X), cuda(Y), mixed_opts())
    s.sketch(seed, S.spcg_default_schedule(N, d))
    sched = OS.default_schedule(N, d)
    mK = sched["m"][-1]
    ZX, _ = OR.srht_transform(X, Y, seed)
    pi = OR.nested_order(sched["n_pad"], mK, seed)
    A_g, _ = (t.cpu().numpy() for t in s.export_sketch(0, mK))
    Zo = ZX[pi]
    # BF16 keeps 8 significant bits: relative rounding <= 2^-8, plus the
    # transform's own error (far smaller)
    assert np.all(np.abs(A_g - Zo) <= 2.0 ** -8 * np.abs(Zo) + 1e-12 * np.abs(Zo).max())
    s.close()


@pytest.mark.parametrize("N,d,kappa,sigma,seed", [(20000, 50, None, 1.0, 1), (16384, 40, 1e6, 0.1, 2),
                                                  (5000, 37, 1e3, 1.0, 6), (70000, 129, 1e5, 0.5, 8)])
def test_mixed_solve_meets_1e6(N, d, kappa, sigma, seed):
    if kappa is None:
        X, Y, _ = gaussian_problem(N, d, sigma, seed=seed)
    else:
        X, Y, _ = svd_problem(N, d, kappa, sigma, seed=seed)
    bh = OL.ols(X, Y)
    s = S.Solver(cuda(X), cuda(Y), mixed_opts())
    sc = S.spcg_default_schedule(N, d)
    sc.tol = 1e-6
    beta, info, st = s.solve(seed, sc)
    assert st == S.SPCG_OK and info.converged == 1
    assert rel_pred_error(X, beta.cpu().numpy(), bh) <= 1e-6
    s.close()


def test_mixed_c2_full_size():
    N, d = 1 << 20, 500
    X, Y, _ = svd_problem(N, d, 1e6, 0.1, seed=1)
    bh = OL.ols(X, Y)
    s = S.Solver(cuda(X), cuda(Y), mixed_opts())
    sc = S.spcg_default_schedule(N, d)
    beta, info, st = s.solve(1, sc)
    assert st == S.SPCG_OK
    assert rel_pred_error(X, beta.cpu().numpy(), bh) <= 1e-6
    s.close()


def _split_pair(A):
    """A (float64) -> (Ah, Al) FP32 with Ah = fl32(A), Al = fl32(A - Ah)."""
    Ah = A.astype(np.float32)
    Al = (A - Ah.astype(np.float64)).astype(np.float32)
    return Ah, Al


@pytest.mark.parametrize("m,d", [(1, 1), (1000, 33), (4097, 256), (3001, 257), (100003, 50),
                                 (20000, 500), (513, 1000)])
def test_pair_pass_parity(m, d):
    """Double-FP32 pass against FP64 on the same pair: products are exact
    (TwoProd) but for the dropped Al*pl term and the FP32 cross terms, both
    near 2^-48 relative; sums are TwoSum-compensated.  Bound: 2^-40 of the
    magnitude sum, a margin of 2^8 over that analysis, still 2^16 below the
    FP32 pass's error."""
    rng = np.random.default_rng(7 * m + d)
    A = rng.standard_normal((m, d)) * np.exp(rng.uniform(-3, 3, size=d))[None, :]
    p = rng.standard_normal(d)
    Ah, Al = _split_pair(A)
    ld = (d + 3) // 4 * 4
    buf = torch.zeros(2 * m * ld, dtype=torch.float32, device="cuda")
    v = buf.view(2, m, ld)
    v[0, :, :d] = cuda(Ah)
    v[1, :, :d] = cuda(Al)
    s = S.Solver(cuda(rng.standard_normal((d + 2, d))), cuda(np.zeros(d + 2)))
    w = s.gram_apply_pair(buf, m, ld, cuda(p)).cpu().numpy()
    s.close()
    Apair = Ah.astype(np.float64) + Al.astype(np.float64)
    ref = Apair.T @ (Apair @ p)
    mag = np.abs(Apair).T @ (np.abs(Apair) @ np.abs(p))
    assert np.all(np.abs(w - ref) <= 2.0 ** -40 * mag + 1e-300)


def _exact_nu(R):
    D = np.sqrt((R * R).sum(axis=0))
    return np.linalg.norm(D[:, None] * np.linalg.inv(R), 2)


@pytest.mark.parametrize("N,d,kappa,seed", [(20000, 50, 1e4, 1), (30000, 200, 1e8, 2),
                                            (16384, 40, 1e2, 3)])
def test_condition_estimate_brackets_exact_norm(N, d, kappa, seed):
    """cond_est is a power-iteration lower bound of ||D R^{-1}||_2."""
    X, Y, _ = svd_problem(N, d, kappa, 0.1, seed=seed)
    s = S.Solver(cuda(X), cuda(Y), mixed_opts())
    sc = S.spcg_default_schedule(N, d)
    beta, info, st = s.solve(seed, sc, raise_on_error=False)
    R = s.export_precond()[0].cpu().numpy()
    s.close()
    nu = _exact_nu(R)
    assert 0.3 * nu <= info.cond_est <= nu * (1 + 1e-9)


@pytest.mark.parametrize("inner", [0, 2])
def test_mixed_kappa_1e8_converges(inner):
    """At kappa = 1e8 the FP32 copy of X perturbs the preconditioned operator
    by about 2^-24 nu > 1; the automatic rule must take the double-FP32 pair
    and still meet 1e-6 against the oracle's OLS estimator."""
    N, d, seed = 65536, 200, 4
    X, Y, _ = svd_problem(N, d, 1e8, 1.0, seed=seed, leverage_df=3)
    bh = OL.ols(X, Y)
    o = mixed_opts()
    o.inner_prec = inner
    s = S.Solver(cuda(X), cuda(Y), o)
    sc = S.spcg_default_schedule(N, d)
    beta, info, st = s.solve(seed, sc, raise_on_error=False)
    s.close()
    assert info.cond_est * 2.0 ** -24 > 1.0 / 32
    assert info.inner_prec == S.INNER_DF
    # 2^-48 nu > tol / 64: the stopping rule must see FP64 true gradients
    assert info.grad_prec == S.GRAD_F64
    assert st == S.SPCG_OK and info.converged == 1
    assert rel_pred_error(X, beta.cpu().numpy(), bh) <= 1e-6


def test_auto_rule_keeps_fp32_when_well_conditioned():
    N, d, seed = 16384, 40, 2
    X, Y, _ = svd_problem(N, d, 1e3, 0.1, seed=seed)
    s = S.Solver(cuda(X), cuda(Y), mixed_opts())
    beta, info, st = s.solve(seed, S.spcg_default_schedule(N, d))
    s.close()
    assert st == S.SPCG_OK
    assert info.cond_est * 2.0 ** -24 <= 1.0 / 32
    assert info.inner_prec == S.INNER_F32
    assert info.grad_prec == S.GRAD_DF


def _split_cases():
    rng = np.random.default_rng(11)
    parts = [rng.standard_normal(4000) * 10.0 ** rng.uniform(-20, 20, 4000),
             rng.standard_normal(1000) * 2.0 ** rng.integers(-80, -60, 1000),   # near 2^-74
             rng.standard_normal(1000) * 2.0 ** rng.integers(120, 127, 1000),   # near 2^127
             np.array([0.0, -0.0, 1.0, -1.0, 2.0 ** -74, 2.0 ** -75, 2.0 ** 126, 3e-320])]
    # exact ties of the float rounding (the 29 dropped bits are 100...0), both parities
    base = rng.standard_normal(1000)
    bits = base.view(np.uint64) & ~np.uint64(0x1FFFFFFF) | np.uint64(0x10000000)
    parts.append(bits.view(np.float64))
    # values whose rounding carries into the exponent (fraction bits all ones)
    ones = rng.standard_normal(500).view(np.uint64) | np.uint64(0xFFFFFFFFFFFFF)
    parts.append(ones.view(np.float64))
    return np.concatenate(parts)


@pytest.mark.parametrize("N,d", [(5000, 37), (20000, 50), (70000, 129), (9000, 300)])
def test_split_fused_column_maxima_give_the_same_sketch(N, d):
    """A mixed solve takes the column maxima of the fixed-point scales from its
    FP32 split; a bare spcg_sketch computes them in a pass of its own.  Both
    must give the same scales, hence the same sketch and R, bit for bit
    (columns spanning 1e-3..1e3, negative extremes, an odd last column)."""
    X, Y, _ = scaled_columns_problem(N, d, 1e-3, 1e3, 0.5, seed=d)
    X[:, 0] = -np.abs(X[:, 0])               # the largest magnitude is negative
    Y = -3.0 * Y
    s = S.Solver(cuda(X), cuda(Y), mixed_opts())
    sc = S.spcg_default_schedule(N, d)
    sc.tol = 1e-6
    s.solve(3, sc, raise_on_error=False)   # the sketch is what is compared
    mK = sc.m[sc.K - 1] if sc.K else 1
    A1, b1 = (t.cpu().numpy() for t in s.export_sketch(0, mK))
    R1 = s.export_precond()[0].cpu().numpy()
    s.sketch(3, sc)
    A2, b2 = (t.cpu().numpy() for t in s.export_sketch(0, mK))
    R2 = s.export_precond()[0].cpu().numpy()
    s.close()
    assert np.array_equal(A1.view(np.uint64), A2.view(np.uint64))
    assert np.array_equal(b1.view(np.uint64), b2.view(np.uint64))
    assert np.array_equal(R1.view(np.uint64), R2.view(np.uint64))


@pytest.mark.parametrize("d", [1, 7, 64, 257, 1100])
def test_split_f32_is_round_to_nearest(d):
    """Xh = fl32(x), Xl = fl32(x - Xh), bit for bit against numpy's rounding."""
    v = _split_cases()
    N = (len(v) + d - 1) // d
    x = np.resize(v, N * d).reshape(N, d)
    ld = (d + 1) // 2 * 2
    Xd = torch.zeros((N, ld), dtype=torch.float64, device="cuda")
    Xd[:, :d] = cuda(x)
    Xh, Xl = S.spcg_split_f32(Xd[:, :d])
    h_ref = x.astype(np.float32)
    l_ref = (x - h_ref.astype(np.float64)).astype(np.float32)
    assert np.array_equal(Xh.cpu().numpy().view(np.uint32), h_ref.view(np.uint32))
    assert np.array_equal(Xl.cpu().numpy().view(np.uint32), l_ref.view(np.uint32))
