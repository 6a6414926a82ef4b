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
from paper_2607_25272_b300.inputs import gaussian_problem, svd_problem

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
                                 (20000, 500), (513, 1000)])
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


@pytest.mark.parametrize("m,d", [(1, 1), (1000, 33), (4097, 256), (100003, 50), (20000, 500)])
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
