"""Parity of the SPCG variants of Sec. 4.3 with the FP64 oracle: the
CountSketch initialisation (SPCG-CS) and the tuned sketch-size schedule.

CountSketch buckets are exact 64-bit fixed-point sums on the GPU: bucket b of
column c is off by at most n_b quanta / 2 with n_b rows in the bucket and a
quantum of at most max_j |x_jc| 2^{n-61} (n = log2 N'), plus one rounding to
FP64; the oracle's own scatter-add (numpy add.at, sequential) is off by at
most gamma_{n_b} sum_{j in b} |x_jc|.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import countsketch as CS
from oracle import linalg as OL
from oracle import spcg as OS
from oracle.metrics import rel_pred_error
from paper_2607_25272_b300 import spcg as S
from paper_2607_25272_b300.inputs import gaussian_problem, svd_problem

pytestmark = pytest.mark.gpu
U = np.finfo(np.float64).eps / 2


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    S.lib()


def cs_schedule(N, d, tol):
    sc = S.spcg_default_schedule(N, d)
    sc.sketch = S.SKETCH_COUNT
    sc.tol = tol
    return sc


@pytest.mark.parametrize("N,d,seed", [(20000, 50, 1), (3000, 37, 5), (9000, 300, 4)])
def test_countsketch_buckets_match_oracle(N, d, seed):
    X, Y, _ = gaussian_problem(N, d, 1.0, seed=seed)
    sc = cs_schedule(N, d, 1e-6)
    s = S.Solver(cuda(X), cuda(Y))
    s.sketch(seed, sc)
    mK = sc.m[sc.K - 1]
    A_g, b_g = (t.cpu().numpy() for t in s.export_sketch(0, mK))
    h, sg = CS.stage_hash(N, mK, seed)
    XY = np.concatenate([X, Y[:, None]], axis=1)
    top = CS.countsketch_apply(XY, h, sg, mK)
    l1 = CS.countsketch_apply(np.abs(XY), h, np.ones(N), mK)
    cnt = np.bincount(h, minlength=mK).astype(float)[:, None]
    nb = int(math.log2(1 << (N - 1).bit_length()))
    mx = np.abs(XY).max(0)[None, :]
    tol = cnt * mx * 2.0 ** (nb - 62) + (cnt * U / (1 - cnt * U)) * l1 + 2 * U * np.abs(top)
    G = np.concatenate([A_g, b_g[:, None]], axis=1)
    assert np.all(np.abs(G - top) <= tol)
    # the preconditioner factor from the independent CountSketch
    _, A_hat = CS.cs_sketches(X, Y, seed, [mK], sc.r)
    R_g = s.export_precond()[0].cpu().numpy()
    R_o = OL.r_factor(A_hat)
    kappa = np.linalg.cond(A_hat)
    rd = sc.r * d
    tol_R = 2 * math.sqrt(2) * kappa * (rd * U / (1 - rd * U)) * (
        np.linalg.norm(A_hat) / np.linalg.norm(A_hat, 2)) + 1e-13
    assert np.linalg.norm(R_g - R_o) <= tol_R * np.linalg.norm(R_o, 2)
    s.close()


@pytest.mark.parametrize("precision,tol", [(S.PREC_FP64, 1e-10), (S.PREC_FP64, 1e-6),
                                           (S.PREC_MIXED, 1e-6)])
@pytest.mark.parametrize("N,d,kappa,seed", [(20000, 50, None, 1), (16384, 40, 1e6, 2),
                                            (70000, 129, 1e5, 8)])
def test_spcg_cs_solve_meets_tolerance(precision, tol, N, d, kappa, seed):
    if kappa is None:
        X, Y, _ = gaussian_problem(N, d, 1.0, seed=seed)
    else:
        X, Y, _ = svd_problem(N, d, kappa, 0.1, seed=seed)
    o = S.Opts()
    o.precision = precision
    s = S.Solver(cuda(X), cuda(Y), o)
    beta, info, st = s.solve(seed, cs_schedule(N, d, tol))
    assert st == S.SPCG_OK and info.converged == 1
    assert rel_pred_error(X, beta.cpu().numpy(), OL.ols(X, Y)) <= tol
    s.close()


def test_spcg_cs_stage_iterates_match_oracle():
    N, d, seed = 20000, 50, 3
    X, Y, _ = gaussian_problem(N, d, 1.0, seed=seed)
    sched = OS.default_schedule(N, d)
    stages, A_hat = CS.cs_sketches(X, Y, seed, sched["m"], sched["r"])
    R = OL.r_factor(A_hat)
    s = S.Solver(cuda(X), cuda(Y))
    s.sketch(seed, cs_schedule(N, d, 1e-6))
    beta_g = torch.zeros(d, dtype=torch.float64, device="cuda")
    beta_o = np.zeros(d)
    for i, ((A_i, b_i), a_i) in enumerate(zip(stages, sched["a"])):
        beta_o, _ = OS.pcg(A_i, b_i, R, beta_o, a_i)
        s.pcg_stage(i, a_i, beta_g)
        assert rel_pred_error(X, beta_g.cpu().numpy(), beta_o) <= 1e-10, i
    s.close()


@pytest.mark.parametrize("precision,tol", [(S.PREC_FP64, 1e-10), (S.PREC_MIXED, 1e-6)])
def test_tuned_schedule_solve(precision, tol):
    N, d = 1 << 17, 64
    X, Y, _ = svd_problem(N, d, 1e4, 0.1, seed=4)
    sc = S.spcg_tuned_schedule(N, d)
    sc.tol = tol
    o = S.Opts()
    o.precision = precision
    s = S.Solver(cuda(X), cuda(Y), o)
    beta, info, st = s.solve(2, sc)
    assert st == S.SPCG_OK and rel_pred_error(X, beta.cpu().numpy(), OL.ols(X, Y)) <= tol
    assert info.K == sc.K and list(info.stage_iters[: sc.K]) == [4] * sc.K
    s.close()


def test_countsketch_schedule_validation():
    X, Y, _ = gaussian_problem(5000, 20, 1.0, seed=3)
    s = S.Solver(cuda(X), cuda(Y))
    bad = S.make_schedule([300, 600], [3, 3], 120, sketch=S.SKETCH_COUNT)   # not powers of two
    with pytest.raises(S.SpcgError) as e:
        s.sketch(1, bad)
    assert e.value.status == S.SPCG_E_INVALID_ARG
    s.close()
