"""The premise of the mixed form's operand rule (CPU, no GPU).

Rounding X to FP32, X~ = X + E with |E_ij| <= 2^-24 |X_ij|, perturbs the
preconditioned Gram operator by
    R^{-T} (X~^T X~ - X^T X) R^{-1} = 2 sym(Q^T E R^{-1}) + (E R^{-1})^T (E R^{-1}),
Q = X R^{-1}, so its norm is at most 2 ||E R^{-1}|| + ||E R^{-1}||^2, and
||E R^{-1}|| <= ||E D^{-1}|| ||D R^{-1}|| with D the column norms.  The rule
compares 2^-24 nu, nu = ||D R^{-1}||_2, with a threshold; these checks pin
that 2^-24 nu tracks ||E R^{-1}|| within a modest factor on the workloads'
SVD construction, and that the perturbation bound holds.
"""
import numpy as np
import pytest

from paper_2607_25272_b300.inputs import svd_problem

U32 = 2.0 ** -24


@pytest.mark.parametrize("N,d,kappa", [(4096, 32, 1e3), (4096, 32, 1e6), (8192, 64, 1e8),
                                       (8192, 64, 1e10)])
def test_fp32_rounding_perturbs_the_preconditioned_operator_by_about_u_nu(N, d, kappa):
    X, _, _ = svd_problem(N, d, kappa, 0.1, seed=3)
    R = np.linalg.qr(X)[1]
    Rinv = np.linalg.inv(R)
    D = np.sqrt((R * R).sum(axis=0))
    nu = np.linalg.norm(D[:, None] * Rinv, 2)
    E = X.astype(np.float32).astype(np.float64) - X
    assert np.all(np.abs(E) <= U32 * np.abs(X))
    er = np.linalg.norm(E @ Rinv, 2)
    # ||E R^{-1}|| <= ||E D^{-1}||_F nu <= 2^-24 sqrt(d) nu, and in practice near 2^-24 nu
    assert er <= U32 * np.sqrt(d) * nu
    assert 0.1 * U32 * nu <= er <= U32 * nu
    Xt = X + E
    M = Rinv.T @ (Xt.T @ Xt - X.T @ X) @ Rinv
    pert = np.linalg.norm(M, 2)
    assert pert <= 2 * er + er * er + 1e-12
    # where 2^-24 nu exceeds one the FP32 operator is no longer a contraction's
    # worth of accurate (the rule moves to the double-FP32 pair there)
    if U32 * nu > 50:
        assert pert > 1.0


# ---- the true-gradient rule: double-FP32 arithmetic in the stopping metric ----
F32 = np.float32


def _two_sum(a, b):
    s = (a + b).astype(F32)
    bb = (s - a).astype(F32)
    return s, ((a - (s - bb)).astype(F32) + (b - bb).astype(F32)).astype(F32)


def _fma32(a, b, c):
    # the product of two FP32 values is exact in FP64; one rounding to FP32
    return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(F32)


def _split(v):
    h = v.astype(F32)
    return h, (v - h.astype(np.float64)).astype(F32)


def _pair_gradient(X, b, x, nseq=256):
    """X^T (b - X x) in double-FP32 arithmetic: X, b and x split into FP32
    pairs, products by TwoProd, sums by TwoSum (the low words plainly), the
    row sums over nseq interleaved sequences renormalised every eight rows."""
    N, d = X.shape
    Xh, Xl = _split(X)
    ph, pl = _split(x)
    bh, bl = _split(b)
    sh = np.zeros(N, F32)
    sl = np.zeros(N, F32)
    for j in range(d):
        pr = (Xh[:, j] * ph[j]).astype(F32)
        pe = _fma32(Xh[:, j], np.full(N, ph[j], F32), -pr)
        sh, se = _two_sum(sh, pr)
        cross = _fma32(Xh[:, j], np.full(N, pl[j], F32), (Xl[:, j] * ph[j]).astype(F32))
        sl = (sl + ((pe + se).astype(F32) + cross).astype(F32)).astype(F32)
    th, tl = _two_sum(bh, -sh)
    tl = (tl + (bl - sl).astype(F32)).astype(F32)
    th, tl = _two_sum(th, tl)
    wh = np.zeros((nseq, d), F32)
    wl = np.zeros((nseq, d), F32)
    for k in range(N // nseq):
        rows = slice(k * nseq, (k + 1) * nseq)
        T = np.broadcast_to(th[rows][:, None], (nseq, d))
        pr = (T * Xh[rows]).astype(F32)
        pe = _fma32(T, Xh[rows], -pr)
        wh, se = _two_sum(wh, pr)
        cross = _fma32(T, Xl[rows], (tl[rows][:, None] * Xh[rows]).astype(F32))
        wl = (wl + ((pe + se).astype(F32) + cross).astype(F32)).astype(F32)
        if k % 8 == 7:
            wh, wl = _two_sum(wh, wl)
    return wh.astype(np.float64).sum(0) + wl.astype(np.float64).sum(0)


@pytest.mark.parametrize("kappa", [1e4, 1e6, 1e8])
def test_pair_gradient_error_in_the_stopping_metric_scales_with_nu(kappa):
    """At the OLS solution the double-FP32 gradient's error, measured as the
    stopping rule measures it (sqrt(dg^T H^{-1} dg) with H = R^T R), stays
    within a small multiple of 2^-48 nu ||R beta||; where 2^-48 nu <= tol/64
    (the rule's condition for using it) that is far below the threshold
    (tol/2) ||R beta||."""
    from scipy.linalg import solve_triangular
    N, d, tol = 16384, 64, 1e-6
    X, Y, _ = svd_problem(N, d, kappa, 1.0, seed=5)
    Q, R = np.linalg.qr(X)
    beta = np.linalg.solve(R, Q.T @ Y)
    XL = X.astype(np.longdouble)
    g_exact = (XL.T @ (Y.astype(np.longdouble) - XL @ beta.astype(np.longdouble))).astype(np.float64)
    D = np.sqrt((R * R).sum(axis=0))
    nu = np.linalg.norm(D[:, None] * np.linalg.inv(R), 2)
    err = np.linalg.norm(solve_triangular(R.T, _pair_gradient(X, Y, beta) - g_exact, lower=True))
    rb = np.linalg.norm(R @ beta)
    assert err <= 4 * 2.0 ** -48 * nu * rb
    if 2.0 ** -48 * nu <= tol / 64:
        assert err <= (tol / 2) * rb / 8
