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
