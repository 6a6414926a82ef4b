"""PCG and SPCG, Algorithm 1 (oracle side; test infrastructure).

* ``default_schedule`` - the experimental schedule of Sec. 4: m_1 = 8d,
  m_{i+1} = 2 m_i, m_K = N/2, r = 6d, a_i = 3 (the choice of Sec. 4.1).
  Readings: N' = 2^ceil(log2 N); m_1 = 2^ceil(log2 8d) because Theorem 3.1
  takes m_1 a power of two; m_K = N'/2 so that m_K < N holds.
* ``pcg`` - PCG(A, b, H-hat, beta_init, a) of Sec. 2.2 on the normal
  equations A^T A beta = A^T b preconditioned by H-hat = R^T R.  The paper
  prints no recurrence; this is the d-space form whose per-iteration cost
  is the (4m + 13)d + 2d^2 flops that Sec. 2.2 charges: one product
  w = A^T (A p), two triangular solves, three dot products and three axpys.
* ``spcg`` - Algorithm 1: Stage I runs a_i PCG iterations on each sketched
  pair, warm-started from the previous beta; Stage II runs PCG on (X, Y).
* ``full_pcg`` - Stage II with a stopping rule (the paper fixes T = 100 and
  judges with the true beta, Sec. 4; this oracle needs a rule that uses
  only computable quantities).  Reading: stop when
  sqrt(gamma) <= tau * ||R beta|| with tau = tol / 2, where
  gamma = g^T H-hat^{-1} g; then recompute g from the true residual
  X^T (Y - X beta) and stop only if the test still holds (else restart PCG
  from that gradient).  By Lemma A.4, H-hat^{-1/2} X^T X H-hat^{-1/2} has its
  spectrum in [1/(1+eps), 1/(1-eps)], so ||X(beta - beta-hat)|| <=
  sqrt(gamma) / sqrt(1 - eps) and ||X beta|| >= ||R beta|| / sqrt(1 + eps);
  with tau = tol/2 the relative prediction error is below tol whenever
  eps <= 0.6 (r = 6d gives eps near sqrt(d/r) ~ 0.4).  A tighter tau would
  sit on the FP64 rounding floor of the true gradient at kappa = 1e6.
* ``thm33_bound`` - the unrounded lower bound on a_i of Theorem 3.3.

Pins (tests/test_oracle_spcg.py): finite termination of PCG within d
iterations on small well-conditioned problems; the CG bound of Lemma A.2
with the exactly computed condition number; the stage contraction of
Eq. (app-stage-intermediate) with the exactly measured embedding distortion
epsilon; the full-sampling special case (m = N', I-hat = all rows: the
sketched solution is the OLS solution and Stage II needs one iteration);
the Theorem 3.3 values of the Fig. 1a discussion (below 3 on
omega in [2^-4, 1], decreasing in omega, a_2 and a_K nearly equal);
the final error reaching the OLS level (Theorem 3.2); the Table 1 SPCG
iteration counts to within a loose band.
"""
import math

import numpy as np

from .linalg import apply_precond, r_factor
from .srht import nested_sketches, padded_rows, srht_transform


class PCGBreakdown(RuntimeError):
    """p^T w <= 0 or a non-finite value inside PCG."""


def default_schedule(N, d, a=3):
    """{m_i}, {a_i}, r of Sec. 4 with the readings stated above."""
    n_pad = padded_rows(N)
    m1 = 1 << (8 * d - 1).bit_length()
    m = []
    mi = m1
    while mi <= n_pad // 2:
        m.append(mi)
        mi *= 2
    return {"m": m, "a": [a] * len(m), "r": 6 * d, "n_pad": n_pad}


def thm33_bound(m_prev, m_cur, d, omega):
    """ln{[(1 + omega) r + 1] / omega} / ln 4, r = sqrt((m_i - d)/(m_{i-1} - d))."""
    ratio = math.sqrt((m_cur - d) / (m_prev - d))
    return math.log(((1.0 + omega) * ratio + 1.0) / omega) / math.log(4.0)


def pcg(A, b, R, beta0, a, callback=None):
    """a iterations of PCG on min ||A beta - b|| preconditioned by R^T R.

    Returns (beta, gammas) with gammas[k] = g_k^T z_k before iteration k+1.
    callback(beta) is called after every iteration (for error histories).
    """
    beta = np.array(beta0, dtype=np.float64, copy=True)
    g = A.T @ (b - A @ beta)
    z = apply_precond(R, g)
    p = z.copy()
    gamma = g @ z
    gammas = [gamma]
    for _ in range(a):
        if gamma == 0.0:
            break
        w = A.T @ (A @ p)
        pw = p @ w
        if not np.isfinite(pw) or pw <= 0.0:
            raise PCGBreakdown("p^T A^T A p <= 0 or not finite")
        alpha = gamma / pw
        beta += alpha * p
        g -= alpha * w
        z = apply_precond(R, g)
        gamma_new = g @ z
        p = z + (gamma_new / gamma) * p
        gamma = gamma_new
        gammas.append(gamma)
        if callback is not None:
            callback(beta)
    return beta, gammas


def full_pcg(X, Y, R, beta0, tol, max_iters=100, max_restarts=5, callback=None):
    """Stage II until the stopping rule holds (see module docstring).

    Returns (beta, iterations, converged)."""
    tau = tol / 2.0
    beta = np.array(beta0, dtype=np.float64, copy=True)
    g = X.T @ (Y - X @ beta)
    true_gradient = True
    z = apply_precond(R, g)
    p = z.copy()
    gamma = g @ z
    iters = 0
    restarts = 0
    while True:
        if math.sqrt(max(gamma, 0.0)) <= tau * np.linalg.norm(R @ beta):
            if true_gradient:
                return beta, iters, True
            if restarts >= max_restarts:
                return beta, iters, False
            restarts += 1
            g = X.T @ (Y - X @ beta)
            true_gradient = True
            z = apply_precond(R, g)
            p = z.copy()
            gamma = g @ z
            continue
        if gamma == 0.0:
            return beta, iters, True
        if iters >= max_iters:
            return beta, iters, False
        w = X.T @ (X @ p)
        pw = p @ w
        if not np.isfinite(pw) or pw <= 0.0:
            raise PCGBreakdown("p^T X^T X p <= 0 or not finite")
        alpha = gamma / pw
        beta += alpha * p
        g -= alpha * w
        true_gradient = False
        z = apply_precond(R, g)
        gamma_new = g @ z
        p = z + (gamma_new / gamma) * p
        gamma = gamma_new
        iters += 1
        if callback is not None:
            callback(beta)


def sketch_all(X, Y, seed, schedule):
    """Nested sketches and the preconditioner factor R (Sec. 2.2)."""
    ZX, ZY = srht_transform(X, Y, seed)
    stages, A_hat = nested_sketches(ZX, ZY, schedule["m"], schedule["r"], seed)
    R = r_factor(A_hat)
    return stages, A_hat, R


def spcg(X, Y, seed, schedule=None, tol=1e-6, beta0=None, max_iters=100,
         max_restarts=5, callback=None):
    """Algorithm 1 with the Stage II stopping rule of ``full_pcg``.

    Returns a dict with beta, R, the per-stage betas and iteration counts."""
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    N, d = X.shape
    if schedule is None:
        schedule = default_schedule(N, d)
    stages, A_hat, R = sketch_all(X, Y, seed, schedule)
    beta = np.zeros(d) if beta0 is None else np.array(beta0, dtype=np.float64)
    stage_betas = []
    for (A_i, b_i), a_i in zip(stages, schedule["a"]):
        beta, _ = pcg(A_i, b_i, R, beta, a_i, callback=callback)
        stage_betas.append(beta.copy())
    beta, s_iters, converged = full_pcg(X, Y, R, beta, tol, max_iters,
                                        max_restarts, callback=callback)
    return {"beta": beta, "R": R, "A_hat": A_hat, "stage_betas": stage_betas,
            "stage_iters": list(schedule["a"]), "refine_iters": s_iters,
            "converged": converged, "schedule": schedule}


def tuned_schedule(N, d, a=4):
    """The tuned sketch-size schedule of Sec. 4.3, generalised in d and N.

    For N = 2^22, d = 2^6 the paper uses m_i in {2^10, ..., 2^16} followed by a
    single subproblem of size 2^20 and a_i = 4.  Reading: m_1 = 2^ceil(log2 16d)
    (= 2^10 at d = 64), seven doublings at most, all below N'/4, then one
    transition stage of size N'/4 (= 2^20 at N = 2^22); r = 6d.
    """
    n_pad = 1 << (int(N) - 1).bit_length()
    m = []
    mi = 1 << (16 * d - 1).bit_length()
    while len(m) < 7 and mi < n_pad // 4:
        m.append(mi)
        mi *= 2
    if n_pad // 4 > (m[-1] if m else 0) and n_pad // 4 > 6 * d:
        m.append(n_pad // 4)
    return {"m": m, "a": [a] * len(m), "r": 6 * d, "n_pad": n_pad}
