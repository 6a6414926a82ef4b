"""CountSketch variant of SPCG, SPCG-CS (oracle side; test infrastructure).

Sec. 3 (after Theorem 3.4) and Sec. 4.3: the sketches of the initialisation
stage are CountSketches instead of SRHTs, so the initialisation costs O(Nd).
A CountSketch S (m x N) has one nonzero per column: S_{h(j), j} = s(j) with a
uniform bucket h(j) in [m] and a Rademacher sign s(j); E[S^T S] = I with no
scale factor.

Readings (the paper gives no construction details):
* Nesting: one hash h_K into m_K buckets; stage i uses h_i(j) = h_K(j) mod m_i
  (m_i powers of two), which is again uniform and independent over j, so S_i
  is a CountSketch and S_i X is obtained by folding the buckets of S_K X
  (bucket t of stage i collects buckets t, t + m_i, ... of stage K).
* The preconditioner uses an independent CountSketch with r = 6d rows (the
  paper replaces the SRHT throughout the initialisation; its sketched Hessian
  is r = 6d in every experiment).
* Draws: for row j < N, w = philox(ctr = (j lo, j hi, TAG, 0), key = seed);
  stage hash h_K(j) = w0 mod m_K (m_K a power of two) with TAG = 4; the
  preconditioner bucket is floor(w0 r / 2^32) with TAG = 5; the sign is
  +1 iff bit 0 of w1 is clear.

Pins (tests/test_oracle_countsketch.py): the scatter equals the product with
the explicit matrix S; folding equals the CountSketch with h mod m_i built
directly; E[S^T S] = I over seeds; SPCG-CS reaches the OLS estimator under the
stopping rule.
"""
import numpy as np

from .linalg import r_factor
from .philox import MASK32, philox4x32_10
from .spcg import full_pcg, pcg

TAG_CS = 4
TAG_CS_HAT = 5


def _draws(n_rows, seed, tag):
    j = np.arange(n_rows, dtype=np.uint64)
    w0, w1, _, _ = philox4x32_10(j & MASK32, j >> np.uint64(32), tag, 0, seed)
    sign = np.where((w1 & np.uint32(1)) == 0, 1.0, -1.0)
    return w0.astype(np.uint64), sign


def stage_hash(n_rows, m_top, seed):
    if m_top & (m_top - 1):
        raise ValueError("m_K must be a power of two")
    w0, sign = _draws(n_rows, seed, TAG_CS)
    return (w0 & np.uint64(m_top - 1)).astype(np.int64), sign


def hat_hash(n_rows, r, seed):
    w0, sign = _draws(n_rows, seed, TAG_CS_HAT)
    return ((w0 * np.uint64(r)) >> np.uint64(32)).astype(np.int64), sign


def countsketch_apply(M, buckets, signs, m):
    """S M for the CountSketch (buckets, signs) with m rows (scatter-add)."""
    out = np.zeros((m,) + M.shape[1:])
    np.add.at(out, buckets, signs.reshape((-1,) + (1,) * (M.ndim - 1)) * M)
    return out


def explicit_matrix(buckets, signs, m):
    S = np.zeros((m, len(buckets)))
    S[buckets, np.arange(len(buckets))] = signs
    return S


def fold(SM, m):
    """Buckets of a CountSketch with SM.shape[0] rows folded modulo m."""
    out = np.zeros((m,) + SM.shape[1:])
    for start in range(0, SM.shape[0], m):
        out += SM[start:start + m]
    return out


def cs_sketches(X, Y, seed, m_list, r):
    """(S_i X, S_i Y) for every m_i and the preconditioner sketch S-hat X."""
    N = X.shape[0]
    XY = np.concatenate([X, Y[:, None]], axis=1)
    m_top = max(m_list)
    h, s = stage_hash(N, m_top, seed)
    top = countsketch_apply(XY, h, s, m_top)
    stages = []
    for m in m_list:
        SM = fold(top, m)
        stages.append((SM[:, :-1], SM[:, -1]))
    hh, hs = hat_hash(N, r, seed)
    A_hat = countsketch_apply(X, hh, hs, r)
    return stages, A_hat


def spcg_cs(X, Y, seed, schedule, tol=1e-6, max_iters=100, max_restarts=5, callback=None):
    """Algorithm 1 with CountSketch sketches (SPCG-CS)."""
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    stages, A_hat = cs_sketches(X, Y, seed, schedule["m"], schedule["r"])
    R = r_factor(A_hat)
    beta = np.zeros(X.shape[1])
    stage_betas = []
    for (A_i, b_i), a_i in zip(stages, schedule["a"]):
        beta, _ = pcg(A_i, b_i, R, beta, a_i, callback=callback)
        stage_betas.append(beta.copy())
    beta, s_iters, converged = full_pcg(X, Y, R, beta, tol, max_iters, max_restarts,
                                        callback=callback)
    return {"beta": beta, "R": R, "stage_betas": stage_betas, "refine_iters": s_iters,
            "converged": converged}
