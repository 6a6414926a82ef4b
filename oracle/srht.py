"""Nested SRHT sketches (oracle side; test infrastructure).

Follows Sec. 2.1 (SRHT definition S = sqrt(N/m) (H D P)_{I,:}) and Sec. 2.2
(the nested construction: Z_X = H D P X and Z_Y = H D P Y are formed once,
the row sets I_1 c ... c I_K are nested with m_{i+1} = 2 m_i, and
S_i X = sqrt(N/m_i) (Z_X)_{I_i,:}).  The preconditioner uses an independent
r-row sample I-hat of the same transform (Sec. 2.2; the cost count of the
proof of Theorem 3.4 charges a single Hadamard transform plus O(r d^2 + d^3)).

Readings where the paper is silent:
* N not a power of two: rows are zero-padded to N' = 2^ceil(log2 N)
  (the SRHT of Sec. 2.1 is stated for N a power of two).
* H is the normalised Walsh-Hadamard matrix in Sylvester (natural) order,
  H_jk = (-1)^popcount(j & k) / sqrt(N').
* P, the nested order pi and I-hat are Feistel permutations keyed by
  Philox (see ``oracle.philox``): (P X')_j = X'_{P(j)}, I_i = {pi(t): t < m_i},
  I-hat = {sigma_hat(t): t < r}; sampling is without replacement.

Pins (tests/test_oracle_srht.py): the fast transform equals the explicit
Sylvester matrix product for N' <= 2^10 and the one-row brute-force formula
``srht_row`` at any size; H H = I; norms are preserved; the full-sampling
special case m = N' gives S^T S = I.
"""
import numpy as np

from .philox import (TAG_HAT, TAG_P, TAG_PI, feistel_permute,
                     rademacher_signs)


def padded_rows(n_rows):
    """N' = 2^ceil(log2 N) for N >= 1."""
    if n_rows < 1:
        raise ValueError("N must be >= 1")
    return 1 << (int(n_rows) - 1).bit_length()


def log2_exact(n):
    k = int(n).bit_length() - 1
    if (1 << k) != n:
        raise ValueError("not a power of two")
    return k


def fwht_rows(M):
    """In place: M <- H M with H the normalised Sylvester Walsh-Hadamard
    matrix of order M.shape[0] (a power of two).  Radix-2 butterflies."""
    n_rows = M.shape[0]
    log2_exact(n_rows)
    cols = M.shape[1:]
    h = 1
    while h < n_rows:
        view = M.reshape((n_rows // (2 * h), 2, h) + cols)
        a = view[:, 0].copy()
        b = view[:, 1]
        view[:, 0] = a + b
        view[:, 1] = a - b
        h *= 2
    M *= 1.0 / np.sqrt(n_rows)
    return M


def sylvester_matrix(n_rows):
    """Explicit normalised H of order n_rows (small sizes; test pin)."""
    j = np.arange(n_rows)
    bits = np.bitwise_and.outer(j, j)
    parity = np.zeros_like(bits)
    while np.any(bits):
        parity ^= bits & 1
        bits >>= 1
    return np.where(parity == 0, 1.0, -1.0) / np.sqrt(n_rows)


def srht_transform(X, Y, seed):
    """(Z_X, Z_Y) = (H D P X', H D P Y') of Sec. 2.2, with X' = [X; 0].

    Returns Z_X (N' x d) and Z_Y (N',)."""
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    n_rows, d = X.shape
    n_pad = padded_rows(n_rows)
    nbits = log2_exact(n_pad)
    perm = feistel_permute(np.arange(n_pad), nbits, TAG_P, seed)
    signs = rademacher_signs(n_pad, seed)
    W = np.zeros((n_pad, d + 1))
    W[:n_rows, :d] = X
    W[:n_rows, d] = Y
    W = signs[:, None] * W[perm]          # (D P X')_k = D_k X'_{P(k)}
    fwht_rows(W)
    return W[:, :d].copy(), W[:, d].copy()


def srht_row(X, Y, seed, j):
    """Row j of (Z_X, Z_Y) by the defining sum (brute force, O(N' d))."""
    X = np.asarray(X, dtype=np.float64)
    n_rows, d = X.shape
    n_pad = padded_rows(n_rows)
    nbits = log2_exact(n_pad)
    k = np.arange(n_pad)
    perm = feistel_permute(k, nbits, TAG_P, seed)
    signs = rademacher_signs(n_pad, seed)
    bits = np.bitwise_and(k, j)
    parity = np.zeros(n_pad, dtype=np.int64)
    while np.any(bits):
        parity ^= bits & 1
        bits >>= 1
    h = np.where(parity == 0, 1.0, -1.0) / np.sqrt(n_pad)
    coef = h * signs
    src = perm
    valid = src < n_rows
    zx = coef[valid] @ X[src[valid]]
    zy = coef[valid] @ np.asarray(Y, dtype=np.float64)[src[valid]]
    return zx, zy


def nested_order(n_pad, count, seed):
    """pi(0..count-1): the first rows of the nested order (I_i = pi[:m_i])."""
    return feistel_permute(np.arange(count), log2_exact(n_pad), TAG_PI, seed)


def hat_order(n_pad, r, seed):
    """I-hat = sigma_hat(0..r-1): the preconditioner rows."""
    return feistel_permute(np.arange(r), log2_exact(n_pad), TAG_HAT, seed)


def nested_sketches(ZX, ZY, m_list, r, seed):
    """Sketched pairs (S_i X, S_i Y) for every m_i in m_list and the
    preconditioner sketch S-hat X (Sec. 2.2), scaled as in the paper:
    S_i X = sqrt(N'/m_i) (Z_X)_{I_i,:}, S-hat X = sqrt(N'/r) (Z_X)_{I-hat,:}.
    """
    n_pad = ZX.shape[0]
    m_max = max(m_list) if len(m_list) else 0
    pi = nested_order(n_pad, m_max, seed)
    stages = []
    for m in m_list:
        scale = np.sqrt(n_pad / m)
        rows = pi[:m]
        stages.append((scale * ZX[rows], scale * ZY[rows]))
    hat = hat_order(n_pad, r, seed)
    A_hat = np.sqrt(n_pad / r) * ZX[hat]
    return stages, A_hat
