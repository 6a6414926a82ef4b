"""Counter-based random draws for the SRHT (oracle side; test infrastructure).

Philox4x32-10 is written from its published definition: J. K. Salmon,
M. A. Moraes, R. O. Dror, D. E. Shaw, "Parallel random numbers: as easy as
1, 2, 3", SC'11.  A 4x32-bit counter and a 2x32-bit key go through ten
rounds; each round multiplies counter words 0 and 2 by two odd constants
into 64-bit products and mixes the high halves with the key and the other
two words, and the key is bumped by two Weyl constants between rounds.

On top of Philox this module defines the permutations that the SRHT of
Sec. 2.1 needs (P, and the uniformly sampled row sets I_i and I-hat of
Sec. 2.2): an alternating (possibly unbalanced) Feistel network on n-bit
indices whose round function is Philox.  Every Feistel round XORs one half
with a function of the other half, so the map is a bijection of
[0, 2^n) for any round function, and its inverse runs the rounds backwards.

Counter layout (the CUDA side implements the same definition separately):

* sign of row k (the Rademacher diagonal D):
      word0(philox(ctr=(k mod 2^32, k >> 32, TAG_SIGN, 0), key=seed)) & 1
      -> D_k = +1 if the bit is 0, -1 if it is 1
* Feistel round i of permutation ``tag`` on n bits, applied to half-value v:
      F = word0(philox(ctr=(v, i, tag, n), key=seed))

Parity: the CPU and GPU generators are compared bit for bit (integer work).
Pins: Philox4x32-10 word for word against an independent implementation of
the same published generator (Triton's, run by its CPU interpreter; the
published known-answer vectors themselves are not available offline), which
fixes the multipliers, Weyl constants, round count, key split and word
order; bijectivity and inverse on exhaustive small domains, bit balance and
chi-square uniformity of Philox words, uniform position distribution of the
permutation over seeds, avalanche of the round function.
"""
import numpy as np

PHILOX_M0 = np.uint64(0xD2511F53)
PHILOX_M1 = np.uint64(0xCD9E8D57)
PHILOX_W0 = np.uint64(0x9E3779B9)
PHILOX_W1 = np.uint64(0xBB67AE85)
MASK32 = np.uint64(0xFFFFFFFF)

TAG_P = 0      # permutation P applied before the Hadamard transform
TAG_SIGN = 1   # Rademacher diagonal D
TAG_PI = 2     # order pi of the nested row sets I_1 c ... c I_K
TAG_HAT = 3    # independent preconditioner row sample I-hat

FEISTEL_ROUNDS = 8


def philox4x32_10(c0, c1, c2, c3, seed):
    """Philox4x32-10 on arrays of counters; returns four uint32 arrays.

    seed is a Python int < 2^64: key = (seed mod 2^32, seed >> 32).
    """
    c0 = np.asarray(c0, dtype=np.uint64) & MASK32
    c1 = np.asarray(c1, dtype=np.uint64) & MASK32
    c2 = np.asarray(c2, dtype=np.uint64) & MASK32
    c3 = np.asarray(c3, dtype=np.uint64) & MASK32
    c0, c1, c2, c3 = np.broadcast_arrays(c0, c1, c2, c3)
    c0, c1, c2, c3 = c0.copy(), c1.copy(), c2.copy(), c3.copy()
    k0 = np.uint64(seed & 0xFFFFFFFF)
    k1 = np.uint64((seed >> 32) & 0xFFFFFFFF)
    for rnd in range(10):
        if rnd > 0:
            k0 = (k0 + PHILOX_W0) & MASK32
            k1 = (k1 + PHILOX_W1) & MASK32
        prod0 = PHILOX_M0 * c0          # < 2^64, exact in uint64
        prod1 = PHILOX_M1 * c2
        hi0, lo0 = prod0 >> np.uint64(32), prod0 & MASK32
        hi1, lo1 = prod1 >> np.uint64(32), prod1 & MASK32
        c0, c1, c2, c3 = (hi1 ^ c1 ^ k0), lo1, (hi0 ^ c3 ^ k1), lo0
    return (c0.astype(np.uint32), c1.astype(np.uint32),
            c2.astype(np.uint32), c3.astype(np.uint32))


def rademacher_signs(n_rows, seed):
    """D_k for k in [0, n_rows): +1.0 / -1.0 (Sec. 2.1, the diagonal D)."""
    k = np.arange(n_rows, dtype=np.uint64)
    w0, _, _, _ = philox4x32_10(k & MASK32, k >> np.uint64(32), TAG_SIGN, 0, seed)
    return np.where((w0 & np.uint32(1)) == 0, 1.0, -1.0)


def _split(nbits):
    b = nbits // 2          # low half width
    a = nbits - b           # high half width
    return a, b


def _round_fn(v, rnd, tag, nbits, seed):
    w0, _, _, _ = philox4x32_10(v, rnd, tag, nbits, seed)
    return w0.astype(np.uint64)


def feistel_permute(x, nbits, tag, seed, rounds=FEISTEL_ROUNDS):
    """sigma_tag(x): a pseudorandom bijection of [0, 2^nbits)."""
    x = np.asarray(x, dtype=np.uint64)
    a, b = _split(nbits)
    mask_a = np.uint64((1 << a) - 1)
    mask_b = np.uint64((1 << b) - 1)
    left = (x >> np.uint64(b)) & mask_a
    right = x & mask_b
    for rnd in range(rounds):
        if rnd % 2 == 0:
            left = left ^ (_round_fn(right, rnd, tag, nbits, seed) & mask_a)
        else:
            right = right ^ (_round_fn(left, rnd, tag, nbits, seed) & mask_b)
    return ((left << np.uint64(b)) | right).astype(np.int64)


def feistel_inverse(y, nbits, tag, seed, rounds=FEISTEL_ROUNDS):
    """sigma_tag^{-1}(y): the rounds of feistel_permute in reverse order."""
    y = np.asarray(y, dtype=np.uint64)
    a, b = _split(nbits)
    mask_a = np.uint64((1 << a) - 1)
    mask_b = np.uint64((1 << b) - 1)
    left = (y >> np.uint64(b)) & mask_a
    right = y & mask_b
    for rnd in reversed(range(rounds)):
        if rnd % 2 == 0:
            left = left ^ (_round_fn(right, rnd, tag, nbits, seed) & mask_a)
        else:
            right = right ^ (_round_fn(left, rnd, tag, nbits, seed) & mask_b)
    return ((left << np.uint64(b)) | right).astype(np.int64)
