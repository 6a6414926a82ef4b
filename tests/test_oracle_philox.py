"""Pins for the oracle's counter-based generator and Feistel permutations
(Sec. 2.1: D is a Rademacher diagonal, P a random permutation, I a uniformly
sampled row set).  Published known-answer vectors are not available offline;
the checks below are properties that a wrong constant, a dropped round, a
swapped word or a broken inverse would fail."""
import numpy as np
import pytest
from scipy import stats

from oracle.philox import (FEISTEL_ROUNDS, TAG_HAT, TAG_P, TAG_PI, TAG_SIGN,
                           feistel_inverse, feistel_permute, philox4x32_10,
                           rademacher_signs)


def _bits(words):
    w = np.asarray(words, dtype=np.uint64)
    return ((w[..., None] >> np.arange(32, dtype=np.uint64)) & np.uint64(1)).astype(np.int8)


def test_bit_balance_all_words():
    n = 1 << 16
    k = np.arange(n, dtype=np.uint64)
    words = philox4x32_10(k, 0, 5, 0, seed=0x1234_5678_9ABC)
    for w in words:
        frac = _bits(w).mean(axis=0)
        # each bit is fair: 6 sigma band of a Binomial(n, 1/2) fraction
        assert np.all(np.abs(frac - 0.5) < 6 * 0.5 / np.sqrt(n))


def test_uniform_top_byte_chi_square():
    n = 1 << 18
    k = np.arange(n, dtype=np.uint64)
    w0, w1, w2, w3 = philox4x32_10(k, 7, 1, 2, seed=99)
    for w in (w0, w1, w2, w3):
        counts = np.bincount((w >> np.uint32(24)).astype(np.int64), minlength=256)
        p = stats.chisquare(counts).pvalue
        assert p > 1e-6


def test_avalanche_on_counter_and_key():
    rng = np.random.default_rng(3)
    base = rng.integers(0, 2**32, size=(4, 2000), dtype=np.uint64)
    ref = np.stack(philox4x32_10(*base, seed=42))
    flips = []
    for word in range(4):
        for bit in (0, 13, 31):
            ctr = base.copy()
            ctr[word] ^= np.uint64(1 << bit)
            out = np.stack(philox4x32_10(*ctr, seed=42))
            flips.append(_bits(out ^ ref).sum(axis=(0, 2)).mean())
    out_key = np.stack(philox4x32_10(*base, seed=43))
    flips.append(_bits(out_key ^ ref).sum(axis=(0, 2)).mean())
    flips = np.array(flips)
    # 128 output bits: a good mixer flips 64 on average
    assert np.all(np.abs(flips - 64.0) < 1.0)


def test_streams_differ_by_tag_and_seed():
    k = np.arange(4096, dtype=np.uint64)
    a = philox4x32_10(k, 0, TAG_SIGN, 0, seed=1)[0]
    b = philox4x32_10(k, 0, TAG_PI, 0, seed=1)[0]
    c = philox4x32_10(k, 0, TAG_SIGN, 0, seed=2)[0]
    assert np.mean(a == b) < 0.01 and np.mean(a == c) < 0.01


def test_rademacher_signs_fair_and_seeded():
    s = rademacher_signs(1 << 16, seed=5)
    assert set(np.unique(s)) == {-1.0, 1.0}
    assert abs(s.mean()) < 6 / np.sqrt(s.size)
    assert np.array_equal(s, rademacher_signs(1 << 16, seed=5))


@pytest.mark.parametrize("nbits", list(range(0, 15)))
def test_feistel_is_a_bijection_with_inverse(nbits):
    n = 1 << nbits
    x = np.arange(n)
    for tag in (TAG_P, TAG_PI, TAG_HAT):
        y = feistel_permute(x, nbits, tag, seed=11 + nbits)
        assert np.array_equal(np.sort(y), x)
        assert np.array_equal(feistel_inverse(y, nbits, tag, seed=11 + nbits), x)


def test_feistel_position_and_pair_uniformity():
    # sigma(0) uniform over 16 positions and (sigma(0), sigma(1)) uniform
    # over the 240 ordered pairs, across seeds.
    nbits, seeds = 4, 12000
    first = np.empty(seeds, dtype=np.int64)
    pair = np.empty(seeds, dtype=np.int64)
    for s in range(seeds):
        y = feistel_permute(np.array([0, 1]), nbits, TAG_PI, seed=s)
        first[s] = y[0]
        pair[s] = y[0] * 16 + y[1]
    c1 = np.bincount(first, minlength=16)
    assert stats.chisquare(c1).pvalue > 1e-6
    c2 = np.bincount(pair, minlength=256)
    valid = np.array([a != b for a in range(16) for b in range(16)])
    assert np.all(c2[~valid] == 0)
    assert stats.chisquare(c2[valid]).pvalue > 1e-6


def test_feistel_rounds_matter():
    # fewer rounds give a different permutation (every round is used)
    x = np.arange(1 << 10)
    full = feistel_permute(x, 10, TAG_P, seed=8)
    for r in range(FEISTEL_ROUNDS):
        assert not np.array_equal(full, feistel_permute(x, 10, TAG_P, seed=8, rounds=r))
