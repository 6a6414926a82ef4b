"""Pins for the oracle's counter-based generator and Feistel permutations
(Sec. 2.1: D is a Rademacher diagonal, P a random permutation, I a uniformly
sampled row set).  Philox4x32-10 itself is pinned word for word against an
independent implementation, Triton's generator run by its CPU interpreter
(a wrong multiplier, Weyl constant, round count, key split or word order
changes every word); the other checks are properties that a swapped word or
a broken inverse would fail."""
import os
import subprocess
import sys

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


def _triton_words(tmp_path, ctr, seeds, rounds):
    src, dst = tmp_path / "in.npz", tmp_path / "out.npz"
    np.savez(src, ctr=ctr.astype(np.uint32), seeds=np.array(seeds, dtype=np.uint64),
             rounds=np.int64(rounds))
    helper = os.path.join(os.path.dirname(os.path.abspath(__file__)), "philox_triton_ref.py")
    subprocess.run([sys.executable, helper, str(src), str(dst)], check=True, timeout=600,
                   capture_output=True)
    return np.load(dst)["words"]


def test_philox_matches_an_independent_implementation(tmp_path):
    """Philox4x32-10 (Salmon et al., SC'11) word for word against Triton's
    implementation of the same generator, over random counters plus the
    all-zero and all-ones counters, and keys whose halves are zero, small,
    mixed and all ones.  The same comparison with Triton at 7 rounds must
    disagree in every word, so the pin sees the round count."""
    pytest.importorskip("triton")
    rng = np.random.default_rng(2024)
    ctr = rng.integers(0, 2**32, size=(128, 4), dtype=np.uint64)
    ctr[0] = 0
    ctr[1] = 0xFFFFFFFF
    seeds = [0, 1, 2, 0x1234_5678_9ABC, 2**63 - 1, 2**63 + 12345, 2**64 - 1]
    ours = np.stack([np.stack(philox4x32_10(ctr[:, 0], ctr[:, 1], ctr[:, 2], ctr[:, 3], sd),
                              axis=1) for sd in seeds])
    ref = _triton_words(tmp_path, ctr, seeds, 10)
    assert ref.shape == ours.shape
    assert np.array_equal(ref, ours)
    ref7 = _triton_words(tmp_path, ctr, seeds, 7)
    assert not np.any(ref7 == ours)
