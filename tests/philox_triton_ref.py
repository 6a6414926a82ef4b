"""Philox4x32 words from an implementation written independently of the
oracle: Triton's own generator (``tl.random.philox``, key = (seed mod 2^32,
seed >> 32), counter = four 32-bit words), run on the CPU by Triton's
interpreter.  Test infrastructure: tests/test_oracle_philox.py runs this
file in a subprocess (the interpreter is chosen by an environment variable
read when the kernel is defined) and compares its words with the oracle's.

Usage: python philox_triton_ref.py IN.npz OUT.npz
IN holds ``ctr`` (n x 4 uint32), ``seeds`` (uint64) and ``rounds`` (int);
OUT gets ``words`` (len(seeds) x n x 4 uint32).
"""
import os
import sys

os.environ["TRITON_INTERPRET"] = "1"

import numpy as np  # noqa: E402
import torch  # noqa: E402
import triton  # noqa: E402
import triton.language as tl  # noqa: E402


@triton.jit
def _philox_words(c_ptr, o_ptr, seed, BLOCK: tl.constexpr, ROUNDS: tl.constexpr):
    i = tl.arange(0, BLOCK)
    c0 = tl.load(c_ptr + 4 * i + 0)
    c1 = tl.load(c_ptr + 4 * i + 1)
    c2 = tl.load(c_ptr + 4 * i + 2)
    c3 = tl.load(c_ptr + 4 * i + 3)
    r0, r1, r2, r3 = tl.random.philox(seed, c0, c1, c2, c3, ROUNDS)
    tl.store(o_ptr + 4 * i + 0, r0.to(tl.int32, bitcast=True))
    tl.store(o_ptr + 4 * i + 1, r1.to(tl.int32, bitcast=True))
    tl.store(o_ptr + 4 * i + 2, r2.to(tl.int32, bitcast=True))
    tl.store(o_ptr + 4 * i + 3, r3.to(tl.int32, bitcast=True))


def main(src, dst):
    z = np.load(src)
    ctr = np.ascontiguousarray(z["ctr"].astype(np.uint32))
    n = ctr.shape[0]
    assert n > 0 and n & (n - 1) == 0, "the block is a power of two"
    rounds = int(z["rounds"])
    c = torch.from_numpy(ctr.view(np.int32).copy())
    words = []
    for seed in z["seeds"].tolist():
        out = torch.zeros_like(c)
        _philox_words[(1,)](c, out, int(seed), BLOCK=n, ROUNDS=rounds)
        words.append(out.numpy().view(np.uint32).copy())
    np.savez(dst, words=np.stack(words))


if __name__ == "__main__":
    main(sys.argv[1], sys.argv[2])
