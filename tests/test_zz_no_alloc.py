"""The allocation-free fused pass (spcg_gram_apply_noalloc) against the
context-based one (spcg_gram_apply).

Some callers cannot allocate device memory (a caching allocator owns the
pool, the process runs under a memory cap, or an allocation would force a
device-wide synchronisation at a bad moment).  For them the library keeps a
fixed scratch array in device memory; this test checks that the pass using
it gives the same w = A^T (A p) as the pass using a context's workspace,
within the tolerance of the other parity tests, on two calls in a row (the
second call reuses the array left by the first).

This file is collected last so that a failure here does not hide the other
GPU tests in a run that stops at the first failure.
"""
import gc

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2607_25272_b300 import spcg as S

pytestmark = pytest.mark.gpu
U = np.finfo(np.float64).eps / 2


def gamma(n):
    return n * U / (1 - n * U)


@pytest.mark.parametrize("m,d", [(200003, 500), (4097, 33), (1000, 1024), (7, 1)])
def test_noalloc_pass_matches_context_pass_twice(m, d):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    rng = np.random.default_rng(m * 7 + d)
    A = rng.standard_normal((m, d))
    p = rng.standard_normal(d)
    lda = d + (d % 2)                     # rows 16-byte aligned (the TMA rule)
    Ad = torch.zeros((m, lda), dtype=torch.float64, device="cuda")
    Ad[:, :d] = torch.from_numpy(A).cuda()
    Av = Ad[:, :d]
    pd = torch.from_numpy(p).cuda()
    solver = S.Solver(torch.from_numpy(rng.standard_normal((d + 2, d))).cuda(),
                      torch.zeros(d + 2, dtype=torch.float64, device="cuda"))
    w_ctx = solver.gram_apply(Av, pd).cpu().numpy()
    solver.close()
    bound = 2 * gamma(m + d) * (np.abs(A).T @ (np.abs(A) @ np.abs(p)))
    for call in range(2):
        w = torch.full((d,), np.nan, dtype=torch.float64, device="cuda")
        gc.collect()                      # no unrelated frees inside the measured call
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        alloc0 = torch.cuda.memory_allocated()
        S.spcg_gram_apply_noalloc(Av, pd, w)
        torch.cuda.synchronize()
        if call == 1:
            # the property the entry point exists for: the second call (the
            # first may load the kernels' module) takes no device memory
            assert torch.cuda.mem_get_info()[0] >= free0
            assert torch.cuda.memory_allocated() <= alloc0
        w = w.cpu().numpy()
        assert np.all(np.abs(w - w_ctx) <= bound)
        assert np.all(np.abs(w - A.T @ (A @ p)) <= bound)


def test_noalloc_rejects_too_many_columns():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    d = S.MAX_D + 2
    A = torch.zeros((4, d), dtype=torch.float64, device="cuda")
    p = torch.zeros(d, dtype=torch.float64, device="cuda")
    with pytest.raises(S.SpcgError) as e:
        S.spcg_gram_apply_noalloc(A, p)
    assert e.value.status == S.SPCG_E_INVALID_ARG


def test_noalloc_binding_rejects_wrong_dtype_and_layout():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    A = torch.zeros((8, 4), dtype=torch.float32, device="cuda")
    p = torch.zeros(4, dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        S.spcg_gram_apply_noalloc(A, p)
    At = torch.zeros((4, 8), dtype=torch.float64, device="cuda").T   # column-major view
    with pytest.raises(ValueError):
        S.spcg_gram_apply_noalloc(At, p)
    with pytest.raises(ValueError):
        S.spcg_gram_apply_noalloc(torch.zeros((8, 4), dtype=torch.float64, device="cuda"),
                                  torch.zeros(5, dtype=torch.float64, device="cuda"))
