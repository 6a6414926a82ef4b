"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Integer work (Philox words, Feistel permutations, signs) must match bit for
bit.  Floating-point tolerances are derived from the arithmetic:

* fused pass w = A^T (A p): both sides sum products in FP64, so
  |w_gpu - w_ref| <= 2 gamma_{m+d} (|A|^T (|A| |p|)), gamma_n = n u / (1 - n u);
* transform rows: the GPU converts column c to 64-bit fixed point with a
  quantum of at most max_k |X_kc| 2^{n-61} (n = log2 N'), adds exactly, and
  rounds once back to FP64, so |dZ_jc| <= (N max_c 2^{n-62} + 2 u |Z_jc|
  sqrt(N')) / sqrt(N') against exact arithmetic; the oracle's own FP64
  transform adds (n + 2) u sum_k |X'_kc| / sqrt(N');
* preconditioner factor: Householder QR is backward stable with
  ||dA||_F <= gamma_{rd} ||A||_F, and R moves by at most
  sqrt(2) kappa(A) ||dA||_F / ||A||_2 relative to ||R||_2 (first order);
* stage iterates and the final estimate: the FP64 tolerance 1e-10 on the
  relative prediction error ||X(beta - beta_ref)|| / ||X beta_ref||.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import linalg as OL
from oracle import philox as OP
from oracle import spcg as OS
from oracle import srht as OR
from oracle.metrics import rel_pred_error
from paper_2607_25272_b300 import spcg as S
from paper_2607_25272_b300.inputs import gaussian_problem, svd_problem

pytestmark = pytest.mark.gpu
U = np.finfo(np.float64).eps / 2


def gamma(n):
    return n * U / (1 - n * U)


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    S.lib()


# ---------------------------------------------------------------- draws ----
def test_philox_bitwise():
    rng = np.random.default_rng(0)
    ctr = rng.integers(0, 2**32, size=(1 << 18, 4), dtype=np.uint64).astype(np.uint32)
    seed = 0xDEADBEEF12345678
    out = S.spcg_philox(cuda(ctr.view(np.int32)), seed).cpu().numpy().view(np.uint32)
    ref = np.stack(OP.philox4x32_10(ctr[:, 0], ctr[:, 1], ctr[:, 2], ctr[:, 3], seed), axis=1)
    assert np.array_equal(out, ref)


@pytest.mark.parametrize("nbits", [1, 2, 7, 12, 15, 20, 23])
def test_feistel_bitwise(nbits):
    count = min(1 << nbits, 1 << 20)
    for tag in (OP.TAG_P, OP.TAG_PI, OP.TAG_HAT):
        for inv in (False, True):
            out = S.spcg_feistel(77 + nbits, nbits, tag, count, inverse=inv).cpu().numpy()
            f = OP.feistel_inverse if inv else OP.feistel_permute
            ref = f(np.arange(count), nbits, tag, 77 + nbits)
            assert np.array_equal(out, ref)


def test_signs_bitwise():
    out = S.spcg_signs(12345, 1 << 20).cpu().numpy()
    assert np.array_equal(out, OP.rademacher_signs(1 << 20, 12345))


# ------------------------------------------------------------ fused pass ----
@pytest.mark.parametrize("m,d", [(1, 1), (7, 3), (1000, 33), (4097, 256), (3001, 257),
                                 (100003, 50), (20000, 500), (2048, 1024), (513, 1000)])
def test_gram_apply_parity(m, d):
    rng = np.random.default_rng(m + d)
    A = rng.standard_normal((m, d))
    p = rng.standard_normal(d)
    X = cuda(rng.standard_normal((d + 2, d)))
    s = S.Solver(X, cuda(np.zeros(d + 2)))
    # the pass takes rows 16-byte aligned: odd d uses a padded leading dimension
    lda = d + (d % 2)
    Ad = torch.zeros((m, lda), dtype=torch.float64, device="cuda")
    Ad[:, :d] = cuda(A)
    w = s.gram_apply(Ad[:, :d], cuda(p)).cpu().numpy()
    ref = A.T @ (A @ p)
    bound = 2 * gamma(m + d) * (np.abs(A).T @ (np.abs(A) @ np.abs(p)))
    assert np.all(np.abs(w - ref) <= bound)
    s.close()


def test_gram_apply_empty_and_strided():
    d = 40
    s = S.Solver(cuda(np.ones((50, d)) + np.eye(50, d)), cuda(np.zeros(50)))
    p = cuda(np.ones(d))
    w = s.gram_apply(torch.empty((0, d), dtype=torch.float64, device="cuda"), p)
    assert torch.all(w == 0)
    rng = np.random.default_rng(3)
    big = rng.standard_normal((300, 64))
    A = cuda(big)[:, :d]          # leading dimension 64 > d
    w = s.gram_apply(A, p).cpu().numpy()
    Ab = big[:, :d]
    ref = Ab.T @ (Ab @ np.ones(d))
    assert np.all(np.abs(w - ref) <= 2 * gamma(300 + d) * (np.abs(Ab).T @ np.abs(Ab).sum(1)))
    # a row stride that breaks the 16-byte rule is rejected, not misread
    with pytest.raises(S.SpcgError) as e:
        s.gram_apply(cuda(np.ones((10, 41)))[:, :d], p)
    assert e.value.status == S.SPCG_E_INVALID_ARG
    s.close()


# ---------------------------------------------------------------- sketch ----
def _transform_tol(X, Y, n_pad, Z):
    """Per-element bound on |Z_gpu - Z_oracle| for rows of the transform."""
    N = X.shape[0]
    nb = int(math.log2(n_pad))
    mx = np.concatenate([np.abs(X).max(0), [np.abs(Y).max()]])
    l1 = np.concatenate([np.abs(X).sum(0), [np.abs(Y).sum()]])
    per_col = (N * mx * 2.0 ** (nb - 62) + 2 * (nb + 2) * U * l1) / np.sqrt(n_pad)
    return per_col[None, : Z.shape[1]] + 4 * U * np.abs(Z)


def _oracle_sketch(X, Y, seed, sched):
    ZX, ZY = OR.srht_transform(X, Y, seed)
    stages, A_hat = OR.nested_sketches(ZX, ZY, sched["m"], sched["r"], seed)
    return ZX, ZY, stages, A_hat


# Besides the default r = 6d: preconditioner sketches of 12800 and 13000 rows.
@pytest.mark.parametrize("N,d,seed,r", [(20000, 50, 1, None), (3000, 37, 5, None),
                                        (4097, 20, 9, None), (600, 20, 2, None),
                                        (9000, 300, 4, None), (40000, 70, 6, 12800),
                                        (40000, 70, 7, 13000), (5000, 161, 8, None)])
def test_sketch_rows_and_preconditioner(N, d, seed, r):
    X, Y, _ = gaussian_problem(N, d, 1.0, seed=seed)
    sched = OS.default_schedule(N, d)
    if r is not None:
        sched["r"] = r
    sched["r"] = min(sched["r"], sched["n_pad"])
    s = S.Solver(cuda(X), cuda(Y))
    sc = S.spcg_default_schedule(N, d)
    sc.r = sched["r"]
    s.sketch(seed, sc)
    n_pad = sched["n_pad"]
    ZX, ZY, stages, A_hat = _oracle_sketch(X, Y, seed, sched)
    if sched["m"]:
        mK = sched["m"][-1]
        A_g, b_g = (t.cpu().numpy() for t in s.export_sketch(0, mK))
        pi = OR.nested_order(n_pad, mK, seed)
        Zo = np.concatenate([ZX[pi], ZY[pi][:, None]], axis=1)
        Zg = np.concatenate([A_g, b_g[:, None]], axis=1)
        assert np.all(np.abs(Zg - Zo) <= _transform_tol(X, Y, n_pad, Zo))
    R_g, Rinv_g, Ahat_g = s.export_precond(r=sched["r"])
    R_g, Rinv_g, Ahat_g = R_g.cpu().numpy(), Rinv_g.cpu().numpy(), Ahat_g.cpu().numpy()
    hs = np.sqrt(n_pad / sched["r"])
    tol_hat = _transform_tol(X, Y, n_pad, A_hat / hs) * hs
    assert np.all(np.abs(Ahat_g - A_hat) <= tol_hat)
    R_o = OL.r_factor(A_hat)
    kappa = np.linalg.cond(A_hat)
    r = sched["r"]
    tol_R = 2 * math.sqrt(2) * kappa * gamma(r * d) * (np.linalg.norm(A_hat) / np.linalg.norm(A_hat, 2))
    assert np.linalg.norm(R_g - R_o) <= tol_R * np.linalg.norm(R_o, 2)
    assert np.all(np.diag(R_g) > 0) and np.array_equal(R_g, np.triu(R_g))
    # R^{-1}: R Rinv = I to the accuracy of a triangular inverse (kappa(R) u d)
    assert np.linalg.norm(R_g @ Rinv_g - np.eye(d)) <= 4 * d * U * np.linalg.cond(R_g) * math.sqrt(d)
    s.close()


# Stage sizes that are not powers of two keep the prefix in nested order (the
# bucketed storage needs power-of-two stages): rows against the oracle, and
# every stage iterate against the oracle's PCG on the same rows.
def test_sketch_and_stages_with_uneven_stage_sizes():
    N, d, seed = 40000, 50, 13
    X, Y, _ = svd_problem(N, d, 1e3, 0.1, seed=seed)
    sched = OS.default_schedule(N, d)
    sched["m"], sched["a"] = [3000, 7000, 12000], [3, 3, 3]
    sc = S.spcg_default_schedule(N, d)
    sc.K = 3
    for i, (m, a) in enumerate(zip(sched["m"], sched["a"])):
        sc.m[i], sc.a[i] = m, a
    s = S.Solver(cuda(X), cuda(Y))
    s.sketch(seed, sc)
    n_pad = sched["n_pad"]
    ZX, ZY, stages, A_hat = _oracle_sketch(X, Y, seed, sched)
    mK = sched["m"][-1]
    A_g, b_g = (t.cpu().numpy() for t in s.export_sketch(0, mK))
    pi = OR.nested_order(n_pad, mK, seed)
    Zo = np.concatenate([ZX[pi], ZY[pi][:, None]], axis=1)
    Zg = np.concatenate([A_g, b_g[:, None]], axis=1)
    assert np.all(np.abs(Zg - Zo) <= _transform_tol(X, Y, n_pad, Zo))
    R = OL.r_factor(A_hat)
    beta_g = torch.zeros(d, dtype=torch.float64, device="cuda")
    beta_o = np.zeros(d)
    for i, ((A_i, b_i), a_i) in enumerate(zip(stages, sched["a"])):
        beta_o, _ = OS.pcg(A_i, b_i, R, beta_o, a_i)
        s.pcg_stage(i, a_i, beta_g)
        assert rel_pred_error(X, beta_g.cpu().numpy(), beta_o) <= 1e-10, i
    s.close()


# The transform's kernels and pass plans: the 64-bit fixed-point butterflies
# are exact, so every tile variant and every split of the index bits into two
# passes must give the same bits; one of them is checked against the oracle's
# FP64 transform row by row.  N' = 2^19 (ragged N, 33 + 1 columns: partial
# column tiles), plans 10 + 9 (default), 9 + 10, 12 + 7 (the 7-level pass on
# the per-round kernel), and 11 + 8, 12 + 7, 8 + 11 and 7 + 12 with every
# pass on the per-round kernel (its 11- and 12-level tiles, 2048 x 8 and
# 4096 x 4, as the gathering first pass and as the scattering last pass).
def test_transform_variants_and_plans_are_bit_identical():
    N, d, seed = (1 << 18) + 37, 33, 12
    X, Y, _ = gaussian_problem(N, d, 1.0, seed=seed)
    sched = OS.default_schedule(N, d)
    mK = sched["m"][-1]
    outs = []
    for tile, first in ((0, 0), (1, 0), (2, 0), (3, 0), (1, 9), (2, 9), (1, 12),
                        (3, 11), (3, 12), (3, 8), (3, 7)):
        o = S.Opts()
        o.fwht_tile = tile
        o.fwht_first_levels = first
        s = S.Solver(cuda(X), cuda(Y), o)
        s.sketch(seed, S.spcg_default_schedule(N, d))
        A_g, b_g = (t.cpu().numpy() for t in s.export_sketch(0, mK))
        R_g = s.export_precond()[0].cpu().numpy()
        s.close()
        outs.append((A_g, b_g, R_g))
    for A_g, b_g, R_g in outs[1:]:
        assert np.array_equal(A_g, outs[0][0]) and np.array_equal(b_g, outs[0][1])
        assert np.array_equal(R_g, outs[0][2])
    n_pad = sched["n_pad"]
    ZX, ZY, _, _ = _oracle_sketch(X, Y, seed, sched)
    pi = OR.nested_order(n_pad, mK, seed)
    Zo = np.concatenate([ZX[pi], ZY[pi][:, None]], axis=1)
    Zg = np.concatenate([outs[0][0], outs[0][1][:, None]], axis=1)
    assert np.all(np.abs(Zg - Zo) <= _transform_tol(X, Y, n_pad, Zo))


# The factorisations of the preconditioner sketch: the blocked cooperative QR
# with look-ahead and without (panels of 32 columns; widths below, at and just
# above one panel, ragged last panels, 16 panels; panel groups of the default
# size, one CTA and five CTAs) and the per-column steps, each against the
# oracle's R within the Householder backward-error bound; a sketch of 120000
# rows takes the per-column path either way (its panel rows do not fit in
# shared memory).
@pytest.mark.parametrize("N,d,r,seed", [(20000, 50, None, 1), (4000, 32, None, 2), (4000, 33, None, 3),
                                        (9000, 300, None, 4), (70000, 129, None, 8),
                                        (3000, 7, None, 6), (1 << 17, 8, 120000, 5),
                                        (20000, 500, None, 9)])
def test_qr_blocked_and_per_column_agree(N, d, r, seed):
    X, Y, _ = gaussian_problem(N, d, 1.0, seed=seed)
    sched = OS.default_schedule(N, d)
    if r is not None:
        sched["r"] = r
    sched["r"] = min(sched["r"], sched["n_pad"])
    r = sched["r"]
    _, _, _, A_hat = _oracle_sketch(X, Y, seed, sched)
    R_o = OL.r_factor(A_hat)
    kappa = np.linalg.cond(A_hat)
    tol_R = 2 * math.sqrt(2) * kappa * gamma(r * d) * (np.linalg.norm(A_hat) / np.linalg.norm(A_hat, 2))
    Rs = []
    # blocked QR with look-ahead (automatic panel group, one panel CTA, five),
    # per column, blocked without look-ahead (automatic, five)
    for by_col, panel_ctas in ((0, 0), (0, 1), (0, 5), (1, 0), (2, 0), (2, 5)):
        o = S.Opts()
        o.qr_by_column = by_col
        o.qr_panel_ctas = panel_ctas
        s = S.Solver(cuda(X), cuda(Y), o)
        sc = S.spcg_default_schedule(N, d)
        sc.r = r
        s.sketch(seed, sc)
        R_g, Rinv_g, _ = (t.cpu().numpy() if t is not None else None for t in s.export_precond())
        s.close()
        assert np.linalg.norm(R_g - R_o) <= tol_R * np.linalg.norm(R_o, 2), by_col
        assert np.all(np.diag(R_g) > 0) and np.array_equal(R_g, np.triu(R_g))
        assert np.array_equal(Rinv_g, np.triu(Rinv_g))
        assert np.linalg.norm(R_g @ Rinv_g - np.eye(d)) <= 4 * d * U * np.linalg.cond(R_g) * math.sqrt(d)
        Rs.append(R_g)
    for R_g in Rs[1:]:
        assert np.linalg.norm(Rs[0] - R_g) <= 2 * tol_R * np.linalg.norm(R_o, 2)


# ---------------------------------------------------------------- stages ----
@pytest.mark.parametrize("N,d,kappa,seed,ds", [(20000, 50, None, 1, 0), (20000, 50, None, 1, 4),
                                               (30000, 24, 1e4, 3, 0), (30000, 24, 1e4, 3, 2),
                                               (12000, 96, 1e3, 4, 0), (12000, 96, 1e3, 4, 12),
                                               (12000, 97, 1e3, 4, 0), (12000, 97, 1e3, 4, 1)])
def test_stage_iterates_match_oracle(N, d, kappa, seed, ds):
    """Every stage's iterate against the oracle's PCG at 1e-10, with the d-space
    step in one CTA (shared-memory kernel up to d = 96, else the cooperative
    kernel on one CTA) or spread over several CTAs (ds = spcg_opts.dspace_ctas)."""
    if kappa is None:
        X, Y, _ = gaussian_problem(N, d, 1.0, seed=seed)
    else:
        X, Y, _ = svd_problem(N, d, kappa, 0.1, seed=seed)
    sched = OS.default_schedule(N, d)
    stages, A_hat, R = OS.sketch_all(X, Y, seed, sched)
    o = S.Opts()
    o.dspace_ctas = ds
    s = S.Solver(cuda(X), cuda(Y), o)
    s.sketch(seed, S.spcg_default_schedule(N, d))
    beta_g = torch.zeros(d, dtype=torch.float64, device="cuda")
    beta_o = np.zeros(d)
    for i, ((A_i, b_i), a_i) in enumerate(zip(stages, sched["a"])):
        beta_o, _ = OS.pcg(A_i, b_i, R, beta_o, a_i)
        s.pcg_stage(i, a_i, beta_g)
        assert rel_pred_error(X, beta_g.cpu().numpy(), beta_o) <= 1e-10, i
    s.close()


# ----------------------------------------------------------------- solve ----
@pytest.mark.parametrize("tol", [1e-6, 1e-10])
def test_solve_gaussian_c1(tol):
    X, Y, _ = gaussian_problem(20000, 50, 1.0, seed=1)
    bh = OL.ols(X, Y)
    sc = S.spcg_default_schedule(20000, 50)
    sc.tol = tol
    s = S.Solver(cuda(X), cuda(Y))
    beta, info, st = s.solve(1, sc)
    assert st == S.SPCG_OK and info.converged == 1
    assert rel_pred_error(X, beta.cpu().numpy(), bh) <= tol
    assert info.K == 6 and list(info.stage_iters[:6]) == [3] * 6
    out = OS.spcg(X, Y, seed=1, tol=tol)
    assert abs(info.refine_iters - out["refine_iters"]) <= 1
    s.close()


@pytest.mark.parametrize("N,d,kappa,sigma,seed", [(16384, 40, 1e6, 0.1, 2), (5000, 37, 1e3, 1.0, 6),
                                                  (70000, 129, 1e5, 0.5, 8), (5000, 1, 1.0, 1.0, 9),
                                                  (6000, 2, 1e2, 1.0, 10)])
def test_solve_ill_conditioned_ragged(N, d, kappa, sigma, seed):
    X, Y, _ = svd_problem(N, d, kappa, sigma, seed=seed)
    bh = OL.ols(X, Y)
    sc = S.spcg_default_schedule(N, d)
    sc.tol = 1e-10
    s = S.Solver(cuda(X), cuda(Y))
    beta, info, st = s.solve(seed, sc)
    assert st == S.SPCG_OK
    assert rel_pred_error(X, beta.cpu().numpy(), bh) <= 1e-10
    s.close()


def test_full_sampling_special_case():
    # m = N' and I-hat = all rows: the stage solves the OLS problem exactly and
    # H-hat = X^T X, so one iteration reaches beta-hat (Sec. 2.2 with S^T S = I).
    X, Y, _ = svd_problem(1024, 6, 1e4, 0.1, seed=5)
    bh = OL.ols(X, Y)
    s = S.Solver(cuda(X), cuda(Y))
    sc = S.make_schedule([1024], [1], 1024, tol=1e-10)
    s.sketch(3, sc)
    beta = torch.zeros(6, dtype=torch.float64, device="cuda")
    s.pcg_stage(0, 1, beta)
    assert rel_pred_error(X, beta.cpu().numpy(), bh) < 1e-9
    st, iters = s.refine(1e-10, 10, beta)
    assert st == S.SPCG_OK and iters <= 1
    s.close()


def test_solve_is_deterministic():
    X, Y, _ = svd_problem(40000, 64, 1e4, 0.2, seed=11)
    s = S.Solver(cuda(X), cuda(Y))
    b1, _, _ = s.solve(4)
    b1 = b1.clone()
    b2, _, _ = s.solve(4)
    assert torch.equal(b1, b2)
    s.close()


@pytest.mark.parametrize("prec", [S.PREC_FP64, S.PREC_MIXED])
def test_capture_safe_solve_replays_as_a_cuda_graph(prec):
    """spcg_solve_enqueue launches the stages and a fixed Stage II schedule with
    no host read, so the sequence can be captured into a CUDA graph: the
    replayed graph meets the target against the oracle's OLS estimator, bit
    for bit like the same sequence run uncaptured."""
    N, d, seed = 40000, 64, 11
    X, Y, _ = svd_problem(N, d, 1e4, 0.2, seed=seed)
    bh = OL.ols(X, Y)
    cs = torch.cuda.Stream()
    o = S.Opts()
    o.precision = prec
    s = S.Solver(cuda(X), cuda(Y), o, stream=cs)
    s.sketch(4, S.spcg_default_schedule(N, d))          # synchronises: outside the capture
    beta = torch.zeros(d, dtype=torch.float64, device="cuda")
    with torch.cuda.stream(cs):
        s.solve_enqueue(beta, rounds=6, iters_per_round=20)
        info, st = s.solve_result()
    assert st == S.SPCG_OK and info.converged == 1
    assert rel_pred_error(X, beta.cpu().numpy(), bh) <= 1e-6
    b_direct = beta.clone()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=cs):
        s.solve_enqueue(beta, rounds=6, iters_per_round=20)
    for _ in range(2):
        with torch.cuda.stream(cs):        # the context's stream: solve_result syncs it
            beta.fill_(float("nan"))
            g.replay()
        info, st = s.solve_result()
        assert st == S.SPCG_OK and info.converged == 1
        assert torch.equal(beta, b_direct)
    s.close()


def test_plain_pcg_when_no_stage_fits():
    # K = 0 (m_1 > N'/2): Algorithm 1 reduces to full-data PCG
    X, Y, _ = gaussian_problem(500, 60, 1.0, seed=2)
    sc = S.spcg_default_schedule(500, 60)
    assert sc.K == 0
    sc.tol = 1e-10
    s = S.Solver(cuda(X), cuda(Y))
    beta, info, st = s.solve(1, sc)
    assert st == S.SPCG_OK and rel_pred_error(X, beta.cpu().numpy(), OL.ols(X, Y)) <= 1e-10
    s.close()


# ---------------------------------------------------------------- errors ----
def test_error_paths_and_recovery():
    X, Y, _ = gaussian_problem(5000, 20, 1.0, seed=3)
    s = S.Solver(cuda(X), cuda(Y))
    beta = torch.zeros(20, dtype=torch.float64, device="cuda")
    with pytest.raises(S.SpcgError) as e:
        s.pcg_stage(0, 3, beta)
    assert e.value.status == S.SPCG_E_STATE
    bad = S.make_schedule([512, 256], [3, 3], 120)
    with pytest.raises(S.SpcgError) as e:
        s.sketch(1, bad)
    assert e.value.status == S.SPCG_E_INVALID_ARG
    s.sketch(1, S.spcg_default_schedule(5000, 20))
    st, iters = s.refine(1e-12, 1, beta, raise_on_error=False)
    assert st == S.SPCG_E_NOT_CONVERGED and iters == 1
    s.close()
    # a zero column: X is not of full column rank, R is singular
    Xs = X.copy()
    Xs[:, 7] = 0.0
    s = S.Solver(cuda(Xs), cuda(Y))
    with pytest.raises(S.SpcgError) as e:
        s.sketch(1)
    assert e.value.status == S.SPCG_E_BREAKDOWN
    s.close()


def test_bounded_wait_times_out_and_context_survives():
    X, Y, _ = gaussian_problem(50000, 64, 1.0, seed=4)
    opts = S.Opts()
    opts.spin_budget = 20_000_000          # ~10 ms at 2 GHz
    opts.inject_stall = 1                  # CTA 0 never issues its first tile
    s = S.Solver(cuda(X), cuda(Y), opts)
    p = cuda(np.ones(64))
    with pytest.raises(S.SpcgError) as e:
        s.gram_apply(cuda(X), p)
    assert e.value.status == S.SPCG_E_TIMEOUT
    s.close()
    s = S.Solver(cuda(X), cuda(Y))
    w = s.gram_apply(cuda(X), p).cpu().numpy()
    assert np.allclose(w, X.T @ (X @ np.ones(64)), rtol=1e-12)
    s.close()


# ------------------------------------------------------- full size (C2) ----
def test_c2_full_size_solve_and_sampled_transform_rows():
    """N = 2^20, d = 500, kappa = 1e6, sigma = 0.1 in the launch configuration
    bench.py times: the solve meets 1e-6 and 1e-10 against the oracle's OLS
    estimator, and sampled rows of the transform match the defining sum."""
    N, d = 1 << 20, 500
    X, Y, _ = svd_problem(N, d, 1e6, 0.1, seed=1)
    bh = OL.ols(X, Y)
    s = S.Solver(cuda(X), cuda(Y))
    for tol in (1e-6, 1e-10):
        sc = S.spcg_default_schedule(N, d)
        sc.tol = tol
        beta, info, st = s.solve(1, sc)
        assert st == S.SPCG_OK
        assert rel_pred_error(X, beta.cpu().numpy(), bh) <= tol
    mK = 1 << 19
    pi = OR.nested_order(N, mK, 1)
    for t in (0, 12345, mK - 1):
        zx, zy = OR.srht_row(X, Y, 1, int(pi[t]))
        A_g, b_g = (v.cpu().numpy() for v in s.export_sketch(t, 1))
        zo = np.concatenate([zx, [zy]])[None, :]
        zg = np.concatenate([A_g[0], b_g])[None, :]
        assert np.all(np.abs(zg - zo) <= _transform_tol(X, Y, N, zo))
    s.close()
