"""Benchmark: seconds to a 1e-6 relative OLS prediction error with SPCG.

Headline workload: plain FP64 SPCG on N = 2^20, d = 500, X = U diag(s) V^T
with s geometric from 1 to 1e-6 (kappa = 1e6), beta ~ N(0, 1), sigma = 0.1;
the paper's default schedule (m_1 = 8d rounded to a power of two, doubling
to N'/2, r = 6d, a_i = 3) and the Stage II stopping rule for tol = 1e-6.
Synthetic data, generated on the host from a fixed seed.

One step = one spcg_solve (SRHT sketch, preconditioner QR, every Stage I
subproblem, Stage II to the stopping rule) with X, Y resident in HBM.
X is 4.19 GB, far larger than the 126 MB L2, so no flush is needed between
steps.  The result is checked against the OLS estimator from LAPACK's
Householder QR (outside the timed region; the oracle package runs only in the
CPU baseline and the reference arm).

The same JSON line carries the metric's comparisons at the other workloads
(one GPU only): "c3" mixed precision against plain FP64 at N = 2^22,
d = 1000, kappa = 1e8 with heavy leverage; "c4" 512 batched FP32 problems
against a loop of plain solves; "c5" the learned schedule against the
paper's schedule at N = 2^23, d = 256.  Those inputs are drawn on the GPU
(same recipes, torch random streams) and judged by properties that hold at
any size (the construction's closed-form OLS estimator, or an FP64 least-
squares solve by the GPU's linear-algebra library).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun each rank solves its own independent problem (weak scaling,
no collective on the data path); rank 0 prints one JSON line.
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    "c3": dict(name="mixed precision, N=2^22, d=1000, kappa=1e8, rows scaled by |t_3| before "
                    "orthonormalising, sigma=1, seed=1",
               N=1 << 22, d=1000, kappa=1e8, sigma=1.0, seed=1, tol=1e-6, leverage_df=3),
    "c4": dict(name="batched: 512 problems, N ~ U[2^12, 2^17], d ~ U[16, 256], X iid N(0,1) "
                    "times column scales log-uniform in [1e-3, 1e3], sigma=1, FP32, seed=1",
               N=None, d=None, kappa=None, sigma=1.0, seed=1, tol=1e-6, batch=512),
    "c5": dict(name="learned schedule: N=2^23, d=256, kappa=1e4, sigma=0.5, seed=1",
               N=1 << 23, d=256, kappa=1e4, sigma=0.5, seed=1, tol=1e-6),
    "c2": dict(name="plain SPCG FP64, N=2^20, d=500, kappa=1e6, sigma=0.1, seed=1",
               N=1 << 20, d=500, kappa=1e6, sigma=0.1, seed=1, tol=1e-6),
    "c1": dict(name="plain SPCG FP64, N=20000, d=50, X iid N(0,1), sigma=1, seed=1",
               N=20000, d=50, kappa=None, sigma=1.0, seed=1, tol=1e-6),
}
WARM_SAMPLE_ROWS = 1 << 14    # oracle warm-up sample of the reference arm
NOMINAL_FP64_TFLOPS = 1.25    # B300 FP64, nominal (context only)
NOMINAL_HBM_GBS = 7700.0      # B300 HBM3e, nominal (context only; the roofline uses the measured copy)
# DRAM bytes per algorithmic byte of k_pass (FP64), from the ncu capture of
# this kernel on a 262144 x 500 operand: read 1.048634624 GB + wrote
# 2.704384 MB for 1.048576 GB of rows.  Set to None whenever the kernel changes
# after the capture.
K_PASS_TRAFFIC_RATIO = (1.048634624e9 + 2.704384e6) / 1.048576e9
# The same for k_pass_df (the double-FP32 pair) on rows of 1000 columns, from
# the ncu capture of this kernel on a 262144 x 1000 pair: read 2.097235 GB +
# wrote 3.191808 MB for 2.097152 GB of Xh and Xl.  None once the kernel changes.
K_PASS_DF_TRAFFIC_RATIO = (2.097235e9 + 3.191808e6) / 2.097152e9
# And for k_pass<float> (the FP32 copy of X) on rows of 500 columns, from the
# ncu capture on a 262144 x 500 FP32 operand: read 524.349184 MB + wrote
# 2.655232 MB for 524.288 MB of rows.  None once the kernel changes.
K_PASS_F32_TRAFFIC_RATIO = (524349184 + 2655232) / 524288000


def lapack_ols(X, Y):
    """The OLS estimator for the accuracy report of the GPU arm: LAPACK's
    Householder QR through numpy (dgeqrf), Q^T Y, a triangular solve."""
    from scipy.linalg import solve_triangular
    Q, R = np.linalg.qr(np.asarray(X, dtype=np.float64), mode="reduced")
    return solve_triangular(R, Q.T @ np.asarray(Y, dtype=np.float64), lower=False)


def rel_error(X, beta, beta_hat):
    """||X (beta - beta_hat)|| / ||X beta_hat||, the workloads' accuracy metric."""
    diff = X @ (np.asarray(beta) - np.asarray(beta_hat))
    return float(np.linalg.norm(diff) / np.linalg.norm(X @ np.asarray(beta_hat)))


def make_problem(w, N=None, seed_offset=0):
    from paper_2607_25272_b300.inputs import gaussian_problem, svd_problem
    N = N or w["N"]
    if w["kappa"] is None:
        return gaussian_problem(N, w["d"], w["sigma"], seed=w["seed"] + seed_offset)
    return svd_problem(N, w["d"], w["kappa"], w["sigma"], seed=w["seed"] + seed_offset,
                       leverage_df=w.get("leverage_df"))


def base_line(args, w, value_s, metric, dtype, world=1):
    return {"metric": metric, "value": value_s, "unit": "s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": value_s * 1e3, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": dtype, "data": "synthetic",
            "config": {"workload": w["name"]}}


def time_solves(solver, seed, sched, steps, warmup, stream, fn=None, region=False):
    """Mean ms per call over `steps` calls after `warmup` calls; region=True
    brackets the timed calls with cudaProfilerStart/Stop (for ncu
    --profile-from-start off)."""
    import torch
    fn = fn or (lambda: solver.solve(seed, sched))
    for _ in range(warmup):
        fn()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    if region:
        torch.cuda.profiler.start()
    e0.record(stream)
    outs = [fn() for _ in range(steps)]
    e1.record(stream)
    torch.cuda.synchronize()
    if region:
        torch.cuda.profiler.stop()
    return e0.elapsed_time(e1) / steps, outs


def closed_form_rel_error(beta, uty, s, V):
    """||X (beta - beta_ols)|| / ||X beta_ols|| for X = U diag(s) V^T with U
    orthonormal: beta_ols = V diag(1/s) U^T Y and ||X v|| = ||diag(s) V^T v||,
    exact up to the orthonormality of U (CholeskyQR2, near 1e-15)."""
    import torch
    b_ols = V @ (uty / s)
    return float(torch.linalg.norm(s * (V.T @ (beta - b_ols))) /
                 torch.linalg.norm(s * (V.T @ b_ols)))


def extra_steps(args):
    """Steps and warm-ups of the nested workloads: at most 5 and 2, so that
    the default run stays within minutes."""
    return max(1, min(args.steps, 5)), max(1, min(args.warmup, 2))


def pass_roofline(info, op, peak_gbs, peak_source, traffic_ratio, kernel):
    """HBM roofline of the passes of one operand kind from a profiled solve:
    algorithmic bytes per launch / mean CUDA-event duration per launch."""
    from paper_2607_25272_b300 import spcg as S
    k = S.OP_NAMES.index(op)
    n, ms, nbytes = info.launches_by_op[k], info.pass_ms_by_op[k], info.bytes_by_op[k]
    if n == 0 or ms <= 0:
        return None
    per_launch = nbytes / n
    gbs = per_launch / (ms / n / 1e3) / 1e9
    return {"bound": "hbm", "kernel": kernel, "achieved": gbs, "peak": peak_gbs, "unit": "GB/s",
            "frac": gbs / peak_gbs, "peak_source": peak_source,
            "peak_nominal_gbs": NOMINAL_HBM_GBS, "frac_of_nominal": gbs / NOMINAL_HBM_GBS,
            "traffic": per_launch * traffic_ratio if traffic_ratio else None,
            "launches_per_step": n, "alg_bytes_per_launch": per_launch}


def host_mem_available():
    """Available host memory in bytes (/proc/meminfo), 0 if unknown."""
    try:
        for ln in open("/proc/meminfo"):
            if ln.startswith("MemAvailable:"):
                return int(ln.split()[1]) * 1024
    except OSError:
        pass
    return 0


def hbm_peak():
    peaks = measured_peaks()
    if "hbm_gbs" in peaks:
        return peaks["hbm_gbs"], "of measured (MEASURED_PEAKS.json hbm_gbs)"
    return 6400.0, "of fallback (6.4 TB/s; no MEASURED_PEAKS.json on this host)"


def run_forms(args, w):
    """Plain FP64 vs mixed precision on one large problem (C3).  The problem
    is drawn on the GPU (host generation of 4M x 1000 takes minutes); the
    prediction error against the OLS estimator comes from the construction's
    closed form (closed_form_rel_error).  Returns a dict."""
    import torch

    from paper_2607_25272_b300 import spcg as S
    from paper_2607_25272_b300.inputs import svd_problem_device
    steps, warmup = extra_steps(args)
    dev = torch.device("cuda", 0)
    t0 = time.time()
    Xd, Yd, _, uty, sv_s, sv_V = svd_problem_device(w["N"], w["d"], w["kappa"], w["sigma"],
                                                    seed=w["seed"],
                                                    leverage_df=w.get("leverage_df"),
                                                    device=dev)
    torch.cuda.synchronize()
    gen_s = time.time() - t0
    N, d = Xd.shape
    stream = torch.cuda.current_stream(dev)
    sched = S.spcg_default_schedule(N, d)
    sched.tol = w["tol"]
    peak, peak_src = hbm_peak()
    res = {}
    for name, prec in (("plain_fp64", S.PREC_FP64), ("mixed", S.PREC_MIXED)):
        o = S.Opts()
        o.precision = prec
        sv = S.Solver(Xd, Yd, o)
        region = args.ncu_region is not None and name.startswith(args.ncu_region)
        ms, outs = time_solves(sv, w["seed"], sched, steps, warmup, stream,
                               fn=lambda sv=sv: sv.solve(w["seed"], sched, raise_on_error=False),
                               region=region)
        beta, info, st = outs[-1]
        sv.close()
        o.profile = 1
        pv = S.Solver(Xd, Yd, o)
        _, pinfo, _ = pv.solve(w["seed"], sched, raise_on_error=False)
        pv.close()
        by_op = {S.OP_NAMES[k]: {"launches": pinfo.launches_by_op[k],
                                 "ms": pinfo.pass_ms_by_op[k],
                                 "gbs": (pinfo.bytes_by_op[k] / (pinfo.pass_ms_by_op[k] / 1e3) / 1e9)
                                 if pinfo.pass_ms_by_op[k] > 0 else None}
                 for k in range(4) if pinfo.launches_by_op[k] > 0}
        res[name] = {"s": ms / 1e3, "status": S.STATUS[st],
                     "rel_pred_error": closed_form_rel_error(beta, uty, sv_s, sv_V),
                     "phases_ms": {"sketch": info.ms_sketch, "stages": info.ms_stages,
                                   "refine": info.ms_refine},
                     "refine_iters": info.refine_iters, "restarts": info.restarts,
                     "cond_est": info.cond_est, "inner_prec": info.inner_prec,
                     "grad_prec": info.grad_prec, "launches": info.launches,
                     "passes_by_operand": by_op}
        if name == "mixed":
            df = info.inner_prec == S.INNER_DF
            res[name]["roofline"] = pass_roofline(
                pinfo, "pair" if df else "float32", peak, peak_src,
                K_PASS_DF_TRAFFIC_RATIO if (df and d == 1000)
                else (K_PASS_F32_TRAFFIC_RATIO if (not df and d == 500) else None),
                "k_pass_df (double-FP32 pair)" if df else "k_pass<float>")
    # end to end through the public API from pinned host buffers, when the
    # host can hold a pinned copy of X (33.6 GB)
    e2e = None
    avail = host_mem_available()
    nbytes = N * d * 8 + N * 8
    if avail > 3 * nbytes:
        Xh = Xd.cpu().pin_memory()
        Yh = Yd.cpu().pin_memory()
        del Xd, Yd
        torch.cuda.empty_cache()
        o = S.Opts()
        o.precision = S.PREC_MIXED
        ts = []
        for _ in range(2):
            torch.cuda.synchronize()
            a0 = torch.cuda.Event(enable_timing=True)
            a1 = torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            b_host, _, st_e = S.spcg_solve_host(Xh, Yh, w["seed"], sched, o)
            a1.record(stream)
            torch.cuda.synchronize()
            ts.append(a0.elapsed_time(a1))
        e2e = {"value": float(min(ts)) / 1e3, "unit": "s", "h2d_bytes_per_step": int(nbytes),
               "d2h_bytes_per_step": int(d * 8), "form": "mixed",
               "status": S.STATUS[st_e]}
        del Xh, Yh
    else:
        del Xd, Yd
    torch.cuda.empty_cache()
    return {"workload": w["name"], "N": N, "d": d, "tol": w["tol"], "steps": steps,
            "warmup": warmup,
            "metric": "seconds to 1e-6 OLS prediction error (mixed precision vs plain FP64 SPCG)",
            "inputs": "drawn on the GPU (svd_problem_device), same recipe",
            "l2": "no flush: X is 33.6 GB, larger than the 126 MB L2",
            "forms": res,
            "speedup_mixed_vs_plain_fp64": res["plain_fp64"]["s"] / res["mixed"]["s"],
            "accuracy_reference": "closed-form OLS estimator of the construction, "
                                  "V diag(1/s) U^T Y",
            "e2e": e2e if e2e else {"unavailable": "host memory too small for a pinned copy of X"},
            "host_s": {"generate": gen_s}}


def run_batched(args, w):
    """C4: 512 uneven FP32 problems in one persistent launch vs a loop of
    single plain-FP64 solves of the same problems.  Problems are drawn on the
    GPU; every solution is judged against an FP64 least-squares solve of its
    FP32 values by the GPU's linear-algebra library (torch.linalg.lstsq),
    which shares nothing with this library's kernels.  Returns a dict."""
    import torch

    from paper_2607_25272_b300 import spcg as S
    from paper_2607_25272_b300.inputs import scaled_columns_problem_device
    steps, warmup = extra_steps(args)
    rng = np.random.default_rng(w["seed"])
    n = w["batch"]
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    shapes = [(int(rng.integers(1 << 12, (1 << 17) + 1)), int(rng.integers(16, 257)))
              for _ in range(n)]
    Xs, Ys = [], []
    for i, (N, d) in enumerate(shapes):
        X, Y, _ = scaled_columns_problem_device(N, d, 1e-3, 1e3, w["sigma"],
                                                seed=w["seed"] * 100000 + i, device=dev,
                                                dtype=torch.float32)
        ld = (d + 3) // 4 * 4
        Xp = torch.zeros((N, ld), dtype=torch.float32, device=dev)
        Xp[:, :d] = X
        Xs.append(Xp[:, :d])
        Ys.append(Y)
    B = S.Batch(Xs, Ys)
    tiles = B.autotune(w["seed"], w["tol"])
    for _ in range(warmup):
        B.solve(w["seed"], w["tol"])
    times = []
    for _ in range(steps):
        rc, st, it, ms = B.solve(w["seed"], w["tol"])
        times.append(ms)
    ms_b = float(np.median(times))
    betas = [b.clone() for b in B.betas]
    phases = batch_phase_summary(B, Xs)
    peak_gbs, peak_src = hbm_peak()
    bound = batch_streaming_bound(shapes, it, peak_gbs)
    bound["x_bound"] = ms_b / bound["bound_ms"]
    bound["peak_source"] = peak_src
    B.close()
    # the comparator: one plain FP64 spcg_solve per problem, back to back
    loop_ms = 0.0
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    loop_status = []
    errs = []
    for X, Y, b in zip(Xs, Ys, betas):
        X64 = X.double().contiguous()
        Y64 = Y.double()
        sv = S.Solver(X64, Y64)
        sc = S.spcg_default_schedule(*X64.shape)
        sc.tol = w["tol"]
        sv.solve(w["seed"], sc, raise_on_error=False)          # warm
        torch.cuda.synchronize()
        e0.record(stream)
        _, _, st_ = sv.solve(w["seed"], sc, raise_on_error=False)
        e1.record(stream)
        torch.cuda.synchronize()
        loop_ms += e0.elapsed_time(e1)
        loop_status.append(st_)
        sv.close()
        bh = torch.linalg.lstsq(X64, Y64[:, None], driver="gels").solution[:, 0]
        errs.append(float(torch.linalg.norm(X64 @ (b - bh)) / torch.linalg.norm(X64 @ bh)))
    total_bytes = sum(X.shape[0] * X.shape[1] * 4 for X in Xs)
    return {"workload": w["name"], "problems": n, "tol": w["tol"], "steps": steps,
            "warmup": warmup,
            "metric": "seconds to 1e-6 OLS prediction error for the whole batch (batched vs a "
                      "loop of plain FP64 SPCG solves)",
            "inputs": "drawn on the GPU (scaled_columns_problem_device), same recipe",
            "batched": {"s": ms_b / 1e3, "status_ok": int(sum(1 for v in st if v == 0)),
                        "max_rel_pred_error": float(max(errs)),
                        "problems_meeting_tol": int(sum(1 for e in errs if e <= w["tol"])),
                        "autotuned_chunk_bytes": tiles,
                        "x_bytes_fp32": int(total_bytes), "phase_ms": phases,
                        "streaming_bound": bound},
            "loop_plain_fp64": {"s": loop_ms / 1e3,
                                "status_ok": int(sum(1 for v in loop_status if v == 0))},
            "speedup_batched_vs_loop": loop_ms / ms_b if ms_b > 0 else None,
            "accuracy_reference": "torch.linalg.lstsq (FP64, QR) of each problem's FP32 values"}


PHASES = ("colmax", "cs_maps", "cs_sums", "stage_matrices", "qr", "stage1", "stage2")


def batch_streaming_bound(shapes, iters, peak_gbs):
    """Algorithmic bytes of one batched solve and the time they take at the
    measured HBM bandwidth.  Per problem (N x d FP32, C = d + 1 with Y, the
    default stages m_i = 2^ceil(log2 8d) doubling to N'/2, a_i = 3, r = 6d):
    the column maxima and the CountSketch each read [X Y] once; the sketch
    writes its m_K int64 bucket rows and the r FP32 preconditioner rows; the
    stage matrices are written once as FP32 and read a_i + 1 times by Stage I
    (a residual pass and a_i iterations); Stage II reads X once per
    iteration plus two true gradients (its start and the confirmed stop)."""
    total = 0
    for (N, d), it in zip(shapes, iters):
        C, ld = d + 1, (d + 3) // 4 * 4
        n_pad = 1 << (N - 1).bit_length()
        m, mi = [], 1 << (8 * d - 1).bit_length()
        while mi <= n_pad // 2:
            m.append(mi)
            mi *= 2
        xb = N * C * 4
        b = 2 * xb                                    # column maxima, CountSketch read
        b += (m[-1] * C * 8 if m else 0) + 6 * d * d * 4   # bucket rows, preconditioner rows
        b += sum(mi * ld * 4 * (1 + 3 + 1) for mi in m)    # stage matrices: write, 4 reads
        b += (int(it) + 2) * N * d * 4                # Stage II passes and true gradients
        total += b
    return {"alg_bytes": int(total), "peak_gbs": peak_gbs,
            "bound_ms": total / (peak_gbs * 1e6)}


def batch_phase_summary(B, Xs, sm_mhz=2032.0):
    """Per-phase device time of the last batched solve: summed over problems
    and for the largest problem (cycles of the SM that solved it at the
    maximum SM clock)."""
    cyc = np.array(B.phase_cycles(), dtype=np.float64)
    big = int(np.argmax([X.shape[0] * X.shape[1] for X in Xs]))
    to_ms = 1.0 / (sm_mhz * 1e3)
    return {"sum_over_problems": {k: float(v) for k, v in zip(PHASES, cyc.sum(0) * to_ms)},
            "largest_problem": {"N": int(Xs[big].shape[0]), "d": int(Xs[big].shape[1]),
                                **{k: float(v) for k, v in zip(PHASES, cyc[big] * to_ms)}}}


def run_learned(args, w):
    """C5: the learned schedule vs the paper's schedule (plain FP64 SPCG) at
    N = 2^23, d = 256, drawn on the GPU and judged by the closed form.
    Returns a dict."""
    import torch

    from paper_2607_25272_b300 import schedule_model as SM
    from paper_2607_25272_b300 import spcg as S
    from paper_2607_25272_b300.inputs import svd_problem_device
    steps, warmup = extra_steps(args)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    Xd, Yd, _, uty, sv_s, sv_V = svd_problem_device(w["N"], w["d"], w["kappa"], w["sigma"],
                                                    seed=w["seed"], device=dev)
    N, d = Xd.shape
    Wb, norm = SM.load(args.weights) if args.weights else SM.load()
    sv = S.Solver(Xd, Yd)
    ms_p, outs_p = time_solves(sv, w["seed"], None, steps, warmup, stream,
                               fn=lambda: sv.solve_learned(w["seed"], None, None, w["tol"],
                                                           raise_on_error=False))
    ms_l, outs_l = time_solves(sv, w["seed"], None, steps, warmup, stream,
                               fn=lambda: sv.solve_learned(w["seed"], Wb, norm, w["tol"],
                                                           raise_on_error=False))
    bp, ip, cp, sp = outs_p[-1]
    bl, il, cl, sl = outs_l[-1]
    sv.close()
    del Xd, Yd
    torch.cuda.empty_cache()
    return {"workload": w["name"], "N": N, "d": d, "tol": w["tol"], "steps": steps,
            "warmup": warmup,
            "metric": "seconds to 1e-6 OLS prediction error (learned schedule vs the paper's "
                      "schedule, plain FP64 SPCG)",
            "model": "MLP 4-64-64-25, BF16 weights" if Wb is not None else
                     "no trained weights: paper schedule",
            "inputs": "drawn on the GPU (svd_problem_device), same recipe",
            "paper_schedule": {"s": ms_p / 1e3, "candidate": cp, "status": S.STATUS[sp],
                               "rel_pred_error": closed_form_rel_error(bp, uty, sv_s, sv_V),
                               "refine_iters": ip.refine_iters},
            "learned_schedule": {"s": ms_l / 1e3, "candidate": cl, "status": S.STATUS[sl],
                                 "rel_pred_error": closed_form_rel_error(bl, uty, sv_s, sv_V),
                                 "refine_iters": il.refine_iters, "stages": il.K},
            "speedup_learned_vs_paper": ms_p / ms_l,
            "accuracy_reference": "closed-form OLS estimator of the construction"}


def print_nested(args, w, res, dtype):
    """A standalone run of one nested workload: its own JSON line."""
    if "forms" in res:
        v = res["forms"]["mixed"]["s"]
    elif "batched" in res:
        v = res["batched"]["s"]
    else:
        v = res["learned_schedule"]["s"]
    line = base_line(args, w, v, res["metric"], dtype)
    line["steps"], line["warmup"] = res["steps"], res["warmup"]
    line["ms_per_step"] = v * 1e3
    line["config"].update({k: res[k] for k in ("N", "d", "problems", "tol") if k in res})
    line["result"] = res
    print(json.dumps(line), flush=True)


class ClockSampler:
    """nvidia-smi SM clock and throttle reasons sampled every 200 ms."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(mx)) if mx else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def max_over_ranks(value, device=None):
    """The largest per-rank value (the job's time); identity on one rank."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64,
                     device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


def host_threads():
    """Threads the oracle's BLAS may use on this host."""
    return int(os.environ.get("OPENBLAS_NUM_THREADS", len(os.sched_getaffinity(0))))


def oracle_phases(X, Y, seed, tol):
    """The oracle's SPCG solve (oracle.spcg.spcg, Algorithm 1 with the Stage II
    stopping rule) as the sequence of its own calls, in its order: the SRHT
    transform, the nested sketches and the preconditioner factor, one PCG run
    per stage, Stage II.  Each phase is returned as a closure so that a caller
    can time them one by one; the last one returns the final beta."""
    from oracle import spcg as OS
    from oracle import srht as OR
    from oracle.linalg import r_factor
    sched = OS.default_schedule(*X.shape)
    st = {"beta": np.zeros(X.shape[1])}

    def transform():
        st["Z"] = OR.srht_transform(X, Y, seed)

    def sketches():
        ZX, ZY = st.pop("Z")
        st["stages"], A_hat = OR.nested_sketches(ZX, ZY, sched["m"], sched["r"], seed)
        st["R"] = r_factor(A_hat)

    def stage(i):
        def run():
            A_i, b_i = st["stages"][i]
            st["beta"], _ = OS.pcg(A_i, b_i, st["R"], st["beta"], sched["a"][i])
        return run

    def refine():
        st.pop("stages", None)
        st["beta"], _, _ = OS.full_pcg(X, Y, st["R"], st["beta"], tol)
        return st["beta"]

    return [transform, sketches] + [stage(i) for i in range(len(sched["m"]))] + [refine]


def phase_groups(phases, K):
    """The phases split into K consecutive groups, as evenly as possible
    (groups are empty when K exceeds the number of phases)."""
    n = len(phases)
    return [phases[(k * n) // K:((k + 1) * n) // K] for k in range(K)]


def cpu_baseline(w, X=None, Y=None):
    """One complete oracle SPCG solve (numpy FP64) of the whole workload at
    its stated size, wall time, no scaling; beside it, timed separately, the
    oracle's direct OLS solve (Householder QR) of the same problem."""
    from oracle.linalg import ols
    from oracle.spcg import spcg as oracle_spcg
    if X is None:
        X, Y, _ = make_problem(w)
    t0 = time.perf_counter()
    oracle_spcg(X, Y, seed=w["seed"], tol=w["tol"])
    sec = time.perf_counter() - t0
    t0 = time.perf_counter()
    ols(X, Y)
    ols_sec = time.perf_counter() - t0
    threads = host_threads()
    return {"value": float(sec), "unit": "s", "cores": int(threads), "kind": "oracle",
            "ols_seconds": float(ols_sec),
            "sample": f"one complete oracle SPCG solve of the whole workload (N={X.shape[0]}, "
                      f"d={X.shape[1]}, same recipe, schedule rule and tol), numpy FP64 with "
                      f"BLAS on {threads} threads (numpy's elementwise transform runs on one); "
                      f"wall time of that solve, not scaled"}


def run_reference(args, w, rank, world):
    """The oracle arm: K timed steps that together run ONE complete oracle
    solve of the stated workload, split at the oracle's own call boundaries
    (transform | sketches + QR | one step per stage | Stage II; with K
    smaller than the number of phases a step runs several, with K larger the
    remaining steps have no work).  value = the sum of the K step times = the
    wall time of that full-size solve; the warm-up steps solve a small sample
    of the same recipe."""
    if rank != 0:
        return
    threads = host_threads()
    for _ in range(args.warmup):                              # warm-ups: small sample
        Xs, Ys, _ = make_problem(w, N=min(WARM_SAMPLE_ROWS, w["N"]))
        for ph in oracle_phases(Xs, Ys, w["seed"], w["tol"]):
            ph()
    X, Y, _ = make_problem(w)                                 # data generation: untimed
    phases = oracle_phases(X, Y, w["seed"], w["tol"])
    K = max(args.steps, 1)
    groups = phase_groups(phases, K)
    step_s = []
    for grp in groups:
        t0 = time.perf_counter()
        for ph in grp:
            ph()
        step_s.append(time.perf_counter() - t0)
    v = float(sum(step_s))
    base = {"value": v, "unit": "s", "cores": int(threads), "kind": "oracle",
            "sample": f"one complete oracle SPCG solve of the whole workload (N={X.shape[0]}, "
                      f"d={X.shape[1]}) run as {K} timed steps split at the oracle's call "
                      f"boundaries ({len(phases)} phases); numpy FP64, BLAS on {threads} "
                      f"threads; warm-ups on a {min(WARM_SAMPLE_ROWS, w['N'])}-row sample"}
    line = {"impl": "reference", "metric": "seconds to 1e-6 OLS prediction error (plain FP64 SPCG)",
            "value": v, "unit": "s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": v * 1e3 / K, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w["name"], "N": w["N"], "d": w["d"], "tol": w["tol"],
                       "step": f"1/{K} of one full-size solve (value = one whole solve)"},
            "step_seconds": [round(t, 3) for t in step_s],
            "cpu_baseline": base,
            "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_pass_only(args, w, local_rank):
    """The fused pass alone: w = X^T (X p) over a rows x d FP64 matrix."""
    import torch

    from paper_2607_25272_b300 import spcg as S
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    g = torch.Generator(device=dev)
    g.manual_seed(1)
    m, d = args.rows, (args.cols or w["d"])
    pair = args.pass_dtype == "pair"
    dt = torch.float32 if pair else getattr(torch, args.pass_dtype)
    align = 16 // torch.empty(0, dtype=dt).element_size()     # rows 16-byte aligned (TMA)
    ld = (d + align - 1) // align * align
    if pair:   # hi block then lo block of a double-FP32 split
        X64 = torch.randn((m, d), dtype=torch.float64, device=dev, generator=g)
        A = torch.zeros(2 * m * ld, dtype=dt, device=dev)
        v = A.view(2, m, ld)
        v[0, :, :d] = X64.float()
        v[1, :, :d] = (X64 - v[0, :, :d].double()).float()
        del X64
    else:
        A = torch.zeros((m, ld), dtype=dt, device=dev)
        A[:, :d] = torch.randn((m, d), dtype=torch.float64, device=dev, generator=g).to(dt)
        A = A[:, :d]
    p = torch.randn(d, dtype=torch.float64, device=dev, generator=g)
    opts = S.Opts()
    opts.profile = 1
    s = S.Solver(torch.randn((d + 2, d), dtype=torch.float64, device=dev, generator=g),
                 torch.zeros(d + 2, dtype=torch.float64, device=dev))
    out = torch.empty(d, dtype=torch.float64, device=dev)
    if pair:
        def call(A, p, out):
            return s.gram_apply_pair(A, m, ld, p, out)
    else:
        call = s.gram_apply if args.pass_dtype == "float64" else s.gram_apply_typed
    for _ in range(args.warmup):
        call(A, p, out)
    stream = torch.cuda.current_stream(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        call(A, p, out)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    nbytes = m * d * (8 if pair else A.element_size())
    kname = "k_pass_df (double-FP32 pair)" if pair else f"k_pass<{args.pass_dtype}>"
    print(json.dumps({"kernel": f"{kname} via spcg_gram_apply (pass + reduce + sync)",
                      "rows": m, "d": d, "ms_per_call": ms, "alg_bytes": nbytes,
                      "gbs": nbytes / ms / 1e6, "tflops": 4 * m * d / ms / 1e9}), flush=True)
    s.close()


def run_sketch_only(args, w, local_rank):
    """spcg_sketch alone (column scales, transform, preconditioner QR) on a rows x d
    problem drawn on the GPU."""
    import torch

    from paper_2607_25272_b300 import spcg as S
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    g = torch.Generator(device=dev)
    g.manual_seed(1)
    m, d = args.rows, (args.cols or w["d"])
    X = torch.randn((m, d), dtype=torch.float64, device=dev, generator=g)
    Y = torch.randn(m, dtype=torch.float64, device=dev, generator=g)
    o = S.Opts()
    o.fwht_tile = args.fwht_tile
    o.fwht_first_levels = args.fwht_first
    o.qr_by_column = args.qr_by_column
    o.qr_panel_ctas = args.qr_panel_ctas
    s = S.Solver(X, Y, o)
    sc = S.spcg_default_schedule(m, d)
    for _ in range(args.warmup):
        s.sketch(1, sc)
    stream = torch.cuda.current_stream(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        s.sketch(1, sc)
    e1.record(stream)
    torch.cuda.synchronize()
    print(json.dumps({"kernel": "spcg_sketch", "rows": m, "d": d, "fwht_tile": args.fwht_tile,
                      "fwht_first_levels": args.fwht_first, "qr_by_column": args.qr_by_column,
                      "qr_panel_ctas": args.qr_panel_ctas,
                      "ms_per_call": e0.elapsed_time(e1) / args.steps}), flush=True)
    s.close()


def run_solve_only(args, w, local_rank):
    """spcg_solve alone on a rows x d Gaussian problem drawn on the GPU (for
    profiling the solve's kernels at a chosen size)."""
    import torch

    from paper_2607_25272_b300 import spcg as S
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    g = torch.Generator(device=dev)
    g.manual_seed(1)
    m, d = args.rows, (args.cols or w["d"])
    X = torch.randn((m, d), dtype=torch.float64, device=dev, generator=g)
    Y = torch.randn(m, dtype=torch.float64, device=dev, generator=g)
    o = S.Opts()
    o.dspace_ctas = args.dspace_ctas
    s = S.Solver(X, Y, o)
    stream = torch.cuda.current_stream(dev)
    ms, outs = time_solves(s, 1, None, args.steps, args.warmup, stream)
    _, info, st = outs[-1]
    print(json.dumps({"kernel": "spcg_solve", "rows": m, "d": d, "ms_per_call": ms,
                      "dspace_ctas": args.dspace_ctas,
                      "status": S.STATUS[st], "launches": info.launches,
                      "refine_iters": info.refine_iters}), flush=True)
    s.close()


def run_batched_only(args, w, local_rank):
    """The batched persistent kernel alone on a batch of args.batch problems of
    the batched workload's recipe, drawn on the GPU (default chunk sizes)."""
    import torch

    from paper_2607_25272_b300 import spcg as S
    from paper_2607_25272_b300.inputs import scaled_columns_problem_device
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    rng = np.random.default_rng(w["seed"])
    Xs, Ys = [], []
    for i in range(args.batch):
        N = int(rng.integers(1 << 12, (1 << 17) + 1))
        d = int(rng.integers(16, 257))
        X, Y, _ = scaled_columns_problem_device(N, d, 1e-3, 1e3, w["sigma"],
                                                seed=w["seed"] * 100000 + i, device=dev,
                                                dtype=torch.float32)
        ld = (d + 3) // 4 * 4
        Xp = torch.zeros((N, ld), dtype=torch.float32, device=dev)
        Xp[:, :d] = X
        Xs.append(Xp[:, :d])
        Ys.append(Y)
    B = S.Batch(Xs, Ys)
    for _ in range(args.warmup):
        B.solve(w["seed"], w["tol"])
    times = [B.solve(w["seed"], w["tol"])[3] for _ in range(args.steps)]
    rc, st, it, _ = B.solve(w["seed"], w["tol"])
    nbytes = sum(X.shape[0] * X.shape[1] * 4 for X in Xs)
    print(json.dumps({"kernel": "k_batched_spcg", "problems": args.batch,
                      "ms_per_call": float(np.median(times)), "status_ok": sum(v == 0 for v in st),
                      "x_bytes_fp32": nbytes, "stage2_iters_sum": int(sum(it)),
                      "phase_ms": batch_phase_summary(B, Xs)}), flush=True)
    B.close()


def run_ours(args, w, rank, world, local_rank):
    import torch

    from paper_2607_25272_b300 import spcg as S

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    X, Y, _ = make_problem(w, seed_offset=rank)
    N, d = X.shape
    Xh = torch.from_numpy(X).pin_memory()
    Yh = torch.from_numpy(Y).pin_memory()
    Xd = Xh.to(dev)
    Yd = Yh.to(dev)
    stream = torch.cuda.current_stream(dev)
    sched = S.spcg_default_schedule(N, d)
    sched.tol = w["tol"]
    solver = S.Solver(Xd, Yd)
    beta = torch.empty(d, dtype=torch.float64, device=dev)

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    for _ in range(args.warmup):
        solver.solve(w["seed"], sched, beta)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    launches = 0
    infos = []
    with ClockSampler(local_rank) as clk:
        barrier()
        torch.cuda.synchronize()
        if args.ncu_region == "plain":
            torch.cuda.profiler.start()
        e0.record(stream)
        for _ in range(args.steps):
            _, info, st = solver.solve(w["seed"], sched, beta)
            launches += info.launches
            infos.append(info)
        e1.record(stream)
        torch.cuda.synchronize()
        if args.ncu_region == "plain":
            torch.cuda.profiler.stop()
        barrier()
    ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, dev)
    beta_h = beta.cpu().numpy()

    # the mixed-precision form on the same problem and schedule (BF16 stages,
    # FP32 compensated refinement, FP64 true gradients)
    mopts = S.Opts()
    mopts.precision = S.PREC_MIXED
    msolver = S.Solver(Xd, Yd, mopts)
    mbeta = torch.empty(d, dtype=torch.float64, device=dev)
    for _ in range(args.warmup):
        msolver.solve(w["seed"], sched, mbeta)
    torch.cuda.synchronize()
    if args.ncu_region == "mixed":
        torch.cuda.profiler.start()
    e0.record(stream)
    minfos = []
    for _ in range(args.steps):
        _, minfo, _ = msolver.solve(w["seed"], sched, mbeta)
        minfos.append(minfo)
    e1.record(stream)
    torch.cuda.synchronize()
    if args.ncu_region == "mixed":
        torch.cuda.profiler.stop()
    ms_mixed = e0.elapsed_time(e1) / args.steps
    mbeta_h = mbeta.cpu().numpy()
    mopts.profile = 1
    mpsolver = S.Solver(Xd, Yd, mopts)
    _, mpinfo, _ = mpsolver.solve(w["seed"], sched)
    mpsolver.close()
    msolver.close()

    # fused-pass timing: the same solves with CUDA events around every pass
    opts = S.Opts()
    opts.profile = 1
    psolver = S.Solver(Xd, Yd, opts)
    pass_ms, pass_bytes, pass_n = 0.0, 0, 0
    for _ in range(args.steps):
        _, pinfo, _ = psolver.solve(w["seed"], sched)
        pass_ms += pinfo.pass_ms
        pass_bytes += pinfo.bytes_pass
        pass_n += pinfo.pass_launches
    psolver.close()

    # end to end through the C ABI from pinned host buffers (spcg_solve_host:
    # H2D of X and Y, the solve, D2H of beta, all inside the timed region)
    e2e_steps = max(1, min(args.steps, 3))
    solver.close()
    del Xd, Yd
    torch.cuda.synchronize()
    t_e2e = []
    for _ in range(e2e_steps):
        torch.cuda.synchronize()
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        bh2, _, st2 = S.spcg_solve_host(Xh, Yh, w["seed"], sched)
        a1.record(stream)
        torch.cuda.synchronize()
        assert st2 == S.SPCG_OK, S.STATUS[st2]
        t_e2e.append(a0.elapsed_time(a1))
    if rank != 0:
        return

    # accuracy against LAPACK's OLS estimator (outside the timed region)
    beta_ols = lapack_ols(X, Y)
    e_rel = rel_error(X, beta_h, beta_ols)
    e_rel_mixed = rel_error(X, mbeta_h, beta_ols)

    hbm_peak_gbs, hbm_src = hbm_peak()
    # the plain pass is bound by FP64 FMA issue: its denominator is the FP64
    # FMA rate measured on this GPU now (a kernel of independent FMA chains)
    fp64_peak_tflops = S.spcg_probe_fma_tflops("float64", 1 << 16)
    avg_pass_s = pass_ms / max(pass_n, 1) / 1e3
    bytes_per_launch = pass_bytes / max(pass_n, 1)
    flops_per_launch = bytes_per_launch / 8 * 4       # 2 FMA per element read
    ach_tflops = flops_per_launch / avg_pass_s / 1e12
    hbm_gbs = bytes_per_launch / avg_pass_s / 1e9
    roofline = {"bound": "alu", "kernel": "k_pass (fused X^T(Xp), FP64)",
                "achieved": ach_tflops, "peak": fp64_peak_tflops, "unit": "TFLOP/s",
                "frac": ach_tflops / fp64_peak_tflops,
                "peak_source": "of measured: FP64 FMA rate of this GPU in this run "
                               "(spcg_probe_fma_tflops, independent FMA chains on every SM)",
                "peak_nominal_tflops": NOMINAL_FP64_TFLOPS,
                # DRAM read+write bytes per launch from the ncu capture of this kernel on a
                # 262144 x 500 operand, scaled by rows to the average launch of the solve
                # (traffic grows with the rows read); None once the kernel changes.
                "traffic": bytes_per_launch * K_PASS_TRAFFIC_RATIO if K_PASS_TRAFFIC_RATIO else None,
                "hbm_gbs": hbm_gbs, "hbm_peak_gbs": hbm_peak_gbs, "hbm_frac": hbm_gbs / hbm_peak_gbs,
                "hbm_peak_source": hbm_src, "hbm_peak_nominal_gbs": NOMINAL_HBM_GBS,
                "hbm_frac_of_nominal": hbm_gbs / NOMINAL_HBM_GBS,
                "pass_launches_per_step": pass_n / args.steps,
                "alg_bytes_per_launch": bytes_per_launch}
    last = infos[-1]
    line = {
        "metric": "seconds to 1e-6 OLS prediction error (plain FP64 SPCG)",
        "value": ms / 1e3, "unit": "s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w["name"], "N": N, "d": d, "tol": w["tol"],
                   "schedule": {"K": sched.K, "m1": sched.m[0] if sched.K else None,
                                "mK": sched.m[sched.K - 1] if sched.K else None,
                                "r": sched.r, "a_i": 3},
                   "l2": "no flush: X is 4.19 GB, larger than the 126 MB L2",
                   "parallelism": f"{world} independent problem(s), one per GPU"},
        "accuracy": {"rel_pred_error_vs_lapack_ols": e_rel,
                     "refine_iters": last.refine_iters, "restarts": last.restarts,
                     "converged": last.converged},
        "phases_ms": {"sketch": last.ms_sketch, "stages": last.ms_stages,
                      "refine": last.ms_refine},
        "forms": {
            "plain_fp64": {"s": ms / 1e3, "rel_pred_error": e_rel},
            "mixed": {"s": ms_mixed / 1e3, "rel_pred_error": e_rel_mixed,
                      "speedup_vs_plain_fp64": ms / ms_mixed,
                      "phases_ms": {"sketch": minfos[-1].ms_sketch, "stages": minfos[-1].ms_stages,
                                    "refine": minfos[-1].ms_refine},
                      "refine_iters": minfos[-1].refine_iters, "restarts": minfos[-1].restarts,
                      "cond_est": minfos[-1].cond_est, "inner_prec": minfos[-1].inner_prec,
                      "grad_prec": minfos[-1].grad_prec,
                      "roofline": pass_roofline(mpinfo, "float32", hbm_peak_gbs, hbm_src,
                                                K_PASS_F32_TRAFFIC_RATIO if w["d"] == 500 else None,
                                                "k_pass<float> (Stage II on the FP32 copy)")}},
        "gpu_launches": launches,
        "roofline": roofline,
        "e2e": {"value": float(np.median(t_e2e)) / 1e3, "unit": "s",
                "h2d_bytes_per_step": int(Xh.numel() * 8 + Yh.numel() * 8),
                "d2h_bytes_per_step": int(d * 8)},
        "clocks": clk.summary(),
    }
    del Xh, Yh
    # the metric's comparisons at the other workloads (one GPU only)
    if world == 1 and not args.headline_only:
        for key in ("c3", "c4", "c5"):
            fn = {"c3": run_forms, "c4": run_batched, "c5": run_learned}[key]
            try:
                line[key] = fn(args, WORKLOADS[key])
            except Exception as e:   # a failed extra must not lose the headline line
                line[key] = {"error": f"{type(e).__name__}: {e}"}
            torch.cuda.empty_cache()
    line["cpu_baseline"] = None if args.no_cpu_baseline else cpu_baseline(w, X, Y)
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c2", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--headline-only", action="store_true",
                    help="skip the nested c3/c4/c5 comparisons of the default run")
    ap.add_argument("--kernel", default=None, choices=[None, "pass", "sketch", "solve", "batched"],
                    help="time one kernel alone instead of the solve")
    ap.add_argument("--rows", type=int, default=1 << 18)
    ap.add_argument("--cols", type=int, default=0,
                    help="columns for --kernel pass|sketch|solve (0: the workload's d)")
    ap.add_argument("--batch", type=int, default=32, help="problems for --kernel batched")
    ap.add_argument("--weights", default=None, help="schedule model weights (npz) for c5")
    ap.add_argument("--ncu-region", default=None, choices=[None, "plain", "mixed"],
                    help="bracket the timed solves of this form with cudaProfilerStart/Stop "
                         "(for ncu --profile-from-start off)")
    ap.add_argument("--fwht-tile", type=int, default=0,
                    help="spcg_opts.fwht_tile for --kernel sketch (0 default, 1, 2, 3)")
    ap.add_argument("--fwht-first", type=int, default=0,
                    help="spcg_opts.fwht_first_levels for --kernel sketch")
    ap.add_argument("--qr-by-column", type=int, default=0,
                    help="spcg_opts.qr_by_column for --kernel sketch")
    ap.add_argument("--qr-panel-ctas", type=int, default=0,
                    help="spcg_opts.qr_panel_ctas for --kernel sketch")
    ap.add_argument("--dspace-ctas", type=int, default=0,
                    help="spcg_opts.dspace_ctas for --kernel solve")
    ap.add_argument("--pass-dtype", default="float64",
                    choices=["float64", "float32", "bfloat16", "pair"])
    args = ap.parse_args()
    w = WORKLOADS[args.workload]
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1 and args.impl == "ours":
        import torch
        torch.distributed.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    if args.kernel == "pass":
        run_pass_only(args, w, local_rank)
    elif args.kernel == "sketch":
        run_sketch_only(args, w, local_rank)
    elif args.kernel == "solve":
        run_solve_only(args, w, local_rank)
    elif args.kernel == "batched":
        run_batched_only(args, w, local_rank)
    elif args.impl == "ours" and args.workload == "c3":
        print_nested(args, w, run_forms(args, w), "bf16/f32/f64")
    elif args.impl == "ours" and args.workload == "c4":
        print_nested(args, w, run_batched(args, w), "f32 (compensated) / f64 scalars")
    elif args.impl == "ours" and args.workload == "c5":
        print_nested(args, w, run_learned(args, w), "f64")
    elif args.impl == "reference":
        run_reference(args, w, rank, world)
    else:
        run_ours(args, w, rank, world, local_rank)
    if world > 1 and args.impl == "ours":
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
