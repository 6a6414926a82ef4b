"""Benchmark: seconds to a 1e-6 relative OLS prediction error with SPCG.

Workload (default): plain FP64 SPCG on N = 2^20, d = 500, X = U diag(s) V^T
with s geometric from 1 to 1e-6 (kappa = 1e6), beta ~ N(0, 1), sigma = 0.1;
the paper's default schedule (m_1 = 8d rounded to a power of two, doubling
to N'/2, r = 6d, a_i = 3) and the Stage II stopping rule for tol = 1e-6.
Synthetic data, generated on the host from a fixed seed.

One step = one spcg_solve (SRHT sketch, preconditioner QR, every Stage I
subproblem, Stage II to the stopping rule) with X, Y resident in HBM.
X is 4.19 GB, far larger than the 126 MB L2, so no flush is needed between
steps.  The result is checked against the oracle's OLS estimator (outside
the timed region).

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
    "c2": dict(name="plain SPCG FP64, N=2^20, d=500, kappa=1e6, sigma=0.1, seed=1",
               N=1 << 20, d=500, kappa=1e6, sigma=0.1, seed=1, tol=1e-6),
    "c1": dict(name="plain SPCG FP64, N=20000, d=50, X iid N(0,1), sigma=1, seed=1",
               N=20000, d=50, kappa=None, sigma=1.0, seed=1, tol=1e-6),
}
CPU_SAMPLE_ROWS = 1 << 17     # oracle row sample for the CPU baseline
# ncu: k_pass (FP64) on 262144 x 500 read 1.048667 GB + wrote 3.14 MB for 1.048576 GB of rows
K_PASS_TRAFFIC_RATIO = (1.048667e9 + 3.142912e6) / 1.048576e9


def make_problem(w, N=None, seed_offset=0):
    from paper_2607_25272_b300.inputs import gaussian_problem, svd_problem
    N = N or w["N"]
    if w["kappa"] is None:
        return gaussian_problem(N, w["d"], w["sigma"], seed=w["seed"] + seed_offset)
    return svd_problem(N, w["d"], w["kappa"], w["sigma"], seed=w["seed"] + seed_offset)


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


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


def cpu_baseline(w, steps=1):
    """The oracle (numpy FP64) on a row sample of the workload, scaled to N."""
    from oracle.spcg import spcg as oracle_spcg
    n_s = min(CPU_SAMPLE_ROWS, w["N"])
    X, Y, _ = make_problem(w, N=n_s)
    times = []
    for _ in range(steps):
        t0 = time.perf_counter()
        oracle_spcg(X, Y, seed=w["seed"], tol=w["tol"])
        times.append(time.perf_counter() - t0)
    threads = int(os.environ.get("OPENBLAS_NUM_THREADS", len(os.sched_getaffinity(0))))
    scale = w["N"] / n_s
    return {"value": float(np.mean(times) * scale), "unit": "s", "cores": int(threads),
            "kind": "oracle",
            "sample": f"oracle SPCG (numpy FP64, BLAS on {threads} threads) on the same recipe "
                      f"with N={n_s} rows, same d, kappa, sigma, schedule rule and tol; "
                      f"wall time x N/{n_s} (measured {np.mean(times):.2f} s per sample solve)"}


def run_reference(args, w, rank, world):
    if rank != 0:
        return
    base = cpu_baseline(w, steps=1)                        # warm-up of the oracle arm
    vals = []
    for _ in range(args.steps):
        vals.append(cpu_baseline(w, steps=1)["value"])
    v = float(np.mean(vals))
    base["value"] = v
    line = {"impl": "reference", "metric": "seconds to 1e-6 OLS prediction error (plain FP64 SPCG)",
            "value": v, "unit": "s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": v * 1e3, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w["name"], "N": w["N"], "d": w["d"], "tol": w["tol"]},
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
    m, d = args.rows, w["d"]
    A = torch.randn((m, d), dtype=torch.float64, device=dev, generator=g)
    p = torch.randn(d, dtype=torch.float64, device=dev, generator=g)
    opts = S.Opts()
    opts.profile = 1
    s = S.Solver(A[: d + 1], torch.zeros(d + 1, dtype=torch.float64, device=dev))
    out = torch.empty(d, dtype=torch.float64, device=dev)
    for _ in range(args.warmup):
        s.gram_apply(A, p, out)
    stream = torch.cuda.current_stream(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        s.gram_apply(A, p, out)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    nbytes = m * d * 8
    print(json.dumps({"kernel": "k_pass via spcg_gram_apply (pass + reduce + sync)",
                      "rows": m, "d": d, "ms_per_call": ms, "alg_bytes": nbytes,
                      "gbs": nbytes / ms / 1e6, "tflops": 4 * m * d / ms / 1e9}), flush=True)
    s.close()


def run_ours(args, w, rank, world, local_rank):
    import torch

    from oracle.linalg import ols
    from oracle.metrics import rel_pred_error
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
        e0.record(stream)
        for _ in range(args.steps):
            _, info, st = solver.solve(w["seed"], sched, beta)
            launches += info.launches
            infos.append(info)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
    ms = e0.elapsed_time(e1) / args.steps
    if world > 1:
        t = torch.tensor([ms], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
    beta_h = beta.cpu().numpy()

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

    # end to end through the public API: pinned host -> device, solve, beta -> host
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
        Xd2 = Xh.to(dev, non_blocking=True)
        Yd2 = Yh.to(dev, non_blocking=True)
        s2 = S.Solver(Xd2, Yd2)
        b2, _, _ = s2.solve(w["seed"], sched)
        bh2 = b2.to("cpu", non_blocking=False)
        a1.record(stream)
        torch.cuda.synchronize()
        s2.close()
        del Xd2, Yd2
        t_e2e.append(a0.elapsed_time(a1))
    if rank != 0:
        return

    # accuracy against the oracle's OLS estimator (outside the timed region)
    e_rel = rel_pred_error(X, beta_h, ols(X, Y))

    peaks = measured_peaks()
    hbm_peak = peaks.get("hbm_gbs", 6400.0)
    avg_pass_s = pass_ms / max(pass_n, 1) / 1e3
    bytes_per_launch = pass_bytes / max(pass_n, 1)
    flops_per_launch = bytes_per_launch / 8 * 4       # 2 FMA per element read
    fp64_peak_tflops = 1.25                            # nominal B300 FP64 (recipe table)
    ach_tflops = flops_per_launch / avg_pass_s / 1e12
    hbm_gbs = bytes_per_launch / avg_pass_s / 1e9
    roofline = {"bound": "alu", "kernel": "k_pass (fused X^T(Xp), FP64)",
                "achieved": ach_tflops, "peak": fp64_peak_tflops, "unit": "TFLOP/s",
                "frac": ach_tflops / fp64_peak_tflops,
                "peak_source": "nominal B300 FP64 1.25 TFLOP/s (recipe table); FP64 FMA probe "
                               "measured 1.13 TFLOP/s",
                # DRAM read+write bytes per launch from the ncu capture of this kernel on a
                # 262144 x 500 operand (profiles/k_pass_fp64_gram_262144x500.md), scaled by
                # rows to the average launch of the solve; None once the kernel changes.
                "traffic": bytes_per_launch * K_PASS_TRAFFIC_RATIO if K_PASS_TRAFFIC_RATIO else None,
                "hbm_gbs": hbm_gbs, "hbm_peak_gbs": hbm_peak, "hbm_frac": hbm_gbs / hbm_peak,
                "hbm_peak_source": "of measured (MEASURED_PEAKS.json hbm_gbs)",
                "pass_launches_per_step": pass_n / args.steps,
                "alg_bytes_per_launch": bytes_per_launch}
    cpu = None if args.no_cpu_baseline else cpu_baseline(w, steps=1)
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
        "accuracy": {"rel_pred_error_vs_oracle_ols": e_rel,
                     "refine_iters": last.refine_iters, "restarts": last.restarts,
                     "converged": last.converged},
        "phases_ms": {"sketch": last.ms_sketch, "stages": last.ms_stages,
                      "refine": last.ms_refine},
        "gpu_launches": launches,
        "roofline": roofline,
        "e2e": {"value": float(np.median(t_e2e)) / 1e3, "unit": "s",
                "h2d_bytes_per_step": int(Xh.numel() * 8 + Yh.numel() * 8),
                "d2h_bytes_per_step": int(d * 8)},
        "clocks": clk.summary(),
        "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c2", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--kernel", default=None, choices=[None, "pass"],
                    help="time one kernel alone instead of the solve")
    ap.add_argument("--rows", type=int, default=1 << 18)
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
    elif args.impl == "reference":
        run_reference(args, w, rank, world)
    else:
        run_ours(args, w, rank, world, local_rank)
    if world > 1 and args.impl == "ours":
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
