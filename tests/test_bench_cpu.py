"""Host-side checks of bench.py's oracle arm: the phase-by-phase run of the
oracle's SPCG solve (the reference arm splits one full-size solve over its
timed steps at these boundaries) gives the same beta as one call of the
oracle's own spcg, bit for bit, and every phase runs exactly once."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from oracle.spcg import spcg as oracle_spcg  # noqa: E402
from paper_2607_25272_b300.inputs import svd_problem  # noqa: E402


def test_phase_split_equals_one_oracle_call():
    X, Y, _ = svd_problem(5000, 20, 1e4, 0.1, seed=3)
    phases = bench.oracle_phases(X, Y, 7, 1e-6)
    out = None
    for ph in phases:
        out = ph()
    ref = oracle_spcg(X, Y, seed=7, tol=1e-6)["beta"]
    assert np.array_equal(out, ref)


def test_phase_groups_cover_every_phase_once():
    for n_phases in (3, 11, 15):
        for K in (1, 2, 5, 11, 20):
            ph = list(range(n_phases))
            groups = bench.phase_groups(ph, K)
            assert sum(groups, []) == ph and len(groups) == K


def test_batched_streaming_bound_counts_every_phase():
    """The batch's streaming bound for one problem, counted by hand: N = 5000,
    d = 20 (C = 21, ld = 20, N' = 8192, stages 256, 512, ..., 4096, r = 120)
    and 7 Stage II iterations."""
    import bench
    N, d, it = 5000, 20, 7
    C, ld = 21, 20
    m = [256, 512, 1024, 2048, 4096]
    want = 2 * N * C * 4                       # column maxima, CountSketch read
    want += 4096 * C * 8 + 6 * d * d * 4       # S_K bucket rows, preconditioner rows
    want += sum(mi * ld * 4 * 5 for mi in m)   # stage matrices written once, read 4 times
    want += (it + 2) * N * d * 4               # Stage II passes and two true gradients
    b = bench.batch_streaming_bound([(N, d)], [it], 1000.0)
    assert b["alg_bytes"] == want
    assert abs(b["bound_ms"] - want / 1e9) < 1e-12


def test_reference_arm_prints_one_contract_line():
    """`bench.py --impl reference` (the oracle arm, host only) on the small
    workload: exactly one JSON line on stdout, with the keys of the bench
    contract, the oracle named as the baseline and no host-device bytes."""
    import json
    import subprocess
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--workload", "c1", "--steps", "3", "--warmup", "1"],
                         cwd=ROOT, check=True, capture_output=True, text=True, timeout=600).stdout
    lines = [ln for ln in out.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference"
    assert line["steps"] == 3 and line["warmup"] == 1 and line["n_gpus"] == 1
    assert line["higher_is_better"] is False and line["unit"] == "s"
    assert line["value"] > 0 and abs(line["ms_per_step"] * 3 / 1e3 - line["value"]) < 1e-9
    assert "workload" in line["config"]
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == line["value"] and cb["cores"] >= 1
    assert cb["sample"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["unit"] == line["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_bench_accuracy_helpers_agree_with_the_oracle():
    """The GPU arm's accuracy report uses its own LAPACK least squares (the
    oracle package runs only in the CPU baseline and the reference arm);
    on the same problem it agrees with the oracle's OLS estimator and error
    metric."""
    from oracle.linalg import ols
    from oracle.metrics import rel_pred_error
    X, Y, beta_true = svd_problem(5000, 40, 1e6, 0.1, seed=3)
    b_lapack = bench.lapack_ols(X, Y)
    b_oracle = ols(X, Y)
    assert rel_pred_error(X, b_lapack, b_oracle) <= 1e-9
    assert abs(bench.rel_error(X, beta_true, b_oracle) - rel_pred_error(X, beta_true, b_oracle)) \
        <= 1e-12 * rel_pred_error(X, beta_true, b_oracle)


def test_pass_roofline_arithmetic():
    """The HBM roofline of a pass kind from a profiled solve's counters:
    algorithmic bytes per launch over the mean event time per launch, against
    the measured peak and, for context, the nominal 7.7 TB/s."""
    from types import SimpleNamespace

    from paper_2607_25272_b300 import spcg as S
    k = S.OP_NAMES.index("float32")
    launches, ms, nbytes = [0] * 4, [0.0] * 4, [0] * 4
    launches[k], ms[k], nbytes[k] = 10, 5.0, 10 * 3_000_000_000    # 3 GB in 0.5 ms each
    info = SimpleNamespace(launches_by_op=launches, pass_ms_by_op=ms, bytes_by_op=nbytes)
    r = bench.pass_roofline(info, "float32", 6000.0, "test peak", 1.01, "k_pass<float>")
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert abs(r["achieved"] - 6000.0) < 1e-9 and abs(r["frac"] - 1.0) < 1e-12
    assert abs(r["frac_of_nominal"] - 6000.0 / 7700.0) < 1e-12
    assert abs(r["traffic"] - 3.03e9) < 1.0 and r["alg_bytes_per_launch"] == 3e9
    assert r["launches_per_step"] == 10
    other = S.OP_NAMES.index("float64")
    assert bench.pass_roofline(info, S.OP_NAMES[other], 6000.0, "x", None, "k") is None


def test_cpu_baseline_on_the_small_workload():
    """The CPU baseline leg on the small workload: one oracle solve timed at
    full size, the direct OLS solve timed beside it, cores stated."""
    b = bench.cpu_baseline(bench.WORKLOADS["c1"])
    assert b["kind"] == "oracle" and b["unit"] == "s" and b["cores"] >= 1
    assert b["value"] > 0 and b["ols_seconds"] > 0 and b["sample"]
