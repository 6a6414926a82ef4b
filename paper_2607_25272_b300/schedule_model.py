"""The learned sketch-size schedule: data, training and the trained weights.

Sec. 4.3 leaves the automatic choice of the schedule open.  Here a small MLP
(4 -> 64 -> 64 -> 25, BF16 weights; kernels in csrc/mlp.cu) predicts the
log10 cost of each of the 25 candidate schedules of spcg_candidate_schedule
from four features taken after the paper's first stage (spcg_features:
log2 N, log2 d, log10 of the condition estimate max R_ii / min R_ii, log10 of
the unexplained share of b_1), and spcg_solve_learned runs the cheapest.

Training data are SPCG runs on the GPU: for every sampled problem, each
candidate runs from the same sketch to the same Stage II tolerance and its
stage-plus-refinement device time is recorded (a candidate that does not
converge costs ten times the slowest).  Problems follow the experimental
design of Sec. 4, X = G diag(s) with s geometric from 1 to 1/kappa, with
N log-uniform in [2^14, 2^20], d log-uniform in [32, 512], kappa log-uniform
in [1e2, 1e8] and sigma log-uniform in [1e-3, 1]; they are drawn on the GPU
from a seeded torch generator (inputs only).  The training loop calls the
library's forward/backward (spcg_mlp_grad) and Adam (spcg_mlp_adam) kernels;
this module only moves data and keeps the loop.

Usage (GPU): python -m paper_2607_25272_b300.schedule_model --problems 800 \
    --out paper_2607_25272_b300/schedule_mlp.npz
"""
import argparse
import json
import math
import os
import time

import numpy as np

from . import spcg as S

N_OUT = 25
PAPER_CANDIDATE = 2
HERE = os.path.dirname(os.path.abspath(__file__))
WEIGHTS = os.path.join(HERE, "schedule_mlp.npz")


def sample_problem(rng_np, gen, device):
    """One training problem drawn on the GPU; returns (X, Y, meta)."""
    import torch
    N = int(round(2.0 ** rng_np.uniform(14, 20)))
    d = int(round(2.0 ** rng_np.uniform(5, 9)))
    d = min(d, N // 8)
    kappa = 10.0 ** rng_np.uniform(2, 8)
    sigma = 10.0 ** rng_np.uniform(-3, 0)
    s = kappa ** (-torch.arange(d, dtype=torch.float64, device=device) / max(d - 1, 1))
    X = torch.randn((N, d), dtype=torch.float64, device=device, generator=gen) * s[None, :]
    beta = torch.randn(d, dtype=torch.float64, device=device, generator=gen)
    Y = X @ beta + sigma * torch.randn(N, dtype=torch.float64, device=device, generator=gen)
    return X, Y, {"N": N, "d": d, "kappa": kappa, "sigma": sigma}


def problem_costs(X, Y, seed, tol=1e-6, precision=S.PREC_FP64):
    """Features and the stage + Stage II device time (ms) of every candidate."""
    import torch
    opts = S.Opts()
    opts.precision = precision
    solver = S.Solver(X, Y, opts)
    try:
        d = X.shape[1]
        beta = torch.zeros(d, dtype=torch.float64, device=X.device)
        # features: the paper's first stage from the paper's sketch
        solver.sketch(seed, S.spcg_default_schedule(*X.shape))
        solver.pcg_stage(0, 3, beta)
        feats = solver.features(beta)
        costs = np.full(N_OUT, np.nan)
        conv = np.zeros(N_OUT, dtype=bool)
        for idx in range(N_OUT):
            _, info, st = solver.solve_candidate(seed, idx, tol, reuse_sketch=True,
                                                 raise_on_error=False)
            costs[idx] = info.ms_stages + info.ms_refine
            conv[idx] = (st == S.SPCG_OK and info.converged == 1)
        worst = np.nanmax(costs[conv]) if conv.any() else np.nanmax(costs)
        costs[~conv] = 10.0 * worst
        return np.array(feats, dtype=np.float64), costs
    finally:
        solver.close()


def collect(n_problems, seed0=1, log_every=50):
    import torch
    rng = np.random.default_rng(seed0)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed0)
    feats, costs, metas = [], [], []
    t0 = time.time()
    for i in range(n_problems):
        X, Y, meta = sample_problem(rng, gen, "cuda")
        f, c = problem_costs(X, Y, seed=seed0 + i)
        feats.append(f)
        costs.append(c)
        metas.append(meta)
        del X, Y
        if log_every and (i + 1) % log_every == 0:
            print(f"[collect] {i + 1}/{n_problems} problems, {time.time() - t0:.0f} s", flush=True)
    return np.array(feats), np.array(costs), metas


class Trainer:
    """Full-batch Adam on the MLP through the library's kernels."""

    def __init__(self, n_out=N_OUT, seed=0):
        import torch
        self.n_out = n_out
        self.P = S.spcg_mlp_params(n_out)
        g = np.random.default_rng(seed)
        theta = np.zeros(self.P, dtype=np.float32)
        # He-style initial weights, zero biases (layout of spcg_mlp_params)
        o = 0
        for rows, cols in ((64, 4), (64, 64), (n_out, 64)):
            theta[o:o + rows * cols] = g.standard_normal(rows * cols) * math.sqrt(2.0 / cols)
            o += rows * cols + rows
        self.theta = torch.from_numpy(theta).cuda()
        self.m = torch.zeros_like(self.theta)
        self.v = torch.zeros_like(self.theta)
        self.grad = torch.zeros_like(self.theta)
        self.Wb = torch.zeros(self.P, dtype=torch.int16, device="cuda")
        S.spcg_mlp_to_bf16(self.theta, self.Wb)
        self.loss = torch.zeros(1, dtype=torch.float32, device="cuda")
        self.step_no = 0

    def fit(self, x, t, steps=3000, lr=3e-3):
        import torch
        xd = torch.as_tensor(x, dtype=torch.float32).cuda().contiguous()
        td = torch.as_tensor(t, dtype=torch.float32).cuda().contiguous()
        ws = torch.zeros(int(S.lib().spcg_mlp_workspace_floats(self.n_out, xd.shape[0])),
                         dtype=torch.float32, device="cuda")
        hist = []
        for k in range(steps):
            S.spcg_mlp_grad(self.Wb, self.n_out, xd, td, self.grad, self.loss, ws)
            self.step_no += 1
            S.spcg_mlp_adam(self.theta, self.grad, self.m, self.v, lr, self.step_no, self.Wb)
            if k % 100 == 0 or k == steps - 1:
                hist.append((k, float(self.loss.item())))
        return hist

    def predict(self, x):
        import torch
        xd = torch.as_tensor(x, dtype=torch.float32).cuda().contiguous()
        return S.spcg_mlp_forward(self.Wb, self.n_out, xd).cpu().numpy()


def train(feats, costs, steps=3000, lr=3e-3, val_frac=0.2, seed=0):
    n = len(feats)
    rng = np.random.default_rng(seed)
    perm = rng.permutation(n)
    nv = max(1, int(val_frac * n))
    val, tr = perm[:nv], perm[nv:]
    fmean, fstd = feats[tr].mean(0), feats[tr].std(0) + 1e-6
    logc = np.log10(costs)
    tmean, tstd = float(logc[tr].mean()), float(logc[tr].std() + 1e-6)
    x = (feats - fmean) / fstd
    t = (logc - tmean) / tstd
    trainer = Trainer(seed=seed)
    hist = trainer.fit(x[tr], t[tr], steps=steps, lr=lr)

    def evaluate(idx):
        pred = trainer.predict(x[idx])
        choice = pred.argmin(1)
        chosen = costs[idx, choice]
        best = costs[idx].min(1)
        paper = costs[idx, PAPER_CANDIDATE]
        return {"regret": float(np.mean(chosen / best)),
                "gain_vs_paper": float(np.sum(paper) / np.sum(chosen)),
                "mean_gain_vs_paper": float(np.mean(paper / chosen)),
                "oracle_gain_vs_paper": float(np.sum(paper) / np.sum(best))}

    stats = {"train": evaluate(tr), "val": evaluate(val), "loss_history": hist,
             "n_train": int(len(tr)), "n_val": int(len(val))}
    norm = np.concatenate([fmean, fstd]).astype(np.float32)
    return trainer, norm, (tmean, tstd), stats


def save(path, trainer, norm, tnorm, stats):
    np.savez(path, theta=trainer.theta.cpu().numpy(), Wb=trainer.Wb.cpu().numpy(),
             norm=norm, target_mean=tnorm[0], target_std=tnorm[1], n_out=N_OUT,
             stats=json.dumps(stats))


def load(path=WEIGHTS):
    """(Wb device tensor, norm floats) of the trained model, or (None, None)."""
    import torch
    if not os.path.exists(path):
        return None, None
    z = np.load(path)
    return torch.from_numpy(z["Wb"]).cuda(), [float(v) for v in z["norm"]]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--problems", type=int, default=800)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--out", default=WEIGHTS)
    ap.add_argument("--data", default=None, help="save the collected data (npz) here")
    args = ap.parse_args()
    feats, costs, metas = collect(args.problems, seed0=args.seed)
    if args.data:
        np.savez(args.data, feats=feats, costs=costs, metas=json.dumps(metas))
    trainer, norm, tnorm, stats = train(feats, costs, steps=args.steps)
    save(args.out, trainer, norm, tnorm, stats)
    print(json.dumps({k: v for k, v in stats.items() if k != "loss_history"}), flush=True)
    print(json.dumps({"runs": int(costs.size), "loss_first_last": [stats["loss_history"][0],
                                                                  stats["loss_history"][-1]]}))


if __name__ == "__main__":
    main()
