"""The multi-process path of bench.py on CPU (gloo, world size 2): each rank
solves its own problem (distinct seeds, no collective on the data path) and
the job time is the maximum over ranks."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist

    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = dict(bench.WORKLOADS["c1"])
        w["N"] = 2000
        X, Y, _ = bench.make_problem(w, seed_offset=rank)
        local = 10.0 + rank
        out[rank] = (bench.max_over_ranks(local), float(X[0, 0]))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_max_and_distinct_problems():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert out[0][0] == 11.0 and out[1][0] == 11.0
    assert out[0][1] != out[1][1]


def test_reference_arm_under_torchrun_prints_once():
    """`bench.py --impl reference` launched as the bench contract launches it
    for N > 1 (torchrun, two ranks): rank 0 alone runs the oracle and prints
    one JSON line; the other rank exits 0 without work."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           os.path.join(root, "bench.py"), "--impl", "reference", "--workload", "c1",
           "--gpus", "2", "--steps", "2", "--warmup", "1"]
    res = subprocess.run(cmd, cwd=root, capture_output=True, text=True, timeout=600)
    assert res.returncode == 0, res.stderr[-2000:]
    lines = [ln for ln in res.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
