"""The multi-process (N > 1) path of bench.py on CPU with the gloo backend, world size 2:
process-group set-up, the max over ranks of the timed region, per-rank independent inputs
(replicas: no data-path collective), and the reference arm under torchrun (rank 0 alone
reports)."""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, port, out):
    os.environ.update({"RANK": str(rank), "LOCAL_RANK": str(rank), "WORLD_SIZE": "2",
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    import bench
    r, ws, local, dist = bench._dist()
    try:
        assert (r, ws) == (rank, 2)
        m = bench._max_over_ranks(1.5 + rank, dist, torch.device("cpu"))
        b = bench._batches(rank, 2000)
        out.put((rank, m, float(b[0].sum())))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_rank_gloo_max_and_independent_replicas():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=240) for _ in range(2))
    for p in ps:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert [m for _, m, _ in res] == [2.5, 2.5]      # the slowest rank's time, on every rank
    assert res[0][2] != res[1][2]                      # each replica draws its own batches


def test_reference_arm_under_torchrun_reports_on_rank0_only():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "2", "--warmup", "3", "--ref-budget", "2"]
    p = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [l for l in p.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle"
