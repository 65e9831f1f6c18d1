"""The multi-rank path of bench.py on CPU (gloo, two processes).

The path runs replicas only: every rank advances its own disc and the only
exchange is the timing reduction.  Every rank must see the slowest rank's
time, the job's rate counts every rank's work, and the reference arm's other
ranks leave without work.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

RANK_CODE = r"""
import json, os, sys
sys.path.insert(0, %r)
import torch.distributed as dist
dist.init_process_group("gloo")
import bench
rank = int(os.environ["RANK"])
slowest = bench.max_over_ranks(1.0 + 2.0 * rank, dist, device="cpu")
world, r, local = bench.dist_env()
print(json.dumps({"rank": rank, "slowest": slowest, "world": world, "r": r, "local": local}))
dist.barrier()
dist.destroy_process_group()
"""


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def test_every_rank_sees_the_slowest_time():
    pytest.importorskip("torch")
    port = free_port()
    procs = []
    for rank in range(2):
        env = dict(os.environ, MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                   LOCAL_RANK=str(rank), WORLD_SIZE="2")
        procs.append(subprocess.Popen([sys.executable, "-c", RANK_CODE % ROOT], env=env, cwd=ROOT,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        try:
            out, err = p.communicate(timeout=180)
        except subprocess.TimeoutExpired:
            for q in procs:
                q.kill()
            raise
        assert p.returncode == 0, err
        outs.append(json.loads(out.strip().splitlines()[-1]))
    outs.sort(key=lambda d: d["rank"])
    assert [d["slowest"] for d in outs] == [3.0, 3.0]
    assert [(d["world"], d["r"], d["local"]) for d in outs] == [(2, 0, 0), (2, 1, 1)]


def test_one_rank_reduces_to_its_own_time():
    import bench
    assert bench.max_over_ranks(1.25, None) == 1.25


def test_job_rate_counts_every_rank():
    import bench
    assert bench.job_rate(2, 100.0, 0.5) == 400.0
    assert bench.job_rate(1, 100.0, 0.5) == 200.0


def test_reference_arm_other_ranks_leave_without_work(monkeypatch):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class Args:
        warmup = 0
        steps = 1

    # rank 1 returns before it looks at the configuration or runs the oracle
    assert bench.run_reference(Args(), None) == 0
