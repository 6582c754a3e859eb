"""The bench's N>1 replica path on CPU: two gloo ranks (127.0.0.1), the
max-over-ranks timing and the whole-job rate, and the reference arm's
rank > 0 exit without work."""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r'''
import os, sys, json
sys.path.insert(0, sys.argv[1])
import torch.distributed as dist
import bench
dist.init_process_group("gloo")
ws, rank, local = bench.dist_info()
dist.barrier()
t = bench.max_over_ranks(1.5 + rank, ws, "cpu")      # rank 1 is the slowest
v = bench.whole_job_rate(1000.0, ws, t)
print(json.dumps({"rank": rank, "ws": ws, "max": t, "rate": v}), flush=True)
dist.barrier()
dist.destroy_process_group()
'''


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_two_gloo_ranks_max_and_rate(tmp_path):
    pytest.importorskip("torch.distributed")
    w = tmp_path / "worker.py"
    w.write_text(WORKER)
    port = free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, WORLD_SIZE="2", RANK=str(r), LOCAL_RANK=str(r), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, str(w), ROOT], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = [p.communicate(timeout=120) for p in procs]
    for p, (o, e) in zip(procs, outs):
        assert p.returncode == 0, e
    import json
    res = [json.loads(o.strip().splitlines()[-1]) for o, _ in outs]
    for r in res:
        assert r["ws"] == 2
        assert r["max"] == 2.5  # every rank reports the slowest rank's time
        assert abs(r["rate"] - 2 * 1000.0 / 2.5) < 1e-9  # units of both ranks over the slowest time


def test_reference_arm_other_ranks_exit_without_work():
    sys.path.insert(0, ROOT)
    import bench

    class A:
        steps, warmup = 1, 1

    assert bench.run_reference(A(), 2, 1) == 0  # returns before building or running the oracle
