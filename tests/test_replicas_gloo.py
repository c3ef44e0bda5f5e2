"""The N > 1 (replicas) path of bench.py on CPU ranks with the gloo backend: the
job time is the slowest rank's, the value counts every rank's updates, and the
reference arm runs on rank 0 only."""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


_WORKER = r"""
import os, sys, json
sys.path.insert(0, {root!r})
import torch.distributed as dist
dist.init_process_group("gloo", init_method="env://")
import bench
r = dist.get_rank()
ms, glups = bench.replica_throughput(10.0 + 5.0 * r, 2e9, "cpu")
print(json.dumps({{"rank": r, "ms": ms, "glups": glups}}))
dist.destroy_process_group()
"""


def _launch(code, world=2):
    port = _free_port()
    procs = []
    for r in range(world):
        env = dict(os.environ, RANK=str(r), LOCAL_RANK=str(r), WORLD_SIZE=str(world),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", code], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE,
                                      text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=120)
        assert p.returncode == 0, err[-2000:]
        outs.append(out)
    return outs


def test_replica_throughput_max_over_ranks_gloo():
    import json
    outs = _launch(_WORKER.format(root=ROOT))
    res = [json.loads(o.strip().splitlines()[-1]) for o in outs]
    for r in res:
        assert r["ms"] == 15.0  # the slowest rank's time on every rank
        assert abs(r["glups"] - 2 * 2e9 / 0.015 / 1e9) < 1e-9


def test_single_process_throughput():
    sys.path.insert(0, ROOT)
    import bench
    ms, glups = bench.replica_throughput(20.0, 1e9)
    assert ms == 20.0 and abs(glups - 50.0) < 1e-12


def test_reference_arm_runs_on_rank0_only():
    """Rank 1 of the reference arm exits 0 without work or output."""
    env = dict(os.environ, RANK="1", LOCAL_RANK="1", WORLD_SIZE="2")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--gpus", "2", "--steps", "1", "--warmup", "0"], env=env,
                       capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""
