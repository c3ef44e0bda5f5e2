"""The multi-rank form of the z-slab decomposition on CPU ranks (gloo): each
rank owns one slab, exchanges its h+1 halo planes with its neighbours by
send/recv every h sweeps, sweeps its slab with the CPU oracle, and rank 0
assembles the cores; the result equals the oracle's single-grid sweep."""
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_WORKER = r"""
import sys, json
sys.path.insert(0, {root!r})
import numpy as np, torch, torch.distributed as dist
import oracle
from paper_0912_4506_gb300 import inputs, slabs
dist.init_process_group("gloo", init_method="env://")
r, P = dist.get_rank(), dist.get_world_size()
nx, ny, nz, h, n = 12, 9, {nz}, {h}, {n}
a = inputs.uniform_grid_f64(nx, ny, nz)          # every rank draws the same grid
z0, z1 = slabs.slab_ranges(nz, P)[r]
lo, hi = slabs.slab_extent(z0, z1, nz, h)
mine = a[lo:hi + 1].copy()
plan = slabs.halo_plan(nz, P, h)
done = 0
while done < n:
    d = min(h, n - done)
    reqs = []
    for dst, gp, src, k in plan:                  # post sends of my core planes
        if src == r:
            buf = torch.from_numpy(np.ascontiguousarray(mine[gp - lo:gp - lo + k]))
            reqs.append(dist.isend(buf, dst))
    for dst, gp, src, k in plan:                  # receive my halo planes
        if dst == r:
            buf = torch.empty((k, ny + 2, nx + 2), dtype=torch.float64)
            dist.recv(buf, src)
            mine[gp - lo:gp - lo + k] = buf.numpy()
    for q in reqs:
        q.wait()
    mine = oracle.sweeps(mine, d, nx=nx)
    done += d
core = mine[(z0 if r > 0 else 0) - lo:(z1 if r < P - 1 else nz + 1) - lo + 1]
parts = [None] * P
dist.all_gather_object(parts, (r, core.tolist()))
if r == 0:
    full = np.concatenate([np.array(c) for _, c in sorted(parts, key=lambda x: x[0])])
    print(json.dumps({{"equal": bool(np.array_equal(full, oracle.sweeps(a, n, nx=nx)))}}))
dist.destroy_process_group()
"""


def _port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _run(world, nz, h, n):
    import json
    port = _port()
    code = _WORKER.format(root=ROOT, nz=nz, h=h, n=n)
    procs = []
    for r in range(world):
        env = dict(os.environ, RANK=str(r), WORLD_SIZE=str(world), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", code], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=180)
        assert p.returncode == 0, err[-3000:]
        outs.append(out)
    return json.loads(outs[0].strip().splitlines()[-1])


def test_two_ranks_multi_layer_halo():
    assert _run(2, 16, 3, 10)["equal"]


def test_three_ranks_deep_halo():
    assert _run(3, 24, 5, 12)["equal"]
