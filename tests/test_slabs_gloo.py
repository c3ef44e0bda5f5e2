"""The multi-rank z-slab decomposition (slabs.RankSlab, the class a multi-GPU run
uses) on CPU ranks over gloo: each rank draws its own planes, exchanges its h+1
halo planes with its neighbours by send/recv before every pass, sweeps its slab
with the CPU oracle in place of the library, and rank 0 assembles the cores; the
result equals the oracle's single-grid sweep."""
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
z0, z1 = slabs.slab_ranges(nz, P)[r]
lo, hi = slabs.slab_extent(z0, z1, nz, h)
# each rank draws only its own planes (the counter-based generator gives the
# values the single grid has there)
mine = torch.from_numpy(inputs.uniform_grid_f64(nx, ny, nz, planes=(lo, hi)))
sweeper = lambda t, d: torch.from_numpy(oracle.sweeps(t.numpy(), d, nx=nx))
rs = slabs.RankSlab(nx, ny, nz, h, mine, r, P, sweeper=sweeper)
rs.sweep(n, {t})
parts = [None] * P
dist.all_gather_object(parts, (r, rs.core().numpy().tolist()))
if r == 0:
    full = np.concatenate([np.array(c) for _, c in sorted(parts, key=lambda x: x[0])])
    a = inputs.uniform_grid_f64(nx, ny, nz)
    print(json.dumps({{"equal": bool(np.array_equal(full, oracle.sweeps(a, n, nx=nx)))}}))
dist.destroy_process_group()
"""


def _port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _run(world, nz, h, n, t=None):
    import json
    port = _port()
    code = _WORKER.format(root=ROOT, nz=nz, h=h, n=n, t=t)
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


def test_four_ranks_shallower_passes_than_halo():
    # passes of depth 2 with 4-plane halos: the exchange still happens every pass
    assert _run(4, 32, 4, 9, t=2)["equal"]


def test_single_rank_is_the_plain_sweep():
    assert _run(1, 10, 3, 7)["equal"]
