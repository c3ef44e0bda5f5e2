"""Every compiled shape of the temporally-blocked kernel (warps per CTA, rows per
thread, CTAs per SM) gives the oracle's bits.  The planner serves each depth with
one shape, so the shapes it does not pick by default are reached through
JACOBI_TB_SHAPE in a fresh process (the choice is read once per process)."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CODE = r"""
import sys; sys.path.insert(0, %(root)r)
import numpy as np, torch, oracle
from paper_0912_4506_gb300 import api, inputs
from tests.helpers import make_grid, to_dev, to_host

want_threads = %(threads)r
for dtype in ("f32", "bf16"):
    for (nx, ny, nz) in ((130, 47, 9), (37, 29, 23), (67, 70, 31)):
        a = make_grid(nx, ny, nz, dtype)
        n = 13
        want = oracle.sweeps(a, n, nx=nx, dtype=dtype)[:, :, :nx + 2]
        for t in (1, 2, 3, 4):
            j = api.Jacobi(api.as_grid(to_dev(a, dtype), nx))
            if t in want_threads:
                assert j.plan(n, t, api.JAC_KERNEL_TB)["threads"] == want_threads[t], t
            got = to_host(j.sweep(n, t, api.JAC_KERNEL_TB), dtype)
            j.check(); j.close()
            assert np.array_equal(got, want), (dtype, nx, t)
        # correction sweeps (zero boundary, right-hand side rho)
        rng = np.random.default_rng(5)
        px = inputs.row_pitch(nx, dtype)
        e = np.zeros((nz + 2, ny + 2, px)); e[1:-1, 1:-1, 1:nx + 1] = rng.random((nz, ny, nx))
        r = np.zeros_like(e); r[1:-1, 1:-1, 1:nx + 1] = 0.1 * rng.random((nz, ny, nx))
        e = inputs.to_dtype(e, dtype, px=px); r = inputs.to_dtype(r, dtype, px=px)
        want = oracle.rhs_sweeps(e, r, n, nx=nx, dtype=dtype)[:, :, :nx + 2]
        for t in (2, 3, 4):
            j = api.Jacobi(api.as_grid(to_dev(e, dtype), nx))
            got = to_host(j.sweep_rhs(api.as_grid(to_dev(r, dtype), nx), n, t), dtype)
            j.check(); j.close()
            assert np.array_equal(got, want), ("rhs", dtype, nx, t)
# adjoint sweeps (FP32): the same bits at every depth, sweep result and gradient
nx, ny, nz, n = 67, 70, 31, 11
W = inputs.to_dtype(inputs.normal_grid_f64(nx, ny, nz), "f32", px=inputs.row_pitch(nx, "f32"))
res = {}
for t in (1, 2, 3, 4):
    lam = api.as_grid(to_dev(W, "f32"), nx)
    lam[0] = 0; lam[-1] = 0; lam[:, 0] = 0; lam[:, -1] = 0; lam[:, :, 0] = 0; lam[:, :, nx + 1] = 0
    gb = api.alloc_like(lam)
    gb.zero_()
    j = api.Jacobi(lam)
    out = j.adjoint(gb, n, t)
    j.check()
    res[t] = (to_host(out, "f32"), to_host(gb, "f32"))
    j.close()
for t in (2, 3, 4):
    assert np.array_equal(res[t][0], res[1][0]) and np.array_equal(res[t][1], res[1][1]), t
print("ok")
"""

# (JACOBI_TB_SHAPE, {depth: threads per CTA the planner must report})
SHAPES = [
    (None, {2: 512, 3: 512, 4: 1024}),     # defaults: two rows per thread at 2 and 3
    ("32,1,1", {2: 1024, 3: 1024, 4: 1024}),  # one row per thread everywhere
    ("16,2,1", {2: 512}),
    ("16,2,2", {3: 512}),
]


@pytest.mark.parametrize("shape,threads", SHAPES, ids=lambda v: str(v))
def test_every_tb_shape_bit_exact(shape, threads):
    env = dict(os.environ)
    env.pop("JACOBI_TB_SHAPE", None)
    if shape:
        env["JACOBI_TB_SHAPE"] = shape
    r = subprocess.run([sys.executable, "-c", CODE % {"root": ROOT, "threads": threads}],
                       env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and "ok" in r.stdout, r.stderr[-3000:]
