"""Blocked sweeps of every kind give the same bits at every depth: correction
sweeps (right-hand side staged through its own TMA ring) against the oracle at
the deepest compiled depths, and adjoint sweeps (sweep result and accumulated
boundary gradient) against the depth-1 run."""
import numpy as np
import pytest

import oracle
from paper_0912_4506_gb300 import inputs
from tests.helpers import make_grid, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
@pytest.mark.parametrize("shape", [(130, 47, 9), (67, 70, 31)], ids=lambda s: "x".join(map(str, s)))
def test_rhs_every_depth_matches_oracle(dtype, shape):
    from paper_0912_4506_gb300 import api
    nx, ny, nz = shape
    rng = np.random.default_rng(5)
    px = inputs.row_pitch(nx, dtype)
    e = np.zeros((nz + 2, ny + 2, px))
    e[1:-1, 1:-1, 1:nx + 1] = rng.random((nz, ny, nx))
    r = np.zeros_like(e)
    r[1:-1, 1:-1, 1:nx + 1] = 0.1 * rng.random((nz, ny, nx))
    e = inputs.to_dtype(e, dtype, px=px)
    r = inputs.to_dtype(r, dtype, px=px)
    n = 17  # remainders at every depth
    want = oracle.rhs_sweeps(e, r, n, nx=nx, dtype=dtype)[:, :, :nx + 2]
    for t in (1, 2, 3, 4, 5, 6):
        j = api.Jacobi(api.as_grid(to_dev(e, dtype), nx))
        got = to_host(j.sweep_rhs(api.as_grid(to_dev(r, dtype), nx), n, t), dtype)
        j.check()
        j.close()
        assert np.array_equal(got, want), t


@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("shape", [(67, 70, 31), (9, 40, 2), (3, 2, 19)],
                         ids=lambda s: "x".join(map(str, s)))
def test_adjoint_same_bits_every_depth(dtype, shape):
    """Adjoint sweeps at every depth give the bits of depth 1, the swept lambda and
    the boundary gradient (face bands thicker than the grid included)."""
    import torch
    from paper_0912_4506_gb300 import api
    nx, ny, nz = shape
    n = 11
    W = inputs.to_dtype(inputs.normal_grid_f64(nx, ny, nz), dtype, px=inputs.row_pitch(nx, dtype))
    res = {}
    for t in range(1, 9):
        lam = api.as_grid(to_dev(W, dtype), nx)
        lam[0] = 0
        lam[-1] = 0
        lam[:, 0] = 0
        lam[:, -1] = 0
        lam[:, :, 0] = 0
        lam[:, :, nx + 1] = 0
        gb = api.alloc_like(lam)
        j = api.Jacobi(lam)
        out = j.adjoint(gb, n, t)
        j.check()
        torch.cuda.synchronize()
        res[t] = (to_host(out, dtype), to_host(gb, dtype))
        j.close()
    for t in range(2, 9):
        assert np.array_equal(res[t][0], res[1][0]), t
        assert np.array_equal(res[t][1], res[1][1]), t


def test_plan_reports_default_depth():
    from paper_0912_4506_gb300 import api
    a = make_grid(96, 40, 30, "f32")
    j = api.Jacobi(api.as_grid(to_dev(a, "f32"), 96))
    p = j.plan(13, 0, api.JAC_KERNEL_AUTO)
    j.close()
    assert p["t"] == 3 and p["remainder_t"] == 1 and p["passes"] == 5
    assert p["threads"] == 32 * p["ext_y"]
