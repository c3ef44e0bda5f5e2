"""z-slab decomposition with multi-layer halos (Sect. 2.1): the slabs' sweeps,
exchanging h halo planes every h sweeps, give the single-grid result bit for
bit."""
import numpy as np
import pytest

import oracle
from tests.helpers import make_grid, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype,shape,nslabs,h,t,n", [
    ("f64", (40, 33, 60), 3, 2, 2, 9),
    ("f64", (40, 33, 60), 4, 4, 4, 13),
    ("f32", (70, 40, 64), 2, 4, 3, 11),
    ("f32", (70, 40, 64), 5, 6, 6, 25),
    ("bf16", (50, 37, 48), 3, 4, 4, 10),
    ("f32", (64, 64, 64), 8, 4, 4, 16),
    ("f64", (33, 21, 30), 1, 3, 3, 7),
])
def test_slabs_equal_single_grid(dtype, shape, nslabs, h, t, n):
    from paper_0912_4506_gb300 import api, slabs
    nx, ny, nz = shape
    a = make_grid(nx, ny, nz, dtype)
    A = api.as_grid(to_dev(a, dtype), nx)
    sj = slabs.SlabJacobi(A, nslabs, h)
    sj.sweep(n, t)
    got = to_host(sj.gather(), dtype)
    sj.close()
    want = oracle.sweeps(a, n, nx=nx, dtype=dtype)[:, :, :nx + 2]
    assert np.array_equal(got, want)


def test_slab_plan_rejects_thin_cores():
    from paper_0912_4506_gb300 import slabs
    with pytest.raises(ValueError):
        slabs.halo_plan(10, 4, 3)


@pytest.mark.parametrize("dtype,shape,ranks,h,t,n", [
    ("f64", (40, 33, 60), 3, 1, 1, 9),
    ("f64", (40, 33, 60), 2, 3, 2, 11),
    ("f32", (70, 40, 64), 4, 4, 3, 13),
    ("bf16", (50, 37, 48), 3, 2, 2, 7),
])
def test_rank_slabs_on_one_gpu_equal_single_grid(dtype, shape, ranks, h, t, n):
    """The per-rank slab class with its library sweeps, every rank's slab drawn
    from its own planes; the messages of a multi-GPU run replaced by in-process
    copies of the same planes (exchange_in_process)."""
    import torch
    from paper_0912_4506_gb300 import inputs, slabs
    nx, ny, nz = shape
    px = inputs.row_pitch(nx, dtype)
    parts = []
    for r in range(ranks):
        z0, z1 = slabs.slab_ranges(nz, ranks)[r]
        lo, hi = slabs.slab_extent(z0, z1, nz, h)
        a = inputs.to_dtype(inputs.uniform_grid_f64(nx, ny, nz, planes=(lo, hi)), dtype, px=px)
        parts.append(slabs.RankSlab(nx, ny, nz, h, to_dev(a, dtype), r, ranks))
    for d in parts[0].passes(n, t):
        slabs.exchange_in_process(parts)
        for p in parts:
            p.local_pass(d)
    torch.cuda.synchronize()
    got = np.concatenate([to_host(p.core(), dtype) for p in parts])[:, :, :nx + 2]
    for p in parts:
        p.close()
    a = make_grid(nx, ny, nz, dtype)
    want = oracle.sweeps(a, n, nx=nx, dtype=dtype)[:, :, :nx + 2]
    assert np.array_equal(got, want)
