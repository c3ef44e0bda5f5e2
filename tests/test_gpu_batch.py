"""Batched grids in one persistent launch: every grid bit-exact against the CPU
oracle and against the single-grid path; graph and direct launch agree; a
missing producer ends in a bounded-wait timeout reported to the host."""
import numpy as np
import pytest

import oracle
from paper_0912_4506_gb300 import inputs
from tests.helpers import make_grid, to_dev, to_host

pytestmark = pytest.mark.gpu

SPECS = [((40, 32, 48), 13, 4), ((33, 70, 9), 7, 3), ((64, 64, 64), 20, 6),
         ((8, 8, 8), 5, 2), ((100, 30, 25), 11, 5), ((57, 41, 36), 1, 4),
         ((72, 96, 40), 0, 4), ((130, 20, 12), 9, 1), ((48, 48, 100), 16, 6)]


def _make(dtype, specs, g0=0):
    from paper_0912_4506_gb300 import api
    hosts, grids = [], []
    for i, ((nx, ny, nz), n, t) in enumerate(specs):
        a = make_grid(nx, ny, nz, dtype, g=g0 + i)
        hosts.append(a)
        grids.append(api.as_grid(to_dev(a, dtype), nx))
    return hosts, grids


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
@pytest.mark.parametrize("graph,wide", [(True, None), (False, None), (True, 64)])
def test_batch_bit_exact_vs_oracle(dtype, graph, wide):
    """Default widths (128-wide tiles for depths 1-2, 64 otherwise) and all grids
    on 64-wide tiles."""
    from paper_0912_4506_gb300 import api
    hosts, grids = _make(dtype, SPECS)
    tx = None if wide is None else [wide] * len(SPECS)
    b = api.Batch(grids, [s[1] for s in SPECS], t=[s[2] for s in SPECS], graph=graph,
                  tile_x=tx)
    outs = b.run()
    b.check()
    info = b.info()
    want_tx = [(128 if max(1, min(s[2], max(1, s[1]))) <= 2 else 64) if wide is None else wide
               for s in SPECS]
    assert info["tile_x"] == want_tx
    for (shape, n, t), a, out, tu in zip(SPECS, hosts, outs, info["t"]):
        nx = shape[0]
        want = oracle.sweeps(a, n, nx=nx, dtype=dtype)[:, :, :nx + 2]
        assert np.array_equal(to_host(out, dtype), want), (shape, n, t, tu)
    b.close()


def test_batch_matches_single_grid_path():
    from paper_0912_4506_gb300 import api
    hosts, grids = _make("f32", SPECS, g0=20)
    b = api.Batch(grids, [s[1] for s in SPECS], t=[s[2] for s in SPECS])
    outs = [to_host(o, "f32") for o in b.run()]
    b.close()
    for (shape, n, t), a, got in zip(SPECS, hosts, outs):
        nx = shape[0]
        j = api.Jacobi(api.as_grid(to_dev(a, "f32"), nx))
        want = to_host(j.sweep(n, t), "f32")
        j.close()
        assert np.array_equal(got, want), shape


def test_missing_producer_times_out_and_context_survives():
    """A work item waits for a tile that no item produces: the bounded wait runs
    out, the status reaches the host as a timeout, the real grids are still
    right, and the context keeps working."""
    from paper_0912_4506_gb300 import api, _lib
    specs = SPECS[:4]
    hosts, grids = _make("f32", specs)
    b = api.Batch(grids, [s[1] for s in specs], t=[s[2] for s in specs],
                  test_missing_producer=True, wait_limit_s=0.05)
    outs = b.run()
    with pytest.raises(_lib.JacobiError) as ei:
        b.check()
    assert ei.value.code == _lib.JAC_ETIMEOUT
    for (shape, n, t), a, out in zip(specs, hosts, outs):
        nx = shape[0]
        assert np.array_equal(to_host(out, "f32"),
                              oracle.sweeps(a, n, nx=nx, dtype="f32")[:, :, :nx + 2])
    b.close()
    # the device is still usable
    a = make_grid(20, 20, 20, "f64")
    j = api.Jacobi(api.as_grid(to_dev(a, "f64"), 20))
    assert np.array_equal(to_host(j.sweep(3, 2, api.JAC_KERNEL_TB), "f64"),
                          oracle.sweeps(a, 3)[:, :, :22])
    j.close()


def test_batch_workload_64_grids_vs_single_path():
    """The 64-grid FP32 workload (shapes multiples of 8 in [32, 256], sweep counts in
    [10, 200], seed 2): every grid equal to the single-grid path, the three smallest
    also against the oracle."""
    import torch
    from paper_0912_4506_gb300 import api
    specs = inputs.batch_specs()
    grids, hosts = [], []
    for i, (nx, ny, nz, n) in enumerate(specs):
        a = make_grid(nx, ny, nz, "f32", g=i)
        hosts.append(a)
        grids.append(api.as_grid(to_dev(a, "f32"), nx))
    b = api.Batch(grids, [s[3] for s in specs], t=[4] * len(specs))
    outs = b.run()
    b.check()
    order = sorted(range(len(specs)), key=lambda i: np.prod(specs[i][:3]))
    for i in range(len(specs)):
        nx, ny, nz, n = specs[i]
        got = to_host(outs[i], "f32")
        j = api.Jacobi(api.as_grid(to_dev(hosts[i], "f32"), nx))
        want = to_host(j.sweep(n, 4), "f32")
        j.close()
        assert np.array_equal(got, want), specs[i]
        if i in order[:3]:
            assert np.array_equal(got, oracle.sweeps(hosts[i], n, nx=nx, dtype="f32")
                                  [:, :, :nx + 2]), specs[i]
    b.close()
    torch.cuda.empty_cache()


def test_autotuner_picks_a_candidate(tmp_path, monkeypatch):
    from paper_0912_4506_gb300 import autotune
    monkeypatch.setenv("JACOBI_GB300_CACHE", str(tmp_path))
    cands = ((128, 2), (64, 4))
    best, table = autotune.tune([(64, 48, 40), (32, 32, 32)], candidates=cands, sweeps=8)
    assert all(tuple(c) in cands for c in best)
    again, _ = autotune.tune([(64, 48, 40)], candidates=cands, sweeps=8)
    assert again[0] == best[0]  # served from the cache


def test_wide_tiles_deeper_than_built_rejected():
    from paper_0912_4506_gb300 import _lib, api
    hosts, grids = _make("f32", SPECS[:2])
    with pytest.raises(_lib.JacobiError) as ei:
        api.Batch(grids, [10, 10], t=[3, 2], tile_x=[128, 128])
    assert ei.value.code == _lib.JAC_EUNSUPPORTED
    with pytest.raises(_lib.JacobiError) as ei:
        api.Batch(grids, [10, 10], t=[7, 2])
    assert ei.value.code == _lib.JAC_EUNSUPPORTED
