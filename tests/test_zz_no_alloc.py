"""jacobi_sweep_noalloc: the sweep for callers that cannot allocate device memory
(code that runs where cudaMalloc is not allowed or not wanted, e.g. a host
framework that owns all device memory through its own pool, or a plug-in that
must not grow the process's device footprint).  Called through the C ABI, it
must give the same grid as the handle-based jacobi_sweep (the library's sweeps
are bit-exact, so the tolerance is zero), on two calls in a row that share the
library's static scratch array, and a call after the first one on the device
must leave the free device memory unchanged.  This file is collected last on
purpose: it must pass alone in a fresh process and after every other test."""
import ctypes

import numpy as np
import pytest

from tests.helpers import make_grid, to_dev, to_host

pytestmark = pytest.mark.gpu


def _via_handle(a, nx, dtype, n, t):
    from paper_0912_4506_gb300 import api
    j = api.Jacobi(api.as_grid(to_dev(a, dtype), nx))
    out = to_host(j.sweep(n, t), dtype)
    j.check()
    j.close()
    return out


def _via_noalloc(a, nx, dtype, n, t):
    import torch
    from paper_0912_4506_gb300 import _lib
    full = to_dev(a, dtype)
    nz2, ny2, px = full.shape
    code = {"f64": _lib.JAC_F64, "f32": _lib.JAC_F32, "bf16": _lib.JAC_BF16}[dtype]
    stream = torch.cuda.current_stream().cuda_stream
    _lib.jacobi_sweep_noalloc(nx, ny2 - 2, nz2 - 2, code, full.data_ptr(), px, n, t, stream, 1)
    pad_before = a[:, :, nx + 2:]
    host = to_host(full, dtype)
    assert np.array_equal(host[:, :, nx + 2:].view(np.uint8), pad_before.view(np.uint8))
    return host[:, :, :nx + 2]


@pytest.mark.parametrize("dtype,shape,n,t", [
    ("f64", (64, 64, 64), 100, 0),
    ("f64", (37, 29, 23), 13, 3),
    ("f32", (61, 50, 40), 17, 4),
    ("f32", (61, 50, 40), 5, 1),
    ("bf16", (70, 33, 20), 9, 8),
])
def test_noalloc_matches_handle_sweep_twice(dtype, shape, n, t):
    nx, ny, nz = shape
    for g in (0, 1):  # two calls in a row on different inputs share the scratch
        a = make_grid(nx, ny, nz, dtype, g=g)
        got = _via_noalloc(a, nx, dtype, n, t)
        want = _via_handle(a, nx, dtype, n, t)
        assert np.array_equal(got, want), (dtype, shape, n, t, g)


def test_noalloc_rejects_grid_larger_than_scratch():
    import torch
    from paper_0912_4506_gb300 import _lib
    small = torch.zeros(16, dtype=torch.float64, device="cuda")
    lib = _lib.load()
    # 256^3 FP64 needs ~136 MB: beyond the 32 MiB scratch, rejected before any launch
    rc = lib.jacobi_sweep_noalloc(256, 256, 256, _lib.JAC_F64,
                                  ctypes.c_void_p(small.data_ptr()), 258, 1, 0, None, 1)
    assert rc == _lib.JAC_EINVAL
    assert b"invalid" in lib.jacobi_strerror(rc)


@pytest.mark.parametrize("dtype,t", [("f64", 0), ("f64", 4), ("f32", 3), ("bf16", 2)])
def test_noalloc_call_reserves_no_device_memory(dtype, t):
    """After a first call of the same kind (which loads the kernels and commits the
    scratch array), a further call leaves the device's free memory unchanged."""
    import torch
    nx, ny, nz = 48, 40, 30
    a = make_grid(nx, ny, nz, dtype)
    _via_noalloc(a, nx, dtype, 7, t)  # first call: kernels and scratch array loaded
    full = to_dev(a, dtype)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    from paper_0912_4506_gb300 import _lib
    code = {"f64": _lib.JAC_F64, "f32": _lib.JAC_F32, "bf16": _lib.JAC_BF16}[dtype]
    _lib.jacobi_sweep_noalloc(nx, ny, nz, code, full.data_ptr(), full.shape[2], 7, t,
                              torch.cuda.current_stream().cuda_stream, 1)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
