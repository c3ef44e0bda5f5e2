"""GPU parity of the mixed-precision refinement pieces against the CPU oracle:
correction sweeps (FP32 and bf16 storage, every depth), the FP64 residual step,
and the whole refinement driver (all bit-exact: same operations, same order)."""
import numpy as np
import pytest

import oracle
from paper_0912_4506_gb300 import inputs
from tests.helpers import NP_DT, to_dev, to_host

pytestmark = pytest.mark.gpu


def _rand_interior(nx, ny, nz, dtype, seed, scale=1.0):
    rng = np.random.default_rng(seed)
    px = inputs.row_pitch(nx, dtype)
    a = np.zeros((nz + 2, ny + 2, px), dtype=np.float64)
    a[1:-1, 1:-1, 1:nx + 1] = (rng.random((nz, ny, nx)) - 0.5) * scale
    return inputs.to_dtype(a, dtype, px=px)


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
@pytest.mark.parametrize("shape", [(45, 38, 17), (64, 64, 64), (3, 70, 5)],
                         ids=lambda s: "x".join(map(str, s)))
def test_rhs_sweeps_bit_exact(dtype, shape):
    from paper_0912_4506_gb300 import api
    nx, ny, nz = shape
    e = _rand_interior(nx, ny, nz, dtype, 1)
    rho = _rand_interior(nx, ny, nz, dtype, 2, scale=0.1)
    for n in (1, 7, 13):
        want = oracle.rhs_sweeps(e, rho, n, nx=nx, dtype=dtype)[:, :, :nx + 2]
        for t in (1, 2, 3, 4, 5, 6):
            j = api.Jacobi(api.as_grid(to_dev(e, dtype), nx))
            out = j.sweep_rhs(api.as_grid(to_dev(rho, dtype), nx), n, t)
            j.check()
            got = to_host(out, dtype)
            j.close()
            assert np.array_equal(got, want), (n, t)
    # deeper than the deepest correction-sweep kernel: rejected, nothing launched
    from paper_0912_4506_gb300 import _lib
    j = api.Jacobi(api.as_grid(to_dev(e, dtype), nx))
    with pytest.raises(_lib.JacobiError) as ei:
        j.sweep_rhs(api.as_grid(to_dev(rho, dtype), nx), 13, 8)
    assert ei.value.code == _lib.JAC_EUNSUPPORTED
    j.close()


def _special_interior(nx, ny, nz, dtype, seed):
    """Corrections mixing zeros of both signs, subnormal and huge values with
    ordinary ones (the widening of e to FP64 has separate paths for them)."""
    rng = np.random.default_rng(seed)
    px = inputs.row_pitch(nx, dtype)
    vals = np.array([0.0, -0.0, 1e-40, -3e-42, 2.0 ** -149, 1e30, -1e30, 0.5, -0.25,
                     1.2e-38, 3.0e38], dtype=np.float64)
    a = np.zeros((nz + 2, ny + 2, px), dtype=np.float64)
    pick = rng.integers(0, 3 * len(vals), (nz, ny, nx))
    reg = (rng.random((nz, ny, nx)) - 0.5) * 1e-3
    a[1:-1, 1:-1, 1:nx + 1] = np.where(pick < len(vals), vals[np.minimum(pick, len(vals) - 1)],
                                       reg)
    return inputs.to_dtype(a, dtype, px=px)


def _rounding_grid(nx, ny, nz):
    """FP64 grid whose interior exercises the exact-rounding paths of the residual
    step, in z-slabs so that neighbours share a kind: values on a 2^-24 lattice
    (their residuals hit binary32 rounding ties), tiny values (residuals in the
    binary32 subnormal range), x*6 with 1 or 2 dropped bits and exact ties
    (m = 2^52 + j and 1.5 * 2^52 + j, both signs, exponents -40..40), and large
    values (residuals near and above the largest binary32)."""
    rng = np.random.default_rng(11)
    px = inputs.row_pitch(nx, "f64")
    a = np.zeros((nz + 2, ny + 2, px), dtype=np.float64)
    shape = (ny, nx)
    for k in range(1, nz + 1):
        kind = (k - 1) * 4 // nz
        j = rng.integers(1, 4096, shape).astype(np.float64)
        if kind == 0:
            v = rng.integers(-8, 9, shape) + j * 2.0 ** -24
        elif kind == 1:
            v = (rng.random(shape) - 0.5) * 1e-39
        elif kind == 2:
            base = np.where(rng.random(shape) < 0.5, 1.0, 1.5)
            sign = np.where(rng.random(shape) < 0.5, -1.0, 1.0)
            e = rng.integers(-40, 41, shape).astype(np.float64)
            v = sign * (base + j * 2.0 ** -52) * 2.0 ** e
        else:
            v = (rng.random(shape) - 0.5) * 1.2e38
        a[k, 1:-1, 1:nx + 1] = v
    return a


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_residual_rounding_edge_cases(dtype):
    from paper_0912_4506_gb300 import api
    nx, ny, nz = 61, 33, 24
    u = _rounding_grid(nx, ny, nz)
    px = inputs.row_pitch(nx, dtype)
    e = inputs.to_dtype(np.zeros((nz + 2, ny + 2, px)), dtype, px=px)
    e_same = np.zeros(u.shape, dtype=e.dtype)
    w = min(u.shape[2], e.shape[2])
    e_same[:, :, :w] = e[:, :, :w]
    want_u, want_rho = oracle.residual_accumulate(u, e_same, nx=nx, dtype=dtype)
    ug = api.as_grid(to_dev(u, "f64"), nx)
    uo = api.alloc_like(ug)
    uo.copy_(ug)
    eg = api.as_grid(to_dev(e, dtype), nx)
    rho = api.alloc_like(eg)
    api.residual_accumulate(ug, uo, eg, rho)
    got_u = to_host(uo, "f64")
    got_rho = to_host(rho, dtype)
    assert np.array_equal(got_u, want_u[:, :, :nx + 2])
    assert np.array_equal(got_rho[1:-1, 1:-1, 1:-1], want_rho[1:-1, 1:-1, 1:nx + 1])


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
@pytest.mark.parametrize("case", ["random", "special", "ragged"])
def test_residual_accumulate_bit_exact(dtype, case):
    from paper_0912_4506_gb300 import api
    nx, ny, nz = (97, 50, 33) if case == "ragged" else (53, 41, 19)
    u = inputs.uniform_grid_f64(nx, ny, nz, px=inputs.row_pitch(nx, "f64")) * 100.0 - 50.0
    if case == "special":
        e = _special_interior(nx, ny, nz, dtype, 4)
    else:
        e = _rand_interior(nx, ny, nz, dtype, 3, scale=1e-3)
    e_same = np.zeros(u.shape, dtype=e.dtype)  # the oracle takes one row pitch for both
    w = min(u.shape[2], e.shape[2])
    e_same[:, :, :w] = e[:, :, :w]
    want_u, want_rho = oracle.residual_accumulate(u, e_same, nx=nx, dtype=dtype)
    ug = api.as_grid(to_dev(u, "f64"), nx)
    uo = api.alloc_like(ug)
    uo.copy_(ug)
    eg = api.as_grid(to_dev(e, dtype), nx)
    rho = api.alloc_like(eg)
    api.residual_accumulate(ug, uo, eg, rho)
    got_u = to_host(uo, "f64")
    got_rho = to_host(rho, dtype)
    assert np.array_equal(got_u, want_u[:, :, :nx + 2])
    assert np.array_equal(got_rho[1:-1, 1:-1, 1:-1], want_rho[1:-1, 1:-1, 1:nx + 1])


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_refine_solve_bit_exact(dtype):
    """Laplace problem (boundary u = x^2 - y^2 + 0.5 z, zero interior): 3 outer
    steps of 7 correction sweeps, GPU vs oracle, bit for bit."""
    from paper_0912_4506_gb300 import api
    nx, ny, nz = 40, 30, 22
    u0 = inputs.laplace_boundary_f64(nx, ny, nz, px=inputs.row_pitch(nx, "f64"))
    want = oracle.refine_solve(u0, 3, 7, dtype=dtype)[:, :, :nx + 2]
    for t in (0, 3, 6):
        got = to_host(api.refine_solve(api.as_grid(to_dev(u0, "f64"), nx), 3, 7, dtype, t),
                      "f64")
        assert np.array_equal(got, want), t


def test_refinement_tracks_fp64_sweeps():
    """Exact arithmetic makes O outer x m inner refinement equal O*m FP64 sweeps;
    in FP32 storage the difference stays at FP32 rounding size."""
    from paper_0912_4506_gb300 import api
    nx, ny, nz = 48, 40, 36
    u0 = inputs.laplace_boundary_f64(nx, ny, nz, px=inputs.row_pitch(nx, "f64"))
    plain = to_host(api.sweep(api.as_grid(to_dev(u0, "f64"), nx), 60, 1), "f64")
    ir = to_host(api.refine_solve(api.as_grid(to_dev(u0, "f64"), nx), 4, 15, "f32"), "f64")
    scale = np.abs(u0).max()
    assert np.abs(ir - plain).max() <= 4 * 60 * 2.0 ** -24 * scale
