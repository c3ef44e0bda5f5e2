"""Gradients through the Jacobi map: the GPU adjoint sweeps against the CPU
oracle's FP64 reverse mode, against central finite differences (exact up to
rounding because the loss is affine), and with/without checkpoints."""
import numpy as np
import pytest

import oracle
from paper_0912_4506_gb300 import inputs
from tests.helpers import to_dev, to_host

pytestmark = pytest.mark.gpu


def _grad_gpu(x64, W, n, t, dtype, checkpoint=False):
    import torch
    from paper_0912_4506_gb300 import api
    nx = x64.shape[2] - 2
    px = inputs.row_pitch(nx, dtype)
    X = api.as_grid(to_dev(inputs.to_dtype(x64, dtype, px=px), dtype), nx)
    X.requires_grad_(True)
    Wt = api.as_grid(to_dev(inputs.to_dtype(W, dtype, px=px), dtype), nx)
    Y = api.jacobi_fn(X, n, t, checkpoint)
    loss = (Y * Wt).sum()
    loss.backward()
    return to_host(X.grad.contiguous(), dtype).astype(np.float64)


@pytest.mark.parametrize("dtype,tol", [("f64", 1e-13), ("f32", 2e-6)])
@pytest.mark.parametrize("shape", [(23, 17, 13), (5, 30, 3)], ids=lambda s: "x".join(map(str, s)))
def test_adjoint_matches_oracle_reverse_mode(dtype, tol, shape):
    nx, ny, nz = shape
    n = 10
    x = inputs.uniform_grid_f64(nx, ny, nz)
    W = inputs.normal_grid_f64(nx, ny, nz)
    want = oracle.grad_f64(W, n)
    scale = np.abs(want).max()
    for t in (1, 2, 3, 4, 6, 8):
        got = _grad_gpu(x, W, n, t, dtype)
        assert np.abs(got - want).max() <= tol * scale, (t, np.abs(got - want).max())


def test_adjoint_edges_and_corners_are_w():
    nx, ny, nz, n = 12, 10, 9, 6
    x = inputs.uniform_grid_f64(nx, ny, nz)
    W = inputs.normal_grid_f64(nx, ny, nz)
    got = _grad_gpu(x, W, n, 3, "f64")
    k, j, i = np.indices(W.shape)
    nb = ((i == 0) | (i == nx + 1)).astype(int) + ((j == 0) | (j == ny + 1)) + \
        ((k == 0) | (k == nz + 1))
    assert np.array_equal(got[nb >= 2], W[nb >= 2])


def test_adjoint_central_differences_16cubed():
    """Central differences with step 1 through the GPU forward sweeps (FP64) on
    the 16^3 instance, on sampled cells of the interior and of every face."""
    import torch
    from paper_0912_4506_gb300 import api
    nx = ny = nz = 16
    n = 8
    x = inputs.uniform_grid_f64(nx, ny, nz)
    W = inputs.normal_grid_f64(nx, ny, nz)
    g = _grad_gpu(x, W, n, 4, "f64")
    Wt = torch.from_numpy(W).cuda()
    rng = np.random.default_rng(0)
    cells = [tuple(rng.integers(1, 17, 3)) for _ in range(24)]
    cells += [(0, 5, 7), (17, 3, 3), (4, 0, 9), (6, 17, 2), (8, 8, 0), (2, 11, 17)]

    def loss(a):
        out = api.sweep(torch.from_numpy(a).cuda(), n, 4)
        return float((out * Wt).sum())

    for (k, j, i) in cells:
        ap = x.copy(); ap[k, j, i] += 1.0
        am = x.copy(); am[k, j, i] -= 1.0
        fd = 0.5 * (loss(ap) - loss(am))
        assert abs(fd - g[k, j, i]) <= 1e-11 * max(1.0, np.abs(W).sum()), (k, j, i)


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_checkpoints_do_not_change_gradient(dtype):
    nx, ny, nz, n = 30, 21, 19, 11
    x = inputs.uniform_grid_f64(nx, ny, nz)
    W = inputs.normal_grid_f64(nx, ny, nz)
    a = _grad_gpu(x, W, n, 4, dtype, checkpoint=False)
    b = _grad_gpu(x, W, n, 4, dtype, checkpoint=True)
    assert np.array_equal(a, b)


def test_forward_of_autograd_fn_is_the_sweep():
    import torch
    from paper_0912_4506_gb300 import api
    nx, ny, nz, n = 26, 20, 18, 9
    x = inputs.uniform_grid_f64(nx, ny, nz)
    X = torch.from_numpy(x).cuda()
    for ck in (False, True):
        Y = api.jacobi_fn(X, n, 4, ck)
        assert np.array_equal(to_host(Y.contiguous(), "f64"), oracle.sweeps(x, n))


@pytest.mark.parametrize("dtype,tol", [("f64", 1e-13), ("f32", 2e-6)])
def test_adjoint_every_pass_count(dtype, tol):
    """Passes rotate through three grids and the last one writes A or B: every
    pass count from 1 to 7 at depths 1 and 2 (each position of the rotation, and
    the last pass redirected away from the third grid) against the oracle; a
    second call on the same handle, which reuses the third grid, gives the same
    bits."""
    import torch
    from paper_0912_4506_gb300 import api
    nx, ny, nz = 19, 11, 7
    x = inputs.uniform_grid_f64(nx, ny, nz)
    W = inputs.normal_grid_f64(nx, ny, nz)
    px = inputs.row_pitch(nx, dtype)
    for n in range(1, 8):
        want = oracle.grad_f64(W, n)
        scale = np.abs(want).max()
        for t in (1, 2):
            got = _grad_gpu(x, W, n, t, dtype)
            assert np.abs(got - want).max() <= tol * scale, (n, t)
            outs = []
            lam0 = api.as_grid(to_dev(inputs.to_dtype(W, dtype, px=px), dtype), nx)
            for face in (0, -1):
                lam0[face] = 0
                lam0[:, face] = 0
            lam0[:, :, 0] = 0
            lam0[:, :, nx + 1] = 0
            j = api.Jacobi(api.alloc_like(lam0))
            for _ in range(2):
                j.A.copy_(lam0)
                gb = api.alloc_like(lam0)
                gb.zero_()
                out = j.adjoint(gb, n, t)
                j.check()
                torch.cuda.synchronize()
                outs.append((to_host(out, dtype), to_host(gb, dtype)))
            j.close()
            assert np.array_equal(outs[0][0], outs[1][0]), (n, t)
            assert np.array_equal(outs[0][1], outs[1][1]), (n, t)
