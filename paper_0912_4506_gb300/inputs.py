"""Seeded synthetic inputs for the Jacobi workloads.

This module only draws numbers; it holds none of the stencil arithmetic.  The
CPU oracle and the GPU library both receive the arrays it returns, so the two
sides never generate their own random data.

Generator (counter based, integer exact on every machine):
    mix64(x)         = the splitmix64 output function applied to the state
                       x + 0x9E3779B97F4A7C15 (Steele, Lea, Flood 2014)
    u01(seed, g, i)  = (mix64((seed << 56) ^ (g << 40) ^ i) >> 11) * 2**-53
with ``i`` the cell's linear index in the compact padded layout
``i + (nx+2) * (j + (ny+2) * k)`` (independent of any row padding), ``g`` the grid
number (0 for a single grid).  FP32 values are RN(double), bf16 values RNE(FP32).

Workloads (the paper's synthetic cubic grids, Sect. 1.5 uses 600^3):
  * uniform grids: interior U[0,1) from seed 0, boundary layer U[0,1) from seed 1;
  * the Laplace problem: boundary data u = x^2 - y^2 + 0.5 z on the padded
    index lattice, interior zero;
  * batches: grid shapes (multiples of 8 in [32, 256]) and sweep counts
    (uniform in [10, 200]) from seed 2;
  * adjoint weights: N(0,1) by Box-Muller from seed 3.
"""
import math

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_TWO_M53 = 2.0 ** -53

SEED_INTERIOR, SEED_BOUNDARY, SEED_BATCH, SEED_WEIGHTS = 0, 1, 2, 3


def mix64(x):
    """splitmix64 output for state ``x`` (uint64 array), wrapping arithmetic."""
    with np.errstate(over="ignore"):
        z = np.asarray(x, dtype=np.uint64) + _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def u01(seed, g, idx):
    """Uniform [0,1) doubles for counters ``idx`` (uint64 array)."""
    key = (np.uint64(seed) << np.uint64(56)) ^ (np.uint64(g) << np.uint64(40))
    bits = mix64(np.asarray(idx, dtype=np.uint64) ^ key) >> np.uint64(11)
    return bits.astype(np.float64) * _TWO_M53


def row_pitch(nx, dtype):
    """Row pitch (elements) of the library's padded layout: nx+2 rounded up so
    that one row is a multiple of 16 bytes."""
    per16 = {"f64": 2, "f32": 4, "bf16": 8}[dtype]
    return -(-(nx + 2) // per16) * per16


def _boundary_mask(nx, ny, nz):
    k = np.arange(nz + 2)[:, None, None]
    j = np.arange(ny + 2)[None, :, None]
    i = np.arange(nx + 2)[None, None, :]
    return ((i == 0) | (i == nx + 1) | (j == 0) | (j == ny + 1) |
            (k == 0) | (k == nz + 1))


def uniform_grid_f64(nx, ny, nz, g=0, px=None, planes=None):
    """Padded FP64 grid (nz+2, ny+2, px): interior U[0,1) (seed 0), boundary layer
    U[0,1) (seed 1); the row padding beyond nx+2 is zero.  ``planes=(lo, hi)``
    returns only the global planes lo..hi (the same values, drawn by counter)."""
    px = nx + 2 if px is None else px
    lo, hi = (0, nz + 1) if planes is None else planes
    out = np.zeros((hi - lo + 1, ny + 2, px), dtype=np.float64)
    plane = (nx + 2) * (ny + 2)
    j = np.arange(ny + 2, dtype=np.uint64)[:, None]
    i = np.arange(nx + 2, dtype=np.uint64)[None, :]
    base = i + np.uint64(nx + 2) * j
    jj = np.arange(ny + 2)[:, None]
    ii = np.arange(nx + 2)[None, :]
    edge = (ii == 0) | (ii == nx + 1) | (jj == 0) | (jj == ny + 1)
    for k in range(lo, hi + 1):
        idx = base + np.uint64(plane * k)
        vi = u01(SEED_INTERIOR, g, idx)
        vb = u01(SEED_BOUNDARY, g, idx)
        bnd = edge | (k == 0) | (k == nz + 1)
        out[k - lo, :, :nx + 2] = np.where(bnd, vb, vi)
    return out


def laplace_boundary_f64(nx, ny, nz, px=None):
    """Padded FP64 grid with boundary data u = x^2 - y^2 + 0.5 z (x=i, y=j, z=k
    padded indices, so the boundary sits at 0 and n+1) and a zero interior.  The
    field is discrete-harmonic, so it is also the exact discrete solution."""
    px = nx + 2 if px is None else px
    out = np.zeros((nz + 2, ny + 2, px), dtype=np.float64)
    k = np.arange(nz + 2, dtype=np.float64)[:, None, None]
    j = np.arange(ny + 2, dtype=np.float64)[None, :, None]
    i = np.arange(nx + 2, dtype=np.float64)[None, None, :]
    full = i * i - j * j + 0.5 * k
    bnd = _boundary_mask(nx, ny, nz)
    out[:, :, :nx + 2] = np.where(bnd, full, 0.0)
    return out


def normal_grid_f64(nx, ny, nz, seed=SEED_WEIGHTS, g=0, px=None):
    """Padded FP64 grid of N(0,1) values (Box-Muller on counters 2c and 2c+1)."""
    px = nx + 2 if px is None else px
    n = (nx + 2) * (ny + 2) * (nz + 2)
    c = np.arange(n, dtype=np.uint64)
    u1 = 1.0 - u01(seed, g, c * np.uint64(2))          # (0, 1]
    u2 = u01(seed, g, c * np.uint64(2) + np.uint64(1))
    z = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)
    out = np.zeros((nz + 2, ny + 2, px), dtype=np.float64)
    out[:, :, :nx + 2] = z.reshape(nz + 2, ny + 2, nx + 2)
    return out


def batch_specs(count=64, lo=32, hi=256, step=8, nmin=10, nmax=200,
                seed=SEED_BATCH):
    """Shapes (nx, ny, nz) and sweep counts for a batch of independent grids.

    Axis sizes are drawn uniformly from {lo, lo+step, ..., hi}; sweep counts
    uniformly from [nmin, nmax].  Counter order: nx, ny, nz, n per grid.
    """
    nsizes = (hi - lo) // step + 1
    ctr = np.arange(4 * count, dtype=np.uint64)
    u = u01(seed, 0, ctr).reshape(count, 4)
    sizes = lo + step * np.floor(u[:, :3] * nsizes).astype(np.int64)
    sweeps = nmin + np.floor(u[:, 3] * (nmax - nmin + 1)).astype(np.int64)
    return [(int(a), int(b), int(c), int(n)) for (a, b, c), n in zip(sizes, sweeps)]


def to_dtype(a64, dtype, px=None):
    """Convert a padded FP64 grid to "f64"/"f32"/"bf16" storage (bf16 returned as
    a torch tensor's bit pattern in uint16), re-padding rows to ``px``."""
    nz2, ny2, _ = a64.shape
    if dtype == "f64":
        src = a64
    else:
        src = a64.astype(np.float32)
        if dtype == "bf16":
            import torch
            src = (torch.from_numpy(np.ascontiguousarray(src)).to(torch.bfloat16)
                   .view(torch.int16).numpy().view(np.uint16))
    if px is None or px == src.shape[2]:
        return np.ascontiguousarray(src)
    out = np.zeros((nz2, ny2, px), dtype=src.dtype)
    w = min(px, src.shape[2])
    out[:, :, :w] = src[:, :, :w]
    return out


def laplace_boundary_torch(nx, ny, nz, dtype=None, device="cuda", px=None):
    """The Laplace-problem grid of `laplace_boundary_f64`, built directly on a
    torch device (for grids too large to stage through host memory): returns a
    (nz+2, ny+2, px) float64 tensor, boundary u = x^2 - y^2 + 0.5 z, interior 0."""
    import torch
    px = nx + 2 if px is None else px
    out = torch.zeros((nz + 2, ny + 2, px), dtype=torch.float64, device=device)
    i = torch.arange(nx + 2, dtype=torch.float64, device=device)
    j = torch.arange(ny + 2, dtype=torch.float64, device=device)
    for k in range(nz + 2):
        plane = (i * i)[None, :] - (j * j)[:, None] + 0.5 * k
        if k == 0 or k == nz + 1:
            out[k, :, :nx + 2] = plane
        else:
            out[k, 0, :nx + 2] = plane[0]
            out[k, ny + 1, :nx + 2] = plane[ny + 1]
            out[k, 1:ny + 1, 0] = plane[1:ny + 1, 0]
            out[k, 1:ny + 1, nx + 1] = plane[1:ny + 1, nx + 1]
    return out
