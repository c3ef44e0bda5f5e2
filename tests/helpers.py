"""Shared helpers for the GPU parity tests (numpy <-> torch grids)."""
import numpy as np

from paper_0912_4506_gb300 import inputs

NP_DT = {"f64": np.float64, "f32": np.float32, "bf16": np.uint16}


def make_grid(nx, ny, nz, dtype, px=None, g=0):
    """Seeded uniform grid (interior seed 0, boundary seed 1) in `dtype` storage
    with the library's row pitch (or `px`)."""
    px = inputs.row_pitch(nx, dtype) if px is None else px
    return inputs.to_dtype(inputs.uniform_grid_f64(nx, ny, nz, g=g), dtype, px=px)


def to_dev(a, dtype, device="cuda"):
    import torch
    if dtype == "bf16":
        return torch.from_numpy(a.view(np.int16)).to(device).view(torch.bfloat16)
    return torch.from_numpy(a).to(device)


def to_host(t, dtype):
    """Copy a (possibly row-padded view) grid to a contiguous numpy array."""
    import torch
    t = t.contiguous()
    if dtype == "bf16":
        return t.view(torch.int16).cpu().numpy().view(np.uint16)
    return t.cpu().numpy()


def first_diff(got, want):
    bad = np.argwhere(got != want)
    if len(bad) == 0:
        return None
    k, j, i = bad[0]
    return (len(bad), (int(i), int(j), int(k)), got[k, j, i], want[k, j, i])
