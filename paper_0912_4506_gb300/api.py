"""PyTorch-facing API: device memory and streams from torch, every computation in
libjacobi_gb300.so (through the ctypes binding in ``_lib``).

A grid is a CUDA tensor of shape (nz+2, ny+2, nx+2) in the padded layout of
include/jacobi.h (interior 1..n, one boundary layer, x contiguous).  Its rows may
be padded: strides (row_pitch*(ny+2), row_pitch, 1) with row_pitch >= nx+2 and a
row of row_pitch elements a multiple of 16 bytes.  ``alloc_grid`` returns such a
view of a padded allocation.  bf16 grids are ``torch.bfloat16`` tensors.
"""
import torch

from . import _lib
from ._lib import (JAC_BF16, JAC_F32, JAC_F64, JAC_KERNEL_AUTO, JAC_KERNEL_PLAIN,
                   JAC_KERNEL_TB, JAC_KERNEL_WAVE, JacobiError)

_DT = {torch.float64: JAC_F64, torch.float32: JAC_F32, torch.bfloat16: JAC_BF16}
_NAME = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16}


def torch_dtype(dtype):
    return _NAME[dtype] if isinstance(dtype, str) else dtype


def row_pitch(nx, dtype):
    """Row pitch (elements) of the padded layout: nx+2 rounded up to 16 bytes."""
    es = torch.empty((), dtype=torch_dtype(dtype)).element_size()
    per = 16 // es
    return -(-(nx + 2) // per) * per


def alloc_grid(nx, ny, nz, dtype="f64", device="cuda", pitch=None):
    """Zeroed grid (nz+2, ny+2, nx+2), a view of rows padded to ``pitch``."""
    dt = torch_dtype(dtype)
    px = row_pitch(nx, dt) if pitch is None else pitch
    full = torch.zeros((nz + 2, ny + 2, px), dtype=dt, device=device)
    return full[:, :, :nx + 2]


def alloc_like(g):
    """Zeroed grid with the shape, dtype, device and row pitch of ``g``."""
    nx, ny, nz, px = grid_geom(g)
    return alloc_grid(nx, ny, nz, g.dtype, g.device, pitch=px)


def as_grid(full, nx):
    """View an (nz+2, ny+2, row_pitch) tensor as the grid of an nx-wide interior."""
    return full[:, :, :nx + 2]


def from_numpy(a, nx, device="cuda"):
    """Grid view (interior width nx) of a host array of shape (nz+2, ny+2,
    row_pitch): float64/float32 arrays, or uint16 arrays holding bf16 bits."""
    import numpy as np
    if a.dtype == np.uint16:
        t = torch.from_numpy(np.ascontiguousarray(a).view(np.int16)).to(device)
        t = t.view(torch.bfloat16)
    else:
        t = torch.from_numpy(np.ascontiguousarray(a)).to(device)
    return as_grid(t, nx)


def _stream_ptr(device=None):
    return torch.cuda.current_stream(device).cuda_stream


def grid_geom(t):
    """(nx, ny, nz, row_pitch) of a grid tensor; raises on a layout the library
    cannot take."""
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError("grids must be CUDA tensors")
    if t.dim() != 3 or t.dtype not in _DT:
        raise ValueError("grids are 3-D float64/float32/bfloat16 tensors")
    nz2, ny2, nx2 = t.shape
    px = t.stride(1)
    if t.stride(2) != 1 or px < nx2 or t.stride(0) != px * ny2:
        raise ValueError("grid must be (nz+2, ny+2, nx+2) with unit x stride and rows of "
                         "row_pitch >= nx+2 elements")
    if (px * t.element_size()) % 16 or t.data_ptr() % 16:
        raise ValueError("rows must be a multiple of 16 bytes and the data 16-byte aligned")
    return nx2 - 2, ny2 - 2, nz2 - 2, px


class Jacobi:
    """A pair of ping-pong grids bound to a library handle.

    ``A`` holds the initial grid with its boundary layer; ``B`` (allocated with
    A's layout if not given) receives A's boundary layer at construction.  With
    ``inplace=True`` there is no B: the sweeps update A in place (pipelined
    passes of depth >= 2 only, see jacobi_create_inplace).
    """

    def __init__(self, A, B=None, stream=None, inplace=False):
        """``stream``: the torch stream the handle launches on (default: the
        current stream at construction)."""
        nx, ny, nz, px = grid_geom(A)
        self.nx, self.ny, self.nz, self.px = nx, ny, nz, px
        self.A = A
        self.inplace = bool(inplace)
        if self.inplace and B is not None:
            raise ValueError("an in-place handle has no second grid")
        self.B = None if self.inplace else (alloc_like(A) if B is None else B)
        if self.B is not None and (grid_geom(self.B) != (nx, ny, nz, px) or
                                   self.B.dtype != A.dtype):
            raise ValueError("B must match A (shape, dtype, row pitch)")
        self.dtype = _DT[A.dtype]
        self.device = A.device
        with torch.cuda.device(self.device):
            sp = _stream_ptr(self.device) if stream is None else stream.cuda_stream
            if self.inplace:
                self._h = _lib.jacobi_create_inplace(nx, ny, nz, self.dtype, A.data_ptr(),
                                                     px, sp)
            else:
                self._h = _lib.jacobi_create(nx, ny, nz, self.dtype, A.data_ptr(),
                                             self.B.data_ptr(), px, sp)

    # ------------------------------------------------------------------
    def sweep(self, nsweeps, t=0, kernel=JAC_KERNEL_AUTO):
        """Run ``nsweeps`` sweeps; returns the tensor that holds the result."""
        with torch.cuda.device(self.device):
            fb = _lib.jacobi_sweep_ex(self._h, nsweeps, t, kernel)
        return self.B if fb else self.A

    def sweep_rhs(self, rho, nsweeps, t=0):
        """Correction sweeps e' = (sum6(e) + rho) * RN(1/6) (A holds e, zero boundary)."""
        if grid_geom(rho) != grid_geom(self.A) or rho.dtype != self.A.dtype:
            raise ValueError("rho must match the grids (shape, dtype, row pitch)")
        with torch.cuda.device(self.device):
            fb = _lib.jacobi_sweep_rhs(self._h, rho.data_ptr(), nsweeps, t)
        return self.B if fb else self.A

    def adjoint(self, grad_bdry, nsweeps, t=0):
        """Adjoint sweeps on A (= lambda_n, zero boundary); accumulates into grad_bdry."""
        if grid_geom(grad_bdry) != grid_geom(self.A) or grad_bdry.dtype != self.A.dtype:
            raise ValueError("grad_bdry must match the grids (shape, dtype, row pitch)")
        with torch.cuda.device(self.device):
            fb = _lib.jacobi_adjoint(self._h, grad_bdry.data_ptr(), nsweeps, t)
        return self.B if fb else self.A

    def upload(self, host):
        """Copy a host grid (a pinned CPU tensor of A's full padded storage shape
        (nz+2, ny+2, row_pitch)) into A, asynchronously on the handle's stream."""
        with torch.cuda.device(self.device):
            _lib.jacobi_upload(self._h, host.data_ptr())

    def download(self, host, from_b):
        """Copy A (from_b=0) or B (from_b=1) into a host tensor of the full padded
        storage shape, asynchronously on the handle's stream."""
        with torch.cuda.device(self.device):
            _lib.jacobi_download(self._h, host.data_ptr(), int(from_b))

    def run_host(self, host_in, host_out, nsweeps, t=0, kernel=JAC_KERNEL_AUTO):
        """Upload, sweep, download: the end-to-end call on host buffers.  Returns
        after enqueueing; synchronise the stream before reading host_out."""
        self.upload(host_in)
        with torch.cuda.device(self.device):
            fb = _lib.jacobi_sweep_ex(self._h, nsweeps, t, kernel)
        self.download(host_out, fb)
        return fb

    def plan(self, nsweeps, t=0, kernel=JAC_KERNEL_AUTO):
        with torch.cuda.device(self.device):
            return _lib.jacobi_plan(self._h, nsweeps, t, kernel)

    def check(self):
        with torch.cuda.device(self.device):
            _lib.jacobi_check(self._h)

    def close(self):
        if getattr(self, "_h", None) is not None:
            with torch.cuda.device(self.device):
                _lib.jacobi_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass



class HostPipeline:
    """End-to-end sweeps of independent problems held in (pinned) host memory.

    Problem i is uploaded, swept and downloaded through handle i % 2; each handle
    owns a device grid pair and launches on its own stream, so one problem's
    host<->device copies overlap the other problem's sweeps (the host link, about
    200 GB/s each way on GB300, is otherwise idle while the sweeps run).  The
    sweeps themselves run one problem after the other (an event orders problem
    i's sweeps after problem i-1's): two problems sweeping at once only share the
    SMs."""

    def __init__(self, nx, ny, nz, dtype="f64", device="cuda"):
        self.device = torch.device(device)
        self.streams = [torch.cuda.Stream(self.device) for _ in range(2)]
        self.jobs = []
        for st in self.streams:
            with torch.cuda.stream(st):
                self.jobs.append(Jacobi(alloc_grid(nx, ny, nz, dtype, self.device),
                                        stream=st))

    def run(self, host_ins, host_outs, nsweeps, t=0, kernel=JAC_KERNEL_AUTO):
        """Enqueue problem i (host_ins[i] -> host_outs[i]) on handle i % 2.  The
        current stream waits for all of them; synchronise it before reading
        host_outs.  Buffers of problems i and i + 1 must be distinct."""
        with torch.cuda.device(self.device):
            cur = torch.cuda.current_stream(self.device)
            for st in self.streams:
                st.wait_stream(cur)
            prev = None
            for i, (hi, ho) in enumerate(zip(host_ins, host_outs)):
                j, st = self.jobs[i % 2], self.streams[i % 2]
                j.upload(hi)
                if prev is not None:
                    st.wait_event(prev)
                fb = _lib.jacobi_sweep_ex(j._h, nsweeps, t, kernel)
                prev = torch.cuda.Event()
                prev.record(st)
                j.download(ho, fb)
            for st in self.streams:
                cur.wait_stream(st)

    def close(self):
        for j in self.jobs:
            j.close()
        self.jobs = []

def sweep(A, nsweeps, t=0, kernel=JAC_KERNEL_AUTO):
    """``nsweeps`` Jacobi sweeps of the grid ``A`` (not modified); returns a new
    grid with the result."""
    A2 = alloc_like(A)
    A2.copy_(A)
    j = Jacobi(A2)
    out = j.sweep(nsweeps, t, kernel)
    j.close()
    return out


def residual_accumulate(u_in, u_out, e, rho):
    """FP64 refinement step: u_out = u_in + e (interior), rho = s(u_out) - 6 u_out
    (only interior cells of u_out and rho are written)."""
    nx, ny, nz, pu = grid_geom(u_in)
    if grid_geom(u_out) != (nx, ny, nz, pu):
        raise ValueError("u_out must match u_in")
    gx, gy, gz, pl = grid_geom(e)
    if (gx, gy, gz) != (nx, ny, nz) or grid_geom(rho) != (gx, gy, gz, pl) or rho.dtype != e.dtype:
        raise ValueError("e and rho must match u's shape and each other")
    if u_in.dtype != torch.float64 or u_out.dtype != torch.float64:
        raise ValueError("u must be float64")
    with torch.cuda.device(u_in.device):
        _lib.jacobi_residual_accumulate(nx, ny, nz, u_in.data_ptr(), u_out.data_ptr(), pu,
                                        e.data_ptr(), rho.data_ptr(), _DT[e.dtype], pl,
                                        _stream_ptr(u_in.device))


class Refiner:
    """Mixed-precision iterative refinement of the Jacobi solve, with its buffers.

    ``u0`` (float64 grid) holds the boundary data and the initial interior.  Each
    outer step runs the FP64 residual (adding the previous correction), then
    ``inner`` correction sweeps in ``dtype`` ("f32" or "bf16") from a zero
    correction; after the last step the last correction is added.  In exact
    arithmetic the result equals ``outer * inner`` plain sweeps of ``u0``.
    """

    def __init__(self, u0, dtype="f32"):
        nx, ny, nz, _ = grid_geom(u0)
        dt = torch_dtype(dtype)
        self.u0 = u0
        self.u = [alloc_like(u0), alloc_like(u0)]
        self.u[0].copy_(u0)
        self.u[1].copy_(u0)
        self.e0 = alloc_grid(nx, ny, nz, dt, u0.device)
        self.e1 = alloc_like(self.e0)
        self.rho = alloc_like(self.e0)
        self.solver = Jacobi(self.e0, self.e1)

    def run(self, outer, inner, t=0):
        """Refine from u0 (every call starts again from u0); returns the grid that
        holds the result."""
        u, e0, rho = self.u, self.e0, self.rho
        u[0].copy_(self.u0)
        e_cur = e0
        cur = 0
        for _ in range(outer):
            residual_accumulate(u[cur], u[1 - cur], e_cur, rho)
            cur = 1 - cur
            e0.zero_()
            e_cur = self.solver.sweep_rhs(rho, inner, t)
        residual_accumulate(u[cur], u[1 - cur], e_cur, rho)
        return u[1 - cur]

    def close(self):
        self.solver.close()


def refine_solve(u0, outer, inner, dtype="f32", t=0):
    r = Refiner(u0, dtype)
    out = r.run(outer, inner, t)
    r.close()
    return out


__all__ = ["Jacobi", "JacobiFn", "jacobi_fn", "Batch", "Refiner", "sweep", "residual_accumulate", "refine_solve", "alloc_grid",
           "alloc_like", "as_grid", "from_numpy", "grid_geom", "row_pitch", "JacobiError",
           "JAC_KERNEL_AUTO", "JAC_KERNEL_PLAIN", "JAC_KERNEL_TB"]


class JacobiFn(torch.autograd.Function):
    """Differentiable n-sweep Jacobi map: Y = n temporally-blocked sweeps of X.

    X is a grid (interior = initial values, boundary layer = Dirichlet data g).
    The backward pass runs the library's adjoint sweeps: lambda_n = dL/dY on the
    interior (zero boundary), n transpose sweeps (the same stencil on a zero
    boundary, the sweep being symmetric on the interior), while the boundary
    gradient accumulates RN(1/6)*lambda_s at each face cell's interior neighbour,
    plus the direct dL/dY on the boundary layer (Y's boundary is g).  Returns one
    grid: interior dL/dX_interior, boundary layer dL/dg.

    With ``checkpoint=True`` the forward pass keeps the state after every pass of
    depth t in ``ctx.checkpoints`` (a list of grids).  The sweep map is affine in
    (X, g), so the backward pass needs no forward state: the gradients are the
    same with and without checkpoints.
    """

    @staticmethod
    def forward(ctx, X, nsweeps, t=0, checkpoint=False):
        if X.dtype not in (torch.float32, torch.float64):
            raise ValueError("JacobiFn supports float32 and float64 grids")
        A = alloc_like(X)
        A.copy_(X)
        j = Jacobi(A)
        ckpts = []
        if checkpoint and nsweeps > 0:
            step = t if t > 0 else 4
            done = 0
            while done < nsweeps:
                d = min(step, nsweeps - done)
                out = j.sweep(d, d, JAC_KERNEL_TB)
                if out is j.B:
                    j.A.copy_(j.B)
                c = alloc_like(X)
                c.copy_(j.A)
                ckpts.append(c)
                done += d
            Y = j.A
        else:
            Y = j.sweep(nsweeps, t, JAC_KERNEL_TB if nsweeps else JAC_KERNEL_AUTO)
        j.close()
        ctx.nsweeps, ctx.t = nsweeps, t
        ctx.checkpoints = ckpts
        Yc = alloc_like(X)
        Yc.copy_(Y)
        return Yc

    @staticmethod
    def backward(ctx, gY):
        gY = gY.to(torch.float64 if gY.dtype == torch.float64 else torch.float32)
        lam = alloc_like(gY) if _is_grid(gY) else None
        if lam is None:  # gradient arrived densely laid out: re-pad it
            nz2, ny2, nx2 = gY.shape
            lam = alloc_grid(nx2 - 2, ny2 - 2, nz2 - 2, gY.dtype, gY.device)
        lam[1:-1, 1:-1, 1:-1].copy_(gY[1:-1, 1:-1, 1:-1])
        grad = alloc_like(lam)
        grad.copy_(gY)
        grad[1:-1, 1:-1, 1:-1].zero_()
        j = Jacobi(lam)
        out = j.adjoint(grad, ctx.nsweeps, ctx.t)
        j.check()
        grad[1:-1, 1:-1, 1:-1].copy_(out[1:-1, 1:-1, 1:-1])
        j.close()
        return grad, None, None, None


def _is_grid(t):
    try:
        grid_geom(t)
        return True
    except ValueError:
        return False


def jacobi_fn(X, nsweeps, t=0, checkpoint=False):
    """Autograd-aware n-sweep Jacobi map (see JacobiFn)."""
    return JacobiFn.apply(X, nsweeps, t, checkpoint)


class Batch:
    """Many independent grids advanced together by one persistent kernel launch,
    recorded into a CUDA graph (include/jacobi.h, jacobi_batch_*).

    ``grids``: list of float32 or bfloat16 grids (each its own shape); ``nsweeps``:
    sweeps per grid; ``t``: depth per grid (None: 4, or the autotuner's choice);
    ``tile_x``: loaded tile width per grid, 64 or 128 (None: 128 where the depth
    allows it); ``nchunk``: k-chunks per pass per grid (None: planner).  B grids are allocated
    with each A's layout.  ``run()`` returns the list of tensors holding the
    results.
    """

    def __init__(self, grids, nsweeps, t=None, nchunk=None, graph=True, test_missing_producer=False,
                 wait_limit_s=0.0, tile_x=None):
        if not grids:
            raise ValueError("empty batch")
        dt = grids[0].dtype
        if dt not in (torch.float32, torch.bfloat16) or any(g.dtype != dt for g in grids):
            raise ValueError("batched grids are all float32 or all bfloat16")
        self.A = list(grids)
        self.B = [alloc_like(g) for g in grids]
        geo = [grid_geom(g) for g in grids]
        self.device = grids[0].device
        flags = (0 if graph else _lib.JAC_BATCH_NO_GRAPH) | \
            (_lib.JAC_BATCH_TEST_MISSING_PRODUCER if test_missing_producer else 0)
        with torch.cuda.device(self.device):
            self._h = _lib.jacobi_batch_create(
                [g[:3] for g in geo], [g[3] for g in geo], [a.data_ptr() for a in self.A],
                [b.data_ptr() for b in self.B], list(nsweeps), t, nchunk, _DT[dt],
                _stream_ptr(self.device), flags, wait_limit_s, tile_x)
        self.count = len(grids)

    def run(self):
        with torch.cuda.device(self.device):
            fb = _lib.jacobi_batch_run(self._h, self.count)
        return [b if f else a for a, b, f in zip(self.A, self.B, fb)]

    def info(self):
        return _lib.jacobi_batch_info(self._h, self.count)

    def check(self):
        with torch.cuda.device(self.device):
            _lib.jacobi_batch_check(self._h)

    def close(self):
        if getattr(self, "_h", None) is not None:
            with torch.cuda.device(self.device):
                _lib.jacobi_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
