"""CPU oracle for the temporally-blocked 3D 7-point Jacobi library.

TEST INFRASTRUCTURE ONLY: the plain, slow, obviously correct statement of what the
GPU path computes.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import it.  It shares no code with the CUDA library and
never imports it.

Every function works on numpy arrays in the padded layout (one boundary layer,
interior 1..n per axis, x contiguous) of shape ``(nz+2, ny+2, px)`` with
``px >= nx+2``.  The arithmetic lives in ``jacobi_oracle.c``; this module only
marshals arguments and composes the C routines into the iterative-refinement
driver.

Paper passages followed (Wittmann, Hager, Wellein, arXiv:0912.4506):
  * Eq. 1 (Sect. 1.1): one cell update, the mean of the six face neighbours.
  * Sect. 1.1: successive sweeps write grids A and B in turn.
Readings where the paper is silent, as this module implements them: the sum is
taken left to right in the order of Eq. 1 and multiplied by RN(1/6) of the
compute precision (no division, no fused multiply-add); the boundary layer is
fixed; bf16 values are rounded to nearest-even after every sweep; the refinement
iterates corrections e' = (sum6(e) + rho) * RN(1/6) on a zero boundary with
rho = sum6(u) - 6u computed in FP64.
"""
import ctypes

import numpy as np

from . import build as _build

_lib = None


def load(path: str = None):
    """Load (building if needed) the oracle library; ``path`` selects another
    build of the same source (used by the mutation tests)."""
    global _lib
    if path is not None:
        lib = ctypes.CDLL(path)
        _declare(lib)
        return lib
    if _lib is None:
        _lib = ctypes.CDLL(_build.build())
        _declare(_lib)
    return _lib


def _declare(lib):
    P = ctypes.c_void_p
    I = ctypes.c_int
    L = ctypes.c_long
    for name in ("oracle_sweeps_f64", "oracle_sweeps_f32", "oracle_sweeps_bf16"):
        f = getattr(lib, name)
        f.argtypes = [P, P, I, I, I, L, L, I, I]
        f.restype = I
    lib.oracle_rhs_sweeps_f64.argtypes = [P, P, P, I, I, I, L, L, I]
    lib.oracle_rhs_sweeps_f64.restype = I
    for name in ("oracle_rhs_sweeps_f32", "oracle_rhs_sweeps_bf16"):
        f = getattr(lib, name)
        f.argtypes = [P, P, P, I, I, I, L, L, I, I]
        f.restype = I
    lib.oracle_residual_accumulate.argtypes = [P, P, P, I, I, I, I, L, L]
    lib.oracle_residual_accumulate.restype = None
    lib.oracle_grad_f64.argtypes = [P, P, P, P, I, I, I, L, L, I]
    lib.oracle_grad_f64.restype = None
    lib.oracle_f32_to_bf16.argtypes = [P, P, ctypes.c_size_t]
    lib.oracle_bf16_to_f32.argtypes = [P, P, ctypes.c_size_t]
    lib.oracle_max_threads.restype = I


_DT = {"f64": np.float64, "f32": np.float32, "bf16": np.uint16}


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _dims(a, nx):
    assert a.ndim == 3 and a.flags["C_CONTIGUOUS"]
    nz2, ny2, px = a.shape
    assert px >= nx + 2
    return ny2 - 2, nz2 - 2, px, ny2


def sweeps(A, n, nx=None, dtype="f64", nthreads=1, lib=None):
    """Return the grid after ``n`` Jacobi sweeps (Eq. 1) of the padded array ``A``.

    ``A`` is not modified.  ``dtype`` is "f64", "f32" or "bf16" (bf16 arrays are
    passed as uint16 bit patterns).  ``nx`` defaults to ``px - 2``.
    """
    lib = lib or load()
    A = np.ascontiguousarray(A, dtype=_DT[dtype]).copy()
    nx = A.shape[2] - 2 if nx is None else nx
    ny, nz, px, py = _dims(A, nx)
    B = A.copy()
    fn = {"f64": lib.oracle_sweeps_f64, "f32": lib.oracle_sweeps_f32,
          "bf16": lib.oracle_sweeps_bf16}[dtype]
    in_b = fn(_ptr(A), _ptr(B), nx, ny, nz, px, py, int(n), int(nthreads))
    return B if in_b else A


def sweeps_into(A, B, n, nx=None, dtype="f64", nthreads=1, lib=None):
    """``n`` sweeps between the caller's arrays ``A`` (input) and ``B`` (whose
    boundary layer must equal A's), without copying either; returns the array
    that holds the result (A when n is even).  Used where the oracle is timed."""
    lib = lib or load()
    assert A.dtype == _DT[dtype] and B.dtype == A.dtype and A.shape == B.shape
    assert A.flags["C_CONTIGUOUS"] and B.flags["C_CONTIGUOUS"]
    nx = A.shape[2] - 2 if nx is None else nx
    ny, nz, px, py = _dims(A, nx)
    fn = {"f64": lib.oracle_sweeps_f64, "f32": lib.oracle_sweeps_f32,
          "bf16": lib.oracle_sweeps_bf16}[dtype]
    in_b = fn(_ptr(A), _ptr(B), nx, ny, nz, px, py, int(n), int(nthreads))
    return B if in_b else A


def rhs_sweeps(E, rho, n, nx=None, dtype="f32", nthreads=1, lib=None):
    """``n`` correction sweeps e' = (sum6(e) + rho) * RN(1/6) on a grid whose
    boundary layer is zero (the refinement's inner iteration)."""
    lib = lib or load()
    E = np.ascontiguousarray(E, dtype=_DT[dtype]).copy()
    rho = np.ascontiguousarray(rho, dtype=_DT[dtype])
    nx = E.shape[2] - 2 if nx is None else nx
    ny, nz, px, py = _dims(E, nx)
    E2 = E.copy()
    if dtype == "f64":
        in_b = lib.oracle_rhs_sweeps_f64(_ptr(E), _ptr(E2), _ptr(rho), nx, ny, nz,
                                         px, py, int(n))
    else:
        fn = (lib.oracle_rhs_sweeps_f32 if dtype == "f32"
              else lib.oracle_rhs_sweeps_bf16)
        in_b = fn(_ptr(E), _ptr(E2), _ptr(rho), nx, ny, nz, px, py, int(n),
                  int(nthreads))
    return E2 if in_b else E


def residual_accumulate(u, e, nx=None, dtype="f32", lib=None):
    """FP64 residual step: returns (u + e, rho) with rho = s(u') - 6 u' stored in
    ``dtype`` (the storage precision of the correction)."""
    lib = lib or load()
    u = np.ascontiguousarray(u, dtype=np.float64).copy()
    e = np.ascontiguousarray(e, dtype=_DT[dtype])
    assert e.shape == u.shape, "u and e must share the padded shape (row pitch included)"
    nx = u.shape[2] - 2 if nx is None else nx
    ny, nz, px, py = _dims(u, nx)
    rho = np.zeros_like(e)
    elem = {"f64": 8, "f32": 4, "bf16": 2}[dtype]
    lib.oracle_residual_accumulate(_ptr(u), _ptr(e), _ptr(rho), elem, nx, ny, nz,
                                   px, py)
    return u, rho


def refine_solve(u0, outer, inner, dtype="f32", nthreads=1, lib=None):
    """Mixed-precision iterative refinement of the Jacobi solve.

    ``u0`` (f64, padded) carries the boundary data and the initial interior.
    Each outer step: residual in FP64 (with the previous correction added), a
    zeroed correction grid, ``inner`` correction sweeps in ``dtype``; after the
    last step the final correction is added.  In exact arithmetic the result
    equals ``outer * inner`` plain sweeps of ``u0``.
    """
    lib = lib or load()
    u = np.ascontiguousarray(u0, dtype=np.float64).copy()
    e = np.zeros(u.shape, dtype=_DT[dtype])
    for _ in range(outer):
        u, rho = residual_accumulate(u, e, dtype=dtype, lib=lib)
        e = np.zeros(u.shape, dtype=_DT[dtype])
        e = rhs_sweeps(e, rho, inner, dtype=dtype, nthreads=nthreads, lib=lib)
    u, _ = residual_accumulate(u, e, dtype=dtype, lib=lib)
    return u


def grad_f64(W, n, nx=None, lib=None):
    """Reverse-mode gradient of L = sum(W * A_n) with respect to A_0 (interior:
    the initial grid; boundary layer: the Dirichlet data), FP64."""
    lib = lib or load()
    W = np.ascontiguousarray(W, dtype=np.float64)
    nx = W.shape[2] - 2 if nx is None else nx
    ny, nz, px, py = _dims(W, nx)
    grad = np.zeros_like(W)
    lam = np.zeros_like(W)
    lam2 = np.zeros_like(W)
    lib.oracle_grad_f64(_ptr(W), _ptr(grad), _ptr(lam), _ptr(lam2), nx, ny, nz, px,
                        py, int(n))
    return grad


def f32_to_bf16(x, lib=None):
    lib = lib or load()
    x = np.ascontiguousarray(x, dtype=np.float32)
    out = np.empty(x.shape, dtype=np.uint16)
    lib.oracle_f32_to_bf16(_ptr(x), _ptr(out), x.size)
    return out


def bf16_to_f32(x, lib=None):
    lib = lib or load()
    x = np.ascontiguousarray(x, dtype=np.uint16)
    out = np.empty(x.shape, dtype=np.float32)
    lib.oracle_bf16_to_f32(_ptr(x), _ptr(out), x.size)
    return out


def max_threads(lib=None):
    return (lib or load()).oracle_max_threads()


__all__ = ["load", "sweeps", "sweeps_into", "rhs_sweeps", "residual_accumulate", "refine_solve",
           "grad_f64", "f32_to_bf16", "bf16_to_f32", "max_threads"]
