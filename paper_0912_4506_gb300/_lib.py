"""ctypes binding of libjacobi_gb300.so: the C ABI of include/jacobi.h, one
Python function per C entry point with the same name.  Argument marshalling
only; every step of the computation runs in the library's CUDA kernels.  There
is no fallback: a missing library raises."""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libjacobi_gb300.so")

JAC_OK, JAC_EINVAL, JAC_ENOMEM, JAC_ECUDA, JAC_ETIMEOUT, JAC_EUNSUPPORTED = 0, -1, -2, -3, -4, -5
JAC_F64, JAC_F32, JAC_BF16 = 0, 1, 2
JAC_KERNEL_AUTO, JAC_KERNEL_PLAIN, JAC_KERNEL_TB, JAC_KERNEL_WAVE = 0, 1, 2, 3
JAC_OP_SWEEP, JAC_OP_RHS, JAC_OP_ADJOINT = 0, 1, 2
JAC_PROBE_DADD, JAC_PROBE_FADD, JAC_PROBE_LOP3, JAC_PROBE_IMAD, JAC_PROBE_EMU_ADD = 0, 1, 2, 3, 4
JAC_PROBE_ACC_ADD = 5
JAC_PROBE_CHAINS = 8

EXPORTS = ["jacobi_create", "jacobi_sweep", "jacobi_sweep_ex", "jacobi_plan",
           "jacobi_sweep_rhs", "jacobi_residual_accumulate", "jacobi_adjoint",
           "jacobi_upload", "jacobi_download", "jacobi_check", "jacobi_destroy",
           "jacobi_strerror", "jacobi_version", "jacobi_sweep_noalloc",
           "jacobi_batch_create", "jacobi_batch_run", "jacobi_batch_info", "jacobi_batch_check",
           "jacobi_batch_destroy", "jacobi_emulated_add", "jacobi_copy_planes",
           "jacobi_max_depth", "jacobi_pipe_probe", "jacobi_emulated_sum6",
           "jacobi_create_inplace"]

JAC_BATCH_NO_GRAPH, JAC_BATCH_TEST_MISSING_PRODUCER = 1, 2


class JacobiError(RuntimeError):
    def __init__(self, code, what=""):
        self.code = code
        msg = _strerror(code) if _lib is not None else str(code)
        super().__init__(f"{what}: {msg} ({code})" if what else f"{msg} ({code})")


class PlanInfo(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int) for n in (
        "kernel", "t", "passes", "remainder_t", "tile_x", "tile_y", "ext_x", "ext_y",
        "kchunk", "threads", "smem_bytes", "grid_x", "grid_y", "grid_z", "emu_adds")]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


_lib = None


def load(path=None):
    """Load the library (no build step here: see paper_0912_4506_gb300.build)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"CUDA library missing: {p} (run __graft_entry__.build())")
    lib = ctypes.CDLL(p)
    P, I, LL = ctypes.c_void_p, ctypes.c_int, ctypes.c_longlong
    PI = ctypes.POINTER(ctypes.c_int)
    sig = {
        "jacobi_create": ([ctypes.POINTER(P), I, I, I, I, P, P, LL, P], I),
        "jacobi_create_inplace": ([ctypes.POINTER(P), I, I, I, I, P, LL, P], I),
        "jacobi_sweep": ([P, I, I, PI], I),
        "jacobi_sweep_ex": ([P, I, I, I, PI], I),
        "jacobi_plan": ([P, I, I, I, ctypes.POINTER(PlanInfo)], I),
        "jacobi_sweep_rhs": ([P, P, I, I, PI], I),
        "jacobi_residual_accumulate": ([I, I, I, P, P, LL, P, P, I, LL, P], I),
        "jacobi_adjoint": ([P, P, I, I, PI], I),
        "jacobi_upload": ([P, P], I),
        "jacobi_download": ([P, P, I], I),
        "jacobi_check": ([P], I),
        "jacobi_destroy": ([P], I),
        "jacobi_strerror": ([I], ctypes.c_char_p),
        "jacobi_version": ([], I),
        "jacobi_sweep_noalloc": ([I, I, I, I, P, LL, I, I, P, I], I),
        "jacobi_batch_create": ([ctypes.POINTER(P), I, PI, ctypes.POINTER(LL), ctypes.POINTER(P),
                                 ctypes.POINTER(P), PI, PI, PI, PI, I, P, I, ctypes.c_double], I),
        "jacobi_batch_run": ([P, PI], I),
        "jacobi_batch_info": ([P, PI, PI, PI, PI, PI], I),
        "jacobi_batch_check": ([P], I),
        "jacobi_batch_destroy": ([P], I),
        "jacobi_emulated_add": ([P, P, P, LL, P], I),
        "jacobi_copy_planes": ([P, P, LL, I, I, P], I),
        "jacobi_max_depth": ([I, I], I),
        "jacobi_emulated_sum6": ([P, P, LL, P], I),
        "jacobi_pipe_probe": ([I, P, I, I, I, P], I),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    if path is None:
        _lib = lib
    return lib


def _strerror(code):
    return _lib.jacobi_strerror(code).decode()


def _ck(rc, what):
    if rc != JAC_OK:
        raise JacobiError(rc, what)


def jacobi_create(nx, ny, nz, dtype, grid_a, grid_b, row_pitch, stream):
    h = ctypes.c_void_p()
    _ck(load().jacobi_create(ctypes.byref(h), nx, ny, nz, dtype, grid_a, grid_b, row_pitch,
                             stream), "jacobi_create")
    return h


def jacobi_create_inplace(nx, ny, nz, dtype, grid, row_pitch, stream):
    h = ctypes.c_void_p()
    _ck(load().jacobi_create_inplace(ctypes.byref(h), nx, ny, nz, dtype, grid, row_pitch,
                                     stream), "jacobi_create_inplace")
    return h


def jacobi_sweep(h, nsweeps, t=0):
    fb = ctypes.c_int(0)
    _ck(load().jacobi_sweep(h, nsweeps, t, ctypes.byref(fb)), "jacobi_sweep")
    return fb.value


def jacobi_sweep_ex(h, nsweeps, t, kernel):
    fb = ctypes.c_int(0)
    _ck(load().jacobi_sweep_ex(h, nsweeps, t, kernel, ctypes.byref(fb)), "jacobi_sweep_ex")
    return fb.value


def jacobi_plan(h, nsweeps, t=0, kernel=JAC_KERNEL_AUTO):
    info = PlanInfo()
    _ck(load().jacobi_plan(h, nsweeps, t, kernel, ctypes.byref(info)), "jacobi_plan")
    return info.as_dict()


def jacobi_sweep_rhs(h, rho, nsweeps, t=0):
    fb = ctypes.c_int(0)
    _ck(load().jacobi_sweep_rhs(h, rho, nsweeps, t, ctypes.byref(fb)), "jacobi_sweep_rhs")
    return fb.value


def jacobi_residual_accumulate(nx, ny, nz, u_in, u_out, u_pitch, e, rho, lo_dtype, lo_pitch,
                               stream):
    _ck(load().jacobi_residual_accumulate(nx, ny, nz, u_in, u_out, u_pitch, e, rho, lo_dtype,
                                          lo_pitch, stream), "jacobi_residual_accumulate")


def jacobi_adjoint(h, grad_bdry, nsweeps, t=0):
    fb = ctypes.c_int(0)
    _ck(load().jacobi_adjoint(h, grad_bdry, nsweeps, t, ctypes.byref(fb)), "jacobi_adjoint")
    return fb.value


def jacobi_upload(h, host_ptr):
    _ck(load().jacobi_upload(h, host_ptr), "jacobi_upload")


def jacobi_download(h, host_ptr, from_b):
    _ck(load().jacobi_download(h, host_ptr, from_b), "jacobi_download")


def jacobi_check(h):
    _ck(load().jacobi_check(h), "jacobi_check")


def jacobi_destroy(h):
    _ck(load().jacobi_destroy(h), "jacobi_destroy")


def jacobi_max_depth(dtype, op=JAC_OP_SWEEP):
    rc = load().jacobi_max_depth(dtype, op)
    if rc < 0:
        raise JacobiError(rc, "jacobi_max_depth")
    return rc


def jacobi_pipe_probe(kind, out_ptr, blocks, threads, iters, stream):
    _ck(load().jacobi_pipe_probe(kind, out_ptr, blocks, threads, iters, stream),
        "jacobi_pipe_probe")


def jacobi_version():
    return load().jacobi_version()


def jacobi_sweep_noalloc(nx, ny, nz, dtype, grid, row_pitch, nsweeps, t, stream, sync):
    """Sweep that allocates nothing (the library's static scratch holds the second
    grid); the result is left in ``grid``."""
    _ck(load().jacobi_sweep_noalloc(nx, ny, nz, dtype, grid, row_pitch, nsweeps, t, stream,
                                    sync), "jacobi_sweep_noalloc")


def _ints(v):
    return (ctypes.c_int * len(v))(*v)


def jacobi_batch_create(dims, pitches, grids_a, grids_b, nsweeps, t, nchunk, dtype, stream,
                        flags=0, wait_limit_s=0.0, tile_x=None):
    """dims: list of (nx, ny, nz); the other lists have one entry per grid."""
    n = len(dims)
    h = ctypes.c_void_p()
    flat = [int(x) for d in dims for x in d]
    P = ctypes.c_void_p
    rc = load().jacobi_batch_create(
        ctypes.byref(h), n, _ints(flat), (ctypes.c_longlong * n)(*pitches),
        (P * n)(*grids_a), (P * n)(*grids_b), _ints(nsweeps),
        _ints(t) if t is not None else None, _ints(tile_x) if tile_x is not None else None,
        _ints(nchunk) if nchunk is not None else None, dtype, stream, flags, float(wait_limit_s))
    _ck(rc, "jacobi_batch_create")
    return h


def jacobi_batch_run(h, count):
    fb = (ctypes.c_int * count)()
    _ck(load().jacobi_batch_run(h, fb), "jacobi_batch_run")
    return list(fb)


def jacobi_batch_info(h, count):
    t = (ctypes.c_int * count)()
    tx = (ctypes.c_int * count)()
    p = (ctypes.c_int * count)()
    items = ctypes.c_int(0)
    ctas = ctypes.c_int(0)
    _ck(load().jacobi_batch_info(h, t, tx, p, ctypes.byref(items), ctypes.byref(ctas)),
        "jacobi_batch_info")
    return {"t": list(t), "tile_x": list(tx), "passes": list(p), "items": items.value,
            "ctas": ctas.value}


def jacobi_batch_check(h):
    _ck(load().jacobi_batch_check(h), "jacobi_batch_check")


def jacobi_batch_destroy(h):
    _ck(load().jacobi_batch_destroy(h), "jacobi_batch_destroy")


def jacobi_emulated_add(a_ptr, b_ptr, out_ptr, n, stream):
    _ck(load().jacobi_emulated_add(a_ptr, b_ptr, out_ptr, n, stream), "jacobi_emulated_add")


def jacobi_emulated_sum6(x_ptr, out_ptr, n, stream):
    _ck(load().jacobi_emulated_sum6(x_ptr, out_ptr, n, stream), "jacobi_emulated_sum6")


def jacobi_copy_planes(dst_ptr, src_ptr, plane_elems, elem_bytes, nplanes, stream):
    _ck(load().jacobi_copy_planes(dst_ptr, src_ptr, plane_elems, elem_bytes, nplanes, stream),
        "jacobi_copy_planes")
