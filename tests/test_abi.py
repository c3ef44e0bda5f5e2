"""The C ABI library loads and exports every entry point include/jacobi.h declares
(no GPU needed: nothing is called that touches a device)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "jacobi.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(jacobi_[a-z_0-9]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    from paper_0912_4506_gb300 import build, _lib
    build.build()
    return _lib.load()


def test_header_declares_expected(lib):
    decl = _declared()
    assert "jacobi_create" in decl and "jacobi_sweep" in decl and "jacobi_destroy" in decl


def test_every_declared_symbol_exported(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_covers_header():
    from paper_0912_4506_gb300 import _lib
    assert sorted(_lib.EXPORTS) == _declared()


def test_strerror_and_version(lib):
    from paper_0912_4506_gb300 import _lib
    assert lib.jacobi_version() >= 100
    for code in (0, -1, -2, -3, -4, -5):
        assert lib.jacobi_strerror(code)
    assert b"invalid" in lib.jacobi_strerror(_lib.JAC_EINVAL)


def test_create_rejects_bad_arguments_without_device(lib):
    import ctypes
    from paper_0912_4506_gb300 import _lib
    h = ctypes.c_void_p()
    P = ctypes.c_void_p
    # bad shapes / pitch / dtype / pointers are rejected before any CUDA call
    cases = [(0, 4, 4, 0, P(16), P(32), 8), (4, 4, 4, 7, P(16), P(32), 8),
             (4, 4, 4, 0, P(16), P(32), 5), (4, 4, 4, 1, P(16), P(32), 6),
             (4, 4, 4, 0, P(0), P(32), 6), (4, 4, 4, 0, P(16), P(16), 6),
             (4, 4, 4, 0, P(17), P(32), 6)]
    for nx, ny, nz, dt, a, b, pitch in cases:
        rc = lib.jacobi_create(ctypes.byref(h), nx, ny, nz, dt, a, b, pitch, None)
        assert rc == _lib.JAC_EINVAL, (nx, ny, nz, dt, pitch, rc)
    assert lib.jacobi_sweep(None, 1, 0, None) == _lib.JAC_EINVAL
    assert lib.jacobi_destroy(None) == _lib.JAC_OK
    # a two-grid handle needs B; the one-grid handle the same checks on its grid
    assert lib.jacobi_create(ctypes.byref(h), 4, 4, 4, 0, P(16), P(0), 6, None) == _lib.JAC_EINVAL
    for nx, ny, nz, dt, a, pitch in [(0, 4, 4, 0, P(16), 8), (4, 4, 4, 7, P(16), 8),
                                     (4, 4, 4, 0, P(16), 5), (4, 4, 4, 0, P(0), 6),
                                     (4, 4, 4, 0, P(17), 6), (4, 4, 4, 1, P(16), 6)]:
        rc = lib.jacobi_create_inplace(ctypes.byref(h), nx, ny, nz, dt, a, pitch, None)
        assert rc == _lib.JAC_EINVAL, (nx, ny, nz, dt, pitch, rc)
    assert lib.jacobi_create_inplace(None, 4, 4, 4, 0, P(16), 6, None) == _lib.JAC_EINVAL


def test_missing_library_fails_loudly(tmp_path):
    """No CPU fallback: a missing shared library raises at load time."""
    from paper_0912_4506_gb300 import _lib
    with pytest.raises(RuntimeError, match="CUDA library missing"):
        _lib.load(str(tmp_path / "libjacobi_gb300.so"))


def test_max_depth_without_device(lib):
    """The deepest depth per dtype and operation comes from the kernel tables (no
    device call): every depth from 1 up to it exists."""
    from paper_0912_4506_gb300 import _lib
    want = {(_lib.JAC_F64, _lib.JAC_OP_SWEEP): 8, (_lib.JAC_F32, _lib.JAC_OP_SWEEP): 8,
            (_lib.JAC_BF16, _lib.JAC_OP_SWEEP): 8, (_lib.JAC_F32, _lib.JAC_OP_RHS): 6,
            (_lib.JAC_BF16, _lib.JAC_OP_RHS): 6, (_lib.JAC_F64, _lib.JAC_OP_RHS): 0,
            (_lib.JAC_F32, _lib.JAC_OP_ADJOINT): 8, (_lib.JAC_F64, _lib.JAC_OP_ADJOINT): 8,
            (_lib.JAC_BF16, _lib.JAC_OP_ADJOINT): 0}
    for (dt, op), mt in want.items():
        assert lib.jacobi_max_depth(dt, op) == mt, (dt, op)
    assert lib.jacobi_max_depth(3, 0) == _lib.JAC_EINVAL
    assert lib.jacobi_max_depth(0, 3) == _lib.JAC_EINVAL
