"""GPU parity of the pipelined (wavefront) passes against the CPU oracle, bit for
bit: two-grid passes at every depth, the in-place (one-grid) handle, the ring
sizes at their minimum (R = 3 blocks of one plane, the tightest reuse of a ring
slot), the full 512^3 FP64 workload at t in {2, 4, 8, 16}, and the bounded waits
(a withheld producer ends the call with a timeout status, the handle stays
usable)."""
import os

import numpy as np
import pytest

from tests.helpers import first_diff, make_grid, to_dev, to_host
from tests.test_gpu_sweep import SHAPES, _oracle_512, oracle_sweeps

pytestmark = pytest.mark.gpu

WAVE = 3


@pytest.fixture
def wave_env():
    """Set JACOBI_WAVE (planes per item, ring blocks) for one test."""
    old = os.environ.get("JACOBI_WAVE")

    def set_(v):
        if v is None:
            os.environ.pop("JACOBI_WAVE", None)
        else:
            os.environ["JACOBI_WAVE"] = v

    yield set_
    set_(old)


def run_wave(a, n, t, dtype, nx, inplace=False):
    from paper_0912_4506_gb300 import api
    A = api.as_grid(to_dev(a, dtype), nx)
    j = api.Jacobi(A, inplace=inplace)
    out = j.sweep(n, t, WAVE)
    j.check()
    if inplace:
        assert out is j.A
    res = to_host(out, dtype)
    j.close()
    return res


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "x".join(map(str, s)))
@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16"])
def test_wave_bit_exact_every_depth(shape, dtype, wave_env):
    nx, ny, nz = shape
    a = make_grid(nx, ny, nz, dtype)
    n = 13
    want = oracle_sweeps(a, n, nx, dtype)
    for ring in (None, "1,3", "2,3", "3,4", "1,4", "2,5,3"):
        wave_env(ring)
        for t in (1, 2, 3, 4, 7, 13):
            got = run_wave(a, n, t, dtype, nx)
            assert first_diff(got, want) is None, (ring, t, first_diff(got, want))


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "x".join(map(str, s)))
@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16"])
def test_wave_inplace_bit_exact(shape, dtype, wave_env):
    nx, ny, nz = shape
    a = make_grid(nx, ny, nz, dtype)
    for ring in (None, "1,3", "1,4", "2,5,3"):
        wave_env(ring)
        for n, t in ((2, 2), (3, 2), (5, 2), (13, 3), (13, 4), (9, 9)):
            want = oracle_sweeps(a, n, nx, dtype)
            got = run_wave(a, n, t, dtype, nx, inplace=True)
            assert first_diff(got, want) is None, (ring, n, t, first_diff(got, want))


@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16"])
def test_wave_row_padding_untouched(dtype):
    """NaN in the row padding of the grid is never read nor written, in place or
    not (the rings have their own padding)."""
    from paper_0912_4506_gb300 import api
    nx, ny, nz = 11, 9, 8
    px = {"f64": 16, "f32": 20, "bf16": 24}[dtype]
    a = make_grid(nx, ny, nz, dtype, px=px)
    if dtype == "bf16":
        a[:, :, nx + 2:] = 0x7FC0
    else:
        a[:, :, nx + 2:] = np.nan
    want = oracle_sweeps(a, 6, nx, dtype)
    for inplace in (False, True):
        Af = to_dev(a, dtype)
        j = api.Jacobi(api.as_grid(Af, nx), inplace=inplace)
        out = to_host(j.sweep(6, 3, WAVE), dtype)
        j.check()
        grids = [Af] if inplace else [Af, j.B]
        pads = [to_host(g, dtype) for g in grids]
        j.close()
        assert np.array_equal(out, want), inplace
        pad = pads[0][:, :, nx + 2:]
        assert np.array_equal(pad.view(np.uint8), a[:, :, nx + 2:].view(np.uint8)), inplace


def test_wave_inplace_rejections():
    """In place: depth 1 and a single sweep have no safe schedule; correction and
    adjoint sweeps and a download of B do not exist.  Nothing is launched."""
    from paper_0912_4506_gb300 import _lib, api
    nx = 20
    a = make_grid(nx, 20, 20, "f64")
    j = api.Jacobi(api.as_grid(to_dev(a, "f64"), nx), inplace=True)
    before = to_host(j.A, "f64")
    for call, code in ((lambda: j.sweep(4, 1, WAVE), _lib.JAC_EUNSUPPORTED),
                       (lambda: j.sweep(1, 2, WAVE), _lib.JAC_EUNSUPPORTED),
                       (lambda: j.sweep(4, 2, 2), _lib.JAC_EUNSUPPORTED),
                       (lambda: j.sweep(4, 2, 1), _lib.JAC_EUNSUPPORTED),
                       (lambda: j.plan(1, 2, WAVE), _lib.JAC_EUNSUPPORTED)):
        with pytest.raises(_lib.JacobiError) as ei:
            call()
        assert ei.value.code == code
    import ctypes
    buf = (ctypes.c_double * 8)()
    assert _lib.load().jacobi_download(j._h, ctypes.addressof(buf), 1) == _lib.JAC_EINVAL
    assert np.array_equal(to_host(j.A, "f64"), before)
    assert j.sweep(0, 2, WAVE) is j.A
    j.close()


def test_wave_plan():
    from paper_0912_4506_gb300 import api
    a = make_grid(40, 30, 50, "f32")
    A = api.as_grid(to_dev(a, "f32"), 40)
    j = api.Jacobi(A)
    p = j.plan(10, 4, WAVE)
    assert (p["kernel"], p["t"], p["passes"], p["remainder_t"]) == (WAVE, 4, 3, 2)
    assert p["ext_x"] == p["tile_x"] and p["ext_y"] == p["tile_y"]  # no halo
    assert p["grid_x"] >= 1 and p["kchunk"] >= 1
    assert j.sweep(10, 4, WAVE) is j.B  # three passes A -> B -> A -> B
    j.close()
    ji = api.Jacobi(api.as_grid(to_dev(a, "f32"), 40), inplace=True)
    p = ji.plan(5, 2, 0)  # remainder of one sweep merged into the last pass
    assert (p["kernel"], p["t"], p["passes"], p["remainder_t"]) == (WAVE, 2, 2, 3)
    p = ji.plan(3, 2, 0)
    assert (p["t"], p["passes"]) == (3, 1)
    ji.close()


def test_wave_missing_producer_times_out_and_recovers(monkeypatch):
    """A producer that never posts (the host withholds the first block of update
    1): the bounded waits end the launch with the timeout status; the next call
    on the same handle is correct again."""
    from paper_0912_4506_gb300 import _lib, api
    nx = 40
    a = make_grid(nx, 24, 30, "f32")
    j = api.Jacobi(api.as_grid(to_dev(a, "f32"), nx))
    monkeypatch.setenv("JACOBI_WAVE_TEST_MISSING_PRODUCER", "1")
    j.sweep(4, 4, WAVE)
    with pytest.raises(_lib.JacobiError) as ei:
        j.check()
    assert ei.value.code == _lib.JAC_ETIMEOUT
    monkeypatch.delenv("JACOBI_WAVE_TEST_MISSING_PRODUCER")
    j.A.copy_(api.as_grid(to_dev(a, "f32"), nx))
    out = to_host(j.sweep(4, 4, WAVE), "f32")
    j.check()
    j.close()
    assert first_diff(out, oracle_sweeps(a, 4, nx, "f32")) is None


@pytest.mark.parametrize("t", [2, 4, 8, 16])
def test_full_size_512cubed_fp64_wave(t):
    """512^3 FP64, 100 sweeps in pipelined passes of depth t (16 included: the
    pipelined kernel has no tile-height limit): every cell equals the oracle's."""
    a, want = _oracle_512()
    from paper_0912_4506_gb300 import api
    A = api.as_grid(to_dev(a, "f64"), 512)
    j = api.Jacobi(A)
    plan = j.plan(100, t, WAVE)
    assert plan["kernel"] == WAVE and plan["t"] == t
    assert plan["emu_adds"] == 8
    out = to_host(j.sweep(100, t, WAVE), "f64")
    j.check()
    j.close()
    assert first_diff(out, want) is None, (t, first_diff(out, want))


def test_full_size_512cubed_fp64_inplace():
    """The same workload on ONE grid (half the memory), depth 4: every cell equals
    the oracle's."""
    a, want = _oracle_512()
    from paper_0912_4506_gb300 import api
    A = api.as_grid(to_dev(a, "f64"), 512)
    j = api.Jacobi(A, inplace=True)
    assert j.B is None
    out = to_host(j.sweep(100, 4), "f64")
    j.check()
    j.close()
    assert first_diff(out, want) is None, first_diff(out, want)


@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16"])
def test_wave_alternate_kernels_bit_exact(dtype, monkeypatch):
    """The alternate instantiations of the pipelined kernel (other register caps
    and load depths, chosen with JACOBI_WAVE_VARIANT) give the same bits."""
    for shape in ((37, 29, 23), (130, 47, 9)):
        nx, ny, nz = shape
        a = make_grid(nx, ny, nz, dtype)
        want = oracle_sweeps(a, 11, nx, dtype)
        for v in ("0", "1", "2"):
            monkeypatch.setenv("JACOBI_WAVE_VARIANT", v)
            for ring in ("1,3", "4,4"):
                monkeypatch.setenv("JACOBI_WAVE", ring)
                for t in (1, 3, 11):
                    got = run_wave(a, 11, t, dtype, nx)
                    assert first_diff(got, want) is None, (v, ring, t, first_diff(got, want))
