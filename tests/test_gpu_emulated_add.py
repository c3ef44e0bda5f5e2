"""The integer-pipe FP64 addition used by the plain FP64 sweep equals the FP64
unit (IEEE-754 round-to-nearest-even) bit for bit, on random pairs across
exponent differences 0..40 and on constructed ties, carries and boundaries;
and the sweep with it stays bit-exact, also when negative values force the
FP64-unit path."""
import numpy as np
import pytest

import oracle
from tests.helpers import make_grid, to_dev, to_host

pytestmark = pytest.mark.gpu


def _gpu_add(a, b):
    import torch
    from paper_0912_4506_gb300 import _lib
    ta = torch.from_numpy(a).cuda()
    tb = torch.from_numpy(b).cuda()
    out = torch.empty_like(ta)
    _lib.jacobi_emulated_add(ta.data_ptr(), tb.data_ptr(), out.data_ptr(), a.size,
                             torch.cuda.current_stream().cuda_stream)
    return out.cpu().numpy()


def _bits(x):
    return x.view(np.uint64)


def test_random_pairs_all_exponent_gaps():
    rng = np.random.default_rng(0)
    n = 4_000_000
    m1 = rng.integers(0, 1 << 52, n, dtype=np.uint64)
    m2 = rng.integers(0, 1 << 52, n, dtype=np.uint64)
    e1 = rng.integers(900, 1100, n, dtype=np.uint64)
    gap = rng.integers(0, 41, n, dtype=np.uint64)
    e2 = e1 - np.minimum(gap, e1 - 1)
    a = ((e1 << np.uint64(52)) | m1).view(np.float64)
    b = ((e2 << np.uint64(52)) | m2).view(np.float64)
    swap = rng.random(n) < 0.5
    a, b = np.where(swap, b, a), np.where(swap, a, b)
    got = _gpu_add(a, b)
    want = a + b
    assert np.array_equal(_bits(got), _bits(want))


def test_constructed_edge_cases():
    cases = []
    one = 1.0
    ulp = 2.0 ** -52
    for k in range(0, 60):
        h = 2.0 ** -k
        cases += [(one, h), (one + ulp, h), (2 - ulp, h), (2 - ulp, 2 - ulp), (one, h * (1 + ulp)),
                  (one + 3 * ulp, h), (1.5, h * 1.5), (np.nextafter(2.0, 0), h)]
    # exact ties at every shift within the integer path
    for d in range(1, 32):
        cases.append((1.0 + ulp, 2.0 ** (-52 - 1)))          # half ulp: tie to even
        cases.append((1.0, 2.0 ** (-52 - 1) * (1 + 2.0 ** -(d % 40))))
    cases += [(3.0, 5.0), (0.75, 0.25), (1e-300, 1e-300), (1e300, 1e300), (6.0, 2.0 ** -30)]
    a = np.array([c[0] for c in cases] + [c[1] for c in cases])
    b = np.array([c[1] for c in cases] + [c[0] for c in cases])
    got = _gpu_add(a, b)
    assert np.array_equal(_bits(got), _bits(a + b))


def test_uniform_unit_interval_sums():
    rng = np.random.default_rng(1)
    n = 2_000_000
    s = np.zeros(n)
    terms = rng.random((6, n))
    for t in terms:  # the partial sums of Eq. 1 on U[0,1) data
        got = _gpu_add(np.where(s == 0, t, s), np.where(s == 0, 0.5, t))
        want = np.where(s == 0, t, s) + np.where(s == 0, 0.5, t)
        assert np.array_equal(_bits(got), _bits(want))
        s = want


def test_sweep_with_negative_values_uses_fp64_unit_and_stays_exact():
    from paper_0912_4506_gb300 import api, inputs
    nx, ny, nz = 40, 33, 21
    u0 = inputs.laplace_boundary_f64(nx, ny, nz, px=inputs.row_pitch(nx, "f64"))
    u0[1:-1, 1:-1, 1:nx + 1] = np.random.default_rng(2).random((nz, ny, nx)) - 0.5
    j = api.Jacobi(api.as_grid(to_dev(u0, "f64"), nx))
    got = to_host(j.sweep(9, 1, api.JAC_KERNEL_PLAIN), "f64")
    j.close()
    assert np.array_equal(got, oracle.sweeps(u0, 9, nx=nx)[:, :, :nx + 2])


def _gpu_sum6(x):
    import torch
    from paper_0912_4506_gb300 import _lib
    n = x.shape[1]
    tx = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    _lib.jacobi_emulated_sum6(tx.data_ptr(), out.data_ptr(), n,
                              torch.cuda.current_stream().cuda_stream)
    return out.cpu().numpy()


def _host_sum6(x):
    s = x[0] + x[1]
    for j in range(2, 6):
        s = s + x[j]
    return s


def test_accumulator_sum6_random_tuples():
    """The unpacked running sum of the FP64 sweeps equals the sequential FP64 sum
    bit for bit: smooth fields (fast path), U[0,1) data, exponent gaps up to 12,
    significands with long runs of trailing zeros (rounding ties) and, mixed in,
    zeros, negatives and subnormals (FP64-unit path)."""
    rng = np.random.default_rng(21)
    n = 1 << 20
    cases = []
    cases.append(0.5 + 0.01 * rng.random((6, n)))
    cases.append(rng.random((6, n)))
    cases.append(np.ldexp(1.0 + rng.random((6, n)), -rng.integers(0, 13, (6, n))))
    m = rng.integers(0, 1 << 52, (6, n), dtype=np.uint64)
    tz = rng.integers(0, 53, (6, n)).astype(np.uint64)
    m = (m >> tz) << tz
    e = (1023 - rng.integers(0, 6, (6, n))).astype(np.uint64)
    cases.append(((e << np.uint64(52)) | m).view(np.float64))
    mixed = rng.random((6, n))
    pick = rng.random((6, n))
    mixed[pick < 0.001] = 0.0
    mixed[(pick >= 0.001) & (pick < 0.002)] *= -1.0
    mixed[(pick >= 0.002) & (pick < 0.003)] = 1e-310
    cases.append(mixed)
    for x in cases:
        got = _gpu_sum6(x)
        assert np.array_equal(_bits(got), _bits(_host_sum6(x)))


def test_accumulator_sum6_rounding_carries_and_ties():
    """Hand cases: carries into a new binade at every addition, sums landing
    exactly half-way between doubles (ties to even both ways), R reaching 2^53."""
    ulp = 2.0 ** -52
    rows = [
        [1.0, 1.0, 2.0, 4.0, 8.0, 16.0],
        [2 - ulp, 2 - ulp, 4 - 2 * ulp, 8 - 4 * ulp, 16 - 8 * ulp, 32 - 16 * ulp],
        [1.0, ulp / 2 * 3, 1.0, 1.0, 1.0, 1.0],
        [1.0 + ulp, 1.0, 2.0 ** -9, 2.0 ** -9 * (1 + ulp), 0.75, 0.75],
        [1.5, 1.5 + ulp, 3 * ulp, 6.0 - 4 * ulp, 0.5 + ulp, 2.0 ** -8],
        [0.3, 0.7, 0.1, 0.9, 0.2, 0.8],
    ]
    x = np.array(rows, dtype=np.float64).T.copy()
    x = np.tile(x, (1, 64))  # several full warps
    got = _gpu_sum6(x)
    assert np.array_equal(_bits(got), _bits(_host_sum6(x)))


def _wide_range_grid(nx, ny, nz, seed):
    """Positive normal values spread over 2^-60 .. 1 (log-uniform): the range
    check passes, and many additions meet exponent gaps above 31, which the
    integer path hands to the FP64 unit lane by lane."""
    from paper_0912_4506_gb300 import inputs
    px = inputs.row_pitch(nx, "f64")
    rng = np.random.default_rng(seed)
    a = np.zeros((nz + 2, ny + 2, px))
    a[:, :, :nx + 2] = 2.0 ** (-60.0 * rng.random((nz + 2, ny + 2, nx + 2)))
    return a


@pytest.mark.parametrize("t", [1, 2, 3, 4, 5, 6, 7, 8])
def test_blocked_fp64_integer_pipe_adds_every_depth(t):
    """FP64 blocked passes with 3 of the 5 additions on the integer pipes: bit-exact
    at every depth on uniform data and on data with a wide exponent range."""
    from paper_0912_4506_gb300 import api
    for a, nx in ((make_grid(70, 45, 23, "f64"), 70), (_wide_range_grid(53, 40, 19, 4), 53)):
        j = api.Jacobi(api.as_grid(to_dev(a, "f64"), nx))
        assert j.plan(11, t, api.JAC_KERNEL_TB)["emu_adds"] == 8  # 4 of 5 additions
        got = to_host(j.sweep(11, t, api.JAC_KERNEL_TB), "f64")
        j.check()
        j.close()
        want = oracle.sweeps(a, 11, nx=nx)[:, :, :nx + 2]
        assert np.array_equal(got, want), t


def test_blocked_fp64_zero_and_negative_values_use_fp64_unit():
    """Values outside [2^-1000, 2^1000] (zeros, negatives) fail the range check, so
    the blocked FP64 pass keeps every addition on the FP64 unit: still bit-exact."""
    from paper_0912_4506_gb300 import api, inputs
    nx, ny, nz = 40, 33, 21
    u0 = inputs.laplace_boundary_f64(nx, ny, nz, px=inputs.row_pitch(nx, "f64"))
    u0[1:-1, 1:-1, 1:nx + 1] = np.random.default_rng(3).random((nz, ny, nx)) - 0.5
    for t in (2, 4, 8):
        j = api.Jacobi(api.as_grid(to_dev(u0, "f64"), nx))
        got = to_host(j.sweep(9, t, api.JAC_KERNEL_TB), "f64")
        j.close()
        assert np.array_equal(got, oracle.sweeps(u0, 9, nx=nx)[:, :, :nx + 2]), t


@pytest.mark.parametrize("nemu", [0, 6, 19, 20, 21, 44, 52, 76])
def test_every_emulation_split_bit_exact(nemu, monkeypatch):
    """Run each split in a fresh process (the split is read once per process)."""
    import subprocess
    import sys
    import os
    code = (
        "import sys; sys.path.insert(0, %r)\n"
        "import numpy as np, oracle\n"
        "from paper_0912_4506_gb300 import api\n"
        "from tests.helpers import make_grid, to_dev, to_host\n"
        "a = make_grid(77, 45, 30, 'f64')\n"
        "j = api.Jacobi(api.as_grid(to_dev(a, 'f64'), 77))\n"
        "assert j.plan(5, 1, api.JAC_KERNEL_PLAIN)['emu_adds'] == %d\n"
        "got = to_host(j.sweep(5, 1, api.JAC_KERNEL_PLAIN), 'f64')\n"
        "assert np.array_equal(got, oracle.sweeps(a, 5, nx=77)[:, :, :79])\n"
        "print('ok')\n" % (os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                            2 * ((nemu - 16) % 8) if nemu >= 16 else nemu))
    env = dict(os.environ, JACOBI_F64_EMU=str(nemu))
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0 and "ok" in r.stdout, r.stderr[-3000:]
