"""Pins for the CPU oracle: facts fixed by the paper and by mathematics, not by
the oracle itself.  Each ``pin_*`` takes a loaded oracle library and raises
AssertionError when the oracle disagrees.  ``test_oracle.py`` runs them on the
real oracle; ``test_oracle_mutations.py`` runs them on copies of the oracle with a
planted mistake and checks that at least one pin fails.
"""
import math
import os

import numpy as np

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
C64 = float.fromhex("0x1.5555555555555p-3")
ULP1 = 2.0 ** -52
HALF = 2.0 ** -53


def _padded(nx, ny, nz, px=None, dtype=np.float64):
    px = nx + 2 if px is None else px
    return np.zeros((nz + 2, ny + 2, px), dtype=dtype)


def pin_hand_4cubed(lib):
    """Eq. 1 on the hand-derived 4^3 case of tests/golden/hand_4cubed.txt."""
    A = _padded(4, 4, 4)
    A[:, :, 0] = 6.0
    expect = {1: {}, 2: {}}
    with open(os.path.join(GOLDEN, "hand_4cubed.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            s, i, j, k, v = line.split()
            expect[int(s)][(int(i), int(j), int(k))] = float.fromhex(v)
    for s in (1, 2):
        out = oracle.sweeps(A, s, lib=lib)
        for k in range(1, 5):
            for j in range(1, 5):
                for i in range(1, 5):
                    want = expect[s].get((i, j, k), 0.0)
                    got = out[k, j, i]
                    assert got == want, (s, i, j, k, got.hex(), want.hex())
        # boundary untouched
        assert np.array_equal(out[:, :, 0], A[:, :, 0])


def pin_sum_order(lib):
    """Eq. 1's operand order i-1, i+1, j-1, j+1, k-1, k+1, summed left to right.

    Neighbours hold (h, h, 1) at three consecutive operand positions and 0
    elsewhere, h = 2^-53 (half an ulp of 1).  Left to right: h + h = 2^-52 exactly,
    then 1 + 2^-52 exactly.  Any order that adds the 1 before either h gives
    1 + h -> 1 (tie to even) and loses both.  So the centre becomes
    RN((1 + 2^-52) * c) exactly when the order is the paper's.
    """
    offs = [(-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0), (0, 0, -1), (0, 0, 1)]
    want = (1.0 + ULP1) * C64
    for start in range(4):
        A = _padded(3, 3, 3)
        for pos, val in zip(range(start, start + 3), (HALF, HALF, 1.0)):
            di, dj, dk = offs[pos]
            A[2 + dk, 2 + dj, 2 + di] = val
        out = oracle.sweeps(A, 1, lib=lib)
        assert out[2, 2, 2] == want, (start, out[2, 2, 2].hex(), want.hex())


def _harmonic_fields(nx, ny, nz):
    k, j, i = np.meshgrid(np.arange(nz + 2), np.arange(ny + 2), np.arange(nx + 2),
                          indexing="ij")
    i, j, k = (x.astype(np.float64) for x in (i, j, k))
    return [3.0 + 2.0 * i - j + 5.0 * k, i * i - j * j, i * j - 4.0 * k,
            i * i - k * k + 2.0 * j, j * j - k * k - 3.0 * i,
            i * i - j * j + 0.5 * k]


def pin_harmonic_fixed_points(lib):
    """Discrete-harmonic fields (linear, x^2-y^2, xy, x^2-z^2, ...) satisfy
    sum6(u) = 6u exactly in small-integer arithmetic, and RN(6u * RN(1/6)) = u
    for every u with 6u exact, so each sweep leaves them unchanged bit for bit
    (f64 and f32; bf16 on fields whose values are bf16-exact)."""
    nx, ny, nz = 7, 6, 5
    for u in _harmonic_fields(nx, ny, nz):
        out = oracle.sweeps(u, 3, nx=nx, dtype="f64", lib=lib)
        assert np.array_equal(out, u)
        u32 = u.astype(np.float32)
        out32 = oracle.sweeps(u32, 3, nx=nx, dtype="f32", lib=lib)
        assert np.array_equal(out32, u32)
    u = _harmonic_fields(nx, ny, nz)[1]  # |u| <= 64, integers: bf16-exact
    ub = oracle.f32_to_bf16(u.astype(np.float32), lib=lib)
    outb = oracle.sweeps(ub, 3, nx=nx, dtype="bf16", lib=lib)
    assert np.array_equal(outb, ub)


def pin_sine_modes(lib):
    """u = sin(p pi i/(N+1)) sin(q pi j/(M+1)) sin(r pi k/(L+1)) with a zero
    boundary is an eigenvector of the sweep: one sweep multiplies it by
    (cos(p pi/(N+1)) + cos(q pi/(M+1)) + cos(r pi/(L+1))) / 3
    (from sin(a(i-1)) + sin(a(i+1)) = 2 sin(ai) cos a).  Non-cubic, padded rows."""
    nx, ny, nz, px = 9, 7, 5, 12
    for (p, q, r) in ((1, 1, 1), (1, 2, 3), (4, 1, 2), (9, 7, 5)):
        k, j, i = np.meshgrid(np.arange(nz + 2), np.arange(ny + 2),
                              np.arange(nx + 2), indexing="ij")
        u = (np.sin(p * math.pi * i / (nx + 1)) * np.sin(q * math.pi * j / (ny + 1))
             * np.sin(r * math.pi * k / (nz + 1)))
        bnd = (i == 0) | (i == nx + 1) | (j == 0) | (j == ny + 1) | (k == 0) | (k == nz + 1)
        u[bnd] = 0.0
        A = _padded(nx, ny, nz, px)
        A[:, :, :nx + 2] = u
        lam = (math.cos(p * math.pi / (nx + 1)) + math.cos(q * math.pi / (ny + 1))
               + math.cos(r * math.pi / (nz + 1))) / 3.0
        n = 10
        out = oracle.sweeps(A, n, nx=nx, lib=lib)
        err = np.abs(out[:, :, :nx + 2] - (lam ** n) * u).max()
        assert err <= 8 * n * 2.0 ** -53, (p, q, r, err)
        assert np.all(out[:, :, nx + 2:] == 0.0)
        out32 = oracle.sweeps(A.astype(np.float32), n, nx=nx, dtype="f32", lib=lib)
        err32 = np.abs(out32[:, :, :nx + 2].astype(np.float64) - (lam ** n) * u).max()
        assert err32 <= 8 * (n + 1) * 2.0 ** -24, (p, q, r, err32)


def pin_bf16_conversion(lib):
    """bf16 storage rounding = round-to-nearest-even on the upper 16 bits of a
    binary32: hand cases at ties, and agreement with torch's conversion."""
    cases = {1.0 + 2.0 ** -8: 0x3F80, 1.0 + 3 * 2.0 ** -8: 0x3F82,
             1.0 + 2.0 ** -8 + 2.0 ** -20: 0x3F81, -2.5: 0xC020, 0.0: 0x0000}
    x = np.array(list(cases), dtype=np.float32)
    got = oracle.f32_to_bf16(x, lib=lib)
    assert [int(v) for v in got] == list(cases.values())
    import torch
    rng = np.random.default_rng(5)
    y = (rng.standard_normal(20000) * 10.0 ** rng.integers(-8, 8, 20000)).astype(np.float32)
    ref = torch.from_numpy(y).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    assert np.array_equal(oracle.f32_to_bf16(y, lib=lib), ref)
    back = oracle.bf16_to_f32(ref, lib=lib)
    assert np.array_equal(back, torch.from_numpy(ref.view(np.int16)).view(torch.bfloat16)
                          .float().numpy())


def pin_bf16_sweep_is_rounded_f32(lib):
    """One bf16 sweep = one f32 sweep of the same (bf16-exact) values, rounded to
    bf16 once (the reading: f32 arithmetic, bf16 storage after every sweep)."""
    rng = np.random.default_rng(11)
    nx, ny, nz = 6, 5, 4
    a = rng.random((nz + 2, ny + 2, nx + 2)).astype(np.float32)
    ab = oracle.f32_to_bf16(a, lib=lib)
    a_exact = oracle.bf16_to_f32(ab, lib=lib)
    one32 = oracle.sweeps(a_exact, 1, dtype="f32", lib=lib)
    oneb = oracle.sweeps(ab, 1, dtype="bf16", lib=lib)
    assert np.array_equal(oneb, oracle.f32_to_bf16(one32, lib=lib))


def pin_residual(lib):
    """rho = s(u) - 6u: zero on a harmonic integer field, exactly 2 on u = x^2
    (sum of the six neighbours of x^2 is 6x^2 + 2); u += e adds e on the interior
    only."""
    nx, ny, nz = 6, 5, 4
    k, j, i = np.meshgrid(np.arange(nz + 2), np.arange(ny + 2), np.arange(nx + 2),
                          indexing="ij")
    interior = ((i >= 1) & (i <= nx) & (j >= 1) & (j <= ny) & (k >= 1) & (k <= nz))
    h = (i * i - j * j + 3.0 * k).astype(np.float64)
    for dt in ("f64", "f32", "bf16"):
        e = np.zeros(h.shape, dtype={"f64": np.float64, "f32": np.float32,
                                     "bf16": np.uint16}[dt])
        u1, rho = oracle.residual_accumulate(h, e, dtype=dt, lib=lib)
        assert np.array_equal(u1, h)
        assert np.all(rho == 0)
    q = (i * i).astype(np.float64)
    u1, rho = oracle.residual_accumulate(q, np.zeros(q.shape, np.float32), lib=lib)
    assert np.all(rho[interior] == 2.0) and np.all(rho[~interior] == 0)
    e = np.where(interior, 0.25, 7.0).astype(np.float32)
    u1, rho = oracle.residual_accumulate(q, e, lib=lib)
    assert np.array_equal(u1, np.where(interior, q + 0.25, q))
    # a constant shift of the interior by 0.25 leaves the x^2 part (2) and adds
    # -0.25 for each boundary neighbour: face cells see fewer interior neighbours
    nb = ((i == 1).astype(float) + (i == nx) + (j == 1) + (j == ny) + (k == 1)
          + (k == nz))
    assert np.array_equal(rho[interior], (2.0 - 0.25 * nb)[interior].astype(np.float32))


def pin_rhs_sweep(lib):
    """The correction sweep with rho = 0 is the plain sweep on a zero-boundary
    grid; with e = 0 and rho = 6 it gives RN(6 * RN(1/6)) = 1 in the interior."""
    rng = np.random.default_rng(3)
    nx, ny, nz = 5, 6, 4
    e = rng.random((nz + 2, ny + 2, nx + 2))
    e[0], e[-1], e[:, 0], e[:, -1], e[:, :, 0], e[:, :, -1] = 0, 0, 0, 0, 0, 0
    for dt, conv in (("f64", np.float64), ("f32", np.float32)):
        a = e.astype(conv)
        got = oracle.rhs_sweeps(a, np.zeros_like(a), 3, dtype=dt, lib=lib)
        assert np.array_equal(got, oracle.sweeps(a, 3, dtype=dt, lib=lib))
        z = np.zeros_like(a)
        six = np.full_like(a, 6.0)
        got = oracle.rhs_sweeps(z, six, 1, dtype=dt, lib=lib)
        assert np.all(got[1:-1, 1:-1, 1:-1] == 1.0) and got[0].sum() == 0


def pin_rhs_sweep_bf16(lib):
    """bf16 correction sweep, values derived by hand (c32 = RN32(1/6) =
    0x1.555556p-3, so 6*c32 = 1 + 2^-25 exactly):
      * e = 0, rho = 6: (0 + 6) * c32 = 1 + 2^-25 -> RN32 1 -> bf16 1.0 (0x3F80);
      * e = 6 at the i-1 neighbour of the centre of a 3^3 interior (zero
        elsewhere), rho = 18 * 2^-8 (bf16-exact): the sum is 6 + 18 * 2^-8 exactly,
        times c32 is (1 + 3 * 2^-8)(1 + 2^-25) -> RN32 1 + 3 * 2^-8, which lies
        half-way between the bf16 values 1 + 2^-7 (0x3F81, odd) and 1 + 2^-6
        (0x3F82, even): nearest-even gives 0x3F82.  Without rho the centre would
        be RN(6 * c32) = 1.0 (0x3F80); truncation would give 0x3F81.
    """
    z = np.zeros((5, 5, 5), dtype=np.uint16)
    six = np.full_like(z, 0x40C0)  # 6.0
    got = oracle.rhs_sweeps(z, six, 1, dtype="bf16", lib=lib)
    assert np.all(got[1:-1, 1:-1, 1:-1] == 0x3F80), got[2, 2, 2]
    assert np.all(got[0] == 0) and np.all(got[:, :, 0] == 0)
    e = np.zeros((5, 5, 5), dtype=np.uint16)
    e[2, 2, 1] = 0x40C0          # 6.0 at (i, j, k) = (1, 2, 2)
    rho = np.zeros_like(e)
    rho[2, 2, 2] = 0x3D90        # 18 * 2^-8 = 1.125 * 2^-4 at the centre
    assert float(oracle.bf16_to_f32(rho[2, 2, 2:3], lib=lib)[0]) == 18 * 2.0 ** -8
    got = oracle.rhs_sweeps(e, rho, 1, dtype="bf16", lib=lib)
    assert int(got[2, 2, 2]) == 0x3F82, hex(int(got[2, 2, 2]))
    # the cell at (2, 2, 2)'s i+1 side sees only its own zero neighbours and rho 0
    assert int(got[2, 2, 3]) == 0


def pin_residual_bf16_store(lib):
    """The bf16 residual store: rho = s(u) - 6u is exactly 2a on u = a * x^2
    (x the padded i index), so choosing a puts the residual on or next to a bf16
    rounding tie (the value is exact in FP64 and FP32, so only the bf16 rounding
    acts):  2a = 1 + 2^-8 is the tie between 0x3F80 and 0x3F81 -> 0x3F80 (even);
    2a = 1 + 3 * 2^-8 ties between 0x3F81 and 0x3F82 -> 0x3F82 (even);
    2a = 1 + 2^-8 + 2^-20 lies just above a tie -> 0x3F81.  A bf16 correction e
    is widened exactly and added on the interior only."""
    nx, ny, nz = 5, 4, 3
    k, j, i = np.meshgrid(np.arange(nz + 2), np.arange(ny + 2), np.arange(nx + 2),
                          indexing="ij")
    interior = ((i >= 1) & (i <= nx) & (j >= 1) & (j <= ny) & (k >= 1) & (k <= nz))
    for two_a, want in ((1 + 2.0 ** -8, 0x3F80), (1 + 3 * 2.0 ** -8, 0x3F82),
                        (1 + 2.0 ** -8 + 2.0 ** -20, 0x3F81)):
        u = (two_a / 2) * (i * i).astype(np.float64)
        e = np.zeros(u.shape, dtype=np.uint16)
        u1, rho = oracle.residual_accumulate(u, e, dtype="bf16", lib=lib)
        assert np.all(rho[interior] == want), (two_a, np.unique(rho[interior]))
        assert np.all(rho[~interior] == 0)
    q = (i * i).astype(np.float64)
    e = np.where(interior, 0x3E80, 0x4000).astype(np.uint16)  # 0.25 inside, 2.0 outside
    u1, _ = oracle.residual_accumulate(q, e, dtype="bf16", lib=lib)
    assert np.array_equal(u1, np.where(interior, q + 0.25, q))


def pin_refinement_equals_plain(lib):
    """In exact arithmetic u + sum_{k<m} J0^k (J u - u) = J^m u, so O outer steps of
    m inner correction sweeps equal O*m plain sweeps (FP64: rounding only)."""
    rng = np.random.default_rng(7)
    nx, ny, nz = 6, 5, 7
    u0 = rng.random((nz + 2, ny + 2, nx + 2))
    u0[1:-1, 1:-1, 1:-1] = 0.0
    ir = oracle.refine_solve(u0, 4, 5, dtype="f64", lib=lib)
    plain = oracle.sweeps(u0, 20, lib=lib)
    assert np.abs(ir - plain).max() < 1e-14
    ir32 = oracle.refine_solve(u0, 4, 5, dtype="f32", lib=lib)
    assert np.abs(ir32 - plain).max() < 1e-5


def _loss(A, W, n, lib):
    return float((W * oracle.sweeps(A, n, lib=lib)).sum())


def pin_gradient_fd(lib):
    """The loss sum(W * A_n) is affine in A_0 (interior and boundary data), so the
    central difference with step 1 equals the gradient up to rounding."""
    rng = np.random.default_rng(9)
    nx, ny, nz, n = 5, 4, 3, 3
    A = rng.random((nz + 2, ny + 2, nx + 2))
    W = rng.standard_normal(A.shape)
    g = oracle.grad_f64(W, n, lib=lib)
    fd = np.zeros_like(A)
    for idx in np.ndindex(A.shape):
        Ap = A.copy(); Ap[idx] += 1.0
        Am = A.copy(); Am[idx] -= 1.0
        fd[idx] = 0.5 * (_loss(Ap, W, n, lib) - _loss(Am, W, n, lib))
    assert np.abs(g - fd).max() < 1e-12 * max(1.0, np.abs(W).sum())


def pin_gradient_structure(lib):
    """Structure of the gradient: edge and corner cells of the boundary layer are
    never read by the 7-point stencil, so their gradient is exactly W there; with
    W zero on the boundary the interior gradient is J0^n W (the sweep is a
    symmetric operator on the interior), i.e. n plain sweeps of W on a zero
    boundary."""
    rng = np.random.default_rng(13)
    nx, ny, nz, n = 6, 5, 4, 4
    W = rng.standard_normal((nz + 2, ny + 2, nx + 2))
    g = oracle.grad_f64(W, n, lib=lib)
    k, j, i = np.indices(W.shape)
    nb = ((i == 0) | (i == nx + 1)).astype(int) + ((j == 0) | (j == ny + 1)) + \
        ((k == 0) | (k == nz + 1))
    edge = nb >= 2
    assert np.array_equal(g[edge], W[edge])
    Wi = W.copy()
    Wi[nb > 0] = 0.0
    gi = oracle.grad_f64(Wi, n, lib=lib)
    fwd = oracle.sweeps(Wi, n, lib=lib)
    interior = nb == 0
    assert np.abs(gi[interior] - fwd[interior]).max() < 1e-14


ALL_PINS = [pin_hand_4cubed, pin_sum_order, pin_harmonic_fixed_points, pin_sine_modes,
            pin_bf16_conversion, pin_bf16_sweep_is_rounded_f32, pin_residual,
            pin_rhs_sweep, pin_rhs_sweep_bf16, pin_residual_bf16_store,
            pin_refinement_equals_plain, pin_gradient_fd,
            pin_gradient_structure]
