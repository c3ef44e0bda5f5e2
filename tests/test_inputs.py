"""The seeded input generators (shared by the oracle tests and the GPU tests)."""
import numpy as np

from paper_0912_4506_gb300 import inputs


def test_splitmix64_published_first_output():
    # splitmix64 started from state 0 first returns 0xE220A8397B1DCDAF
    assert int(inputs.mix64(np.uint64(0))) == 0xE220A8397B1DCDAF


def test_mix64_matches_bigint_definition():
    M = (1 << 64) - 1

    def ref(x):
        z = (x + 0x9E3779B97F4A7C15) & M
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M
        return z ^ (z >> 31)

    xs = [0, 1, 2, 12345, (1 << 63) + 7, M]
    got = inputs.mix64(np.array(xs, dtype=np.uint64))
    assert [int(v) for v in got] == [ref(x) for x in xs]


def test_uniform_grid_deterministic_and_layout():
    a = inputs.uniform_grid_f64(5, 4, 3)
    b = inputs.uniform_grid_f64(5, 4, 3, px=10)
    assert np.array_equal(a, b[:, :, :7]) and np.all(b[:, :, 7:] == 0)
    assert np.array_equal(a, inputs.uniform_grid_f64(5, 4, 3))
    assert a.min() >= 0.0 and a.max() < 1.0
    # interior and boundary come from different seeds
    c = inputs.uniform_grid_f64(5, 4, 3, g=1)
    assert not np.array_equal(a, c)


def test_row_pitch_is_16_bytes():
    for dt, e in (("f64", 8), ("f32", 4), ("bf16", 2)):
        for nx in (1, 4, 62, 64, 255, 256, 1024):
            px = inputs.row_pitch(nx, dt)
            assert px >= nx + 2 and (px * e) % 16 == 0 and px - (nx + 2) < 16 // e


def test_laplace_boundary_is_harmonic_data():
    u = inputs.laplace_boundary_f64(6, 5, 4)
    assert np.all(u[1:-1, 1:-1, 1:-1] == 0.0)
    assert u[0, 2, 3] == 9.0 - 4.0 + 0.0 and u[5, 2, 3] == 9.0 - 4.0 + 2.5


def test_batch_specs_ranges():
    specs = inputs.batch_specs()
    assert len(specs) == 64 and specs == inputs.batch_specs()
    for nx, ny, nz, n in specs:
        for a in (nx, ny, nz):
            assert 32 <= a <= 256 and a % 8 == 0
        assert 10 <= n <= 200
    assert len({s[:3] for s in specs}) > 50


def test_normal_moments():
    w = inputs.normal_grid_f64(30, 30, 30)
    assert abs(w.mean()) < 0.01 and abs(w.std() - 1.0) < 0.01


def test_to_dtype():
    a = inputs.uniform_grid_f64(6, 3, 2)
    f = inputs.to_dtype(a, "f32", px=12)
    assert f.dtype == np.float32 and f.shape == (4, 5, 12)
    assert np.array_equal(f[:, :, :8], a.astype(np.float32))
    b = inputs.to_dtype(a, "bf16", px=16)
    assert b.dtype == np.uint16 and b.shape == (4, 5, 16)


def test_plane_range_equals_slice_of_full_grid():
    """A rank of the z-slab decomposition draws only its planes: the same values
    the full grid has there (counter-based generator)."""
    import numpy as np
    from paper_0912_4506_gb300 import inputs
    full = inputs.uniform_grid_f64(11, 7, 20, px=14)
    for lo, hi in ((0, 4), (3, 12), (15, 21), (0, 21)):
        part = inputs.uniform_grid_f64(11, 7, 20, px=14, planes=(lo, hi))
        assert np.array_equal(part, full[lo:hi + 1])
