"""The CPU oracle against what the paper and mathematics fix (no GPU)."""
import numpy as np
import pytest

import oracle
from tests import oracle_pins


@pytest.mark.parametrize("pin", oracle_pins.ALL_PINS, ids=lambda f: f.__name__)
def test_pin(pin):
    pin(oracle.load())


def test_constants_are_rn_one_sixth():
    # RN64(1/6) and RN32(1/6) = (float) RN64(1/6) (no double rounding issue here)
    assert 1.0 / 6.0 == oracle_pins.C64
    assert float(np.float32(1.0) / np.float32(6.0)) == float(np.float32(oracle_pins.C64))


def test_openmp_bit_identical():
    rng = np.random.default_rng(1)
    a = rng.random((14, 11, 13))
    s1 = oracle.sweeps(a, 7, nx=10, nthreads=1)
    s4 = oracle.sweeps(a, 7, nx=10, nthreads=4)
    assert np.array_equal(s1, s4)
    b = a.astype(np.float32)
    assert np.array_equal(oracle.sweeps(b, 5, dtype="f32", nthreads=1),
                          oracle.sweeps(b, 5, dtype="f32", nthreads=3))


def test_ping_pong_parity_and_zero_sweeps():
    rng = np.random.default_rng(2)
    a = rng.random((6, 7, 8))
    assert np.array_equal(oracle.sweeps(a, 0), a)
    one = oracle.sweeps(a, 1)
    two = oracle.sweeps(a, 2)
    assert np.array_equal(oracle.sweeps(one, 1), two)
    # the row padding beyond nx+2 is never read or written
    a2 = np.concatenate([a, np.full((6, 7, 3), np.nan)], axis=2)
    out = oracle.sweeps(a2, 3, nx=6)
    assert np.array_equal(out[:, :, :8], oracle.sweeps(a, 3))
    assert np.all(np.isnan(out[:, :, 8:]))
