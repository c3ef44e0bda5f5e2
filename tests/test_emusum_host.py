"""The exact binary64 running sum of the FP64 sweeps (emusum.cuh), compiled for
the host and checked against the host's IEEE-754 additions on millions of
6-tuples: uniform, smooth, wide-exponent and tie-heavy data, every word form.
The GPU tests check the device build of the same source against the FP64 unit."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path_factory.mktemp("emusum") / "emusum_check")
    subprocess.run([cxx, "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math",
                    os.path.join(HERE, "emusum_check.cpp"), "-o", exe], check=True)
    return exe


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_running_sum_matches_ieee(checker, seed):
    r = subprocess.run([checker, str(seed), "2000000"], capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    fast = int(r.stdout.split("fast")[1].split()[0])
    assert fast > 1000000  # most tuples take the integer path
