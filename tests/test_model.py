"""The performance model of a blocked pass (Sect. 1.4, Eq. 4-5 restated for the
GPU), checked against the paper's own numbers and hand-computed tile cases."""
import math

import pytest

from paper_0912_4506_gb300 import model


def test_eq5_matches_the_papers_nehalem_prediction():
    """M_s / M_s,1 = 2 and M_c / M_s,1 = 8 give 16T / (7 + 4T) at t = 4, and 1.45
    for one team (Sect. 1.4); the large-tT limit is M_c / M_s = 4."""
    for T in (1, 2, 3, 5):
        assert model.eq5_speedup(4, 1.0, 2.0, 8.0, teams=T) == pytest.approx(16 * T / (7 + 4 * T))
    assert round(model.eq5_speedup(4, 1.0, 2.0, 8.0), 2) == 1.45
    assert model.eq5_speedup(10 ** 7, 1.0, 2.0, 8.0) == pytest.approx(4.0, rel=1e-5)


def test_eq4_is_memory_plus_cache_transfers():
    # t = 1: only the 16 B memory transfer; each further update adds 2 x 8 B of cache traffic
    assert model.eq4_time(1, 10.0, 80.0) == pytest.approx(16 / 10.0)
    assert model.eq4_time(3, 10.0, 80.0) == pytest.approx(16 / 10.0 + 4 * 8 / 80.0)


def test_tile_arithmetic_fp32_depth3_128x32():
    """Hand-computed: output tile 120 x 26 (128 - 6 rounded down to 4 cells of
    16 B), computed cells 128 * (30 + 28 + 26) = 10752 per 3 * 120 * 26 = 9360
    useful updates, HBM 4 * (4096 + 3120) / 9360 bytes, shared memory
    4 * (4096 + 3 * 3840 + 3 * 3584 + 2 * 3328) / 9360 bytes."""
    assert model.tile(3, 128, 32, 4) == (120, 26)
    assert model.recompute(3, 128, 32, 4) == pytest.approx(10752 / 9360)
    assert model.hbm_bytes(3, 128, 32, 4) == pytest.approx(4 * 7216 / 9360)
    assert model.smem_bytes(3, 128, 32, 4) == pytest.approx(4 * 33024 / 9360)
    # the k-chunk's pipeline fill: 2t extra planes per kz output planes
    assert model.hbm_bytes(3, 128, 32, 4, kz=64) == pytest.approx(4 * 7216 / 9360 * 70 / 64)


def test_tile_arithmetic_fp64_depth1_64x32():
    # depth 1: output 62 x 30, one level computed on 30 rows of 64 cells
    assert model.tile(1, 64, 32, 8) == (62, 30)
    assert model.recompute(1, 64, 32, 8) == pytest.approx(64 * 30 / (62 * 30))
    assert model.hbm_bytes(1, 64, 32, 8) == pytest.approx(8 * (2048 + 1860) / 1860)


def test_predict_bounds():
    # a plain-like pass with free instructions is HBM-bound at M_s / bytes
    g, bound = model.predict(1, 128, 32, 4, hbm_gbs=8000.0, sm_mhz=2000.0, sms=152,
                             inst_per_update=0.0)
    assert bound == "hbm"
    assert g == pytest.approx(8000.0 / model.hbm_bytes(1, 128, 32, 4))
    # an expensive update is issue-bound: 152 SMs x 128 inst/clk x 2 GHz / (I r)
    g, bound = model.predict(3, 128, 32, 4, hbm_gbs=8000.0, sm_mhz=2000.0, sms=152,
                             inst_per_update=40.0)
    assert bound == "issue"
    assert g == pytest.approx(152 * 128 * 2e9 / (40.0 * model.recompute(3, 128, 32, 4)) / 1e9)
    # an FP64 pipe of 500 G op/s with 2 operations per update binds at 250 / r
    g, bound = model.predict(2, 64, 32, 8, hbm_gbs=8000.0, sm_mhz=2000.0, sms=152,
                             inst_per_update=1.0, pipe_ops=2.0, pipe_gops=500.0)
    assert bound == "pipe"
    assert g == pytest.approx(250.0 / model.recompute(2, 64, 32, 8))


def test_order_candidates_prefers_narrow_tiles_on_narrow_grids():
    cands = [(128, 2), (64, 2), (64, 4)]
    # 248 columns: two 124-wide output tiles fit exactly, 60-wide ones waste 21 %
    wide = model.order_candidates(cands, (248, 248, 256), 4, 6800.0, 2070.0, 152, 17.0)
    narrow = model.order_candidates(cands, (40, 256, 256), 4, 6800.0, 2070.0, 152, 17.0)
    assert wide.index((128, 2)) < wide.index((64, 2))
    assert narrow.index((64, 2)) < narrow.index((128, 2))
    assert math.isfinite(model.predict(6, 64, 32, 4, 6800.0, 2070.0, 152, 17.0)[0])
