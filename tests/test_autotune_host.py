"""Host logic of the depth autotuner, without a GPU: the measurement is replaced
by a fake whose best depth is known; the first call measures every candidate of
every new shape and caches the result, the second reads the cache only."""
import json
import types

import pytest

torch = pytest.importorskip("torch")


def test_tune_measures_once_then_uses_cache(tmp_path, monkeypatch):
    from paper_0912_4506_gb300 import autotune
    monkeypatch.setenv("JACOBI_GB300_CACHE", str(tmp_path))
    monkeypatch.setattr(torch.cuda, "get_device_name", lambda dev=None: "FakeGPU")
    monkeypatch.setattr(torch.cuda, "get_device_properties",
                        lambda dev=None: types.SimpleNamespace(multi_processor_count=152))
    calls = []

    def fake_time(shape, dtype, cand, sweeps, device, reps):
        calls.append((shape, cand))
        tile_x, t = cand
        # rate peaks at the shape's best (width, depth)
        best = (128, 2) if shape[0] >= 100 else (64, 3)
        return 1e9 * (10.0 - abs(t - best[1]) - (0 if tile_x == best[0] else 0.5))

    monkeypatch.setattr(autotune, "_time_shape", fake_time)
    shapes = [(128, 64, 64), (40, 40, 40), (128, 64, 64)]
    cands = ((128, 1), (128, 2), (64, 2), (64, 3))
    ts, table = autotune.tune(shapes, "f32", candidates=cands, device="cpu")
    assert ts == [(128, 2), (64, 3), (128, 2)]
    # two distinct shapes x four candidates (the repeated shape is measured once)
    assert len(calls) == 8
    cached = json.loads((tmp_path / "autotune.json").read_text())
    cs = "|64x2,64x3,128x1,128x2"  # the candidate set is part of the key
    assert (cached["FakeGPU|f32|128x64x64" + cs]["tile_x"],
            cached["FakeGPU|f32|128x64x64" + cs]["t"]) == (128, 2)
    assert cached["FakeGPU|f32|40x40x40" + cs]["t"] == 3

    calls.clear()
    ts2, _ = autotune.tune(shapes, "f32", candidates=cands, device="cpu")
    assert ts2 == ts and calls == []


def test_model_prunes_the_measured_candidates(tmp_path, monkeypatch):
    """With the model's parameters only the first `keep` candidates in model order
    are measured, and the best of those is chosen."""
    from paper_0912_4506_gb300 import autotune, model
    monkeypatch.setenv("JACOBI_GB300_CACHE", str(tmp_path))
    monkeypatch.setattr(torch.cuda, "get_device_name", lambda dev=None: "FakeGPU")
    monkeypatch.setattr(torch.cuda, "get_device_properties",
                        lambda dev=None: types.SimpleNamespace(multi_processor_count=152))
    calls = []

    def fake_time(shape, dtype, cand, sweeps, device, reps):
        calls.append(cand)
        return 1e9 * (cand[1] + (1 if cand[0] == 64 else 0))

    monkeypatch.setattr(autotune, "_time_shape", fake_time)
    cands = ((128, 1), (128, 2), (64, 2), (64, 3), (64, 4), (64, 5), (64, 6))
    params = dict(hbm_gbs=6800.0, sm_mhz=2070.0, sms=152, inst_per_update=17.0)
    shape = (96, 80, 64)
    order = model.order_candidates(list(cands), shape, 4, **params)
    best, _ = autotune.tune([shape], "f32", candidates=cands, device="cpu",
                            model_params=params, keep=3)
    assert calls == order[:3]
    assert best[0] == max(order[:3], key=lambda c: c[1] + (1 if c[0] == 64 else 0))


def test_candidates_without_a_kernel_are_skipped(tmp_path, monkeypatch):
    """A candidate the batched kernel does not have (128-wide tiles deeper than 2,
    64-wide deeper than 6) is never timed; a cached choice is reused only for the
    same candidate set."""
    from paper_0912_4506_gb300 import autotune
    monkeypatch.setenv("JACOBI_GB300_CACHE", str(tmp_path))
    monkeypatch.setattr(torch.cuda, "get_device_name", lambda dev=None: "FakeGPU")
    monkeypatch.setattr(torch.cuda, "get_device_properties",
                        lambda dev=None: types.SimpleNamespace(multi_processor_count=152))
    calls = []

    def fake_time(shape, dtype, cand, sweeps, device, reps):
        calls.append(cand)
        return 1e9 * cand[1]

    monkeypatch.setattr(autotune, "_time_shape", fake_time)
    shape = (200, 120, 64)
    cands = ((128, 2), (128, 3), (64, 4), (64, 7))
    best, _ = autotune.tune([shape], "f32", candidates=cands, device="cpu")
    assert best == [(64, 4)] and sorted(calls) == [(64, 4), (128, 2)]
    autotune.tune([shape], "f32", candidates=cands, device="cpu")
    assert len(calls) == 2  # cached
    autotune.tune([shape], "f32", candidates=((64, 4), (64, 2)), device="cpu")
    assert len(calls) == 4  # another candidate set is tuned afresh
