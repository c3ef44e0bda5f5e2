"""Autotuner for the tile shape and temporal-blocking depth of batched grids.

For every distinct grid shape it times the batched persistent kernel itself on
enough replicas of that shape to fill the GPU, for each candidate (tile width,
depth), and keeps the fastest (lattice-site updates per second).  Results are cached in a
JSON file keyed by device name, dtype and shape, so a batch is tuned once.
The paper chose its blocking parameters experimentally as well (Sect. 1.5: the
parameter space is large and the best values were found by measurement).
"""
import json
import os
import time

import torch

from . import api

# (loaded tile width, depth): 128-wide tiles exist up to depth 2, 64-wide up to 6
DEFAULT_CANDIDATES = ((128, 1), (128, 2), (64, 2), (64, 3), (64, 4), (64, 5), (64, 6))


def _built(dtype, cand):
    """The batched kernel has this (tile width, depth); other candidates are
    skipped rather than timed."""
    tile_x, t = cand
    return (tile_x == 64 and t <= 6) or (tile_x == 128 and t <= 2)


def cache_path():
    base = os.environ.get("JACOBI_GB300_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "paper_0912_4506_gb300"))
    os.makedirs(base, exist_ok=True)
    return os.path.join(base, "autotune.json")


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _key(dev, dtype, shape, cands):
    """Cache key: device, dtype, shape and the candidate set (a new set retunes)."""
    cs = ",".join(f"{w}x{t}" for w, t in sorted(cands))
    return f"{torch.cuda.get_device_name(dev)}|{dtype}|{shape[0]}x{shape[1]}x{shape[2]}|{cs}"


def _time_shape(shape, dtype, cand, sweeps, device, reps):
    tile_x, t = cand
    nx, ny, nz = shape
    grids = []
    for _ in range(reps):
        g = api.alloc_grid(nx, ny, nz, dtype, device)
        g.uniform_()
        grids.append(g)
    b = api.Batch(grids, [sweeps] * reps, t=[t] * reps, tile_x=[tile_x] * reps)
    b.run()  # warm-up
    torch.cuda.synchronize(device)
    t0 = time.perf_counter()
    b.run()
    torch.cuda.synchronize(device)
    dt = time.perf_counter() - t0
    b.check()
    b.close()
    return reps * nx * ny * nz * sweeps / dt


def tune(shapes, dtype="f32", candidates=DEFAULT_CANDIDATES, sweeps=24, device="cuda",
         use_cache=True, model_params=None, keep=None):
    """Best (tile width, depth) per shape (list aligned with `shapes`) and the
    measurements.  With `model_params` (hbm_gbs, sm_mhz, sms, inst_per_update)
    the candidates of each shape are ordered by the performance model (model.py,
    the paper's Eq. 4-5 restated for the GPU) and only the first `keep` are
    measured."""
    from . import model
    path = cache_path()
    cache = _load(path) if use_cache else {}
    dev = torch.device(device)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    out, table = [], {}
    for shape in shapes:
        key = _key(dev, dtype, shape, [tuple(c) for c in candidates if _built(dtype, c)])
        if key in cache and "tile_x" in cache[key]:
            out.append((cache[key]["tile_x"], cache[key]["t"]))
            table[key] = cache[key]
            continue
        nx, ny, nz = shape
        cells = nx * ny * nz
        # replicas: enough tiles to cover every SM a few times, bounded memory
        reps = max(1, min(64, (4 * sms * 64 * 32) // max(cells // 8, 1) + 1))
        cands = [tuple(c) for c in candidates if _built(dtype, c)]
        if model_params is not None:
            es = {"f32": 4, "bf16": 2}[dtype]
            cands = model.order_candidates(cands, shape, es, **model_params)
            if keep:
                cands = cands[:keep]
        rates = {c: _time_shape(shape, dtype, c, sweeps, dev, reps) for c in cands}
        best = max(rates, key=rates.get)
        cache[key] = {"tile_x": best[0], "t": best[1],
                      "glups": {f"{k[0]}x{k[1]}": v / 1e9 for k, v in rates.items()},
                      "measured": len(rates)}
        table[key] = cache[key]
        out.append(best)
    if use_cache:
        with open(path, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
    return out, table
