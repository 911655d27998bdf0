"""Autotuner for the particle kernel's tile shape and the sort period.

For a run configuration it times a few steps of every supported tile shape
(16x8, 32x8, 8x8, 16x16, 32x4) and sort period (1, 2) on the GPU and keeps the
fastest, caching the choice in a JSON file next to the built library keyed by
(nz, nr, n_modes, particles per cell, periodic).  Timing uses CUDA events on the
library's stream; the state is the run's own plasma and laser.
"""
import json
import os

from . import _build

TILES = [(16, 8), (32, 8), (8, 8), (16, 16), (32, 4)]
SORT_PERIODS = [1, 2]
CACHE = os.path.join(_build.BUILD, "autotune.json")


def _key(nz, nr, n_modes, ppc, periodic):
    return "%d_%d_%d_%d_%d" % (nz, nr, n_modes, ppc, int(periodic))


def _load_cache():
    try:
        return json.load(open(CACHE))
    except Exception:
        return {}


def _save_cache(cache):
    os.makedirs(os.path.dirname(CACHE), exist_ok=True)
    tmp = CACHE + ".tmp%d" % os.getpid()
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, CACHE)


def tune(make_sim, init_state, nz, nr, n_modes, ppc, periodic=True, steps=8, warmup=2,
         use_cache=True, sort_periods=None):
    """make_sim(tile_z, tile_r, sort_period) -> Sim; init_state(sim) loads the
    run's plasma and laser.  sort_periods: the periods to try (default 1 and
    2; a batch needs one common period).  Returns (tile_z, tile_r,
    sort_period, ms_per_step)."""
    import torch
    periods = list(sort_periods) if sort_periods else SORT_PERIODS
    key = _key(nz, nr, n_modes, ppc, periodic) + ("" if periods == SORT_PERIODS else
                                                  "_sp" + "-".join(map(str, periods)))
    cache = _load_cache() if use_cache else {}
    if key in cache:
        c = cache[key]
        return c["tile_z"], c["tile_r"], c["sort_period"], c["ms_per_step"]
    best = None
    stream = torch.cuda.current_stream()
    for tz, tr in TILES:
        for sp in periods:
            sim = make_sim(tz, tr, sp)
            init_state(sim)
            sim.step(warmup)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sim.step(steps)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / steps
            sim.close()
            if best is None or ms < best[3]:
                best = (tz, tr, sp, ms)
    cache[key] = {"tile_z": best[0], "tile_r": best[1], "sort_period": best[2], "ms_per_step": best[3]}
    if use_cache:
        _save_cache(cache)
    return best
