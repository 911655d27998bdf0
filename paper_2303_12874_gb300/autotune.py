"""Autotuner for the particle kernel's tile shape, the sort period and the
particles each thread takes in a row (about ppc / that many threads share a
cell: the threads-per-cell knob).

For a run configuration it times a few steps of every supported tile shape
(16x8, 32x8, 8x8, 16x16, 32x4), sort period (1, 2 by default) and particles
per thread (16 by default) on the GPU and keeps the fastest, caching the choice
in a JSON file next to the built library keyed by (nz, nr, n_modes, particles
per cell, periodic, the candidates, batch).
Timing uses CUDA events; the state is the run's own plasma and laser.  With
batch=True only the combinations a batch accepts are tried (a sort period of
at most min(tile_z, tile_r) - 3, so that a particle never deposits outside the
3 x 3 tiles around the tile it was sorted into).
"""
import json
import os

from . import _build
from . import QpicError

TILES = [(16, 8), (32, 8), (8, 8), (16, 16), (32, 4)]
SORT_PERIODS = [1, 2]
PARTICLES_PER_THREAD = [16]
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


def batch_ok(tile_z, tile_r, sort_period):
    """Whether a batch accepts a run with this tile shape and sort period."""
    return max(1, sort_period) + 3 <= min(tile_z, tile_r)


def _time_one(make_sim, init_state, tz, tr, sp, ppt, steps, warmup, batch_copies):
    """ms per step of one run, or of a batch of batch_copies runs"""
    import torch
    from . import Batch
    sims = [make_sim(tz, tr, sp, ppt) for _ in range(max(1, batch_copies))]
    for sim in sims:
        init_state(sim)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    b = None
    if batch_copies > 0:
        b = Batch(sims)
        n = -(-steps // b.cycle) * b.cycle
        b.step(-(-warmup // b.cycle) * b.cycle)
        run = lambda: b.step(n)
    else:
        n = steps
        sims[0].step(warmup)
        run = lambda: sims[0].step(n)
    torch.cuda.synchronize()
    e0.record(stream)
    run()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / n
    if b is not None:
        b.close()
    for sim in sims:
        sim.close()
    return ms


def tune(make_sim, init_state, nz, nr, n_modes, ppc, periodic=True, steps=8, warmup=2,
         use_cache=True, sort_periods=None, batch=False, batch_copies=0, particles_per_thread=None):
    """make_sim(tile_z, tile_r, sort_period, particles_per_thread) -> Sim;
    init_state(sim) loads the run's plasma and laser.  sort_periods and
    particles_per_thread: the candidates (default 1, 2 and 8).  batch: try
    only what a batch accepts; batch_copies > 0: time a batch of that many
    copies of the run (whose particle phase is one persistent launch) instead
    of the run on its own.  Returns (tile_z, tile_r, sort_period,
    particles_per_thread, ms_per_step)."""
    periods = list(sort_periods) if sort_periods else SORT_PERIODS
    ppts = list(particles_per_thread) if particles_per_thread else PARTICLES_PER_THREAD
    batch = batch or batch_copies > 0
    key = _key(nz, nr, n_modes, ppc, periodic) + "_sp" + "-".join(map(str, periods)) + \
        "_pt" + "-".join(map(str, ppts)) + ("_b%d" % batch_copies if batch else "")
    cache = _load_cache() if use_cache else {}
    if key in cache:
        c = cache[key]
        return c["tile_z"], c["tile_r"], c["sort_period"], c["particles_per_thread"], c["ms_per_step"]
    best = None
    for tz, tr in TILES:
        for sp in periods:
            if batch and not batch_ok(tz, tr, sp):
                continue
            for ppt in ppts:
                try:
                    ms = _time_one(make_sim, init_state, tz, tr, sp, ppt, steps, warmup, batch_copies)
                except QpicError as e:
                    if "EINVAL" not in str(e):
                        raise
                    continue                    # a shape this run cannot take (e.g. too much shared memory)
                if best is None or ms < best[4]:
                    best = (tz, tr, sp, ppt, ms)
    if best is None:
        raise ValueError("no tile shape and sort period to try")
    cache[key] = {"tile_z": best[0], "tile_r": best[1], "sort_period": best[2],
                  "particles_per_thread": best[3], "ms_per_step": best[4]}
    if use_cache:
        _save_cache(cache)
    return best
