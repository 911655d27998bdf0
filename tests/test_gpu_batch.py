"""Batches: independent runs of different sizes advanced by one CUDA graph
launch per cycle give bit-identical results to the same runs stepped one by
one (the int64 deposit makes every run deterministic), and the autotuner
returns a supported, working tile shape."""
import numpy as np
import pytest

import paper_2303_12874_gb300 as q
from paper_2303_12874_gb300 import autotune

pytestmark = pytest.mark.gpu

RUNS = [dict(nz=96, nr=16, n0=0.01, a0=1.0, ppc=(2, 2, 2), tile=(16, 8)),
        dict(nz=160, nr=24, n0=0.02, a0=2.5, ppc=(2, 2, 4), tile=(32, 8)),
        dict(nz=128, nr=20, n0=0.005, a0=1.5, ppc=(2, 2, 8), tile=(8, 8))]


def _make(r):
    sim = q.Sim(r["nz"], r["nr"], 0.2, 0.5, dt=0.12, tile_z=r["tile"][0], tile_r=r["tile"][1])
    sim.load_plasma(r["n0"], 0.0, 0.0, r["ppc"])
    zc = 0.5 * r["nz"] * 0.2
    sim.add_laser(r["a0"], 4.0, 6.0, zc, zc)
    return sim


def test_batch_graph_equals_individual_runs():
    solo = [_make(r) for r in RUNS]
    for s in solo:
        s.step(12)
    batched = [_make(r) for r in RUNS]
    b = q.Batch(batched)
    b.step(12)
    for s, t in zip(solo, batched):
        assert t.diag()["steps"] == 12
        for which in ("E", "B", "J"):
            assert np.array_equal(s.fields(which), t.fields(which)), which
        ps, pt = s.particles(), t.particles()
        ks = np.lexsort((ps["uz"], ps["phi"], ps["r"], ps["z"]))
        kt = np.lexsort((pt["uz"], pt["phi"], pt["r"], pt["z"]))
        for k in ("z", "r", "ux", "uy", "uz", "w"):
            assert np.array_equal(ps[k][ks], pt[k][kt]), k
    b.close()


def test_autotune_picks_a_working_shape():
    r = RUNS[1]

    def make(tz, tr, sp):
        return q.Sim(r["nz"], r["nr"], 0.2, 0.5, dt=0.12, tile_z=tz, tile_r=tr, sort_period=sp)

    def init(sim):
        sim.load_plasma(r["n0"], 0.0, 0.0, r["ppc"])

    tz, tr, sp, ms = autotune.tune(make, init, r["nz"], r["nr"], 2, 16, steps=4, warmup=1,
                                   use_cache=False)
    assert (tz, tr) in autotune.TILES and sp in autotune.SORT_PERIODS and ms > 0
