"""Batches: independent runs of different sizes, tile shapes, mode counts and
sort periods, advanced by one CUDA graph launch per cycle (the particle phase
of every step one persistent launch per group of runs).  A batch is
deterministic (two batches of the same runs are bit-identical: the int64
deposit), agrees with the same runs stepped one by one to FP32 rounding (the
batched particle kernel is compiled on its own, and the compiler may fuse a
different set of its multiply-adds than in the single-run kernel) and tracks
the FP64 oracle.  A
withheld work item makes the bounded waits give up with QPIC_ETIMEOUT instead
of hanging; what a batch cannot run is refused; the autotuner returns a
supported, working shape."""
import numpy as np
import pytest

import paper_2303_12874_gb300 as q
import synth
from paper_2303_12874_gb300 import autotune
from pairs import compare_fields, make_pair, oracle_config1_state, oracle_state_to_gpu

pytestmark = pytest.mark.gpu

RUNS = [dict(nz=96, nr=16, n0=0.01, a0=1.0, ppc=(2, 2, 2), tile=(16, 8)),
        dict(nz=160, nr=24, n0=0.02, a0=2.5, ppc=(2, 2, 4), tile=(32, 8)),
        dict(nz=128, nr=20, n0=0.005, a0=1.5, ppc=(2, 2, 8), tile=(8, 8))]


def _make(r):
    sim = q.Sim(r["nz"], r["nr"], 0.2, 0.5, dt=0.12, tile_z=r["tile"][0], tile_r=r["tile"][1],
                n_modes=r.get("n_modes", 2), sort_period=r.get("sort_period", 2))
    sim.load_plasma(r["n0"], 0.0, 0.0, r["ppc"])
    zc = 0.5 * r["nz"] * 0.2
    if r.get("n_modes", 2) >= 2:                        # the laser is an m = 1 field
        sim.add_laser(r["a0"], 4.0, 6.0, zc, zc)
    return sim


MIXED = [dict(nz=96, nr=16, n0=0.01, a0=1.0, ppc=(2, 2, 2), tile=(16, 8), sort_period=1),
         dict(nz=112, nr=19, n0=0.02, a0=2.0, ppc=(2, 2, 4), tile=(16, 8), sort_period=4),
         dict(nz=80, nr=12, n0=0.01, a0=1.5, ppc=(2, 2, 4), tile=(8, 8), n_modes=1),
         dict(nz=96, nr=20, n0=0.01, a0=1.5, ppc=(2, 2, 2), tile=(16, 8), n_modes=3),
         dict(nz=96, nr=36, n0=0.01, a0=1.5, ppc=(2, 2, 2), tile=(16, 16))]


def _sorted_particles(s):
    p = s.particles()
    k = np.lexsort((p["uz"], p["phi"], p["r"], p["z"]))
    return {f: p[f][k] for f in ("z", "r", "ux", "uy", "uz", "w")}


def _rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("runs,nsteps", [(RUNS, 12), (MIXED, 16)], ids=["tiles", "periods_modes"])
def test_batch_matches_individual_runs(runs, nsteps):
    solo = [_make(r) for r in runs]
    for s in solo:
        s.step(nsteps)
    batched = [[_make(r) for r in runs] for _ in range(2)]
    bs = [q.Batch(x) for x in batched]
    assert nsteps % bs[0].cycle == 0
    for b in bs:
        b.step(nsteps)
    for r, s, t, u in zip(runs, solo, batched[0], batched[1]):
        assert t.diag()["steps"] == nsteps
        for which in ("E", "B", "J"):
            # deterministic: the two batches agree bit for bit
            assert np.array_equal(t.fields(which), u.fields(which)), (r, which)
            # FP32 rounding against the single-run kernel (the current, a
            # difference of nearly equal particle sums, is the most sensitive)
            tol = 1e-4 if which == "J" else 1e-5
            assert _rel(t.fields(which), s.fields(which)) <= tol, (r, which)
        pt, pu, ps = _sorted_particles(t), _sorted_particles(u), _sorted_particles(s)
        for k in ("z", "r", "ux", "uy", "uz", "w"):
            assert np.array_equal(pt[k], pu[k]), (r, k)
        assert np.array_equal(np.sort(pt["w"]), np.sort(ps["w"]))
        # first and second moments over the particle set (independent of the
        # buffer order), against the sum of their magnitudes
        for k in ("z", "r", "ux", "uz"):
            for e in (1, 2):
                mt, ms = np.sum(pt["w"] * pt[k] ** e), np.sum(ps["w"] * ps[k] ** e)
                assert abs(mt - ms) <= 1e-5 * np.sum(ps["w"] * np.abs(ps[k]) ** e), (r, k, e)
    for b in bs:
        b.close()


def test_autotune_picks_a_working_shape():
    r = RUNS[1]

    def make(tz, tr, sp, ppt):
        return q.Sim(r["nz"], r["nr"], 0.2, 0.5, dt=0.12, tile_z=tz, tile_r=tr, sort_period=sp,
                     particles_per_thread=ppt)

    def init(sim):
        sim.load_plasma(r["n0"], 0.0, 0.0, r["ppc"])

    tz, tr, sp, ppt, ms = autotune.tune(make, init, r["nz"], r["nr"], 2, 16, steps=4, warmup=1,
                                        use_cache=False)
    assert (tz, tr) in autotune.TILES and sp in autotune.SORT_PERIODS and ppt in autotune.PARTICLES_PER_THREAD and ms > 0
    # timed as a batch of two copies: only what a batch accepts; threads per cell too
    tz, tr, sp, ppt, ms = autotune.tune(make, init, r["nz"], r["nr"], 2, 16, steps=4, warmup=1,
                                        use_cache=False, sort_periods=(2, 4), batch_copies=2,
                                        particles_per_thread=(2, 8))
    assert autotune.batch_ok(tz, tr, sp) and sp in (2, 4) and ppt in (2, 8) and ms > 0
    q.Batch([make(tz, tr, sp, ppt)]).close()


def test_batch_tracks_oracle():
    """two runs in different groups (2 and 3 modes) from states the oracle
    evolved; after one cycle of the batch each matches the oracle"""
    w = synth.workload("cfg1_small")
    pairs = []
    for n_modes, nz in ((2, w["nz"]), (3, w["nz"] - 24)):
        sim, o = make_pair(nz, w["nr"], w["dz"], w["dr"], 0.13, n_modes=n_modes)
        oracle_config1_state(o, dict(w, nz=nz), 0.13)
        o.step(3)
        oracle_state_to_gpu(o, sim)
        pairs.append((sim, o))
    b = q.Batch([p[0] for p in pairs])
    b.step(b.cycle)
    for sim, o in pairs:
        o.step(b.cycle)
        for which in ("E", "B", "J"):
            compare_fields(sim, o, which, 5e-5)
    b.close()


def test_withheld_item_times_out():
    """the first particle item never publishes: the reductions that wait on it
    give up after a few thousand polls and the step reports QPIC_ETIMEOUT;
    with the default limit and nothing withheld the batch steps again"""
    sims = [_make(r) for r in RUNS[:2]]
    b = q.Batch(sims)
    b.set_wait(2000, 0)
    with pytest.raises(q.QpicError, match="ETIMEOUT"):
        b.step(b.cycle)
    b.set_wait(1 << 24, -1)
    b.step(b.cycle)
    with pytest.raises(q.QpicError, match="EINVAL"):
        b.set_wait(-1, -1)
    b.close()


def test_batch_refuses_what_it_cannot_run():
    r = RUNS[0]
    bad = [dict(r, tile=(32, 4)),                       # sort period 2 > min(TZ, TR) - 3
           dict(r, tile=(16, 8), sort_period=6)]
    for spec in bad:
        with pytest.raises(q.QpicError, match="EINVAL"):
            q.Batch([_make(spec)])
    s = q.Sim(r["nz"], r["nr"], 0.2, 0.5, dt=0.12, precision=q.QPIC_FP64)
    with pytest.raises(q.QpicError, match="EINVAL"):
        q.Batch([s])


def test_more_runs_than_one_launch_holds():
    """70 runs of one shape need two persistent launches per step (at most 64
    runs each); one run holds no particles at all"""
    specs = [dict(nz=32, nr=8, n0=0.01 * (1 + k % 5), a0=1.0, ppc=(1, 1, 2), tile=(16, 8)) for k in range(70)]

    def make(k):
        if k == 17:
            return q.Sim(32, 8, 0.2, 0.5, dt=0.12)
        return _make(specs[k])

    solo = [make(k) for k in range(70)]
    for s in solo:
        s.step(8)
    batched = [make(k) for k in range(70)]
    b = q.Batch(batched)
    assert 8 % b.cycle == 0
    b.step(8)
    assert batched[17].num_particles() == 0
    for s, t in zip(solo, batched):
        assert t.diag()["steps"] == 8
        for which in ("E", "J"):
            assert _rel(t.fields(which), s.fields(which)) <= 1e-4, which
    b.close()
