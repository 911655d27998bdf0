"""Checkpoint and resume (qpic_save_state / qpic_load_state): 40 steps run
without a break equal 20 steps, a save, a load into a new context and 20 more
steps, bit for bit on the FP32 fixed-point path (the current is an integer sum
over particles, so the particle order a load brings does not matter) -- for a
periodic box with a laser and for an open box with a moving window and plasma
injection.  Snapshots from another configuration are refused."""
import numpy as np
import pytest

import paper_2303_12874_gb300 as q
import synth

pytestmark = pytest.mark.gpu


def _make(moving):
    if moving:
        sim = q.Sim(160, 24, 0.2, 0.5, dt=0.12, periodic=False, moving_window=True, seed=3)
        sim.load_plasma(0.01, 5.0, 6.0, (2, 2, 2))
        sim.add_laser(1.5, 5.0, 8.0, 20.0, 24.0)
    else:
        sim = q.Sim(128, 20, 0.2, 0.5, dt=0.12, seed=7)
        sim.load_plasma(0.02, 0.0, 0.0, (2, 2, 2))
        sim.add_laser(1.2, 4.0, 6.0, 12.8, 12.8)
    return sim


def _state(sim):
    f = {(w, c, m): sim.get_field(w, c, m) for w in ("E", "B") for c in ("r", "phi", "z") for m in range(sim.nm)}
    p = sim.particles()
    order = np.lexsort((p["uz"], p["uy"], p["ux"], p["phi"], p["r"], p["z"]))
    return f, {k: v[order] for k, v in p.items()}, sim.diag()


@pytest.mark.parametrize("moving", [False, True])
def test_resume_is_bit_identical(moving):
    a = _make(moving)
    a.step(40)
    fa, pa, da = _state(a)
    b = _make(moving)
    b.step(20)
    snap = b.save_state()
    c = _make(moving)                      # a fresh context of the same configuration
    c.load_state(snap)
    c.step(20)
    fc, pc, dc = _state(c)
    assert dc["steps"] == da["steps"] == 40 and dc["shifts"] == da["shifts"]
    for k in fa:
        assert np.array_equal(fa[k], fc[k]), k
    assert len(pa["z"]) == len(pc["z"])
    for k in pa:
        assert np.array_equal(pa[k], pc[k]), k
    if moving:
        assert da["shifts"] > 5                                  # the window moved and injected


def test_snapshot_of_another_configuration_is_refused():
    a = _make(False)
    snap = a.save_state()
    other = q.Sim(128, 20, 0.2, 0.5, dt=0.11)
    with pytest.raises(q.QpicError, match="EINVAL"):
        other.load_state(snap)
    with pytest.raises(q.QpicError, match="EINVAL"):
        a.load_state(snap[:-8])
