"""Moving window (open box, circular z buffer on the GPU) against the oracle's
window driver: the same shifts, the same injected plasma, the same fields.  Both sides set up
the plasma and the laser themselves from the same recipe."""
import numpy as np
import pytest

import paper_2303_12874_gb300 as q
from oracle import sim as osim
from pairs import COMPS, rel_l2

pytestmark = pytest.mark.gpu


def test_moving_window_tracks_oracle():
    nz, nr, dz, dr, dt = 120, 20, 0.2, 0.5, 0.14
    plasma = dict(n0=0.02, z_start=6.0, ramp_len=10.0, ppc=(2, 2, 2))
    sim = q.Sim(nz, nr, dz, dr, dt=dt, periodic=False, moving_window=True, seed=5)
    sim.load_plasma(plasma["n0"], plasma["z_start"], plasma["ramp_len"], plasma["ppc"])
    sim.add_laser(1.2, 4.0, 6.0, 15.0, 18.0)
    # the oracle's window driver builds the same state from the same recipe on
    # its own (nothing read back from the GPU)
    run = osim.Run(nz, nr, dz, dr, dt=dt, periodic=False, moving_window=True)
    run.load_plasma(plasma["n0"], plasma["z_start"], plasma["ramp_len"], plasma["ppc"], seed=5)
    run.add_laser(1.2, 4.0, 6.0, 15.0, 18.0)
    o = run.o
    nsteps = 16
    sim.step(nsteps)
    run.step(nsteps)
    d = sim.diag()
    assert d["shifts"] == run.shifts > 5
    for which in ("E", "B"):
        for c in COMPS:
            for m in range(2):
                err = rel_l2(sim.get_field(which, c, m), o.get_field(which, c, m))
                assert err < 1e-4, (which, c, m, err)
    g = sim.particles()
    r = o.particles()
    rl = r["w"] > 0
    assert len(g["z"]) == int(rl.sum())
    assert abs(g["w"].sum() / r["w"][rl].sum() - 1) < 1e-6
    assert abs(np.sort(g["z"]).mean() - np.sort(r["z"][rl]).mean()) < 1e-5
