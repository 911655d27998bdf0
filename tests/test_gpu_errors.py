"""Error reporting, made to happen with valid inputs (no GPU fault):
- QPIC_ECAPACITY: a load larger than the capacity the caller fixed
  (max_particles) is refused before anything is written; a moving-window
  run reserves 64 columns of injection on top of its load, so a capacity
  below that is refused too.
- QPIC_EOVERFLOW: 28M equal particles in one cell, each moving 0.4 of a cell
  along z, put about 1.4 x 2^62 fixed-point units into each of two J_z nodes;
  the reduction checks the int64 sums against 2^62 and the step reports it
  (the sums themselves stay below 2^63, so nothing wraps before the check)."""
import numpy as np
import pytest

import paper_2303_12874_gb300 as q

pytestmark = pytest.mark.gpu


def test_loads_beyond_capacity_are_refused():
    nz, nr = 64, 8
    sim = q.Sim(nz, nr, 0.2, 0.5, max_particles=nz * nr - 1)
    with pytest.raises(q.QpicError, match="ECAPACITY"):
        sim.load_plasma(0.01, 0.0, 0.0, (1, 1, 1))
    with pytest.raises(q.QpicError, match="ECAPACITY"):
        n = nz * nr
        sim.load_particles(np.full(n, 1.0), np.full(n, 1.0), np.zeros(n), np.zeros(n), np.zeros(n),
                           np.zeros(n), np.ones(n))
    sim.load_particles(*(np.ones(10) for _ in range(7)))          # within the capacity
    assert sim.num_particles() == 10
    win = q.Sim(nz, nr, 0.2, 0.5, periodic=False, moving_window=True, max_particles=nz * nr + 63 * nr)
    with pytest.raises(q.QpicError, match="ECAPACITY"):
        win.load_plasma(0.01, 0.0, 0.0, (1, 1, 1))
    win = q.Sim(nz, nr, 0.2, 0.5, periodic=False, moving_window=True, max_particles=nz * nr + 64 * nr)
    win.load_plasma(0.01, 0.0, 0.0, (1, 1, 1))
    win.step(20)                                # the window moves and injects within its reserve


def test_fixed_point_overflow_is_reported():
    # charge units at scale 2^38 (1 - 2^-10) / (largest charge): each particle
    # adds that scale x 0.6 (cells moved) x 1 (r weight) to one J_z node
    n = 36 * 2 ** 20
    nz, nr, dz, dr, dt = 32, 8, 0.2, 0.5, 0.13
    assert 1.2 * 2 ** 62 < n * 0.6 * 2 ** 38 * (1023 / 1024) < 1.5 * 2 ** 62
    rng = np.random.default_rng(7)
    z = (10 + 0.1 + 0.2 * rng.random(n)) * dz          # cell 10, offsets 0.1-0.3
    r = np.full(n, 3.0 * dr)                            # on the node row: r weights 1, 0
    vz = 0.6 * dz / dt                                  # 0.6 cell per step
    uz = np.full(n, vz / np.sqrt(1.0 - vz * vz))
    zeros = np.zeros(n)
    sim = q.Sim(nz, nr, dz, dr, dt=dt, max_particles=n)
    sim.load_particles(z, r, zeros, zeros, zeros, uz, np.ones(n))
    with pytest.raises(q.QpicError, match="EOVERFLOW"):
        sim.step(1)
