"""The oracle's multi-threaded mode (oracle/qpic_oracle.c, or_set_partitions).

The particles are deposited in P fixed ranges and the range currents summed
node by node in range order.  Field updates are per node and unchanged.  So:
- with P ranges the result is the same bit for bit for 1 or many threads;
- it differs from the serial oracle only by the order of the current's
  additions (round-off, < 1e-13 relative);
- P = 1 is the serial oracle itself."""
import numpy as np
import pytest

import synth
from oracle import coeffs as C
from oracle import setup


def _box(oracle_mod, partitions, threads):
    nz, nr, dz, dr, dt = 96, 24, 0.2, 0.5, 0.12
    cE, cB = C.dual_coefficients(dt, dz)
    o = oracle_mod.Oracle(nz, nr, 2, dz, dr, dt, cE, cB, C.filter_taps(cB), periodic=True,
                          partitions=partitions, threads=threads)
    p = setup.plasma_cells(np.arange(nz), nr, dz, dr, 0.02, 0.0, 0.0, (2, 2, 2), 5)
    rng = np.random.default_rng(3)
    for k in ("ux", "uy", "uz"):
        p[k] = rng.normal(0.0, 0.2, len(p["z"]))
    o.load_particles(**p)
    setup.add_laser(o, cE, cB, 1.5, 4.0, 5.0, 9.6, 9.6)
    o.step(6)
    return o


def _state(o):
    f = [o.fields(w) for w in ("E", "B", "J")]
    return f, o.particles()


def test_partitions_independent_of_threads_and_close_to_serial(oracle_mod):
    if not oracle_mod.Oracle.has_openmp():
        pytest.skip("oracle built without OpenMP")
    ser = _state(_box(oracle_mod, 1, 0))
    one = _state(_box(oracle_mod, 7, 1))
    many = _state(_box(oracle_mod, 7, 4))
    for a, b in zip(one[0], many[0]):
        assert np.array_equal(a, b)
    for k in one[1]:
        assert np.array_equal(one[1][k], many[1][k])
    for a, b in zip(one[0], ser[0]):
        assert np.max(np.abs(a - b)) <= 1e-13 * np.max(np.abs(b))
    for k in ("z", "r", "ux", "uy", "uz"):
        assert np.max(np.abs(one[1][k] - ser[1][k])) <= 1e-12 * (1 + np.max(np.abs(ser[1][k])))
    again = _state(_box(oracle_mod, 1, 4))          # P = 1 with threads: the serial path
    for a, b in zip(again[0], ser[0]):
        assert np.array_equal(a, b)
