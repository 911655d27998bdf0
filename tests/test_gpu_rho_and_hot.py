"""Charge density and energetic electrons on the GPU against the FP64 oracle.

- The charge density per mode (k_rho, the ion background and the Gauss-law
  diagnostic read it) through qpic_get_field(RHO) and the allocation-free entry
  point, element by element against Oracle.rho() of the same particles, before
  and after a step, on the FP32 and the plain FP64 paths.
- One particle stage with momenta up to |u| = 500 (gamma up to ~870): the
  paper's DLA electrons reach gamma ~ 10^2 - 10^3, above the 10 MeV cut
  (gamma > 20.6) of the spectrum.  The FP32 Boris push with rsqrt and the
  approximate square roots of the move are compared with the oracle there.
- A NaN in a field reaches the diagnostics, which then report QPIC_ENONFINITE."""
import ctypes

import numpy as np
import pytest

import paper_2303_12874_gb300 as q
import synth
from pairs import (compare_fields, distinct_weights, load_same_particles, make_pair,
                   match_by_weight, set_same_random_fields)

pytestmark = pytest.mark.gpu

DZ, DR = 0.2, 0.5


def _noalloc_rho(sim, mode):
    re = np.zeros((sim.nr + 1, sim.nz))
    im = np.zeros((sim.nr + 1, sim.nz))
    D = ctypes.POINTER(ctypes.c_double)
    st = sim.L.qpic_charge_density_noalloc(sim.h, mode, re.ctypes.data_as(D), im.ctypes.data_as(D))
    assert st == 0, sim.L.qpic_last_error(sim.h)
    return re + 1j * im


@pytest.mark.parametrize("precision", [q.QPIC_FP32_FIXED, q.QPIC_FP64])
def test_charge_density_matches_oracle(precision):
    nz, nr, nm = 72, 19, 3
    sim, o = make_pair(nz, nr, DZ, DR, 0.13, n_modes=nm, precision=precision)
    p = synth.random_particles(31, 30000, nz, nr, DZ, DR, umax=0.8)
    load_same_particles(sim, o, p)
    # FP32 path: the particles' offsets are FP32 (about 1e-7 of a cell)
    tol = 1e-5 if precision == q.QPIC_FP32_FIXED else 1e-12
    for stage in range(2):
        ref = o.rho()
        for m in range(nm):
            scale = np.max(np.abs(ref[m]))
            assert scale > 0
            for got in (sim.get_field("rho", "r", m), _noalloc_rho(sim, m)):
                assert np.max(np.abs(got - ref[m])) <= tol * scale, (stage, m)
        if stage == 0:
            # one particle stage on both sides (no fields: a ballistic move)
            sim.run_stages(2)
            o.push_deposit()


def test_particle_stage_with_energetic_electrons():
    nz, nr = 64, 17
    sim, o = make_pair(nz, nr, DZ, DR, 0.13)
    set_same_random_fields(sim, o, 8, amp=0.5)
    p = synth.random_particles(9, 20000, nz, nr, DZ, DR, umax=500.0)
    p["w"] = distinct_weights(len(p["z"]), 9)
    load_same_particles(sim, o, p)
    sim.run_stages(2)
    o.push_deposit()
    compare_fields(sim, o, "J", 1e-5)
    g = sim.particles_raw()
    live = g["w"] > 0
    g = {k: v[live] for k, v in g.items()}
    r = o.particles()
    ig, ir = match_by_weight(g, r)
    g = {k: v[ig] for k, v in g.items()}
    r = {k: v[ir] for k, v in r.items()}
    gamma = np.sqrt(1 + r["ux"] ** 2 + r["uy"] ** 2 + r["uz"] ** 2)
    assert np.max(gamma) > 500
    for k in ("ux", "uy", "uz"):
        # FP32: relative to the particle's own |u|
        assert np.max(np.abs(g[k] - r[k]) / gamma) < 2e-6, k
    Lz = nz * DZ
    dzz = np.abs((g["z"] - r["z"] + 0.5 * Lz) % Lz - 0.5 * Lz)
    assert np.max(dzz) < 1e-5
    assert np.max(np.abs(g["r"] - r["r"])) < 1e-5


def test_non_finite_fields_are_reported():
    sim = q.Sim(48, 12, DZ, DR, dt=0.13)
    sim.load_plasma(0.01, 0.0, 0.0, (1, 1, 2))
    assert sim.diag()["particles"] > 0
    bad = np.zeros((13, 48))
    bad[5, 7] = np.nan
    sim.set_field("E", "z", 0, bad)
    with pytest.raises(q.QpicError, match="ENONFINITE"):
        sim.diag()
