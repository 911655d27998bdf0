"""The plain FP64 GPU path against the oracle (same readings, double
precision: agreement to ~1e-12 per step), and the modal work of Eq. 16
(W_LWFA from the m = 0 field, W_DLA from m = 1) on both GPU paths."""
import numpy as np
import pytest

import paper_2303_12874_gb300 as q
import synth
from oracle import coeffs as C
from pairs import COMPS, compare_fields, make_pair, rel_l2, sync_fields

pytestmark = pytest.mark.gpu


def _fp64_pair(track_work=False, periodic=True, moving_window=False, nz=None):
    w = synth.workload("cfg1_small")
    nz = nz or w["nz"]
    nr, dz, dr, dt = w["nr"], w["dz"], w["dr"], 0.13
    sim = q.Sim(nz, nr, dz, dr, dt=dt, precision=q.QPIC_FP64, track_work=track_work,
                periodic=periodic, moving_window=moving_window)
    import oracle
    cE, cB = C.dual_coefficients(dt, dz)
    o = oracle.Oracle(nz, nr, 2, dz, dr, dt, cE, cB, C.filter_taps(cB), periodic=periodic,
                      track_work=track_work)
    pl, la = w["plasma"], w["laser"]
    sim.load_plasma(pl["n0"], pl["z_start"], pl["ramp_len"], pl["ppc"])
    sim.add_laser(la["a0"], la["w0"], la["fwhm"], la["z_centroid"], la["z_focus"])
    return sim, o


def _inject(sim, o):
    sync_fields(sim, o, ("E", "B"))
    p = sim.particles_raw()
    live = p["w"] > 0
    o.load_particles(*(p[k][live] for k in ("z", "r", "phi", "ux", "uy", "uz", "w")))
    return live


def test_fp64_path_one_step_and_ten():
    sim, o = _fp64_pair()
    sim.step(2)
    _inject(sim, o)
    sim.step(1)
    o.step(1)
    for which in ("E", "B", "J"):
        compare_fields(sim, o, which, 1e-11)
    sim.step(9)
    o.step(9)
    for which in ("E", "B"):
        compare_fields(sim, o, which, 1e-9)


def test_fp64_path_particles_match_oracle():
    sim, o = _fp64_pair()
    sim.step(2)
    live = _inject(sim, o)
    sim.step(1)
    o.step(1)
    g = sim.particles_raw()
    r = o.particles()
    for k in ("z", "r", "ux", "uy", "uz"):
        assert np.max(np.abs(g[k][live] - r[k])) < 1e-11 * (1 + np.abs(r[k]).max()), k


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_modal_work_eq16(precision):
    w = synth.workload("cfg1_small")
    nz, nr, dz, dr, dt = w["nz"], w["nr"], w["dz"], w["dr"], 0.13
    prec = q.QPIC_FP64 if precision == "fp64" else q.QPIC_FP32_FIXED
    sim = q.Sim(nz, nr, dz, dr, dt=dt, precision=prec, track_work=True)
    import oracle
    cE, cB = C.dual_coefficients(dt, dz)
    o = oracle.Oracle(nz, nr, 2, dz, dr, dt, cE, cB, C.filter_taps(cB), periodic=True,
                      track_work=True)
    pl, la = w["plasma"], w["laser"]
    sim.load_plasma(pl["n0"], pl["z_start"], pl["ramp_len"], pl["ppc"])
    sim.add_laser(2.0, la["w0"], la["fwhm"], la["z_centroid"], la["z_focus"])
    sim.step(6)                          # let the plasma respond: an m = 0 wake field appears
    live = _inject(sim, o)
    g0 = sim.particles_raw()
    sim.run_stages(1 | 2 | 4)            # one step without sort: buffer order kept
    o.step(1)
    g = sim.particles_raw()
    r = o.particles()
    tol = 1e-10 if precision == "fp64" else 2e-4
    for k in ("W0", "W1"):
        scale = np.abs(r[k]).max()
        assert scale > 0
        inc = g[k][live] - g0[k][live]
        assert np.max(np.abs(inc - r[k])) <= tol * scale, k
    # the laser (m = 1) does work where it overlaps the plasma; energy bookkeeping:
    # W0 + W1 equals the kinetic energy change to O(dt^2) per particle
    assert np.abs(r["W1"]).max() > 0
