"""The plain FP64 GPU path against the oracle (same readings, double
precision: agreement to ~1e-12 per step), and the per-particle work on both
GPU paths: the modal split of Eq. 16 (W_LWFA from the m = 0 field, W_DLA
from m = 1) and the directional split of Eq. 17 (W_z, W_perp)."""
import numpy as np
import pytest

import paper_2303_12874_gb300 as q
import synth
from oracle import coeffs as C
from pairs import compare_fields, oracle_config1_state, oracle_state_to_gpu

pytestmark = pytest.mark.gpu


def _fp64_pair(track_work=False, a0=None, warm=2):
    """config-1 state evolved by the oracle for `warm` steps, loaded into a
    plain-FP64 GPU context (nothing flows from the GPU to the oracle)"""
    import oracle
    w = synth.workload("cfg1_small")
    if a0 is not None:
        w = dict(w, laser=dict(w["laser"], a0=a0))
    nz, nr, dz, dr, dt = w["nz"], w["nr"], w["dz"], w["dr"], 0.13
    cE, cB = C.dual_coefficients(dt, dz)
    o = oracle.Oracle(nz, nr, 2, dz, dr, dt, cE, cB, C.filter_taps(cB), periodic=True,
                      track_work=track_work)
    oracle_config1_state(o, w, dt)
    if warm:
        o.step(warm)
    sim = q.Sim(nz, nr, dz, dr, dt=dt, precision=q.QPIC_FP64, track_work=track_work)
    oracle_state_to_gpu(o, sim)
    return sim, o


def test_fp64_path_one_step_and_ten():
    sim, o = _fp64_pair()
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
    sim.step(1)
    o.step(1)
    g = sim.particles_raw()                 # the FP64 path keeps the load order
    live = g["w"] > 0
    r = o.particles()
    for k in ("z", "r", "ux", "uy", "uz"):
        assert np.max(np.abs(g[k][live] - r[k])) < 1e-11 * (1 + np.abs(r[k]).max()), k


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("mode", [1, 2])
def test_work_eq16_eq17(precision, mode):
    """the oracle evolves a wake for 6 steps (laser a0 = 2); that state goes to
    the GPU (whose work counters start at 0) and both take one step: the GPU's
    W0, W1 equal the oracle's increments, for the modal split of Eq. 16
    (mode 1) and the directional split of Eq. 17 (mode 2).  The FP64 path
    keeps the particle order and is compared particle by particle; the FP32
    path sorts at load, so it is compared through the sums and the z-moments
    of the increments."""
    import oracle
    w = synth.workload("cfg1_small")
    w = dict(w, laser=dict(w["laser"], a0=2.0))
    nz, nr, dz, dr, dt = w["nz"], w["nr"], w["dz"], w["dr"], 0.13
    prec = q.QPIC_FP64 if precision == "fp64" else q.QPIC_FP32_FIXED
    cE, cB = C.dual_coefficients(dt, dz)
    o = oracle.Oracle(nz, nr, 2, dz, dr, dt, cE, cB, C.filter_taps(cB), periodic=True,
                      track_work=mode)
    oracle_config1_state(o, w, dt)
    o.step(6)                            # let the plasma respond: an m = 0 wake field appears
    r0 = o.particles()
    sim = q.Sim(nz, nr, dz, dr, dt=dt, precision=prec, track_work=mode)
    oracle_state_to_gpu(o, sim)
    sim.run_stages(1 | 2 | 4)            # one step without sort: buffer order kept
    o.step(1)
    g = sim.particles_raw()
    live = g["w"] > 0
    g = {k: v[live] for k, v in g.items()}
    r = o.particles()
    for k in ("W0", "W1"):
        inc = r[k] - r0[k]
        scale = np.abs(inc).max()
        assert scale > 0
        if precision == "fp64":
            assert np.max(np.abs(g[k] - inc)) <= 1e-10 * scale, k
        else:
            tot = np.abs(inc).sum()
            assert abs(g[k].sum() - inc.sum()) <= 1e-4 * tot, k
            assert abs((g[k] * g["z"]).sum() - (inc * r["z"]).sum()) <= 1e-4 * (np.abs(inc * r["z"]).sum()), k
    # the laser (m = 1) does work where it overlaps the plasma; energy bookkeeping:
    # W0 + W1 equals the kinetic energy change to O(dt^2) per particle
    assert np.abs(r["W1"] - r0["W1"]).max() > 0
