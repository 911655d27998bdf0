"""CUDA path vs the FP64 oracle, stage by stage and step by step, from the
same FP64 inputs or from a state the oracle evolved (tests/pairs.py; nothing
read back from the GPU feeds the oracle).  Tolerance: relative L2 <= 1e-5 per field,
component and mode for one step (the FP32 + int64 fixed-point target), particle
coordinates to FP32 precision.  Sizes span several 16 x 8 particle tiles and a
ragged tail (nz, nr not multiples of the tile)."""
import numpy as np
import pytest

import synth
from oracle import setup
from pairs import (COMPS, angle_diff, compare_fields, distinct_weights, load_same_particles,
                   make_pair, match_by_weight, oracle_config1_state, oracle_state_to_gpu, rel_l2,
                   set_same_random_fields)

pytestmark = pytest.mark.gpu

DZ, DR = 0.2, 0.5
TOL = 1e-5


def _random_particles(n, nz, nr, seed, umax=1.0):
    p = synth.random_particles(seed, n, nz, nr, DZ, DR, umax=umax)
    p["w"] = distinct_weights(n, seed)          # lets particles be matched across buffer orders
    return p


def test_faraday_stage():
    sim, o = make_pair(100, 21, DZ, DR, 0.13)
    set_same_random_fields(sim, o, 1)
    sim.run_stages(1)
    o.faraday()
    compare_fields(sim, o, "B", 1e-6)
    compare_fields(sim, o, "Bbar", 1e-6)


@pytest.mark.parametrize("n_modes", [1, 2, 3])
def test_particle_stage(n_modes):
    nz, nr = 70, 19
    sim, o = make_pair(nz, nr, DZ, DR, 0.13, n_modes=n_modes)
    set_same_random_fields(sim, o, 2, amp=0.5)
    load_same_particles(sim, o, _random_particles(20000, nz, nr, 3))
    sim.run_stages(2)                    # gather + push + deposit (+ decode)
    o.push_deposit()
    compare_fields(sim, o, "J", TOL)
    g = sim.particles_raw()
    live = g["w"] > 0
    g = {k: v[live] for k, v in g.items()}
    r = o.particles()
    ig, ir = match_by_weight(g, r)
    gl = {k: v[ig] for k, v in g.items()}
    r = {k: v[ir] for k, v in r.items()}
    Lz = nz * DZ
    dzz = np.abs((gl["z"] - r["z"] + 0.5 * Lz) % Lz - 0.5 * Lz)
    assert np.max(dzz) < 2e-5 * DZ * 50
    assert np.max(np.abs(gl["r"] - r["r"])) < 1e-5
    m = r["r"] > 0.05
    assert np.max(np.abs(angle_diff(gl["phi"][m], r["phi"][m]))) < 1e-4
    for k in ("ux", "uy", "uz"):
        assert np.max(np.abs(gl[k] - r[k])) < 1e-5 * (1 + np.abs(r[k]).max())


def test_ampere_stage():
    nz, nr = 70, 19
    sim, o = make_pair(nz, nr, DZ, DR, 0.13)
    set_same_random_fields(sim, o, 4, amp=0.5)
    load_same_particles(sim, o, _random_particles(20000, nz, nr, 5))
    sim.run_stages(2 | 4)
    o.push_deposit()
    o.ampere()
    compare_fields(sim, o, "J", TOL)
    compare_fields(sim, o, "E", TOL)


def _config1_state(sim, o, nsteps_warm=0):
    w = synth.workload("cfg1_small")
    pl, la = w["plasma"], w["laser"]
    sim.load_plasma(pl["n0"], pl["z_start"], pl["ramp_len"], pl["ppc"])
    sim.add_laser(la["a0"], la["w0"], la["fwhm"], la["z_centroid"], la["z_focus"])
    return w


def test_load_plasma_matches_oracle():
    w = synth.workload("cfg1_small")
    nz, nr = w["nz"], w["nr"]
    sim, o = make_pair(nz, nr, w["dz"], w["dr"], 0.13)
    pl = w["plasma"]
    sim.load_plasma(pl["n0"], pl["z_start"], pl["ramp_len"], pl["ppc"])
    g = sim.particles()
    r = setup.plasma_cells(np.arange(nz), nr, w["dz"], w["dr"], pl["n0"], pl["z_start"],
                           pl["ramp_len"], pl["ppc"], pl["seed"])
    assert len(g["z"]) == len(r["z"]) == nz * nr * 8
    kg = np.lexsort((np.round(np.mod(g["phi"], 2 * np.pi), 5), np.round(g["r"], 6), np.round(g["z"], 6)))
    kr = np.lexsort((np.round(np.mod(r["phi"], 2 * np.pi), 5), np.round(r["r"], 6), np.round(r["z"], 6)))
    assert np.max(np.abs(g["z"][kg] - r["z"][kr])) < 1e-5
    assert np.max(np.abs(g["r"][kg] - r["r"][kr])) < 1e-5
    assert np.max(np.abs(angle_diff(g["phi"][kg], r["phi"][kr]))) < 1e-6
    assert np.max(np.abs(g["w"][kg] / r["w"][kr] - 1)) < 1e-6


def test_laser_matches_oracle():
    w = synth.workload("cfg1_small")
    sim, o = make_pair(w["nz"], w["nr"], w["dz"], w["dr"], 0.13)
    la = w["laser"]
    sim.add_laser(la["a0"], la["w0"], la["fwhm"], la["z_centroid"], la["z_focus"], 0.3)
    setup.add_laser(o, o_cE(o), o_cB(o), la["a0"], la["w0"], la["fwhm"], la["z_centroid"],
                    la["z_focus"], 0.3)
    compare_fields(sim, o, "E", 1e-6, modes=[1])
    compare_fields(sim, o, "B", 1e-6, modes=[1])


def o_cE(o):
    from oracle import coeffs as C
    return C.dual_coefficients(o.dt, o.dz)[0]


def o_cB(o):
    from oracle import coeffs as C
    return C.dual_coefficients(o.dt, o.dz)[1]


@pytest.mark.parametrize("solver,sort_period,ppt", [("dual", 2, 8), ("yee", 2, 8), ("dual", 1, 8),
                                                    ("dual", 3, 8), ("dual", 2, 1), ("dual", 2, 3),
                                                    ("dual", 2, 16)])
def test_full_step_config1(solver, sort_period, ppt):
    """sort_period 3 leaves particles up to 2 cells outside their tile: those
    take the global-memory path of the same kernel.  ppt: particles per thread
    (1: chunks of 256 particles, so a 16 x 8 tile of this plasma (1024
    particles) is deposited in several chunks with a drain between them;
    16: chunks of 4096, the largest the 32-bit planes allow)"""
    w = synth.workload("cfg1_small")
    nz, nr = w["nz"], w["nr"]
    from oracle import coeffs as C
    dt = 0.9 * C.cfl_dt(w["dz"], w["dr"], nr, 2, solver)
    sim, o = make_pair(nz, nr, w["dz"], w["dr"], dt, solver=solver, sort_period=sort_period,
                       particles_per_thread=ppt)
    oracle_config1_state(o, dict(w, solver=solver), dt)
    # the oracle builds up currents and plasma motion; its state goes to the GPU
    o.step(3)
    oracle_state_to_gpu(o, sim)
    # sort period 3: steps 2 and 3 run with particles drifted beyond their tiles
    nst = 3 if sort_period == 3 else 1
    sim.step(nst)
    o.step(nst)
    for which in ("E", "B", "J"):
        compare_fields(sim, o, which, TOL)


def test_particles_per_thread_leaves_results_unchanged():
    """the particles each thread takes in a row only regroup the exact
    integer sums of the deposit: fields bit-identical for 1, 3, 8 and 16"""
    w = synth.workload("cfg1_small")
    out = []
    for ppt in (1, 3, 8, 16):
        sim, _o = make_pair(w["nz"], w["nr"], w["dz"], w["dr"], 0.13, particles_per_thread=ppt)
        _config1_state(sim, _o)
        sim.step(5)
        out.append([sim.fields(f) for f in ("E", "B", "J")])
    for other in out[1:]:
        for a, b in zip(out[0], other):
            assert np.array_equal(a, b)


def test_bit_reproducible():
    """int64 deposit: fields and the particle set are bit-identical run to run.
    The particle buffer order (atomic counting sort) may differ, so particles
    are compared as sorted sets, and FP64 sums over particles to round-off."""
    w = synth.workload("cfg1_small")
    out = []
    for _ in range(2):
        sim, _o = make_pair(w["nz"], w["nr"], w["dz"], w["dr"], 0.13)
        _config1_state(sim, _o)
        sim.step(5)
        p = sim.particles()
        key = np.lexsort((p["uz"], p["phi"], p["r"], p["z"]))
        out.append((sim.fields("E"), sim.fields("B"), sim.fields("J"),
                    np.array([p[k][key] for k in ("z", "r", "phi", "ux", "uy", "uz", "w")]),
                    sim.diag()["kinetic"]))
    for a, b in zip(out[0][:4], out[1][:4]):
        assert np.array_equal(np.asarray(a), np.asarray(b))
    assert abs(out[0][4] - out[1][4]) <= 1e-13 * abs(out[0][4])


def test_multi_step_config1_tracks_oracle():
    w = synth.workload("cfg1_small")
    nz, nr = w["nz"], w["nr"]
    sim, o = make_pair(nz, nr, w["dz"], w["dr"], 0.13)
    oracle_config1_state(o, w, 0.13)
    oracle_state_to_gpu(o, sim)
    sim.step(20)
    o.step(20)
    compare_fields(sim, o, "E", 1e-4)
    compare_fields(sim, o, "B", 1e-4)


@pytest.mark.parametrize("n_modes,tile", [(1, (16, 8)), (2, (32, 8)), (2, (8, 8)), (2, (16, 16)),
                                          (2, (32, 4)), (3, (16, 8)), (4, (16, 8))])
def test_particle_stage_tiled(n_modes, tile):
    """the deposit through the staged shared-memory tiles (register sums for
    moves inside a cell, the queue for moves across cells) for every tile shape
    and one to four modes; nz = 100 and nr = 19 leave ragged tiles for every
    shape"""
    nz, nr = 100, 19
    from oracle import coeffs as C
    dt = min(0.13, 0.9 * C.cfl_dt(DZ, DR, nr, n_modes, "dual"))    # higher m lowers the limit
    sim, o = make_pair(nz, nr, DZ, DR, dt, n_modes=n_modes, tile=tile)
    set_same_random_fields(sim, o, 5, amp=0.5)
    load_same_particles(sim, o, _random_particles(30000, nz, nr, 6))
    sim.run_stages(16)                   # sort into tiles
    sim.run_stages(2)                    # gather + push + deposit (+ reduction)
    o.push_deposit()
    compare_fields(sim, o, "J", TOL)
    ke_g = sim.diag()["kinetic"]
    pr = o.particles()
    ke_o = float(np.sum(pr["w"] * (np.sqrt(1 + pr["ux"] ** 2 + pr["uy"] ** 2 + pr["uz"] ** 2) - 1)))
    assert abs(ke_g / ke_o - 1) < 1e-5


def test_field_copies_check_the_buffer_length():
    """qpic_get_fields / qpic_set_fields refuse buffers shorter than (nr+1)*nz
    and copy nothing; the full length works"""
    import ctypes
    sim, _o = make_pair(40, 9, DZ, DR, 0.13)
    D = ctypes.POINTER(ctypes.c_double)
    n = (sim.nr + 1) * sim.nz
    re = np.full(n, 7.0)
    im = np.zeros(n)
    assert sim.L.qpic_get_fields(sim.h, 0, 2, 0, re.ctypes.data_as(D), im.ctypes.data_as(D), n - 1) == -1
    assert np.all(re == 7.0)
    assert sim.L.qpic_set_fields(sim.h, 0, 2, 0, re.ctypes.data_as(D), im.ctypes.data_as(D), n - 1) == -1
    assert sim.L.qpic_set_fields(sim.h, 0, 2, 0, re.ctypes.data_as(D), im.ctypes.data_as(D), n) == 0
    back = np.zeros(n)
    assert sim.L.qpic_get_fields(sim.h, 0, 2, 0, back.ctypes.data_as(D), None, n) == 0
    assert np.array_equal(back, re)


def test_set_field_takes_re_im_pairs():
    """set_field with a (re, im) pair of float64 arrays stores what the complex
    form stores; a pair of the wrong size is refused"""
    sim, _o = make_pair(40, 9, DZ, DR, 0.13)
    rng = np.random.default_rng(3)
    shape = (sim.nr + 1, sim.nz)
    re, im = rng.standard_normal(shape), rng.standard_normal(shape)
    sim.set_field("B", "phi", 1, (re, im))
    got = sim.get_field("B", "phi", 1)
    sim.set_field("B", "phi", 1, re + 1j * im)
    assert np.array_equal(got, sim.get_field("B", "phi", 1))
    assert np.array_equal(got.real, re.astype(np.float32).astype(np.float64))
    with pytest.raises(ValueError):
        sim.set_field("B", "phi", 1, (re[:-1], im[:-1]))


def test_box_shorter_than_two_staged_tiles():
    """nz = 24 < 2 x (16 + 5): the staged tile would overlap its own wrap, so
    every particle takes the global-memory path of the same kernel"""
    nz, nr = 24, 19
    sim, o = make_pair(nz, nr, DZ, DR, 0.13)
    set_same_random_fields(sim, o, 21, amp=0.5)
    load_same_particles(sim, o, _random_particles(6000, nz, nr, 22))
    sim.step(1)
    o.step(1)
    for which in ("E", "B", "J"):
        compare_fields(sim, o, which, TOL)
