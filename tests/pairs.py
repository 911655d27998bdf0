"""Helpers for GPU-vs-oracle parity tests: build a CUDA context and an oracle
box with the same grid and time step (each side fits its own coefficients),
and give both the same state.  Data only flow towards the GPU: both sides get
the same FP64 seeded inputs (the GPU rounds them to FP32), or the oracle
evolves a state that is then loaded into the GPU.  Nothing read back from the
GPU is ever an oracle input; a one-step comparison therefore includes the FP32
rounding of the inputs (about 1e-7, well inside the 1e-5 tolerance)."""
import numpy as np

import oracle
import paper_2303_12874_gb300 as q
from oracle import coeffs as C

COMPS = ("r", "phi", "z")


def make_pair(nz, nr, dz, dr, dt, n_modes=2, solver="dual", periodic=True, jz_filter=True,
              track_work=False, tile=(16, 8), sort_period=2, moving_window=False,
              precision=q.QPIC_FP32_FIXED, particles_per_thread=16, absorb_cells=0, absorb_sigma=0.0):
    sim = q.Sim(nz, nr, dz, dr, n_modes=n_modes, dt=dt, solver=solver, periodic=periodic,
                jz_filter=jz_filter, track_work=track_work, tile_z=tile[0], tile_r=tile[1],
                sort_period=sort_period, moving_window=moving_window, precision=precision,
                particles_per_thread=particles_per_thread, absorb_cells=absorb_cells,
                absorb_sigma=absorb_sigma)
    cE, cB = C.solver_coefficients(solver, dt, dz)
    taps = C.filter_taps(cB) if (jz_filter and solver != "yee") else None
    o = oracle.Oracle(nz, nr, n_modes, dz, dr, dt, cE, cB, taps, periodic=periodic,
                      track_work=track_work, absorb_cells=absorb_cells, absorb_sigma=absorb_sigma)
    return sim, o


def random_field_arrays(nz, nr, nm, seed, amp=0.3, which_list=("E", "B", "Bbar")):
    """seeded FP64 field planes {(which, comp, mode): [nr+1][nz]} (complex for m >= 1)"""
    rng = np.random.default_rng(seed)
    out = {}
    for which in which_list:
        for c in COMPS:
            for m in range(nm):
                v = rng.standard_normal((nr + 1, nz))
                if m:
                    v = v + 1j * rng.standard_normal((nr + 1, nz))
                out[(which, c, m)] = amp * v
    return out


def set_same_fields(sim, o, arrays):
    for (which, c, m), v in arrays.items():
        sim.set_field(which, c, m, v)
        o.set_field(which, c, m, v)


def set_same_random_fields(sim, o, seed, amp=0.3, which_list=("E", "B", "Bbar")):
    set_same_fields(sim, o, random_field_arrays(sim.nz, sim.nr, sim.nm, seed, amp, which_list))


def load_same_particles(sim, o, parts):
    """the same FP64 particle arrays into both sides"""
    keys = ("z", "r", "phi", "ux", "uy", "uz", "w")
    sim.load_particles(**{k: parts[k] for k in keys})
    o.load_particles(*(np.asarray(parts[k], dtype=np.float64) for k in keys))


def oracle_state_to_gpu(o, sim, which_list=("E", "B")):
    """load the oracle's fields and particles into the GPU context"""
    for which in which_list:
        for c in COMPS:
            for m in range(sim.nm):
                sim.set_field(which, c, m, o.get_field(which, c, m))
    p = o.particles()
    live = p["w"] > 0
    sim.load_particles(*(p[k][live] for k in ("z", "r", "phi", "ux", "uy", "uz", "w")))


def oracle_config1_state(o, w, dt):
    """the config-1 plasma (the oracle's generator) and laser on the oracle"""
    from oracle import setup
    pl, la = w["plasma"], w["laser"]
    parts = setup.plasma_cells(np.arange(w["nz"]), w["nr"], w["dz"], w["dr"], pl["n0"], pl["z_start"],
                               pl["ramp_len"], pl["ppc"], pl["seed"])
    o.load_particles(**parts)
    cE, cB = C.solver_coefficients(w.get("solver", "dual"), dt, w["dz"])
    setup.add_laser(o, cE, cB, la["a0"], la["w0"], la["fwhm"], la["z_centroid"], la["z_focus"])
    return parts


def distinct_weights(n, seed):
    """n weights in (0.5, 1.5), pairwise distinct in FP32 (particles can then be
    matched by weight across buffer orders: the push never changes w)"""
    rng = np.random.default_rng(seed)
    return 0.5 + (rng.permutation(n) + 0.5) / n


def match_by_weight(g, r):
    """index arrays (ig, ir) pairing GPU and oracle particles with equal weights"""
    ig = np.argsort(np.asarray(g["w"], dtype=np.float32), kind="stable")
    ir = np.argsort(np.asarray(r["w"], dtype=np.float32), kind="stable")
    assert np.array_equal(np.asarray(g["w"], np.float32)[ig], np.asarray(r["w"], np.float32)[ir])
    return ig, ir


def rel_l2(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def compare_fields(sim, o, which, tol, modes=None, skip_rows=None):
    out = {}
    for c in COMPS:
        for m in (modes if modes is not None else range(sim.nm)):
            g = sim.get_field(which, c, m)
            r = o.get_field(which, c, m)
            if skip_rows is not None:
                g, r = g[skip_rows], r[skip_rows]
            out[(c, m)] = rel_l2(g, r)
    bad = {k: v for k, v in out.items() if v > tol}
    assert not bad, "%s rel-L2 above %g: %s" % (which, tol, bad)
    return out


def angle_diff(a, b):
    return np.angle(np.exp(1j * (a - b)))
