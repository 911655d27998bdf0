"""Helpers for GPU-vs-oracle parity tests: build a CUDA context and an oracle
box with the same grid and time step (each side fits its own coefficients),
and inject one identical state into both.  The state is first written to the
GPU and read back, so the oracle starts from exactly the FP32-rounded values
the kernels see; a comparison after one step then measures that step only."""
import numpy as np

import oracle
import paper_2303_12874_gb300 as q
from oracle import coeffs as C

COMPS = ("r", "phi", "z")


def make_pair(nz, nr, dz, dr, dt, n_modes=2, solver="dual", periodic=True, jz_filter=True,
              track_work=False, tile=(16, 8), sort_period=2, moving_window=False,
              precision=q.QPIC_FP32_FIXED):
    sim = q.Sim(nz, nr, dz, dr, n_modes=n_modes, dt=dt, solver=solver, periodic=periodic,
                jz_filter=jz_filter, track_work=track_work, tile_z=tile[0], tile_r=tile[1],
                sort_period=sort_period, moving_window=moving_window, precision=precision)
    cE, cB = C.solver_coefficients(solver, dt, dz)
    taps = C.filter_taps(cB) if (jz_filter and solver != "yee") else None
    o = oracle.Oracle(nz, nr, n_modes, dz, dr, dt, cE, cB, taps, periodic=periodic,
                      track_work=track_work)
    return sim, o


def sync_fields(sim, o, which_list=("E", "B", "Bbar")):
    """copy the GPU's (FP32-rounded) fields into the oracle"""
    for which in which_list:
        for c in COMPS:
            for m in range(sim.nm):
                o.set_field(which, c, m, sim.get_field(which, c, m))


def set_random_fields(sim, seed, amp=0.3, which_list=("E", "B", "Bbar")):
    rng = np.random.default_rng(seed)
    for which in which_list:
        for c in COMPS:
            for m in range(sim.nm):
                v = rng.standard_normal((sim.nr + 1, sim.nz))
                if m:
                    v = v + 1j * rng.standard_normal((sim.nr + 1, sim.nz))
                sim.set_field(which, c, m, amp * v)


def load_same_particles(sim, o, parts):
    sim.load_particles(**parts)
    p = sim.particles_raw()
    live = p["w"] > 0
    o.load_particles(p["z"][live], p["r"][live], p["phi"][live], p["ux"][live], p["uy"][live],
                     p["uz"][live], p["w"][live])
    return p, live


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
