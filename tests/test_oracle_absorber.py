"""Pins of the oracle's absorbing radial layer (an extension: the paper's runs
end at a conducting wall).  The layer's conductivity must (a) leave every
row it cannot yet have influenced bit-identical to a run without it (the r
stencil spreads one row per step), (b) damp a uniform field at the lossy-medium
rate e^{-sigma t} to the accuracy of the centred update, and (c) return far
less of an outgoing cylindrical pulse than the conducting wall does, measured
against a box so large that nothing comes back within the run."""
import numpy as np

import oracle
from oracle import coeffs as C


def _box(nz, nr, nm, dt, nabs, sigma=0.0, dz=0.5, dr=0.5, solver="yee"):
    cE, cB = C.solver_coefficients(solver, dt, dz)
    return oracle.Oracle(nz, nr, nm, dz, dr, dt, cE, cB, None, periodic=True, absorb_cells=nabs,
                         absorb_sigma=sigma)


def test_rows_outside_its_reach_are_untouched(oracle_mod):
    nz, nr, nm, nabs, n = 16, 40, 2, 8, 5
    rng = np.random.default_rng(3)
    fields = {(w, c, m): rng.standard_normal((nr + 1, nz)) + (1j * rng.standard_normal((nr + 1, nz)) if m else 0)
              for w in ("E", "B") for c in ("r", "phi", "z") for m in range(nm)}
    out = []
    for cells in (0, nabs):
        o = _box(nz, nr, nm, 0.2, cells, solver="dual")
        for (w, c, m), v in fields.items():
            o.set_field(w, c, m, v)
        o.step(n)
        out.append(o)
    first = nr - nabs                      # first row with a loss (its E_z, E_phi, B_r at r > r0)
    keep = first - n - 1                   # rows the layer cannot have reached after n steps
    changed = False
    for w in ("E", "B"):
        for c in ("r", "phi", "z"):
            for m in range(nm):
                a, b = out[0].get_field(w, c, m), out[1].get_field(w, c, m)
                assert np.array_equal(a[:keep], b[:keep]), (w, c, m)
                changed |= not np.array_equal(a[first:], b[first:])
    assert changed


def test_uniform_field_decays_at_the_lossy_medium_rate(oracle_mod):
    """a uniform E_z with no B: away from the wall the curl stays zero for the
    first step, so each row is multiplied by the update's decay factor, which
    must agree with e^{-sigma dt} to third order in sigma dt"""
    nz, nr, nabs, dt, dr, smax = 4, 40, 20, 0.2, 0.5, 2.0
    o = _box(nz, nr, 1, dt, nabs, smax, dr=dr)
    o.set_field("E", "z", 0, np.ones((nr + 1, nz)))
    o.step(1)
    ez = o.get_field("E", "z", 0).real[:, 0]
    r0 = (nr - nabs) * dr
    for j in range(nr - nabs - 3, nr - 2):
        r = j * dr
        sdt = smax * (max(r - r0, 0.0) / (nabs * dr)) ** 2 * dt
        assert abs(ez[j] - np.exp(-sdt)) <= sdt ** 3 / 12 + 1e-15, (j, ez[j], np.exp(-sdt))
    assert ez[nr - nabs - 3] == 1.0 and ez[nr - 3] < 0.8


def _pulse(nr, nabs, nsteps, sigma=0.0, nz=8, dt=0.3, snap=10):
    o = _box(nz, nr, 1, dt, nabs, sigma)
    r = np.arange(nr + 1) * 0.5
    o.set_field("E", "z", 0, np.exp(-(r / 3.0) ** 2)[:, None] * np.ones((1, nz)))
    out = []
    for k in range(nsteps):
        o.step(1)
        if (k + 1) % snap == 0:
            out.append(np.stack([o.get_field("E", "z", 0).real, o.get_field("B", "phi", 0).real]))
    return out


def test_outgoing_pulse_is_absorbed(oracle_mod):
    """an m = 0 cylindrical pulse uniform in z (k_z = 0) goes out to the wall
    at r = 50 and, with a conducting wall, comes back in full; with a 20-cell
    layer (default sigma_max) what comes back into r < 25 within 99 time units
    stays below 4% of the pulse (the layer is matched only in the continuum)"""
    nr, T, ji = 100, 330, 50
    ref = _pulse(nr + 400, 0, T)
    refn = max(np.linalg.norm(a[:, :ji]) for a in ref)
    back = {}
    for cells in (0, 20):
        x = _pulse(nr, cells, T)
        back[cells] = max(np.linalg.norm(a[:, :ji] - b[:, :ji]) for a, b in zip(x, ref)) / refn
    assert back[0] > 0.5, back
    assert back[20] < 0.04, back
