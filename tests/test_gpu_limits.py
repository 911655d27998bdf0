"""The largest grids allowed (nz + gap < 32768 columns for the packed cell
index; nr < 65535 rows, the field kernels taking one block row per grid
row): accepted one below the limit and stepped with particles in
the last column and next to the wall (the same charge-conserving step as
anywhere else: total charge and particle count kept, fields finite); refused
at the limit."""
import numpy as np
import pytest

import paper_2303_12874_gb300 as q

pytestmark = pytest.mark.gpu


def _particles(n, zmax, rmax, seed):
    rng = np.random.default_rng(seed)
    z = zmax - 0.01 - rng.random(n) * 3.0
    r = rmax - 0.01 - rng.random(n) * 1.5
    u = 0.3 * rng.standard_normal((3, n))
    return z, r, rng.uniform(0, 2 * np.pi, n), u[0], u[1], u[2], np.full(n, 1e-3)


@pytest.mark.parametrize("nz,nr", [(32767, 2), (16, 65534)], ids=["widest", "tallest"])
def test_largest_grid_steps(nz, nr):
    dz, dr = 0.2, 0.5
    sim = q.Sim(nz, nr, dz, dr, tile_z=16, tile_r=8)
    p = _particles(4096, nz * dz, nr * dr, 3)
    sim.load_particles(*p)
    q0 = sim.diag()["charge"]
    sim.step(3)
    d = sim.diag()
    assert d["particles"] == 4096
    assert abs(d["charge"] - q0) <= 1e-12 * abs(q0)
    for which in ("E", "B", "J"):
        f = sim.fields(which)
        assert np.all(np.isfinite(f)) and np.abs(f).max() > 0, which


@pytest.mark.parametrize("nz,nr", [(32768, 2), (16, 65535)])
def test_grid_at_the_limit_is_refused(nz, nr):
    with pytest.raises(q.QpicError, match="EINVAL"):
        q.Sim(nz, nr, 0.2, 0.5)


@pytest.mark.parametrize("n_modes,tile", [(3, (32, 8)), (4, (32, 8)), (4, (16, 16))])
def test_tile_too_large_for_the_modes_is_refused(n_modes, tile):
    """the particle kernel's block (staged fields, accumulators) must fit the
    device's shared memory: these mode counts and tiles would not"""
    with pytest.raises(q.QpicError, match="EINVAL"):
        q.Sim(64, 16, 0.2, 0.5, n_modes=n_modes, tile_z=tile[0], tile_r=tile[1])
    q.Sim(64, 16, 0.2, 0.5, n_modes=n_modes, tile_z=8, tile_r=8, precision=q.QPIC_FP64)   # no tiles: fine


@pytest.mark.parametrize("kw", [dict(particles_per_thread=17), dict(particles_per_thread=-1),
                                dict(tile_z=16, tile_r=4), dict(tile_z=7), dict(sort_period=-3)])
def test_invalid_particle_settings_are_refused(kw):
    with pytest.raises(q.QpicError, match="EINVAL"):
        q.Sim(64, 16, 0.2, 0.5, **kw)
