"""Absorbing radial layer (graded conductivity next to the wall, centred lossy
update): CUDA path against the FP64 oracle, stage by stage and over many
steps, on the FP32 and FP64 paths; rows outside the layer unchanged bit for
bit; the layer's absorption of an outgoing pulse measured on the GPU itself;
invalid settings refused."""
import numpy as np
import pytest

import paper_2303_12874_gb300 as q
import synth
from pairs import (compare_fields, load_same_particles, make_pair, oracle_config1_state,
                   oracle_state_to_gpu, set_same_random_fields)

pytestmark = pytest.mark.gpu

DZ, DR = 0.2, 0.5


@pytest.mark.parametrize("nabs,sigma", [(6, 0.0), (6, 3.0), (19, 0.0)])
def test_field_stages_with_layer(nabs, sigma):
    """nabs = nr: the layer reaches the axis rows (advanced in FP64)"""
    sim, o = make_pair(100, 19, DZ, DR, 0.13, absorb_cells=nabs, absorb_sigma=sigma)
    set_same_random_fields(sim, o, 11)
    sim.run_stages(1)
    o.faraday()
    compare_fields(sim, o, "B", 1e-6)
    compare_fields(sim, o, "Bbar", 1e-6)
    sim.run_stages(4)
    o.ampere()
    compare_fields(sim, o, "E", 1e-6)


def test_full_steps_config1_with_layer():
    w = synth.workload("cfg1_small")
    nz, nr = w["nz"], w["nr"]
    sim, o = make_pair(nz, nr, w["dz"], w["dr"], 0.13, absorb_cells=8)
    oracle_config1_state(o, w, 0.13)
    o.step(3)
    oracle_state_to_gpu(o, sim)
    sim.step(1)
    o.step(1)
    for which in ("E", "B", "J"):
        compare_fields(sim, o, which, 1e-5)
    sim.step(19)
    o.step(19)
    compare_fields(sim, o, "E", 1e-4)
    compare_fields(sim, o, "B", 1e-4)


def test_fp64_path_with_layer():
    sim, o = make_pair(64, 24, DZ, DR, 0.13, absorb_cells=10, precision=q.QPIC_FP64)
    set_same_random_fields(sim, o, 12)
    sim.step(5)
    o.step(5)
    compare_fields(sim, o, "E", 1e-11)
    compare_fields(sim, o, "B", 1e-11)


def test_rows_outside_the_layer_are_unchanged():
    nz, nr, nabs, n = 64, 40, 8, 5
    out = []
    for cells in (0, nabs):
        sim, o = make_pair(nz, nr, DZ, DR, 0.13, absorb_cells=cells)
        set_same_random_fields(sim, o, 13)
        sim.step(n)
        out.append(sim)
    keep = nr - nabs - n - 1
    for which in ("E", "B"):
        a, b = out[0].fields(which), out[1].fields(which)
        assert np.array_equal(a[..., :keep, :], b[..., :keep, :]), which
        assert not np.array_equal(a, b)


def _pulse(nr, nabs, nsteps, snap=10, nz=16, dt=0.3):
    sim = q.Sim(nz, nr, 0.5, 0.5, n_modes=1, dt=dt, solver="yee", absorb_cells=nabs)
    r = np.arange(nr + 1) * 0.5
    sim.set_field("E", "z", 0, np.exp(-(r / 3.0) ** 2)[:, None] * np.ones((1, nz)))
    out = []
    for _ in range(nsteps // snap):
        sim.step(snap)
        out.append(np.stack([sim.get_field("E", "z", 0).real, sim.get_field("B", "phi", 0).real]))
    return out


def test_outgoing_pulse_is_absorbed_on_the_gpu():
    """the oracle's pin, repeated on the FP32 path: what comes back into
    r < 25 from a 20-cell layer stays below 4% of the pulse, against more
    than half from the conducting wall"""
    nr, T, ji = 100, 330, 50
    ref = _pulse(nr + 400, 0, T)
    refn = max(np.linalg.norm(a[:, :ji]) for a in ref)
    back = {}
    for cells in (0, 20):
        x = _pulse(nr, cells, T)
        back[cells] = max(np.linalg.norm(a[:, :ji] - b[:, :ji]) for a, b in zip(x, ref)) / refn
    assert back[0] > 0.5 and back[20] < 0.04, back


@pytest.mark.parametrize("cells,sigma", [(-1, 0.0), (41, 0.0), (4, -1.0), (4, float("nan"))])
def test_invalid_layer_is_refused(cells, sigma):
    with pytest.raises(q.QpicError, match="EINVAL"):
        q.Sim(64, 40, DZ, DR, absorb_cells=cells, absorb_sigma=sigma)
