"""The allocation-free charge-density entry point (qpic_charge_density_noalloc).

It exists for callers that cannot allocate device memory during the call, for
example hosts with a fixed device-memory budget or code running inside a
device allocator's callbacks.  Its result must equal the allocating path
(qpic_get_field with QPIC_FIELD_RHO) -- on two calls in a row, so a second call
does not add onto what the first left in the shared static array -- on the
FP32 fixed-point path and the plain FP64 path, and grids too large for the
static array are refused.

This file is named to be collected last: if it fails, a run that stops at the
first failure has already run every other test."""
import ctypes

import numpy as np
import pytest

import paper_2303_12874_gb300 as q

pytestmark = pytest.mark.gpu


def _noalloc(sim, mode):
    re = np.zeros((sim.nr + 1, sim.nz))
    im = np.zeros((sim.nr + 1, sim.nz))
    D = ctypes.POINTER(ctypes.c_double)
    st = sim.L.qpic_charge_density_noalloc(sim.h, mode, re.ctypes.data_as(D), im.ctypes.data_as(D))
    return st, re + 1j * im


@pytest.mark.parametrize("precision", [q.QPIC_FP32_FIXED, q.QPIC_FP64])
def test_noalloc_matches_allocating_path_twice(precision):
    sim = q.Sim(96, 20, 0.2, 0.5, n_modes=2, dt=0.13, precision=precision)
    sim.load_plasma(0.01, 0.0, 0.0, (2, 2, 4))
    sim.add_laser(1.0, 4.0, 6.0, 9.6, 9.6)
    sim.step(3)
    for call in range(2):
        for mode in range(2):
            ref = sim.get_field("rho", "r", mode)
            st, got = _noalloc(sim, mode)
            assert st == 0, sim.L.qpic_last_error(sim.h)
            scale = np.max(np.abs(ref))
            assert scale > 0
            # same deposit kernel; FP64 atomics may add in another order
            assert np.max(np.abs(got - ref)) <= 1e-12 * scale, (call, mode)


def test_noalloc_refuses_grids_beyond_its_buffer():
    sim = q.Sim(4000, 400, 0.2, 0.8, n_modes=2, dt=0.1)       # 2*2*401*4000 > 2^21 doubles
    st, _ = _noalloc(sim, 0)
    assert q.STATUS[st] == "EINVAL"
    assert b"static buffer holds" in sim.L.qpic_last_error(sim.h)
