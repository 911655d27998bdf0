"""Pins of the oracle's energy diagnostics against closed forms.

- The finite-volume control volumes of the integer rows (quarter cylinder at
  the axis, half annulus at the wall) and of the half rows both tile the
  cylinder: each sums to pi R^2 dz.
- A uniform m = 0 field of value c on any component has energy
  (1/2) c^2 pi R^2 L (L = nz dz), whether it lives on integer or half rows.
- A uniform m = 1 part F_1 is the physical field 2 Re(F_1 e^{i phi}), whose
  azimuthal mean square is 2 |F_1|^2: energy |F_1|^2 pi R^2 L.
- Kinetic energy of one electron with u = (0, 0, 3/4): gamma - 1 = 1/4.
"""
import numpy as np
import pytest

from oracle import coeffs as C
from oracle import diag

NZ, NR, DZ, DR = 12, 7, 0.2, 0.5


def test_control_volumes_tile_the_cylinder():
    R = NR * DR
    V = diag.control_volumes(NR, DR, DZ)
    assert abs(V.sum() / (np.pi * R * R * DZ) - 1) < 1e-14
    Vh = 2 * np.pi * (np.arange(NR) + 0.5) * DR * DR * DZ
    assert abs(Vh.sum() / (np.pi * R * R * DZ) - 1) < 1e-14


def _box(oracle_mod):
    cE, cB = C.dual_coefficients(0.1, DZ)
    return oracle_mod.Oracle(NZ, NR, 2, DZ, DR, 0.1, cE, cB, None, periodic=True)


# (field, component): integer-row components are E_phi, E_z, B_r; half-row ones
# E_r, B_phi, B_z (their last row lies beyond the wall and carries no volume)
@pytest.mark.parametrize("which,comp", [("E", "z"), ("E", "phi"), ("B", "r"),
                                        ("E", "r"), ("B", "phi"), ("B", "z")])
def test_uniform_field_energy(oracle_mod, which, comp):
    o = _box(oracle_mod)
    half = (which, comp) in (("E", "r"), ("B", "phi"), ("B", "z"))
    c0, c1 = 0.7, 0.3 - 0.4j
    v0 = np.full((NR + 1, NZ), c0)
    v1 = np.full((NR + 1, NZ), c1, dtype=complex)
    if half:
        v0[NR] = 0.0
        v1[NR] = 0.0
    o.set_field(which, comp, 0, v0)
    o.set_field(which, comp, 1, v1)
    vol = np.pi * (NR * DR) ** 2 * NZ * DZ
    fe = diag.field_energy(o)
    assert abs(fe[0] / (0.5 * c0 * c0 * vol) - 1) < 1e-13
    assert abs(fe[1] / (abs(c1) ** 2 * vol) - 1) < 1e-13


def test_kinetic_energy_single_electron():
    p = {"ux": np.array([0.0]), "uy": np.array([0.0]), "uz": np.array([0.75]), "w": np.array([2.0])}
    assert abs(diag.kinetic_energy(p) - 2.0 * 0.25) < 1e-15
