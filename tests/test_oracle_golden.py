"""Pins of the oracle against numbers the paper prints (tests/golden/paper_values.json)."""
import json
import os

import numpy as np

from oracle import coeffs as C

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def _w0_over_wp():
    # w0/w_p = sqrt(n_c/n0), n_c = eps0 m w0^2 / e^2 with w0 = 2 pi c / lambda (SI constants)
    lam = GOLD["laser_wavelength_nm"]["value"] * 1e-9
    n0 = GOLD["electron_density_cm3"]["value"] * 1e6
    eps0, me, e, c = 8.8541878128e-12, 9.1093837015e-31, 1.602176634e-19, 299792458.0
    w0 = 2 * np.pi * c / lam
    nc = eps0 * me * w0 ** 2 / e ** 2
    return np.sqrt(nc / n0)


def test_yee_time_staggering_factor_through_the_oracle(oracle_mod):
    """Run the oracle's own Yee Faraday step on a plane wave at the paper's
    resolution and time step; the time-averaged B it produces relative to E is
    the staggering factor cos(w dt/2) of Eq. 13, printed as ~0.994."""
    ratio = _w0_over_wp()
    assert abs(ratio - 10.83) < 0.02                 # conversion used for the paper's numbers
    dt = GOLD["dt_yee_3d_over_wp"]["value"] * ratio  # in 1/w0
    dz = 2 * np.pi / GOLD["points_per_lambda"]["value"]
    nz, nr = 120, 4                                  # 4 wavelengths, periodic
    cE, cB = C.yee_coefficients()
    o = oracle_mod.Oracle(nz, nr, 2, dz, 1.0, dt, cE, cB, periodic=True)
    k = 2 * np.pi * 4 / (nz * dz)
    omega = 2 / dt * np.arcsin(dt / dz * np.sin(k * dz / 2))     # Yee dispersion, Eq. 10
    zi, zh = np.arange(nz) * dz, (np.arange(nz) + 0.5) * dz
    ones = np.ones((nr + 1, 1))
    ex = np.cos(k * zi)[None, :] * ones
    by = np.cos(k * zh + 0.5 * omega * dt)[None, :] * ones      # B at t = -dt/2
    o.set_field("E", "r", 1, 0.5 * ex)
    o.set_field("E", "phi", 1, 0.5j * ex)
    o.set_field("B", "phi", 1, 0.5 * by)
    o.set_field("B", "r", 1, -0.5j * by)
    o.faraday()
    bbar = 2 * o.get_field("Bbar", "phi", 1)[0].real
    # Bbar^n = By(z_{i+1/2}, t=0) cos(w dt/2): compare with the exact wave at t = 0
    fac = np.sum(bbar * np.cos(k * zh)) / np.sum(np.cos(k * zh) ** 2)
    # printed to three digits ("approximately 0.994"): agree to its last digit
    assert abs(fac - GOLD["yee_time_staggering_factor"]["value"]) < 1e-3
    assert abs(fac - np.cos(0.5 * omega * dt)) < 1e-12


def test_dual_removes_staggering_factor(oracle_mod):
    dz = 2 * np.pi / GOLD["points_per_lambda"]["value"]
    dt = 0.6 * dz
    nz, nr = 120, 4
    cE, cB = C.dual_coefficients(dt, dz)
    assert len(cE) == GOLD["dual_coefficients"]["value"]
    o = oracle_mod.Oracle(nz, nr, 2, dz, 1.0, dt, cE, cB, periodic=True)
    k = 2 * np.pi * 4 / (nz * dz)
    kE = C.symbol(cE, k * dz)[0] / dz
    kB = C.symbol(cB, k * dz)[0] / dz
    omega = 2 / dt * np.arcsin(0.5 * dt * np.sqrt(kE * kB))
    zi, zh = np.arange(nz) * dz, (np.arange(nz) + 0.5) * dz
    ones = np.ones((nr + 1, 1))
    ex = np.cos(k * zi)[None, :] * ones
    by = np.sqrt(kE / kB) * np.cos(k * zh + 0.5 * omega * dt)[None, :] * ones
    o.set_field("E", "r", 1, 0.5 * ex)
    o.set_field("E", "phi", 1, 0.5j * ex)
    o.set_field("B", "phi", 1, 0.5 * by)
    o.set_field("B", "r", 1, -0.5j * by)
    o.faraday()
    bbar = 2 * o.get_field("Bbar", "phi", 1)[0].real
    fac = np.sum(bbar * np.cos(k * zh)) / np.sum(np.cos(k * zh) ** 2)
    assert abs(fac - 1.0) < 1e-5
