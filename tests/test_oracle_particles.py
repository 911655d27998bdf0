"""Pins of the oracle's particle side (gather, Boris push, deposit) against
closed forms, invariants and brute force.

- continuity per mode to round-off (the deposit's defining identity; m >= 1
  axis node reported separately), and Gauss's law in the dual form kept over
  many steps with the J_z filter (Eq. 10's i[k]_B.E);
- charge density of a uniform lattice (exact interior value, axis quadrature),
  total charge and dipole moments (fix V_j and the e^{-i m phi} convention),
  and a brute-force azimuthal quadrature of the 3D density projected on modes;
- gather of uniform transverse and linear radial fields (rotation, 2 Re convention,
  axis parity);
- one electron in a vacuum plane wave: u_x = A_x, gamma - u_z = 1 (Eq. 6 closed form);
- betatron frequency w_p / sqrt(2 gamma) in an ion channel (Eq. 1).
"""
import numpy as np
import pytest

from oracle import coeffs as C
from oracle import diag, setup

DZ, DR = 0.2, 0.5


def _random_box(oracle_mod, nz=16, nr=8, nm=2, n=3000, seed=7, periodic=True, dt=0.12,
                amp=0.6, umax=2.0, ktaps=False):
    rng = np.random.default_rng(seed)
    cE, cB = C.dual_coefficients(dt, DZ)
    kt = C.filter_taps(cB) if ktaps else None
    o = oracle_mod.Oracle(nz, nr, nm, DZ, DR, dt, cE, cB, kt, periodic=periodic)
    for which in ("E", "Bbar"):
        for c in ("r", "phi", "z"):
            for m in range(nm):
                v = amp * (rng.standard_normal((nr + 1, nz)) + (1j * rng.standard_normal((nr + 1, nz)) if m else 0))
                o.set_field(which, c, m, v)
    z = rng.uniform(0, nz * DZ, n)
    r = nr * DR * np.sqrt(rng.uniform(0, 1, n))
    r[:20] = rng.uniform(0, 0.3 * DR, 20)                 # near the axis
    r[20:40] = nr * DR - rng.uniform(0, 0.3 * DR, 20)     # near the wall
    phi = rng.uniform(-np.pi, np.pi, n)
    u = rng.uniform(-umax, umax, (3, n))
    w = rng.uniform(0.5, 1.5, n)
    o.load_particles(z, r, phi, u[0], u[1], u[2], w)
    return o, cE, cB


def test_continuity_per_mode_to_roundoff(oracle_mod):
    o, cE, cB = _random_box(oracle_mod, nm=3)
    rho0 = o.rho()
    o.push_deposit()
    rho1 = o.rho()
    J = o.fields("J")
    res = diag.continuity_residual(rho0, rho1, J, DR, DZ, o.dt, True)
    for m in range(3):
        scale = np.max(np.abs(rho1[m] - rho0[m])) / o.dt
        r = res[m][:o.nr].copy()          # wall node included below, axis separate
        if m >= 1:
            axis = r[0].copy()
            r[0] = 0.0
            # physical rho_m(0) = 0 for m >= 1 but the deposit moves modal charge there
            assert np.max(np.abs(axis)) > 1e-6 * scale
        assert np.max(np.abs(r)) < 1e-12 * scale, m
        assert np.max(np.abs(res[m][o.nr])) < 1e-12 * scale


def test_gauss_dual_kept_with_filter(oracle_mod):
    nz, nr, dt = 64, 12, 0.12
    results = {}
    for use_filter in (True, False):
        cE, cB = C.dual_coefficients(dt, DZ)
        kt = C.filter_taps(cB) if use_filter else None
        o = oracle_mod.Oracle(nz, nr, 2, DZ, DR, dt, cE, cB, kt, periodic=True)
        p = setup.plasma_cells(np.arange(nz), nr, DZ, DR, 0.05, 0.0, 0.0, (2, 2, 4), seed=3)
        o.load_particles(**p)
        setup.add_laser(o, cE, cB, a0=1.5, w0=3.0, tau=3.0, z_c=6.4, z_f=6.4)
        rho_ion = -o.rho()
        r0 = diag.gauss_residual(o, cB, rho_ion)
        o.step(30)
        r1 = diag.gauss_residual(o, cB, rho_ion)
        scale = np.nanmax(np.abs(o.rho()[0] + rho_ion[0]))
        d0 = np.nanmax(np.abs((r1[0] - r0[0])[:nr]))
        d1 = np.nanmax(np.abs((r1[1] - r0[1])[1:nr]))
        results[use_filter] = (d0 / scale, d1 / scale)
    assert results[True][0] < 1e-10 and results[True][1] < 1e-10
    # without the current correction the dual divergence drifts visibly
    assert results[False][0] > 1e-6


def test_uniform_lattice_density(oracle_mod):
    nz, nr, n0 = 8, 6, 0.02
    cE, cB = C.yee_coefficients()
    o = oracle_mod.Oracle(nz, nr, 2, DZ, DR, 0.1, cE, cB, periodic=True)
    p = setup.plasma_cells(np.arange(nz), nr, DZ, DR, n0, 0.0, 0.0, (2, 2, 4), seed=1)
    o.load_particles(**p)
    rho = o.rho()
    # interior nodes receive exactly n V_j from a 2-per-cell radial lattice
    assert np.max(np.abs(rho[0][1:nr] + n0)) < 1e-14
    # axis node: charge of r in {dr/4, 3dr/4} weighted (3/4, 1/4) over V_0 = pi dr^2 dz/4
    assert np.max(np.abs(rho[0][0] + 1.5 * n0)) < 1e-14
    # 4 particles evenly spaced in phi: no m = 1 moment
    assert np.max(np.abs(rho[1])) < 1e-15


def test_charge_and_dipole_moments(oracle_mod):
    o, _, _ = _random_box(oracle_mod, nm=3, n=500)
    rho = o.rho()
    p = o.particles()
    V = diag.control_volumes(o.nr, DR, DZ)
    Q = -p["w"]
    assert abs(np.sum(V[:, None] * rho[0]) - Q.sum()) < 1e-12 * abs(Q.sum())
    rj = np.arange(o.nr + 1) * DR
    x, y = p["r"] * np.cos(p["phi"]), p["r"] * np.sin(p["phi"])
    # linear shapes reproduce r: sum_j V_j r_j rho_1 = sum_p Q (x - i y)
    d1 = np.sum((V * rj)[:, None] * rho[1])
    assert abs(d1 - np.sum(Q * (x - 1j * y))) < 1e-11 * np.sum(np.abs(Q) * p["r"])
    # and quadrupole: sum_j V_j r_j^2 rho_2 ~ sum_p Q (x - i y)^2 (shape error O(dr^2))
    d2 = np.sum((V * rj ** 2)[:, None] * rho[2])
    ref2 = np.sum(Q * (x - 1j * y) ** 2)
    assert abs(d2 - ref2) < 0.05 * np.sum(np.abs(Q) * p["r"] ** 2)


def test_brute_force_azimuthal_projection(oracle_mod):
    o, _, _ = _random_box(oracle_mod, nm=3, n=400)
    rho = o.rho()
    p = o.particles()
    nphi = 1 << 13
    nz, nr = o.nz, o.nr
    V = diag.control_volumes(nr, DR, DZ)
    dens = np.zeros((nr + 1, nz, nphi))
    zc = p["z"] / DZ
    rc = p["r"] / DR
    k = np.round((p["phi"] % (2 * np.pi)) / (2 * np.pi) * nphi).astype(int) % nphi
    for q in range(len(zc)):
        i0, j0 = int(np.floor(zc[q])), int(np.floor(rc[q]))
        for a in (0, 1):
            for b in (0, 1):
                wz = 1 - abs(zc[q] - (i0 + a))
                wr = 1 - abs(rc[q] - (j0 + b))
                if wz <= 0 or wr <= 0 or j0 + b > nr:
                    continue
                # charge per control volume in one azimuthal bin (bin width 2 pi / nphi)
                dens[j0 + b, (i0 + a) % nz, k[q]] += -p["w"][q] * wz * wr / (V[j0 + b] / nphi)
    phik = 2 * np.pi * np.arange(nphi) / nphi
    for m in range(3):
        proj = np.sum(dens * np.exp(-1j * m * phik), axis=2) / nphi
        err = np.max(np.abs(proj - rho[m])) / np.max(np.abs(rho[0]))
        assert err < 5 * m * np.pi / nphi + 1e-12


def test_gather_uniform_and_linear_fields(oracle_mod):
    nz, nr = 10, 6
    cE, cB = C.yee_coefficients()
    o = oracle_mod.Oracle(nz, nr, 2, DZ, DR, 0.1, cE, cB, periodic=True)
    ones = np.ones((nr + 1, nz))
    E0x, E0y, Bz0, kr = 0.7, -0.3, 0.25, 0.9
    # uniform (Ex, Ey) in mode 1, linear radial E_r = kr r in mode 0, uniform B_z
    o.set_field("E", "r", 1, 0.5 * (E0x - 1j * E0y) * ones)
    o.set_field("E", "phi", 1, 0.5 * (1j * E0x + E0y) * ones)
    rh = (np.arange(nr + 1) + 0.5)[:, None] * DR * np.ones((1, nz))
    o.set_field("E", "r", 0, kr * rh)
    o.set_field("Bbar", "z", 0, Bz0 * ones)
    rng = np.random.default_rng(2)
    n = 200
    z = rng.uniform(0, nz * DZ, n)
    r = rng.uniform(0, (nr - 0.5) * DR, n)
    r[:10] = rng.uniform(0, 0.25 * DR, 10)
    phi = rng.uniform(-np.pi, np.pi, n)
    g = o.gather(z, r, phi)
    x, y = r * np.cos(phi), r * np.sin(phi)
    assert np.max(np.abs(g[:, 0] - (E0x + kr * x))) < 1e-13
    assert np.max(np.abs(g[:, 1] - (E0y + kr * y))) < 1e-13
    assert np.max(np.abs(g[:, 2])) < 1e-15
    assert np.max(np.abs(g[:, 5] - Bz0)) < 1e-13


def test_electron_in_vacuum_plane_wave(oracle_mod):
    """prescribed wave A_x = a0 cos(k(z - t)); from rest: u_x = A_x(xi) - A_x(xi0),
    gamma - u_z = 1 (Eq. 6 closed form for q = -1)"""
    nz, nr, dt, a0, k = 256, 16, 0.05, 0.5, 0.25   # x excursion a0/k = 2 < wall
    cE, cB = C.yee_coefficients()
    o = oracle_mod.Oracle(nz, nr, 2, DZ, DR, dt, cE, cB, periodic=True)
    ones = np.ones((nr + 1, 1))
    z0 = 20.0
    o.load_particles([z0], [0.0], [0.0], [0.0], [0.0], [0.0], [1e-12])
    zi, zh = np.arange(nz) * DZ, (np.arange(nz) + 0.5) * DZ
    A = lambda xi: a0 * np.cos(k * xi)
    ex = lambda z, t: -a0 * k * np.sin(k * (z - t))      # E_x = -dA/dt = B_y
    worst_inv, worst_ux = 0.0, 0.0
    for n in range(600):
        t = n * dt
        Ez_ = ex(zi, t)[None, :] * ones                    # E_r, E_phi at integer z
        o.set_field("E", "r", 1, 0.5 * Ez_)
        o.set_field("E", "phi", 1, 0.5j * Ez_)
        By = ex(zh, t)[None, :] * ones                     # B_r, B_phi at half z
        o.set_field("Bbar", "r", 1, -0.5j * By)
        o.set_field("Bbar", "phi", 1, 0.5 * By)
        p0 = o.particles()
        o.push_deposit()
        p1 = o.particles()
        # u at n+1/2 against the closed form at the mid-position
        zm = 0.5 * (p0["z"][0] + p1["z"][0])
        if p1["z"][0] < p0["z"][0] - 0.5 * nz * DZ:       # periodic wrap
            zm += 0.5 * nz * DZ
        ux = p1["ux"][0]
        g = np.sqrt(1 + ux ** 2 + p1["uy"][0] ** 2 + p1["uz"][0] ** 2)
        worst_inv = max(worst_inv, abs(g - p1["uz"][0] - 1.0))
        # at rest at t = -dt/2 (u is defined at half steps)
        worst_ux = max(worst_ux, abs(ux - (A(zm - (t + 0.5 * dt)) - A(z0 + 0.5 * dt))))
    assert worst_inv < 2e-4
    assert worst_ux < 3e-3
    assert p1["uz"][0] >= 0.0          # the wave pushes the electron forward


def test_betatron_frequency_eq1(oracle_mod):
    nz, nr, dt, n0, g0 = 16, 8, 0.1, 0.01, 20.0
    cE, cB = C.yee_coefficients()
    o = oracle_mod.Oracle(nz, nr, 1, DZ, DR, dt, cE, cB, periodic=True)
    rh = (np.arange(nr + 1) + 0.5)[:, None] * DR * np.ones((1, nz))
    o.set_field("E", "r", 0, 0.5 * n0 * rh)               # ion channel: E_r = n r / 2
    uz = np.sqrt(g0 ** 2 - 1)
    o.load_particles([0.3], [0.6], [0.0], [0.0], [0.0], [uz], [1e-12])
    xs = []
    for n in range(9000):
        o.push_deposit()
        p = o.particles()
        xs.append(p["r"][0] * np.cos(p["phi"][0]))
    xs = np.array(xs)
    cross = np.nonzero((xs[:-1] > 0) & (xs[1:] <= 0))[0]
    frac = xs[cross] / (xs[cross] - xs[cross + 1])
    tc = (cross + frac) * dt
    period = np.mean(np.diff(tc))
    w_beta = np.sqrt(n0) / np.sqrt(2 * g0)                # Eq. 1 (w_p^2 = n)
    assert abs(2 * np.pi / period / w_beta - 1) < 2e-3
