"""Pins of three oracle functions against physics fixed outside the oracle.

- Azimuthal current of the deposit (Sec. III.B; charge-conserving deposit per
  mode): a charge moving on a circle carries the current density J = rho v.  As
  the azimuthal step goes to zero, J_phi^0 of the deposit equals rho^0 v_phi at
  the mid-point of the move, and J_phi^m (m >= 1) equals rho^m v_phi (r_j/r_p),
  the form fixed by continuity with the (i m / r) divergence.  rho itself is
  pinned by the lattice-density tests, so a wrong sign, control volume or
  azimuthal velocity in the current fails here.
- Laser fields at focus (Eq. 18): with E_x = E0 exp(-r^2/w0^2) sin(theta), the
  longitudinal field is E_z = 2x/(k w0^2) E0 exp(-r^2/w0^2) cos(theta): a
  quarter period apart with amplitude ratio 2x/(k w0^2).  By the same argument
  for div B = 0, B_z at y = x0 follows B_y the same way.  A rotated polarisation
  rotates the whole field.
- Reduced model (Sec. II): the right-hand side of Eq. 8 is the Lorentz force of
  the potentials of Eqs. 2-3 (laser, Coulomb gauge) and Eqs. 5-6 (spherical
  bubble in the gauge A_z = -phi_b, A_perp = 0), E = -dA/dt - grad phi,
  B = curl A, differentiated here by central finite differences.
"""
import numpy as np
import pytest
from scipy import special

from oracle import coeffs as C
from oracle import reduced as R
from oracle import setup

DZ, DR = 0.2, 0.5


# ------------------------------------------------------------ J_phi = rho v_phi
def _circular_box(oracle_mod, z, r, phi, U, w, dt, nm=3):
    cE, cB = C.dual_coefficients(dt, DZ)
    o = oracle_mod.Oracle(24, 10, nm, DZ, DR, dt, cE, cB, None, periodic=True)
    # purely azimuthal momentum: u = U (-sin phi, cos phi, 0), no fields
    o.load_particles(z, r, phi, -U * np.sin(phi), U * np.cos(phi), np.zeros_like(z), w)
    return o


def test_m0_azimuthal_current_is_rho_v(oracle_mod):
    rng = np.random.default_rng(11)
    n, U, dt = 400, 0.6, 1e-3
    z = rng.uniform(0.3, 4.5, n)
    r = rng.uniform(0.7, 4.2, n)
    phi = rng.uniform(-np.pi, np.pi, n)
    w = rng.uniform(0.5, 1.5, n)
    o = _circular_box(oracle_mod, z, r, phi, U, w, dt)
    rho0 = o.rho()
    o.push_deposit()
    rho1 = o.rho()
    vphi = U / np.sqrt(1.0 + U * U)
    J0 = o.get_field("J", "phi", 0)
    expect = 0.5 * (rho0[0] + rho1[0]) * vphi
    scale = np.max(np.abs(expect))
    assert scale > 0
    # the azimuthal step is ~1e-3 rad: the residual is second order in it
    assert np.max(np.abs(J0 - expect)) < 1e-5 * scale


@pytest.mark.parametrize("m", [1, 2])
def test_m_ge_1_azimuthal_current_limit(oracle_mod, m):
    """one particle at a time: J_phi^m at its four nodes equals
    rho^m v_phi r_j / r_p, to second order in the azimuthal step"""
    dt, U = 1e-3, 0.4
    vphi = U / np.sqrt(1.0 + U * U)
    for zp, rp, ph in ((1.33, 1.71, 0.4), (2.07, 3.29, -2.2), (3.9, 0.83, 2.9)):
        o = _circular_box(oracle_mod, np.array([zp]), np.array([rp]), np.array([ph]), U,
                          np.array([1.0]), dt)
        rho0 = o.rho()
        o.push_deposit()
        rho1 = o.rho()
        rj = (np.arange(o.nr + 1) * DR)[:, None]
        expect = 0.5 * (rho0[m] + rho1[m]) * vphi * rj / rp
        J = o.get_field("J", "phi", m)
        scale = np.max(np.abs(expect))
        assert np.max(np.abs(J - expect)) < 2e-5 * scale, (m, zp, rp)


# ------------------------------------------------------------ laser, Eq. 18
def _x_and_z_at_focus(x0, a0, w0, psi, phis, ts):
    """physical E_x, E_y, E_z and B_x, B_y, B_z at (z_f, r = x0, phi) for times ts,
    from laser_fields' m = 1 amplitudes (F = 2 Re(F_1 e^{i phi})) on grids
    placed so that each component's staggered node lies at (z_f, x0)"""
    tau = 1e7                                    # flat envelope
    z_f = 40.0
    out = {k: np.zeros((len(phis), len(ts))) for k in ("Ex", "Ey", "Ez", "Bx", "By", "Bz")}
    # integer-r components (E_phi, E_z, B_r): dr so that j dr = x0, half-r ones: (j+1/2) dr = x0
    dr_int, dr_half = x0 / 8.0, x0 / 8.5
    # integer-z components (E_r, E_phi, B_z): z_f = zmin + 10 dz; half-z: zmin + 10.5 dz
    zmin_int, zmin_half = z_f - 10 * DZ, z_f - 10.5 * DZ
    for it, t in enumerate(ts):
        E_i, B_i = setup.laser_fields(20, 12, DZ, dr_int, zmin_int, t, a0, w0, tau, z_f, z_f, psi)
        E_h, B_h = setup.laser_fields(20, 12, DZ, dr_half, zmin_half, t, a0, w0, tau, z_f, z_f, psi)
        Ei_h, Bi_h = setup.laser_fields(20, 12, DZ, dr_half, zmin_int, t, a0, w0, tau, z_f, z_f, psi)
        Eh_i, Bh_i = setup.laser_fields(20, 12, DZ, dr_int, zmin_half, t, a0, w0, tau, z_f, z_f, psi)
        comp = {  # (array, row, column) of each component's node at (z_f, x0)
            "Er": (Ei_h["r"], 8, 10), "Ephi": (E_i["phi"], 8, 10), "Ez": (Eh_i["z"], 8, 10),
            "Br": (Bh_i["r"], 8, 10), "Bphi": (B_h["phi"], 8, 10), "Bz": (Bi_h["z"], 8, 10),
        }
        for ip, ph in enumerate(phis):
            f = {k: 2.0 * np.real(a[j, i] * np.exp(1j * ph)) for k, (a, j, i) in comp.items()}
            c, s = np.cos(ph), np.sin(ph)
            out["Ex"][ip, it] = f["Er"] * c - f["Ephi"] * s
            out["Ey"][ip, it] = f["Er"] * s + f["Ephi"] * c
            out["Ez"][ip, it] = f["Ez"]
            out["Bx"][ip, it] = f["Br"] * c - f["Bphi"] * s
            out["By"][ip, it] = f["Br"] * s + f["Bphi"] * c
            out["Bz"][ip, it] = f["Bz"]
    return out


def _fit_sin_cos(ts, y):
    A = np.stack([np.sin(ts), np.cos(ts)], axis=1)
    coef, *_ = np.linalg.lstsq(A, y, rcond=None)
    return coef


def test_laser_fields_eq18_at_focus():
    a0, w0, x0 = 1.3, 9.0, 2.5
    ts = np.linspace(0.0, 2 * np.pi, 24, endpoint=False)
    f = _x_and_z_at_focus(x0, a0, w0, 0.0, [0.0, 0.5 * np.pi], ts)
    g = np.exp(-x0 * x0 / (w0 * w0))
    K = 2.0 * x0 / (w0 * w0)                      # 2x/(k w0^2), k = omega0/c = 1
    # phi = 0 (x = x0, y = 0): E_x = E0 g sin(theta), E_z = K E0 g cos(theta)
    a, b = _fit_sin_cos(ts, f["Ex"][0])
    c, d = _fit_sin_cos(ts, f["Ez"][0])
    assert np.hypot(a, b) == pytest.approx(a0 * g, rel=1e-9)
    assert (c, d) == pytest.approx((-K * b, K * a), abs=1e-9 * a0)
    assert np.max(np.abs(f["Ey"][0])) < 1e-12
    # the forward wave: B_y = E_x (c = 1) at the same node
    assert np.max(np.abs(f["By"][0] - f["Ex"][0])) < 1e-9 * a0
    # phi = pi/2 (y = x0): no E_z (it goes with x), B_z follows B_y like E_z follows E_x
    a, b = _fit_sin_cos(ts, f["By"][1])
    c, d = _fit_sin_cos(ts, f["Bz"][1])
    assert np.hypot(a, b) == pytest.approx(a0 * g, rel=1e-9)
    assert (c, d) == pytest.approx((-K * b, K * a), abs=1e-9 * a0)
    assert np.max(np.abs(f["Ez"][1])) < 1e-12


def test_laser_polarisation_rotates_the_field():
    a0, w0, x0, psi = 0.8, 7.0, 1.9, 0.7
    ts = np.linspace(0.0, 2 * np.pi, 8, endpoint=False)
    base = _x_and_z_at_focus(x0, a0, w0, 0.0, [0.3], ts)
    rot = _x_and_z_at_focus(x0, a0, w0, psi, [0.3 + psi], ts)
    c, s = np.cos(psi), np.sin(psi)
    for F in ("E", "B"):
        x, y = base[F + "x"][0], base[F + "y"][0]
        assert np.max(np.abs(rot[F + "x"][0] - (c * x - s * y))) < 1e-12
        assert np.max(np.abs(rot[F + "y"][0] - (s * x + c * y))) < 1e-12
        assert np.max(np.abs(rot[F + "z"][0] - base[F + "z"][0])) < 1e-12


# ------------------------------------------------------------ reduced model
def _potential_force(x, zeta, ux, uz, t, a0, wp, kperp, vphi, h=1e-4):
    """Lorentz force (q = -1) on an electron at (x, y = 0, z = zeta + t) from the
    laser potentials of Eqs. 2-3 and the bubble potentials of Eqs. 5-6 in the
    gauge A_z = -phi_b, by central differences"""
    kz = 1.0 / vphi

    def A(X, Y, Z, T):
        r = np.hypot(X, Y)
        xi = Z - vphi * T
        s = kperp * r
        with np.errstate(invalid="ignore", divide="ignore"):
            j1_over_r = np.where(r > 0, special.j1(s) / np.where(r > 0, r, 1.0), 0.5 * kperp)
        Ax = a0 * special.j0(s) * np.cos(kz * xi)
        Az_l = a0 * (kperp * X / kz) * j1_over_r * np.sin(kz * xi)
        zz = Z - T
        psi = 0.25 * wp * wp * (-zz * zz - r * r)          # Eq. 6 (the constant drops out)
        phi_b = 0.5 * psi                                   # psi = phi_b - A_z with A_z = -phi_b
        return Ax, Az_l - phi_b, phi_b

    def d(f, k):
        args = [x, 0.0, zeta + t, t]
        ap, am = list(args), list(args)
        ap[k] = args[k] + h
        am[k] = args[k] - h
        return [(p - m) / (2 * h) for p, m in zip(f(*ap), f(*am))]

    dAx_dx, dAz_dx, dphi_dx = d(A, 0)
    dAx_dz, dAz_dz, dphi_dz = d(A, 2)
    dAx_dt, dAz_dt, _ = d(A, 3)
    Ex = -dAx_dt - dphi_dx
    Ez = -dAz_dt - dphi_dz
    By = dAx_dz - dAz_dx                     # the x-z plane: B_x = B_z = 0 at y = 0
    gamma = np.sqrt(1 + ux * ux + uz * uz)
    vx, vz = ux / gamma, uz / gamma
    return -(Ex - vz * By), -(Ez + vx * By)


@pytest.mark.parametrize("kperp", [0.0, 0.07, 0.21])
def test_reduced_rhs_is_the_lorentz_force_of_the_potentials(kperp):
    rng = np.random.default_rng(5)
    n = 64
    a0, wp, vphi = 2.3, 0.09, 1.0031
    x = rng.uniform(-4.0, 4.0, n)
    zeta = rng.uniform(-15.0, 5.0, n)
    ux = rng.normal(0.0, 2.0, n)
    uz = rng.uniform(0.0, 40.0, n)
    t = rng.uniform(0.0, 300.0, n)
    got = np.array([R.rhs(t[k], np.array([[x[k]], [zeta[k]], [ux[k]], [uz[k]]]), a0, wp, kperp, vphi)[:, 0]
                    for k in range(n)])
    gamma = np.sqrt(1 + ux * ux + uz * uz)
    assert got[:, 0] == pytest.approx(ux / gamma, abs=1e-15)
    assert got[:, 1] == pytest.approx(uz / gamma - 1.0, abs=1e-15)
    Fx, Fz = _potential_force(x, zeta, ux, uz, t, a0, wp, kperp, vphi)
    # du/dt = F (momentum u = gamma v, m = 1)
    assert np.max(np.abs(got[:, 2] - Fx)) < 1e-7 * (1 + np.max(np.abs(Fx)))
    assert np.max(np.abs(got[:, 3] - Fz)) < 1e-7 * (1 + np.max(np.abs(Fz)))
    if kperp > 0:
        # the k_perp terms matter at this size: dropping them would fail the check
        Fx0, Fz0 = _potential_force(x, zeta, ux, uz, t, a0, wp, 0.0, vphi)
        assert np.max(np.abs(Fz - Fz0)) > 1e-3
