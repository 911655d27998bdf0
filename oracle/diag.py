"""Oracle diagnostics in FP64 numpy.  TEST INFRASTRUCTURE ONLY.

Finite-volume conventions shared with the deposit in qpic_oracle.c: the node
(i, j) owns the annulus between r_{j-1/2} and r_{j+1/2} (a disk of radius dr/2 on
the axis, the inner half-annulus at the wall), volume V_j; densities are charge
per control volume.
"""
import numpy as np

MEC2_MEV = 0.51099895


def control_volumes(nr, dr, dz):
    V = 2.0 * np.pi * np.arange(nr + 1) * dr * dr * dz
    V[0] = np.pi * 0.25 * dr * dr * dz
    R = nr * dr
    V[nr] = np.pi * (R * R - (R - 0.5 * dr) ** 2) * dz
    return V


def _zshift(f, k, periodic):
    """g[..., i] = f[..., i + k] (zero outside an open box)"""
    if periodic:
        return np.roll(f, -k, axis=-1)
    g = np.zeros_like(f)
    n = f.shape[-1]
    if k >= 0:
        g[..., : n - k] = f[..., k:]
    else:
        g[..., -k:] = f[..., : n + k]
    return g


def dzB(f, cB, dz, periodic):
    """D^B_z of a half-z-located array (index i holds i+1/2), result at integer i"""
    out = np.zeros_like(f)
    for l, c in enumerate(cB, start=1):
        out += c * (_zshift(f, l - 1, periodic) - _zshift(f, -l, periodic))
    return out / dz


def dzYee(f, dz, periodic):
    return (f - _zshift(f, -1, periodic)) / dz


def divergence(Fr, Fphi, Fz, m, dr, dz, dz_op):
    """Finite-volume divergence of mode m at nodes (i, j), j = 0..nr:
    (r_{j+1/2} F_r(j+1/2) - r_{j-1/2} F_r(j-1/2)) / (r_j dr) + (i m / r_j) F_phi + D_z F_z,
    with 4 F_r(dr/2)/dr on the axis and only the inner face at the wall node
    (its control volume is the inner half-annulus).  dz_op maps half-z to integer z."""
    nr = Fr.shape[0] - 1
    out = np.zeros_like(Fz)
    j = np.arange(1, nr)[:, None]
    rp, rm, rj = (j + 0.5) * dr, (j - 0.5) * dr, j * dr
    out[1:nr] = (rp * Fr[1:nr] - rm * Fr[0:nr - 1]) / (rj * dr) + 1j * m / rj * Fphi[1:nr]
    out[0] = 4.0 * Fr[0] / dr
    V = control_volumes(nr, dr, dz)
    R = nr * dr
    out[nr] = (-2.0 * np.pi * dz * (R - 0.5 * dr) * Fr[nr - 1]) / V[nr] + 1j * m / R * Fphi[nr]
    out += dz_op(Fz)
    return out


def gauss_residual(o, cB, rho_ion, use_yee=False):
    """per mode: div_B E - (rho_e + rho_ion) at nodes j = 0..nr-1 (for m >= 1 the
    axis node is reported separately).  Returns list of arrays [nr+1][nz]."""
    E = o.fields("E")
    rho = o.rho()
    out = []
    for m in range(o.nm):
        op = (lambda f: dzYee(f, o.dz, o.periodic)) if use_yee else \
             (lambda f: dzB(f, cB, o.dz, o.periodic))
        d = divergence(E[0][m], E[1][m], E[2][m], m, o.dr, o.dz, op)
        d[o.nr] = np.nan                 # conductor node carries induced charge
        out.append(d - rho[m] - rho_ion[m])
    return out


def continuity_residual(rho0, rho1, J, dr, dz, dt, periodic):
    """per mode (rho1 - rho0)/dt + div J with the two-point z difference
    (the deposit's own continuity equation).  J = [3][nm][nr+1][nz]."""
    out = []
    for m in range(rho0.shape[0]):
        d = divergence(J[0][m], J[1][m], J[2][m], m, dr, dz,
                       lambda f: dzYee(f, dz, periodic))
        out.append((rho1[m] - rho0[m]) / dt + d)
    return out


def field_energy(o):
    """per mode: 1/2 sum V(r_loc) (|E|^2 + |B|^2) at each component's own
    location, modes m >= 1 counted twice (F = F_0 + 2 Re F_m e^{i m phi})."""
    nr, dr, dz = o.nr, o.dr, o.dz
    Vint = control_volumes(nr, dr, dz)
    Vhalf = 2.0 * np.pi * (np.arange(nr + 1) + 0.5) * dr * dr * dz
    Vhalf[nr] = 0.0
    E, B = o.fields("E"), o.fields("B")
    # half-r components: E_r, B_phi, B_z; integer-r: E_phi, E_z, B_r
    res = []
    for m in range(o.nm):
        s = 0.0
        for F, c, half in ((E, 0, True), (E, 1, False), (E, 2, False),
                           (B, 0, False), (B, 1, True), (B, 2, True)):
            V = Vhalf if half else Vint
            s += np.sum(V[:, None] * np.abs(F[c][m]) ** 2)
        res.append(0.5 * s * (1.0 if m == 0 else 2.0))
    return res


def kinetic_energy(p):
    g = np.sqrt(1.0 + p["ux"] ** 2 + p["uy"] ** 2 + p["uz"] ** 2)
    return float(np.sum(p["w"] * (g - 1.0)))


def spectrum(p, edges_mev):
    g = np.sqrt(1.0 + p["ux"] ** 2 + p["uy"] ** 2 + p["uz"] ** 2)
    h, _ = np.histogram((g - 1.0) * MEC2_MEV, bins=edges_mev, weights=p["w"])
    return h


def work_f_ratio(gamma, omega_p, w0, omega0=1.0):
    """Eq. 19: ratio f of the cycle-averaged work of the laser's longitudinal
    field to that of its transverse field, for an electron of Lorentz factor
    gamma in betatron resonance near focus (c = 1): f = -2 sqrt(2 gamma) /
    (omega0 omega_p w0^2)."""
    return -2.0 * np.sqrt(2.0 * np.asarray(gamma, dtype=np.float64)) / (omega0 * omega_p * w0 * w0)


def work_f_estimate(gamma, Wz, Wperp, omega_p, w0, omega0=1.0):
    """Eq. 20: the LWFA / DLA split estimated from the directional work of
    Eq. 17, W*_LWFA = W_z - f W_perp and W*_DLA = (1 + f) W_perp, with f of
    Eq. 19 at each particle's gamma."""
    f = work_f_ratio(gamma, omega_p, w0, omega0)
    Wz = np.asarray(Wz, dtype=np.float64)
    Wperp = np.asarray(Wperp, dtype=np.float64)
    return Wz - f * Wperp, (1.0 + f) * Wperp
