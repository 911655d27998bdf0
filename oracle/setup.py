"""Initial conditions for the oracle: plasma lattice and Gaussian laser, FP64 numpy.
TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Plasma (reading of the paper's quasi-3D set-up, Appendix A): a regular
ppc_z x ppc_r x ppc_phi lattice in every cell, cold (u = 0), weights
proportional to r_p and to the local density, one azimuthal offset per cell drawn
from a counter-based SplitMix64 keyed on (seed, cell).

Laser (Eq. 18 near focus, generalised to a paraxial Gaussian beam): linear
polarisation at angle psi, field envelope exp(-2 ln2 xi^2/tau^2) so that the
intensity FWHM is tau, all in the m = 1 mode.
"""
import numpy as np

M64 = (1 << 64) - 1


def splitmix64(x):
    """SplitMix64 output function (Steele, Lea & Flood, OOPSLA 2014) applied to
    state x + golden gamma; x is a numpy uint64 array (wrapping arithmetic)."""
    with np.errstate(over="ignore"):
        z = (x + np.uint64(0x9E3779B97F4A7C15)).astype(np.uint64)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def cell_uniform(seed, iz_abs, jr):
    """uniform [0,1) per (seed, absolute z cell, r cell): key = seed<<40 ^ iz<<20 ^ jr"""
    key = ((np.uint64(seed) << np.uint64(40))
           ^ (np.asarray(iz_abs, dtype=np.uint64) << np.uint64(20))
           ^ np.asarray(jr, dtype=np.uint64))
    return (splitmix64(key) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def density(z, n0, z_start, ramp_len):
    """n0 times a linear up-ramp of length ramp_len starting at z_start, plateau after"""
    z = np.asarray(z, dtype=np.float64)
    if ramp_len <= 0:
        return np.where(z >= z_start, n0, 0.0)
    return n0 * np.clip((z - z_start) / ramp_len, 0.0, 1.0)


def plasma_cells(iz_abs, nr, dz, dr, n0, z_start, ramp_len, ppc, seed, jitter=True):
    """Particles of the given absolute z cells (all r cells).
    Returns dict z, r, phi, ux, uy, uz, w (lab-frame z)."""
    pz, pr, pp = ppc
    iz_abs = np.atleast_1d(np.asarray(iz_abs, dtype=np.int64))
    I, Jr, A, Bq, Cp = np.meshgrid(iz_abs, np.arange(nr), np.arange(pz), np.arange(pr),
                                   np.arange(pp), indexing="ij")
    I, Jr, A, Bq, Cp = [x.ravel() for x in (I, Jr, A, Bq, Cp)]
    z = (I + (A + 0.5) / pz) * dz
    r = (Jr + (Bq + 0.5) / pr) * dr
    jit = cell_uniform(seed, I, Jr) if jitter else np.zeros(len(I))
    phi = 2.0 * np.pi * (Cp + jit) / pp
    n = density(z, n0, z_start, ramp_len)
    w = n * 2.0 * np.pi * r * (dr / pr) * (dz / pz) / pp
    keep = w > 0
    zeros = np.zeros(int(keep.sum()))
    return dict(z=z[keep], r=r[keep], phi=phi[keep], ux=zeros, uy=zeros.copy(),
                uz=zeros.copy(), w=w[keep])


def laser_fields(nz, nr, dz, dr, zmin, t, a0, w0, tau, z_c, z_f, psi=0.0,
                 periodic=False, omega=1.0):
    """m = 1 amplitudes of a paraxial Gaussian beam at time t on the staggered grid.
    Complex beam parameter q(z) = (z - z_f) - i z_R, z_R = w0^2/2 (k0 = 1); the
    x-field is Re[a0 env (-i) A e^{i(z - z_c - omega t)}] with
    A = (-i z_R/q) exp(i r^2/(2q)); E_z = Re[-(x/q) Ex_c] from Gauss's law and
    B_y = Ex, B_z = Re[-(y/q) Ex_c] from Faraday's law for a forward wave.
    Returns (E, B) as dicts comp -> [nr+1][nz] complex m = 1 amplitudes."""
    zR = 0.5 * w0 * w0
    Lz = nz * dz

    def core(zg, rg, tt):
        xi = zg - z_c - tt
        if periodic:
            xi = (xi + 0.5 * Lz) % Lz - 0.5 * Lz
        env = np.exp(-2.0 * np.log(2.0) * xi ** 2 / tau ** 2)
        q = (zg - z_f) - 1j * zR
        A = (-1j * zR / q) * np.exp(1j * rg ** 2 / (2.0 * q))
        exc = a0 * env * (-1j) * A * np.exp(1j * (xi + (1.0 - omega) * tt))
        return exc, q

    i = np.arange(nz)
    j = np.arange(nr + 1)
    rot = np.exp(-1j * psi)

    def at(hz, hr, tt):
        zg = zmin + (i[None, :] + 0.5 * hz) * dz
        rg = (j[:, None] + 0.5 * hr) * dr + 0.0 * zg
        return core(zg + 0.0 * rg, rg, tt), rg

    E, B = {}, {}
    # E_r (i, j+1/2), E_phi (i, j), E_z (i+1/2, j) at time t
    (exc, _), _ = at(0, 1, t)
    E["r"] = 0.5 * exc.real * rot
    (exc, _), _ = at(0, 0, t)
    E["phi"] = 0.5j * exc.real * rot
    (exc, q), rg = at(1, 0, t)
    E["z"] = 0.5 * rg * np.real(-exc / q) * rot
    # B_r (i+1/2, j), B_phi (i+1/2, j+1/2), B_z (i, j+1/2)
    (exc, _), _ = at(1, 0, t)
    B["r"] = -0.5j * exc.real * rot
    (exc, _), _ = at(1, 1, t)
    B["phi"] = 0.5 * exc.real * rot
    (exc, q), rg = at(0, 1, t)
    B["z"] = -0.5j * rg * np.real(-exc / q) * rot
    # half-r rows at index nr lie outside the wall; conductor rows of E_phi, E_z
    for d in (E, B):
        for c in ("r", "phi", "z"):
            d[c] = np.array(d[c], dtype=np.complex128)
    E["r"][nr, :] = 0.0
    B["phi"][nr, :] = 0.0
    B["z"][nr, :] = 0.0
    E["phi"][nr, :] = 0.0
    E["z"][nr, :] = 0.0
    B["r"][nr, :] = 0.0
    E["z"][0, :] = 0.0
    return E, B


def add_laser(o, cE, cB, a0, w0, tau, z_c, z_f, psi=0.0):
    """Add the laser to an Oracle box: E at t = 0, B at t = -dt/2 scaled by
    sqrt([k]_E/[k]_B) at k0 = 1 (the discrete B/E ratio of a wave, Eq. 9), with the
    discrete frequency from Eq. 10 for the time shift."""
    from .coeffs import symbol
    if o.nm < 2:
        raise ValueError("the laser is an m = 1 field: the box needs at least 2 modes")
    kE = symbol(cE, o.dz)[0] / o.dz
    kB = symbol(cB, o.dz)[0] / o.dz
    omega = 2.0 / o.dt * np.arcsin(0.5 * o.dt * np.sqrt(kE * kB))
    ratio = np.sqrt(kE / kB)
    E, _ = laser_fields(o.nz, o.nr, o.dz, o.dr, o.zmin, 0.0, a0, w0, tau, z_c, z_f, psi,
                        o.periodic, omega)
    _, B = laser_fields(o.nz, o.nr, o.dz, o.dr, o.zmin, -0.5 * o.dt, a0, w0, tau, z_c, z_f, psi,
                        o.periodic, omega)
    for c in ("r", "phi", "z"):
        o.set_field("E", c, 1, o.get_field("E", c, 1) + E[c])
        o.set_field("B", c, 1, o.get_field("B", c, 1) + ratio * B[c])
