"""Reduced model of an electron in a bubble wake and a channel-guided laser
(Sec. II, Eqs. 2-8), integrated in FP64 numpy.  TEST INFRASTRUCTURE ONLY: the
tests and the benchmark's CPU baseline use it; the library never does.

Units: c = 1, the laser frequency omega0 = 1 (times in 1/omega0, lengths in
c/omega0), momenta u = gamma v.  Motion stays in the x-z plane (y = 0).

Eq. 8 (spherical bubble of Eq. 6, laser of Eqs. 3-4) in coordinates reads
    x'' + (gamma'/gamma) x' + (w_b^2/2)(1 + z') x = F_x,
    zeta'' + (gamma'/gamma)(zeta' + 1) + w_b^2 (zeta - x x'/2) = F_z,
with w_b^2 = w_p^2/(2 gamma) (Eq. 1), zeta = z - t, xi = z - v_phi t and
    F_x = (a0/gamma) [(1 - k_z z') J0(k_perp x) - (k_perp^2/k_z) z' J1'(k_perp x)] sin(k_z xi),
    F_z = -(a0/gamma) {(k_perp/k_z) J1(k_perp x) cos(k_z xi)
                       - k_z x' [J0(k_perp x) + (k_perp^2/k_z^2) J1'(k_perp x)] sin(k_z xi)}.
Since d(gamma x')/dt = gamma (x'' + (gamma'/gamma) x') and
d(gamma z')/dt = gamma (zeta'' + (gamma'/gamma)(zeta' + 1)), the same system in
the state (x, zeta, u_x, u_z) is explicit:
    dx/dt = u_x/gamma,   dzeta/dt = u_z/gamma - 1,
    du_x/dt = gamma F_x - (w_p^2/4)(1 + z') x,
    du_z/dt = gamma F_z - (w_p^2/2)(zeta - x x'/2),
gamma = sqrt(1 + u_x^2 + u_z^2).

Time-staggering factor (Sec. IV.A): to model a solver whose E and B are
staggered in time, the laser's magnetic terms -- those proportional to
v sin(k_z xi): k_z z' J0 and (k_perp^2/k_z) z' J1' in F_x, k_z x' [J0 +
(k_perp/k_z)^2 J1'] in F_z -- are multiplied by b = cos(omega0 dt_PIC / 2)
(about 0.994 for the paper's Yee runs); b = 1 is the unstaggered model.

Injection (Appendix A): electrons enter the bubble over a time interval.
Electron i is held at its initial state until step start[i] of the fixed step
grid t0 + k dt and integrated from there (start = None: all from step 0).

Readings: k_z = omega0 / v_phi (the laser's longitudinal wavenumber follows the
phase velocity, which the paper takes from a PIC run), k_perp is an input
(Eq. 3's 2.4/(r_b + c/w_p) is the caller's choice), the injection time is
rounded up to the step grid, and the explicit fifth-order Runge-Kutta method
of Appendix A is taken to be Dormand-Prince (Dormand & Prince, J. Comput.
Appl. Math. 6, 1980) at a fixed step, its fifth-order weights.
"""
import numpy as np
from scipy import special

# Dormand-Prince 5(4): nodes, stage coefficients, fifth-order weights
DP_C = np.array([0.0, 1 / 5, 3 / 10, 4 / 5, 8 / 9, 1.0])
DP_A = [
    [],
    [1 / 5],
    [3 / 40, 9 / 40],
    [44 / 45, -56 / 15, 32 / 9],
    [19372 / 6561, -25360 / 2187, 64448 / 6561, -212 / 729],
    [9017 / 3168, -355 / 33, 46732 / 5247, 49 / 176, -5103 / 18656],
]
DP_B = np.array([35 / 384, 0.0, 500 / 1113, 125 / 192, -2187 / 6784, 11 / 84])


def j1_prime(s):
    """dJ1/ds = J0(s) - J1(s)/s, with the limit 1/2 at s = 0"""
    s = np.asarray(s, dtype=np.float64)
    out = np.full(s.shape, 0.5)
    nz = s != 0
    out[nz] = special.j0(s[nz]) - special.j1(s[nz]) / s[nz]
    return out


def rhs(t, y, a0, wp, kperp, vphi, bfac=1.0):
    """time derivative of y = (x, zeta, u_x, u_z) (arrays of n particles);
    bfac multiplies the laser's magnetic (v sin(k_z xi)) terms"""
    x, zeta, ux, uz = y
    gamma = np.sqrt(1.0 + ux * ux + uz * uz)
    vx, vz = ux / gamma, uz / gamma
    kz = 1.0 / vphi
    xi = zeta + t - vphi * t                     # z - v_phi t with z = zeta + t
    s = kperp * x
    J0, J1, J1p = special.j0(s), special.j1(s), j1_prime(s)
    sn, cs = np.sin(kz * xi), np.cos(kz * xi)
    Fx = (a0 / gamma) * ((1.0 - bfac * kz * vz) * J0 - bfac * (kperp * kperp / kz) * vz * J1p) * sn
    Fz = -(a0 / gamma) * ((kperp / kz) * J1 * cs - bfac * kz * vx * (J0 + (kperp * kperp) / (kz * kz) * J1p) * sn)
    dux = gamma * Fx - 0.25 * wp * wp * (1.0 + vz) * x
    duz = gamma * Fz - 0.5 * wp * wp * (zeta - 0.5 * x * vx)
    return np.array([vx, vz - 1.0, dux, duz])


def dp5_step(t, y, dt, *par):
    """one fixed Dormand-Prince step of the fifth-order solution"""
    k = []
    for i in range(6):
        yi = y + dt * sum(a * kj for a, kj in zip(DP_A[i], k)) if i else y
        k.append(rhs(t + DP_C[i] * dt, yi, *par))
    return y + dt * sum(b * kj for b, kj in zip(DP_B, k))


def integrate(x, zeta, ux, uz, a0, wp, kperp, vphi, t0, dt, nsteps, bfac=1.0, start=None):
    """nsteps fixed steps from t0; electron i moves from step start[i] on (all
    from step 0 when start is None); returns the final (x, zeta, u_x, u_z)"""
    y = np.array([np.asarray(v, dtype=np.float64) for v in (x, zeta, ux, uz)])
    st = None if start is None else np.asarray(start)
    t = t0
    for k in range(nsteps):
        if st is None:
            y = dp5_step(t, y, dt, a0, wp, kperp, vphi, bfac)
        else:
            on = st <= k
            if on.any():
                y[:, on] = dp5_step(t, y[:, on], dt, a0, wp, kperp, vphi, bfac)
        t = t0 + (k + 1) * dt
    return y[0], y[1], y[2], y[3]
