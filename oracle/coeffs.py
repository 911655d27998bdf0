"""Extended-stencil ("dual") z-derivative coefficients, CFL limit and the J_z
filter, in FP64 numpy.  TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Operators (Sec. III.A, Eq. 9): a staggered z-derivative with L coefficients,
    D f_{i+1/2} = sum_{l=1}^{L} C_l (f_{i+l} - f_{i+1-l}) / dz,
has the Fourier symbol [k] = (2/dz) sum_l C_l sin((l - 1/2) k dz).

Targets: Eq. 11 ([k]_B [k]_E = (sin(k dt/2)/(dt/2))^2, light moves at c) and
Eq. 15 (sqrt([k]_E/[k]_B) cos(k dt/2) = 1, exact time-averaged Lorentz force)
have the unique positive solution
    [k]_E = (2/dt) tan(k dt/2),   [k]_B = sin(k dt)/dt,
which the coefficients are fitted to (least squares on k dz in (0, band*pi],
uniform weight, with the exact long-wavelength limit sum (2l-1) C_l = 1).
The fit band and weight are a reading: the paper defers them to its Ref. Li2021.
"""
import numpy as np


def symbol(C, theta):
    """[k] dz of a staggered operator with coefficients C at theta = k dz"""
    C = np.asarray(C, dtype=np.float64)
    l = np.arange(1, len(C) + 1) - 0.5
    return 2.0 * np.sin(np.outer(np.atleast_1d(theta), l)) @ C


def target_kE(theta, nu):
    """[k]_E dz = (2/nu) tan(nu theta / 2), nu = dt/dz (solution of Eqs. 11 + 15)"""
    return 2.0 * np.tan(0.5 * nu * theta) / nu


def target_kB(theta, nu):
    """[k]_B dz = sin(nu theta) / nu"""
    return np.sin(nu * theta) / nu


def fit_coefficients(target, L=16, band=0.8, nsamp=4000):
    """Constrained least squares: minimise |A C - g|^2 subject to sum (2l-1) C_l = 1.
    Null-space method: C = e_1 + N y, N an orthonormal basis of the constraint's
    null space (from a QR factorisation), y from lstsq."""
    theta = band * np.pi * np.arange(1, nsamp + 1) / nsamp
    l = np.arange(1, L + 1) - 0.5
    A = 2.0 * np.sin(np.outer(theta, l))
    g = target(theta)
    c = 2.0 * np.arange(1, L + 1) - 1.0
    Cp = np.zeros(L)
    Cp[0] = 1.0                       # satisfies c . Cp = 1
    if L == 1:
        return Cp
    Q, _ = np.linalg.qr(np.column_stack([c, np.eye(L)[:, 1:]]))
    N = Q[:, 1:]
    y, *_ = np.linalg.lstsq(A @ N, g - A @ Cp, rcond=None)
    return Cp + N @ y


def dual_coefficients(dt, dz, L=16, band=0.8):
    """(C^E, C^B) for the dual solver at time step dt."""
    nu = dt / dz
    cE = fit_coefficients(lambda th: target_kE(th, nu), L, band)
    cB = fit_coefficients(lambda th: target_kB(th, nu), L, band)
    return cE, cB


def yee_coefficients():
    """The standard Yee operator: one coefficient, C_1 = 1, for both E and B."""
    return np.array([1.0]), np.array([1.0])


def solver_coefficients(solver, dt, dz, L=16, band=0.8):
    if solver == "yee":
        return yee_coefficients()
    return dual_coefficients(dt, dz, L, band)


def filter_taps(cB, tol=1e-16, n=1 << 14):
    """Taps k_0..k_{K-1} of the symmetric z filter whose symbol is
    [k]_Yee / [k]_B = sin(theta/2) / sum_l C^B_l sin((l-1/2) theta).
    Applying it to the two-point-continuity current J_z gives D^B_z (K*J_z) =
    D^Yee_z J_z, so Gauss's law in the dual form (Eq. 10's i[k]_B . E) holds.
    Taps are truncated after the last one with |k_n| >= tol |k_0|."""
    cB = np.asarray(cB, dtype=np.float64)
    if len(cB) == 1 and cB[0] == 1.0:
        return None                   # Yee: identity
    theta = 2.0 * np.pi * np.arange(n) / n
    theta = np.where(theta > np.pi, theta - 2.0 * np.pi, theta)
    s = symbol(cB, theta) / 2.0
    ratio = np.ones(n)
    nzr = theta != 0.0
    if np.any(np.abs(s[nzr]) < 1e-12):
        raise ValueError("[k]_B has a zero in (0, pi]: the J_z filter does not exist")
    ratio[nzr] = np.sin(theta[nzr] / 2.0) / s[nzr]
    K = np.real(np.fft.ifft(ratio))
    keep = np.nonzero(np.abs(K[: n // 2]) >= tol * abs(K[0]))[0]
    return K[: keep.max() + 1].copy()


def max_z_eigen(cE, cB, dz, ntheta=8192):
    """max over theta in (0, pi] of [k]_E [k]_B (the z part of curl curl)"""
    theta = np.pi * np.arange(1, ntheta + 1) / ntheta
    return float(np.max(symbol(cE, theta) * symbol(cB, theta))) / dz ** 2


def radial_operator_matrix(nr, dr, m, n_modes=None):
    """Matrix of v -> curl_B curl_E v for z-independent fields of mode m, built by
    applying the oracle's own Faraday and Ampere operators (dt = 1, J = 0) on a
    one-cell periodic box (so every z difference vanishes).  Unknowns: E_r at
    j+1/2 (j < nr), E_phi and E_z at j (j <= nr)."""
    from . import Oracle
    nm = (m + 1) if n_modes is None else n_modes
    o = Oracle(1, nr, nm, 1.0, dr, 1.0, [1.0], [1.0], periodic=True)
    idx = [("r", j) for j in range(nr)] + [("phi", j) for j in range(nr + 1)] + \
          [("z", j) for j in range(nr + 1)]
    n = len(idx)
    A = np.zeros((n, n), dtype=np.complex128)
    zero = np.zeros((nr + 1, 1), dtype=np.complex128)
    for col, (c, j) in enumerate(idx):
        for which in ("E", "B", "J"):
            for cc in ("r", "phi", "z"):
                for mm in range(nm):
                    o.set_field(which, cc, mm, zero)
        v = zero.copy()
        v[j, 0] = 1.0
        o.set_field("E", c, m, v)
        o.faraday()                      # B = -curl_E v
        for cc in ("r", "phi", "z"):
            o.set_field("E", cc, m, zero)
        o.ampere()                       # E = curl_B B = -curl_B curl_E v
        for row, (c2, j2) in enumerate(idx):
            A[row, col] = -o.get_field("E", c2, m)[j2, 0]
    return A


def radial_eigen_max(nr, dr, m):
    ev = np.linalg.eigvals(radial_operator_matrix(nr, dr, m))
    return float(np.max(ev.real))


def cfl_dt(dz, dr, nr, n_modes, solver="dual", L=16, band=0.8, tol=1e-10):
    """Largest dt with (dt^2/4) lambda_max(dt) <= 1 (leapfrog stability of the
    discrete curl curl), lambda_max = max_theta [k]_E[k]_B + max_m mu_m, where
    mu_m is the largest eigenvalue of mode m's radial operator.  For the dual
    solver the coefficients are refitted at each trial dt (bisection)."""
    mu = max(radial_eigen_max(nr, dr, m) for m in range(n_modes))

    def ok(dt):
        cE, cB = solver_coefficients(solver, dt, dz, L, band)
        return 0.25 * dt * dt * (max_z_eigen(cE, cB, dz) + mu) <= 1.0

    lo, hi = 0.0, dz          # the fit needs nu = dt/dz < 1 (tan target finite)
    if solver == "yee":
        hi = 2.0 * dz
    while hi - lo > tol * hi:
        mid = 0.5 * (lo + hi)
        if ok(mid):
            lo = mid
        else:
            hi = mid
    return lo
