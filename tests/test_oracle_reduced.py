"""Pins of the reduced-model oracle (Sec. II, Eqs. 1-8; oracle/reduced.py).

- without the laser (a0 = 0) Eq. 8 keeps I = gamma - u_z + (w_p^2/4)(x^2 + zeta^2):
  d(gamma - u_z)/dt = x' u_x' + (z' - 1) u_z' = -(w_p^2/2)(x x' + zeta zeta');
- the plane-wave limit (w_p = 0, k_perp = 0, v_phi = 1) keeps u_x - a0 cos(xi) and
  gamma - u_z, the closed-form plane-wave electron;
- small betatron oscillations in the bubble at w_p / sqrt(2 gamma) (Eq. 1);
- the fixed-step integrator converges at fifth order, and agrees with scipy's
  adaptive DOP853 at tight tolerances on the same right-hand side.
"""
import numpy as np
import pytest
from scipy.integrate import solve_ivp

from oracle import reduced as R

LASER = dict(a0=2.0, wp=1 / 12.0, kperp=0.04, vphi=1.0008)


def _run(y0, par, dt, n, t0=0.0):
    x, z, ux, uz = (np.atleast_1d(np.float64(v)) for v in y0)
    return np.array(R.integrate(x, z, ux, uz, par["a0"], par["wp"], par["kperp"], par["vphi"], t0, dt, n))


def test_wake_invariant_without_laser():
    par = dict(a0=0.0, wp=0.1, kperp=0.05, vphi=1.001)
    y0 = ([1.0, -0.5], [-2.0, 3.0], [0.0, 0.3], [50.0, 5.0])
    def inv(y):
        x, zeta, ux, uz = y
        return np.sqrt(1 + ux ** 2 + uz ** 2) - uz + 0.25 * par["wp"] ** 2 * (x ** 2 + zeta ** 2)
    I0 = inv(np.array(y0))
    y = _run(y0, par, 0.25, 4000)
    assert np.max(np.abs(inv(y) - I0) / I0) < 1e-10
    assert np.max(np.abs(y[0] - np.array(y0[0]))) > 0.1          # it did move


def test_plane_wave_limit():
    par = dict(a0=1.5, wp=0.0, kperp=0.0, vphi=1.0)
    y0 = (0.0, 0.3, 0.0, 0.0)
    y = _run(y0, par, 0.02, 5000)
    x, zeta, ux, uz = y[:, 0]
    gamma = np.sqrt(1 + ux ** 2 + uz ** 2)
    xi = zeta                                                  # xi = zeta at v_phi = c
    assert ux - par["a0"] * np.cos(xi) == pytest.approx(-par["a0"] * np.cos(0.3), abs=1e-10)
    assert gamma - uz == pytest.approx(1.0, abs=1e-10)
    assert uz > 0.1                                            # pushed forward


def test_betatron_frequency_eq1():
    wp, gamma0 = 0.1, 200.0
    par = dict(a0=0.0, wp=wp, kperp=0.05, vphi=1.0)
    dt, n = 0.5, 20000
    x, zeta, ux, uz = (np.array([v]) for v in (0.5, 0.0, 0.0, np.sqrt(gamma0 ** 2 - 1)))
    xs, gs = [], []
    t = 0.0
    y = np.array([x, zeta, ux, uz])
    for k in range(n):
        y = R.dp5_step(t, y, dt, par["a0"], par["wp"], par["kperp"], par["vphi"])
        t = (k + 1) * dt
        xs.append(y[0, 0])
        gs.append(np.sqrt(1 + y[2, 0] ** 2 + y[3, 0] ** 2))
    xs = np.array(xs)
    up = np.nonzero((xs[:-1] < 0) & (xs[1:] >= 0))[0]
    tz = (up + xs[up] / (xs[up] - xs[up + 1])) * dt + dt         # upward zero crossings
    period = np.mean(np.diff(tz))
    assert len(up) >= 5
    # the wake slowly accelerates the electron as it slips behind zeta = 0: take
    # the mean gamma between the first and the last crossing
    g = np.mean(np.array(gs)[up[0]:up[-1] + 1])
    assert 1.005 < g / gamma0 < 1.02
    assert 2 * np.pi / period == pytest.approx(wp / np.sqrt(2 * g), rel=1e-3)


def test_fifth_order_convergence():
    """an electron at rest meets the laser (the phase runs at ~omega0): halving
    the step divides the error by ~2^5 (4th order would give 16)"""
    y0 = (1.0, -20.0, 0.0, 0.0)
    T = 40.0
    ref = _run(y0, LASER, 0.005, int(T / 0.005))
    err = []
    for dt in (0.16, 0.08, 0.04):
        y = _run(y0, LASER, dt, int(round(T / dt)))
        err.append(np.max(np.abs(y - ref)))
    r1, r2 = err[0] / err[1], err[1] / err[2]
    assert 25 < r1 < 64 and 25 < r2 < 45, (err, r1, r2)


def test_matches_scipy_dop853():
    y0 = np.array([1.0, -20.0, 0.0, 20.0])
    T = 200.0
    sol = solve_ivp(lambda t, y: R.rhs(t, y.reshape(4, 1), *LASER.values()).ravel(), (0.0, T), y0,
                    method="DOP853", rtol=1e-12, atol=1e-12)
    y = _run(tuple(y0), LASER, 0.05, int(T / 0.05))[:, 0]
    assert np.max(np.abs(y - sol.y[:, -1]) / (1 + np.abs(sol.y[:, -1]))) < 1e-9
    assert abs(y[2]) > 0.1                                     # the laser drove the x motion


def test_appendix_bunch_and_its_orbits():
    """the seeded bunch follows Appendix A's injection recipe, and the oracle
    integrates it with the appendix's parameters without leaving the model:
    the wake invariant changes only through the laser"""
    import synth
    P = synth.REDUCED_PAPER
    wp = 1.0 / (P["v_phi"] * P["kz_over_wp"])
    Rb = P["R_over_lp"] / wp
    x, zeta, ux, uz = synth.reduced_bunch(3, 4000, v_g=P["v_g"], wp=wp, R_over_lp=P["R_over_lp"])
    assert np.all((zeta >= -Rb + 0.286 / wp) & (zeta <= -Rb + 0.836 / wp))
    assert np.all(np.abs(x) <= np.sqrt(Rb * Rb - zeta * zeta))
    gamma = np.sqrt(1 + ux ** 2 + uz ** 2)
    gg = 1 / np.sqrt(1 - P["v_g"] ** 2)
    assert np.all((gamma >= gg * (1 - 1e-12)) & (gamma <= 2 * gg))
    assert np.all(uz / gamma >= P["v_g"] * (1 - 1e-12))
    y = R.integrate(x[:200], zeta[:200], ux[:200], uz[:200], P["a0"], wp, 2.4 * wp / (P["R_over_lp"] + 1),
                    P["v_phi"], 0.0, 0.1, 300)
    assert np.all(np.isfinite(np.array(y)))
    y0 = R.integrate(x[:200], zeta[:200], ux[:200], uz[:200], 0.0, wp, 0.05, P["v_phi"], 0.0, 0.1, 300)
    I = lambda x_, z_, a_, b_: np.sqrt(1 + a_ ** 2 + b_ ** 2) - b_ + 0.25 * wp * wp * (x_ ** 2 + z_ ** 2)
    I0 = I(x[:200], zeta[:200], ux[:200], uz[:200])
    assert np.max(np.abs(I(*y0) - I0) / I0) < 1e-10            # no laser: invariant kept
    assert np.max(np.abs(I(*y) - I0) / I0) > 1e-6               # the laser changes it


# ---- time-staggering factor and injection (Sec. IV.A, Appendix A)
def _states(n, seed):
    rng = np.random.default_rng(seed)
    return np.array([rng.uniform(-3, 3, n), rng.uniform(-30, 5, n), rng.normal(0, 2, n),
                     rng.uniform(0, 50, n)])


def test_staggering_factor_scales_only_the_magnetic_terms():
    """b multiplies terms that do no work: F(b) - F(0) = b (F(1) - F(0)) and
    v . (F(1) - F(0)) = 0, while b = 1 is the printed Eq. 8 bit for bit"""
    y = _states(200, 3)
    t = 17.3
    par = (2.1, 0.08, 0.11, 1.0025)
    F0 = R.rhs(t, y, *par, bfac=0.0)
    F1 = R.rhs(t, y, *par, bfac=1.0)
    Fb = R.rhs(t, y, *par, bfac=0.9935)
    assert np.array_equal(F1, R.rhs(t, y, *par))
    dm = F1 - F0
    scale = np.max(np.abs(dm[2:]))
    assert scale > 1e-3
    assert np.max(np.abs((Fb - F0) - 0.9935 * dm)) < 1e-12 * (1 + scale)
    gamma = np.sqrt(1 + y[2] ** 2 + y[3] ** 2)
    power = (y[2] * dm[2] + y[3] * dm[3]) / gamma          # v . F_magnetic
    assert np.max(np.abs(power)) < 1e-12 * (1 + scale)
    assert np.array_equal(F0[:2], F1[:2])                  # positions do not see it


def test_paper_staggering_factor_from_its_yee_time_step():
    """Sec. IV.A quotes cos(omega0 dt/2) ~ 0.994 for the Yee runs: with the
    Appendix A time step 0.01875/omega_p and omega0 = v_phi k_z = 12.17 omega_p"""
    import json
    import os
    import synth
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))
    P = synth.REDUCED_PAPER
    w0_over_wp = P["v_phi"] * P["kz_over_wp"]
    b = np.cos(0.5 * w0_over_wp * gold["dt_yee_3d_over_wp"]["value"])
    # the printed value is rounded ("approximately 0.994"): 0.9935 here
    assert b == pytest.approx(gold["yee_time_staggering_factor"]["value"], abs=1e-3)


def test_start_steps_hold_then_integrate():
    y0 = _states(6, 4)
    par = dict(a0=1.7, wp=0.07, kperp=0.05, vphi=1.001)
    t0, dt, n = 2.0, 0.1, 50
    start = np.array([0, 7, 13, 49, 50, 80])
    got = np.array(R.integrate(*y0, par["a0"], par["wp"], par["kperp"], par["vphi"], t0, dt, n,
                               bfac=0.99, start=start))
    for i, k in enumerate(start):
        if k >= n:
            assert np.array_equal(got[:, i], y0[:, i])      # not yet injected
            continue
        ref = np.array(R.integrate(*y0[:, i:i + 1], par["a0"], par["wp"], par["kperp"], par["vphi"],
                                   t0 + k * dt, dt, n - k, bfac=0.99))[:, 0]
        assert np.max(np.abs(got[:, i] - ref)) < 1e-12 * (1 + np.max(np.abs(ref)))
