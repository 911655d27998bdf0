"""Seeded synthetic inputs shared by the oracle side and the CUDA side of the
tests and the benchmark.  This module holds workload descriptions and random
arrays only -- none of the method's arithmetic.

The workloads stand in for the paper's laser-wakefield runs (Table I and
Appendix A), whose data are not available: uniform or up-ramped electron
plasma, a linearly polarised Gaussian laser, normalised units (c = 1, lengths
in c/w0, time in 1/w0, densities in n_c).
"""
import numpy as np

# Each workload: grid, plasma, laser, steps.  "dt": None means 0.9 x the CFL
# limit of the chosen solver.  z_centroid / z_focus are lab-frame positions.
WORKLOADS = {
    # Plain FP64-sized case: 256 x 32, 8 ppc, periodic box.  The laser is
    # centred in the 51.2-long box (launch point z = 60 lies outside it).
    "cfg1_small": dict(nz=256, nr=32, dz=0.2, dr=0.5, n_modes=2, solver="dual",
                       periodic=True, moving_window=False,
                       plasma=dict(n0=0.01, z_start=0.0, ramp_len=0.0, ppc=(2, 2, 2), seed=1),
                       laser=dict(a0=1.0, w0=10.0, fwhm=20.0, z_centroid=25.6, z_focus=25.6),
                       steps=100),
    # LWFA/DLA run: 4000 x 400, 32 ppc (51.2M macroparticles), moving window.
    # The plasma fills the initial box (linear up-ramp over its first 200 c/w0,
    # plateau after); the pulse starts 2 FWHM behind the front edge and is
    # focused 100 c/w0 (half a ramp length) ahead of its launch point.
    "cfg2_lwfa": dict(nz=4000, nr=400, dz=0.2, dr=0.8, n_modes=2, solver="dual",
                      periodic=False, moving_window=True,
                      plasma=dict(n0=0.005, z_start=0.0, ramp_len=200.0, ppc=(2, 2, 8), seed=2),
                      laser=dict(a0=2.0, w0=30.0, fwhm=100.0, z_centroid=600.0, z_focus=700.0),
                      steps=5000),
    # Precision study geometry: 2000 x 200, 16 ppc, config-1 physics, periodic.
    "cfg4_precision": dict(nz=2000, nr=200, dz=0.2, dr=0.5, n_modes=2, solver="dual",
                           periodic=True, moving_window=False,
                           plasma=dict(n0=0.01, z_start=0.0, ramp_len=0.0, ppc=(2, 2, 4), seed=4),
                           laser=dict(a0=1.0, w0=10.0, fwhm=20.0, z_centroid=200.0, z_focus=200.0),
                           steps=2000),
}


def workload(name, **over):
    w = dict(WORKLOADS[name])
    for k, v in over.items():
        w[k] = v
    return w


def random_particles(seed, n, nz, nr, dz, dr, umax=1.0, zmin=0.0, axis_frac=0.02, wall_frac=0.02):
    """n particles uniform in the box volume (r ~ sqrt(U)), a few near the axis
    and the wall, momenta uniform in [-umax, umax]^3, weights in [0.5, 1.5]."""
    rng = np.random.default_rng(seed)
    z = zmin + rng.uniform(0.0, nz * dz, n)
    r = nr * dr * np.sqrt(rng.uniform(0.0, 1.0, n))
    na, nw = int(axis_frac * n), int(wall_frac * n)
    r[:na] = rng.uniform(0.0, 0.3 * dr, na)
    r[na:na + nw] = nr * dr - rng.uniform(1e-6, 0.3 * dr, nw)
    phi = rng.uniform(-np.pi, np.pi, n)
    u = rng.uniform(-umax, umax, (3, n))
    w = rng.uniform(0.5, 1.5, n) * 1e-3
    return dict(z=z, r=r, phi=phi, ux=u[0], uy=u[1], uz=u[2], w=w)


def random_fields(seed, nz, nr, n_modes, amp=0.3):
    """dict comp -> list over modes of [nr+1][nz] complex arrays (mode 0 real)"""
    rng = np.random.default_rng(seed)
    out = {}
    for c in ("r", "phi", "z"):
        out[c] = []
        for m in range(n_modes):
            re = rng.standard_normal((nr + 1, nz))
            im = rng.standard_normal((nr + 1, nz)) if m else np.zeros((nr + 1, nz))
            out[c].append(amp * (re + 1j * im))
    return out


# Appendix A's reduced-model set (measured from the paper's 3D PIC runs):
# v_phi = 1.002565 c, v_g = 0.993583 c, k_z = 12.14 w_p/c, R = 3 c/w_p, a0 = 2.8.
# In units of the local laser frequency w0 = v_phi k_z (= 12.17 w_p):
REDUCED_PAPER = dict(a0=2.8, v_phi=1.002565, v_g=0.993583, kz_over_wp=12.14, R_over_lp=3.0)


def reduced_bunch(seed, n, v_g=0.993583, wp=1.0 / (1.002565 * 12.14), R_over_lp=3.0):
    """Electrons injected into the bubble as Appendix A describes, in units of
    the laser frequency (c = 1): zeta uniform in [-2R + 0.286/w_p, -2R +
    0.836/w_p] shifted by +R (the model's bubble is centred on zeta = 0), x
    uniform in [-r_b, r_b] with r_b = sqrt(R^2 - zeta^2), gamma uniform in
    [gamma_g, 2 gamma_g] with gamma_g = 1/sqrt(1 - v_g^2), and the velocity at
    a random angle to the x axis with v_z >= v_g.  Returns (x, zeta, u_x, u_z):
    the state at injection.  The injection times (the appendix spreads them
    over 200/w_p) are not drawn here; the caller passes each electron's start
    step to the integrator (`start`), as the benchmark's staggering leg and
    the reduced-model tests do."""
    rng = np.random.default_rng([seed, 7])
    R = R_over_lp / wp
    zeta = rng.uniform(-2 * R + 0.286 / wp, -2 * R + 0.836 / wp, n) + R
    rb = np.sqrt(np.maximum(R * R - zeta * zeta, 0.0))
    x = rng.uniform(-1.0, 1.0, n) * rb
    gg = 1.0 / np.sqrt(1.0 - v_g * v_g)
    gamma = rng.uniform(gg, 2 * gg, n)
    v = np.sqrt(1.0 - 1.0 / (gamma * gamma))
    smin = np.minimum(v_g / v, 1.0)                  # sin of the angle to the x axis, v_z >= v_g
    th = rng.uniform(np.arcsin(smin), np.pi - np.arcsin(smin))
    u = gamma * v
    return x, zeta, u * np.cos(th), u * np.sin(th)
