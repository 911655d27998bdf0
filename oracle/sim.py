"""A small FP64 driver around the oracle box: coefficients and time step, plasma,
laser, moving window.  TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Moving window (a reading: the paper's runs move the box with the laser but do
not describe it): after a step that ends at t = n dt, while v t >= (shifts+1) dz
the box moves by one cell; the new front column receives the plasma lattice of
its absolute cell index, particles behind the box are removed.
"""
import numpy as np

from . import Oracle, coeffs, setup


class Run:
    def __init__(self, nz, nr, dz, dr, n_modes=2, dt=None, cfl_frac=0.9, solver="dual",
                 n_coef=16, fit_band=0.8, jz_filter=True, periodic=True,
                 moving_window=False, window_v=1.0, track_work=False, filter_tol=1e-16):
        if moving_window and periodic:
            raise ValueError("a moving window needs an open box")
        if dt is None or dt <= 0:
            dt = cfl_frac * coeffs.cfl_dt(dz, dr, nr, n_modes, solver, n_coef, fit_band)
        self.cE, self.cB = coeffs.solver_coefficients(solver, dt, dz, n_coef, fit_band)
        self.ktaps = coeffs.filter_taps(self.cB, filter_tol) if (jz_filter and solver != "yee") else None
        self.o = Oracle(nz, nr, n_modes, dz, dr, dt, self.cE, self.cB, self.ktaps,
                        periodic=periodic, track_work=track_work)
        self.nz, self.nr, self.dz, self.dr, self.dt = nz, nr, dz, dr, dt
        self.moving_window, self.window_v = moving_window, window_v
        self.nstep = 0
        self.shifts = 0
        self.plasma = None

    def load_plasma(self, n0, z_start, ramp_len, ppc, seed, jitter=True):
        self.plasma = dict(n0=n0, z_start=z_start, ramp_len=ramp_len, ppc=tuple(ppc),
                           seed=seed, jitter=jitter)
        p = setup.plasma_cells(np.arange(self.nz) + self.shifts, self.nr, self.dz, self.dr,
                               n0, z_start, ramp_len, ppc, seed, jitter)
        self.o.load_particles(**p)
        return p

    def add_laser(self, a0, w0, fwhm, z_centroid, z_focus, pol_angle=0.0):
        setup.add_laser(self.o, self.cE, self.cB, a0, w0, fwhm, z_centroid, z_focus, pol_angle)

    def _shift(self):
        self.o.shift_window()
        self.shifts += 1
        if self.plasma is not None:
            pl = self.plasma
            p = setup.plasma_cells([self.nz - 1 + self.shifts], self.nr, self.dz, self.dr,
                                   pl["n0"], pl["z_start"], pl["ramp_len"], pl["ppc"],
                                   pl["seed"], pl["jitter"])
            if len(p["z"]):
                self.o.append_particles(**p)
        self.o.compact()

    def step(self, n=1):
        for _ in range(n):
            self.o.step(1)
            self.nstep += 1
            if self.moving_window:
                while self.window_v * (self.nstep * self.dt) >= (self.shifts + 1) * self.dz:
                    self._shift()
