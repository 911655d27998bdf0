"""Python binding of libqpic, the GB300 quasi-3D dual-solver PIC step.

Argument marshalling only: every step of the method runs in the CUDA library
(include/qpic.h).  There is no CPU fallback: if the library is missing or no
GPU is present, calls raise.

PyTorch is used for plumbing only: an optional device allocator hook (so the
library's buffers come from torch's caching allocator) and the CUDA stream.
"""
import ctypes
import os

import numpy as np

from . import _build

_lib = None

# revision tag of the gather+push+deposit kernel; measured DRAM traffic stored
# under profiles/ is only reported while it matches
KERNEL_REV = "gpd-v21"

QPIC_YEE, QPIC_DUAL = 0, 1
QPIC_FP64, QPIC_FP32_FIXED, QPIC_FP32_FATOMIC = 0, 1, 2
FIELD = {"E": 0, "B": 1, "Bbar": 2, "J": 3, "rho": 4}
COMP = {"r": 0, "phi": 1, "z": 2}
STAGE_FARADAY, STAGE_PARTICLES, STAGE_AMPERE, STAGE_WINDOW, STAGE_SORT = 1, 2, 4, 8, 16
STATUS = {0: "OK", -1: "EINVAL", -2: "ENOMEM", -3: "ECUDA", -4: "ECFL", -5: "EOVERFLOW",
          -6: "ETIMEOUT", -7: "ENONFINITE", -8: "ESTATE", -9: "ECAPACITY", -10: "ECHECK"}

ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class Config(ctypes.Structure):
    _fields_ = [
        ("nz", ctypes.c_int32), ("nr", ctypes.c_int32), ("n_modes", ctypes.c_int32),
        ("dz", ctypes.c_double), ("dr", ctypes.c_double), ("dt", ctypes.c_double),
        ("cfl_frac", ctypes.c_double), ("solver", ctypes.c_int32), ("n_coef", ctypes.c_int32),
        ("fit_band", ctypes.c_double), ("precision", ctypes.c_int32), ("jz_filter", ctypes.c_int32),
        ("filter_tol", ctypes.c_double), ("periodic_z", ctypes.c_int32),
        ("moving_window", ctypes.c_int32), ("window_v", ctypes.c_double),
        ("tile_z", ctypes.c_int32), ("tile_r", ctypes.c_int32), ("sort_period", ctypes.c_int32),
        ("particles_per_thread", ctypes.c_int32), ("absorb_cells", ctypes.c_int32),
        ("absorb_sigma", ctypes.c_double), ("track_work", ctypes.c_int32), ("seed", ctypes.c_uint64), ("max_particles", ctypes.c_int64),
        ("cuda_stream", ctypes.c_void_p), ("dev_alloc", ALLOC_FN), ("dev_free", FREE_FN),
        ("alloc_user", ctypes.c_void_p),
    ]


class QpicError(RuntimeError):
    pass


def _checked():
    return os.environ.get("QPIC_CHECKED") == "1"


def library_path():
    return _build.LIB_CHECK if _checked() else _build.LIB


def load(build_if_needed=True):
    """Load libqpic.so (building it with nvcc first when stale); with
    QPIC_CHECKED=1 in the environment, the checked build (QPIC_CHECK)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build(check=_checked()) if build_if_needed else library_path()
    if not os.path.exists(path):
        raise QpicError("libqpic.so not found at %s (run __graft_entry__.build())" % path)
    L = ctypes.CDLL(path)
    _declare(L)
    _lib = L
    return L


_P = ctypes.c_void_p
_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.c_int32


def _declare(L):
    L.qpic_default_config.argtypes = [ctypes.POINTER(Config)]
    L.qpic_init.argtypes = [ctypes.POINTER(Config), ctypes.POINTER(_P)]
    L.qpic_destroy.argtypes = [_P]
    L.qpic_destroy.restype = None
    L.qpic_last_error.argtypes = [_P]
    L.qpic_last_error.restype = ctypes.c_char_p
    L.qpic_get_solver.argtypes = [_P, _D, ctypes.POINTER(_I), _D, _D, _I, _D, _I, ctypes.POINTER(_I)]
    L.qpic_cfl_limit.argtypes = [_P, _D]
    L.qpic_load_plasma.argtypes = [_P, ctypes.c_double, ctypes.c_double, ctypes.c_double, _I, _I, _I, _I]
    L.qpic_load_particles.argtypes = [_P, ctypes.c_int64] + [_D] * 7
    L.qpic_add_laser.argtypes = [_P] + [ctypes.c_double] * 6
    L.qpic_step.argtypes = [_P, _I]
    L.qpic_run_stages.argtypes = [_P, _I]
    L.qpic_get_field.argtypes = [_P, _I, _I, _I, _D, _D]
    L.qpic_set_field.argtypes = [_P, _I, _I, _I, _D, _D]
    L.qpic_get_fields.argtypes = [_P, _I, _I, _I, _D, _D, ctypes.c_int64]
    L.qpic_set_fields.argtypes = [_P, _I, _I, _I, _D, _D, ctypes.c_int64]
    L.qpic_num_particles.argtypes = [_P, ctypes.POINTER(ctypes.c_int64)]
    L.qpic_get_particles.argtypes = [_P, _D, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)]
    L.qpic_get_particles_raw.argtypes = [_P, _D, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)]
    L.qpic_get_diag.argtypes = [_P, _D, _I]
    L.qpic_fit_coefficients.argtypes = [_I, ctypes.c_double, ctypes.c_double, _I, ctypes.c_double,
                                        _D, _D, ctypes.POINTER(_I)]
    L.qpic_filter_taps.argtypes = [_D, _I, ctypes.c_double, _D, _I, ctypes.POINTER(_I)]
    L.qpic_stability_limit.argtypes = [_I, ctypes.c_double, ctypes.c_double, _I, _I, _I,
                                       ctypes.c_double, _D]
    L.qpic_profile.argtypes = [_P, _I, _I]
    L.qpic_launch_count.argtypes = [_P, ctypes.POINTER(ctypes.c_int64)]
    L.qpic_charge_density_noalloc.argtypes = [_P, _I, _D, _D]
    L.qpic_batch_create.argtypes = [ctypes.POINTER(_P), _I, _P, ctypes.POINTER(_P)]
    L.qpic_batch_create.restype = ctypes.c_int
    L.qpic_batch_step.argtypes = [_P, _I]
    L.qpic_batch_step.restype = ctypes.c_int
    L.qpic_batch_cycle.argtypes = [_P]
    L.qpic_batch_cycle.restype = _I
    L.qpic_batch_last_error.argtypes = [_P]
    L.qpic_batch_last_error.restype = ctypes.c_char_p
    L.qpic_batch_set_wait.argtypes = [_P, ctypes.c_int64, _I]
    L.qpic_batch_set_wait.restype = ctypes.c_int
    L.qpic_batch_destroy.argtypes = [_P]
    L.qpic_batch_destroy.restype = None
    L.qpic_gauss_residual.argtypes = [_P, _D, _I]
    L.qpic_gauss_residual.restype = ctypes.c_int
    L.qpic_spectrum.argtypes = [_P, _D, _I, _D]
    L.qpic_spectrum.restype = ctypes.c_int
    L.qpic_charge_density_noalloc.restype = ctypes.c_int
    L.qpic_launch_count.restype = ctypes.c_int
    L.qpic_reduced_integrate.argtypes = ([ctypes.c_int64] + [_D] * 4 + [ctypes.c_double] * 7 +
                                         [_I, ctypes.POINTER(_I)])
    L.qpic_reduced_integrate.restype = ctypes.c_int
    L.qpic_reduced_integrate_device.argtypes = ([ctypes.c_int64] + [ctypes.c_void_p] * 4 +
                                                [ctypes.c_double] * 7 + [_I, ctypes.c_void_p,
                                                                         ctypes.c_void_p])
    L.qpic_reduced_integrate_device.restype = ctypes.c_int
    L.qpic_work_f_estimate.argtypes = [ctypes.c_int64] + [_D] * 5 + [ctypes.c_double] * 3 + [_D, _D]
    L.qpic_work_f_estimate.restype = ctypes.c_int
    L.qpic_state_size.argtypes = [_P, ctypes.POINTER(ctypes.c_int64)]
    L.qpic_state_size.restype = ctypes.c_int
    L.qpic_save_state.argtypes = [_P, ctypes.c_void_p, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)]
    L.qpic_save_state.restype = ctypes.c_int
    L.qpic_load_state.argtypes = [_P, ctypes.c_void_p, ctypes.c_int64]
    L.qpic_load_state.restype = ctypes.c_int
    L.qpic_kernel_times.argtypes = [_P, _I, _D, ctypes.POINTER(ctypes.c_int64),
                                    ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(_I)]
    for name in ("qpic_default_config", "qpic_init", "qpic_get_solver", "qpic_cfl_limit",
                 "qpic_load_plasma", "qpic_load_particles", "qpic_add_laser", "qpic_step",
                 "qpic_run_stages", "qpic_get_field", "qpic_set_field", "qpic_get_fields",
                 "qpic_set_fields", "qpic_num_particles",
                 "qpic_get_particles", "qpic_get_diag", "qpic_profile", "qpic_kernel_times",
                 "qpic_get_particles_raw", "qpic_fit_coefficients", "qpic_filter_taps",
                 "qpic_stability_limit"):
        getattr(L, name).restype = ctypes.c_int


def _dp(a):
    return a.ctypes.data_as(_D)


def fit_coefficients(solver, dt, dz, n_coef=16, fit_band=0.8):
    """Host-side dual/Yee coefficient fit of the library (no GPU needed)."""
    L = load()
    cE = np.zeros(64)
    cB = np.zeros(64)
    n = _I()
    st = L.qpic_fit_coefficients(QPIC_YEE if solver == "yee" else QPIC_DUAL, dt, dz, n_coef,
                                 fit_band, _dp(cE), _dp(cB), ctypes.byref(n))
    if st != 0:
        raise QpicError("qpic_fit_coefficients: %s" % STATUS.get(st, st))
    return cE[:n.value].copy(), cB[:n.value].copy()


def filter_taps(cB, tol=1e-16):
    L = load()
    cB = np.ascontiguousarray(cB, dtype=np.float64)
    taps = np.zeros(512)
    n = _I()
    st = L.qpic_filter_taps(_dp(cB), len(cB), tol, _dp(taps), 512, ctypes.byref(n))
    if st != 0:
        raise QpicError("qpic_filter_taps: %s" % STATUS.get(st, st))
    return taps[:n.value].copy() if n.value else None


def stability_limit(solver, dz, dr, nr, n_modes, n_coef=16, fit_band=0.8):
    L = load()
    v = ctypes.c_double()
    st = L.qpic_stability_limit(QPIC_YEE if solver == "yee" else QPIC_DUAL, dz, dr, nr, n_modes,
                                n_coef, fit_band, ctypes.byref(v))
    if st != 0:
        raise QpicError("qpic_stability_limit: %s" % STATUS.get(st, st))
    return v.value


def work_f_estimate(ux, uy, uz, Wz, Wperp, omega_p, w0, omega0=1.0):
    """LWFA / DLA work estimated from the directional work of a run with
    track_work=2 (W0 = W_z, W1 = W_perp), by the library's host function
    qpic_work_f_estimate (Eqs. 19-20; no GPU needed).  Returns (lwfa, dla)."""
    L = load()
    a = [np.ascontiguousarray(x, dtype=np.float64) for x in (ux, uy, uz, Wz, Wperp)]
    n = len(a[0])
    if any(len(x) != n for x in a):
        raise ValueError("work_f_estimate: arrays of different lengths")
    lwfa, dla = np.zeros(n), np.zeros(n)
    st = L.qpic_work_f_estimate(n, *[_dp(x) for x in a], omega_p, w0, omega0, _dp(lwfa), _dp(dla))
    if st != 0:
        raise QpicError("qpic_work_f_estimate: %s" % STATUS.get(st, st))
    return lwfa, dla


def reduced_integrate(x, zeta, ux, uz, a0, omega_p, k_perp, v_phi, t0, dt, nsteps, bfac=1.0,
                      start=None):
    """The reduced model of Eq. 8 on the GPU (qpic_reduced_integrate): host
    arrays in, new host arrays (x, zeta, u_x, u_z) out after nsteps steps.
    bfac: factor on the laser's magnetic terms (cos(omega0 dt/2) models a
    time-staggered solver); start: optional per-electron first step."""
    L = load()
    a = [np.array(v, dtype=np.float64, copy=True).reshape(-1) for v in (x, zeta, ux, uz)]
    n = len(a[0])
    if any(len(v) != n for v in a):
        raise ValueError("reduced_integrate: arrays of different lengths")
    sp = None
    if start is not None:
        sa = np.ascontiguousarray(start, dtype=np.int32).reshape(-1)
        if len(sa) != n:
            raise ValueError("reduced_integrate: start has %d entries, need %d" % (len(sa), n))
        sp = sa.ctypes.data_as(ctypes.POINTER(_I))
    st = L.qpic_reduced_integrate(n, *[_dp(v) for v in a], a0, omega_p, k_perp, v_phi, bfac, t0, dt,
                                  int(nsteps), sp)
    if st != 0:
        raise QpicError("qpic_reduced_integrate: %s" % STATUS.get(st, st))
    return tuple(a)


def reduced_integrate_device(ptrs, n, a0, omega_p, k_perp, v_phi, t0, dt, nsteps, stream=None, bfac=1.0,
                             start_ptr=None):
    """Device variant: ptrs = four device addresses of n doubles (x, zeta, u_x,
    u_z), advanced in place on `stream` (an integer cudaStream_t or None);
    start_ptr: optional device address of n int32 first steps."""
    L = load()
    st = L.qpic_reduced_integrate_device(n, *[ctypes.c_void_p(int(p)) for p in ptrs], a0, omega_p, k_perp,
                                         v_phi, bfac, t0, dt, int(nsteps), ctypes.c_void_p(start_ptr or 0),
                                         ctypes.c_void_p(stream or 0))
    if st != 0:
        raise QpicError("qpic_reduced_integrate_device: %s" % STATUS.get(st, st))


class Batch:
    """Independent runs advanced together by one CUDA graph launch per cycle
    (per step: Faraday per run, one persistent particle-phase launch per group
    of runs, then filter, Ampere and sort per run)."""

    def __init__(self, sims, stream=None):
        self.L = load()
        self.sims = list(sims)
        arr = (_P * len(self.sims))(*[sm.h for sm in self.sims])
        st_ptr = None if stream is None else (stream if isinstance(stream, int) else stream.cuda_stream)
        h = _P()
        st = self.L.qpic_batch_create(arr, len(self.sims), st_ptr, ctypes.byref(h))
        self.h = h
        if st != 0:
            msg = self.L.qpic_batch_last_error(h).decode() if h else ""
            self.close()
            raise QpicError("qpic_batch_create: %s %s" % (STATUS.get(st, st), msg))
        self.cycle = int(self.L.qpic_batch_cycle(h))

    def step(self, n):
        st = self.L.qpic_batch_step(self.h, int(n))
        if st != 0:
            raise QpicError("qpic_batch_step: %s %s" % (STATUS.get(st, st),
                                                       self.L.qpic_batch_last_error(self.h).decode()))

    def set_wait(self, polls, withheld_item=-1):
        st = self.L.qpic_batch_set_wait(self.h, int(polls), int(withheld_item))
        if st != 0:
            raise QpicError("qpic_batch_set_wait: %s" % STATUS.get(st, st))

    def close(self):
        if getattr(self, "h", None):
            self.L.qpic_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _TorchAllocator:
    """Device memory from PyTorch's caching allocator, kept alive by pointer."""

    def __init__(self, device=0):
        import torch
        self.torch = torch
        self.device = device
        self.live = {}
        self.alloc_cb = ALLOC_FN(self._alloc)
        self.free_cb = FREE_FN(self._free)

    def _alloc(self, nbytes, user):
        try:
            t = self.torch.empty(int(nbytes), dtype=self.torch.uint8, device="cuda:%d" % self.device)
        except RuntimeError:
            return 0                      # out of memory: the library reports QPIC_ENOMEM
        p = t.data_ptr()
        self.live[p] = t
        return p

    def _free(self, ptr, user):
        self.live.pop(ptr, None)


class Sim:
    """One simulation context (a thin wrapper over the C ABI)."""

    def __init__(self, nz, nr, dz, dr, n_modes=2, dt=0.0, cfl_frac=0.9, solver="dual", n_coef=16,
                 fit_band=0.8, jz_filter=True, filter_tol=1e-16, periodic=True,
                 moving_window=False, window_v=1.0, tile_z=16, tile_r=8, sort_period=2,
                 particles_per_thread=16, absorb_cells=0, absorb_sigma=0.0,
                 track_work=False, seed=1, max_particles=0, stream=None, torch_alloc=False,
                 precision=QPIC_FP32_FIXED):
        self.L = load()
        cfg = Config()
        self.L.qpic_default_config(ctypes.byref(cfg))
        cfg.nz, cfg.nr, cfg.n_modes = nz, nr, n_modes
        cfg.dz, cfg.dr, cfg.dt, cfg.cfl_frac = dz, dr, (dt or 0.0), cfl_frac
        cfg.solver = QPIC_YEE if solver == "yee" else QPIC_DUAL
        cfg.n_coef, cfg.fit_band = n_coef, fit_band
        cfg.precision = precision
        cfg.jz_filter, cfg.filter_tol = int(jz_filter), filter_tol
        cfg.periodic_z, cfg.moving_window, cfg.window_v = int(periodic), int(moving_window), window_v
        cfg.tile_z, cfg.tile_r, cfg.sort_period = tile_z, tile_r, sort_period
        cfg.particles_per_thread = particles_per_thread
        cfg.absorb_cells, cfg.absorb_sigma = absorb_cells, absorb_sigma
        # track_work: False/0 off, True/1 modal work (Eq. 16), 2 directional work (Eq. 17)
        cfg.track_work, cfg.seed, cfg.max_particles = int(track_work), seed, max_particles
        if stream is not None:
            cfg.cuda_stream = stream if isinstance(stream, int) else stream.cuda_stream
        self._alloc = None
        if torch_alloc:
            # True: PyTorch's caching allocator; or an allocator object with
            # alloc_cb / free_cb callbacks (as _TorchAllocator has)
            self._alloc = torch_alloc if hasattr(torch_alloc, "alloc_cb") else _TorchAllocator()
            cfg.dev_alloc, cfg.dev_free = self._alloc.alloc_cb, self._alloc.free_cb
        self.cfg = cfg
        h = _P()
        st = self.L.qpic_init(ctypes.byref(cfg), ctypes.byref(h))
        self.h = h
        if st != 0:
            msg = self.L.qpic_last_error(h).decode() if h else ""
            if h:
                self.L.qpic_destroy(h)
                self.h = None
            raise QpicError("qpic_init: %s %s" % (STATUS.get(st, st), msg))
        self.nz, self.nr, self.nm = nz, nr, n_modes
        self.dz, self.dr = dz, dr
        self.dt = self.solver()["dt"]

    def close(self):
        if getattr(self, "h", None):
            self.L.qpic_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st, what):
        if st != 0:
            raise QpicError("%s: %s %s" % (what, STATUS.get(st, st),
                                           self.L.qpic_last_error(self.h).decode()))

    # ---- solver constants
    def solver(self):
        dt = ctypes.c_double()
        L = _I()
        cE = np.zeros(64)
        cB = np.zeros(64)
        taps = np.zeros(512)
        nt = _I()
        self._check(self.L.qpic_get_solver(self.h, ctypes.byref(dt), ctypes.byref(L), _dp(cE), _dp(cB),
                                           64, _dp(taps), 512, ctypes.byref(nt)), "get_solver")
        return {"dt": dt.value, "cE": cE[:L.value].copy(), "cB": cB[:L.value].copy(),
                "taps": taps[:nt.value].copy() if nt.value else None}

    def cfl_limit(self):
        v = ctypes.c_double()
        self._check(self.L.qpic_cfl_limit(self.h, ctypes.byref(v)), "cfl_limit")
        return v.value

    # ---- initial conditions
    def load_plasma(self, n0, z_start, ramp_len, ppc, jitter=True):
        self._check(self.L.qpic_load_plasma(self.h, n0, z_start, ramp_len, ppc[0], ppc[1], ppc[2],
                                            int(jitter)), "load_plasma")

    def load_particles(self, z, r, phi, ux, uy, uz, w):
        arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (z, r, phi, ux, uy, uz, w)]
        self._check(self.L.qpic_load_particles(self.h, len(arrs[0]), *[_dp(a) for a in arrs]),
                    "load_particles")

    def add_laser(self, a0, w0, fwhm, z_centroid, z_focus, pol_angle=0.0):
        self._check(self.L.qpic_add_laser(self.h, a0, w0, fwhm, z_centroid, z_focus, pol_angle),
                    "add_laser")

    # ---- stepping
    def step(self, n=1):
        self._check(self.L.qpic_step(self.h, int(n)), "step")

    def run_stages(self, stages):
        self._check(self.L.qpic_run_stages(self.h, int(stages)), "run_stages")

    # ---- fields
    def get_field(self, which, comp, mode):
        re = np.zeros((self.nr + 1, self.nz))
        im = np.zeros((self.nr + 1, self.nz))
        self._check(self.L.qpic_get_fields(self.h, FIELD[which], COMP[comp], mode, _dp(re), _dp(im),
                                           re.size), "get_fields")
        return re + 1j * im

    def set_field(self, which, comp, mode, val):
        """val: a complex (nr+1, nz) array, or a (re, im) pair of float64 arrays
        of that size (passed as they are when C-contiguous: pinned host
        buffers are then copied without staging)."""
        if isinstance(val, tuple):
            re, im = (np.ascontiguousarray(x, dtype=np.float64).reshape(-1) for x in val)
        else:
            val = np.asarray(val, dtype=np.complex128).reshape(self.nr + 1, self.nz)
            re = np.ascontiguousarray(val.real)
            im = np.ascontiguousarray(val.imag)
        if re.size != (self.nr + 1) * self.nz or im.size != re.size:
            raise ValueError("set_field: %d values, the grid has %d" % (re.size, (self.nr + 1) * self.nz))
        self._check(self.L.qpic_set_fields(self.h, FIELD[which], COMP[comp], mode, _dp(re), _dp(im),
                                           re.size), "set_fields")

    def fields(self, which):
        return np.array([[self.get_field(which, c, m) for m in range(self.nm)]
                         for c in ("r", "phi", "z")])

    def rho(self):
        return np.array([self.get_field("rho", "r", m) for m in range(self.nm)])

    # ---- particles and diagnostics
    def num_particles(self):
        n = ctypes.c_int64()
        self._check(self.L.qpic_num_particles(self.h, ctypes.byref(n)), "num_particles")
        return n.value

    def particles(self, out=None):
        """Live particles as FP64 arrays z, r, phi, ux, uy, uz, w, W0, W1.  out: an
        optional caller-owned float64 buffer of at least 9 * num_particles()
        (for example in pinned host memory); the arrays returned are then views
        into it, valid until the buffer is reused."""
        n = self.num_particles()
        cap = max(n, 1)
        keys = ("z", "r", "phi", "ux", "uy", "uz", "w", "W0", "W1")
        if out is not None:
            out = np.ascontiguousarray(out, dtype=np.float64).reshape(-1)
            if out.size < 9 * cap:
                raise QpicError("particles: out holds %d doubles, need %d" % (out.size, 9 * cap))
            cap = out.size // 9
        else:
            out = np.zeros(9 * cap)
        nout = ctypes.c_int64()
        self._check(self.L.qpic_get_particles(self.h, _dp(out), cap, ctypes.byref(nout)),
                    "get_particles")
        n = nout.value
        v = out[:9 * cap].reshape(9, cap)[:, :n]
        return {k: v[i] for i, k in enumerate(keys)}

    def particles_raw(self):
        """buffer-order export (no sort): same order across particle stages"""
        cap = max(self.cfg.max_particles, 1)
        n = ctypes.c_int64()
        while True:
            out = np.zeros(9 * cap)
            st = self.L.qpic_get_particles_raw(self.h, _dp(out), cap, ctypes.byref(n))
            if st == -9 and n.value > cap:
                cap = n.value
                continue
            self._check(st, "get_particles_raw")
            break
        out = out.reshape(9, cap)[:, :n.value]
        keys = ("z", "r", "phi", "ux", "uy", "uz", "w", "W0", "W1")
        return {k: out[i].copy() for i, k in enumerate(keys)}

    def save_state(self):
        """the whole simulation state as a bytes-like numpy uint8 array (qpic_save_state)"""
        n = ctypes.c_int64()
        self._check(self.L.qpic_state_size(self.h, ctypes.byref(n)), "state_size")
        buf = np.empty(n.value, dtype=np.uint8)
        w = ctypes.c_int64()
        self._check(self.L.qpic_save_state(self.h, buf.ctypes.data, buf.size, ctypes.byref(w)), "save_state")
        return buf[:w.value]

    def load_state(self, buf):
        """replace this context's state with a snapshot from save_state"""
        buf = np.ascontiguousarray(buf, dtype=np.uint8)
        self._check(self.L.qpic_load_state(self.h, buf.ctypes.data, buf.size), "load_state")

    def diag(self):
        v = np.zeros(7 + self.nm)
        self._check(self.L.qpic_get_diag(self.h, _dp(v), len(v)), "get_diag")
        return {"time": v[0], "steps": int(v[1]), "shifts": int(v[2]), "particles": int(v[3]),
                "charge": v[4], "kinetic": v[5], "field_energy": list(v[6:6 + self.nm]),
                "overflow": bool(v[6 + self.nm])}

    def gauss_residual(self):
        """per mode (|div_B E - rho_net|, |rho_net|) L2 norms"""
        v = np.zeros(2 * self.nm)
        self._check(self.L.qpic_gauss_residual(self.h, _dp(v), len(v)), "gauss_residual")
        return [(v[2 * m], v[2 * m + 1]) for m in range(self.nm)]

    def spectrum(self, edges_mev):
        e = np.ascontiguousarray(edges_mev, dtype=np.float64)
        out = np.zeros(len(e) - 1)
        self._check(self.L.qpic_spectrum(self.h, _dp(e), len(out), _dp(out)), "spectrum")
        return out

    def profile(self, enable=True, reset=True):
        self._check(self.L.qpic_profile(self.h, int(enable), int(reset)), "profile")

    def launch_count(self):
        n = ctypes.c_int64()
        self._check(self.L.qpic_launch_count(self.h, ctypes.byref(n)), "launch_count")
        return n.value

    def kernel_times(self):
        n = 16
        ms = np.zeros(n)
        la = (ctypes.c_int64 * n)()
        names = (ctypes.c_char_p * n)()
        nc = _I()
        self._check(self.L.qpic_kernel_times(self.h, n, _dp(ms), la, names, ctypes.byref(nc)),
                    "kernel_times")
        return {names[k].decode(): (ms[k], la[k]) for k in range(nc.value)}
