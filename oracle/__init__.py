"""FP64 CPU oracle for the quasi-3D dual-solver PIC step (arXiv:2303.12874, Sec. III).

TEST INFRASTRUCTURE ONLY.  Only tests/, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package.  It shares no code with
the CUDA library in ``paper_2303_12874_gb300``.

Layout:
  qpic_oracle.c  the step itself (Faraday, gather, Boris push, deposit, Ampere)
  coeffs.py      extended-stencil coefficients (Eqs. 11, 15), CFL, J_z filter
  setup.py       plasma loading (SplitMix64-keyed jitter) and the Gaussian laser
  diag.py        charge density, Gauss residual, energies, spectrum
  sim.py         a small driver tying the pieces together
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qpic_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lib = None


def build(force=False):
    """Compile the oracle's C core with plain gcc (strict IEEE FP64, no
    fast-math), with OpenMP when the compiler has it (the serial result is the
    same either way; see or_set_partitions)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-o", tmp, _SRC, "-lm"]
    try:
        subprocess.check_call(base[:1] + ["-fopenmp"] + base[1:], stderr=subprocess.DEVNULL)
    except subprocess.CalledProcessError:
        subprocess.check_call(base)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        _declare(_lib)
    return _lib


_D = ctypes.POINTER(ctypes.c_double)
_VP = ctypes.c_void_p


def _declare(L):
    L.or_create.restype = _VP
    L.or_create.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                            ctypes.c_double, ctypes.c_double, ctypes.c_int, _D, _D,
                            ctypes.c_int, _D, ctypes.c_int, ctypes.c_int]
    L.or_destroy.argtypes = [_VP]
    L.or_set_field.argtypes = [_VP, ctypes.c_int, ctypes.c_int, ctypes.c_int, _D, _D]
    L.or_get_field.argtypes = [_VP, ctypes.c_int, ctypes.c_int, ctypes.c_int, _D, _D]
    L.or_set_zmin.argtypes = [_VP, ctypes.c_double]
    L.or_load_particles.argtypes = [_VP, ctypes.c_long] + [_D] * 7
    L.or_append_particles.argtypes = [_VP, ctypes.c_long] + [_D] * 7
    L.or_num_particles.restype = ctypes.c_long
    L.or_num_particles.argtypes = [_VP]
    L.or_get_particles.argtypes = [_VP, _D]
    L.or_faraday.argtypes = [_VP]
    L.or_push_deposit.argtypes = [_VP]
    L.or_ampere.argtypes = [_VP]
    L.or_step.argtypes = [_VP, ctypes.c_int]
    L.or_gather.argtypes = [_VP, ctypes.c_long, _D, _D, _D, _D]
    L.or_deposit_rho.argtypes = [_VP, _D, _D]
    L.or_shift_window.argtypes = [_VP]
    L.or_compact.argtypes = [_VP]
    L.or_set_partitions.argtypes = [_VP, ctypes.c_int, ctypes.c_int]
    L.or_set_absorber.argtypes = [_VP, ctypes.c_int, ctypes.c_double]
    L.or_has_openmp.restype = ctypes.c_int


def _p(a):
    return a.ctypes.data_as(_D)


FIELDS = {"E": 0, "B": 1, "Bbar": 2, "J": 3}
COMPS = {"r": 0, "phi": 1, "z": 2}


class Oracle:
    """One oracle simulation box.  Fields are per mode, complex, [nr+1][nz].
    track_work: 0 off; 1 the modal work of Eq. 16 (W0 from m = 0, W1 from
    m >= 1); 2 the directional work of Eq. 17 (W0 = W_z, W1 = W_perp)."""

    def __init__(self, nz, nr, n_modes, dz, dr, dt, cE, cB, ktaps=None,
                 periodic=True, track_work=False, partitions=1, threads=0, absorb_cells=0,
                 absorb_sigma=0.0):
        cE = np.ascontiguousarray(cE, dtype=np.float64)
        cB = np.ascontiguousarray(cB, dtype=np.float64)
        kt = np.ascontiguousarray(ktaps if ktaps is not None else np.zeros(1), dtype=np.float64)
        nk = 0 if ktaps is None else len(ktaps)
        self.nz, self.nr, self.nm = nz, nr, n_modes
        self.dz, self.dr, self.dt = dz, dr, dt
        self.periodic = periodic
        self.zmin = 0.0
        self.L = lib()
        self.h = self.L.or_create(nz, nr, n_modes, dz, dr, dt, len(cE), _p(cE), _p(cB),
                                  nk, _p(kt), int(periodic), int(track_work))
        if not self.h:
            raise ValueError("oracle: bad configuration")
        if partitions > 1 or threads > 0:
            self.set_partitions(partitions, threads)
        if absorb_cells > 0:
            self.set_absorber(absorb_cells, absorb_sigma)

    def set_absorber(self, ncells, sigma_max=0.0):
        """Absorbing layer of `ncells` cells next to the wall (0: none): both
        fields multiplied after each update by exp(-sigma(r) dt), sigma rising
        as the square of the depth to sigma_max (<= 0: 3 ln(1e4) / (2 ncells
        dr)); see or_set_absorber."""
        self.L.or_set_absorber(self.h, int(ncells), float(sigma_max))

    def set_partitions(self, partitions, threads=0):
        """Deposit the particles in `partitions` fixed ranges (in parallel when
        the library has OpenMP; `threads` > 0 sets the thread count) and sum
        the range currents node by node in range order: the result depends on
        the number of ranges, not on the number of threads.  1 = serial."""
        self.L.or_set_partitions(self.h, int(partitions), int(threads))

    @staticmethod
    def has_openmp():
        return bool(lib().or_has_openmp())

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            self.L.or_destroy(h)
            self.h = None

    # fields
    def _check_field(self, which, comp, mode):
        if which not in FIELDS or comp not in COMPS or not 0 <= int(mode) < self.nm:
            raise ValueError("no field %r %r mode %r in a box of %d modes" % (which, comp, mode, self.nm))

    def set_field(self, which, comp, mode, val):
        self._check_field(which, comp, mode)
        val = np.asarray(val, dtype=np.complex128).reshape(self.nr + 1, self.nz)
        re = np.ascontiguousarray(val.real)
        im = np.ascontiguousarray(val.imag)
        self.L.or_set_field(self.h, FIELDS[which], COMPS[comp], mode, _p(re), _p(im))

    def get_field(self, which, comp, mode):
        self._check_field(which, comp, mode)
        re = np.zeros((self.nr + 1, self.nz))
        im = np.zeros((self.nr + 1, self.nz))
        self.L.or_get_field(self.h, FIELDS[which], COMPS[comp], mode, _p(re), _p(im))
        return re + 1j * im

    def fields(self, which):
        """array [3 comps][nm][nr+1][nz] complex"""
        return np.array([[self.get_field(which, c, m) for m in range(self.nm)]
                         for c in ("r", "phi", "z")])

    def set_fields(self, which, arr):
        for ci, c in enumerate(("r", "phi", "z")):
            for m in range(self.nm):
                self.set_field(which, c, m, arr[ci][m])

    def set_zmin(self, zmin):
        self.zmin = float(zmin)
        self.L.or_set_zmin(self.h, self.zmin)

    # particles
    def load_particles(self, z, r, phi, ux, uy, uz, w):
        arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (z, r, phi, ux, uy, uz, w)]
        self.L.or_load_particles(self.h, len(arrs[0]), *[_p(a) for a in arrs])

    def append_particles(self, z, r, phi, ux, uy, uz, w):
        arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (z, r, phi, ux, uy, uz, w)]
        self.L.or_append_particles(self.h, len(arrs[0]), *[_p(a) for a in arrs])

    def num_particles(self):
        return int(self.L.or_num_particles(self.h))

    def particles(self):
        """dict of arrays z, r, phi, ux, uy, uz, w, W0, W1"""
        n = self.num_particles()
        out = np.zeros(9 * max(n, 1))
        self.L.or_get_particles(self.h, _p(out))
        out = out[:9 * n].reshape(9, n)
        keys = ("z", "r", "phi", "ux", "uy", "uz", "w", "W0", "W1")
        return {k: out[i].copy() for i, k in enumerate(keys)}

    # step pieces
    def faraday(self):
        self.L.or_faraday(self.h)

    def push_deposit(self):
        self.L.or_push_deposit(self.h)

    def ampere(self):
        self.L.or_ampere(self.h)

    def step(self, n=1):
        self.L.or_step(self.h, int(n))

    def gather(self, z, r, phi):
        z, r, phi = [np.ascontiguousarray(a, dtype=np.float64) for a in (z, r, phi)]
        out = np.zeros((len(z), 6))
        self.L.or_gather(self.h, len(z), _p(z), _p(r), _p(phi), _p(out))
        return out

    def rho(self):
        """charge density per mode, [nm][nr+1][nz] complex"""
        shape = (self.nm, self.nr + 1, self.nz)
        re = np.zeros(shape)
        im = np.zeros(shape)
        self.L.or_deposit_rho(self.h, _p(re), _p(im))
        return re + 1j * im

    def shift_window(self):
        self.L.or_shift_window(self.h)
        self.zmin += self.dz

    def compact(self):
        self.L.or_compact(self.h)
