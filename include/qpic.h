/*
 * qpic.h -- C ABI of libqpic, a GB300 (sm_103a) quasi-3D electromagnetic
 * particle-in-cell step with the extended-stencil ("dual") Maxwell solver of
 * arXiv:2303.12874 (Miller et al.), Sec. III.
 *
 * Method (paper sections):
 *   Sec. III.A, Eqs. 9-15  dual solver: z-derivatives with L coefficients fitted
 *                          so that [k]_B[k]_E = (sin(k dt/2)/(dt/2))^2 (Eq. 11)
 *                          and sqrt([k]_E/[k]_B) cos(k dt/2) = 1 (Eq. 15).
 *   Sec. III.B              azimuthal-mode ("quasi-3D") fields F_m e^{i m phi}.
 *   Eq. 6, Eq. 12           relativistic push with E^n and the time-averaged B.
 *   Sec. II (end)           charge-conserving current deposition.
 *   Eq. 16                  modal work W_LWFA (m = 0) and W_DLA (m = 1).
 *
 * Units: c = 1, lengths in c/w0, time in 1/w0, fields in m c w0/e, momenta
 * u = gamma v, densities in n_c (w_p^2 = n); electrons, q = -1, m = 1.
 *
 * Conventions for every call:
 *   - returns a qpic_status; no exception or abort crosses the ABI;
 *     qpic_last_error(ctx) gives a text for the last failure;
 *   - host buffers are owned by the caller and only read/written during the
 *     call; device memory is owned by the context;
 *   - a context is used by one host thread at a time;
 *   - all work is queued on the context's CUDA stream; calls that return
 *     data to the host synchronise that stream.
 *   - field planes are [nr+1][nz] (r index j = 0..nr slowest, z fastest) in
 *     the window's logical order, per component and mode.  Mode 0 is real
 *     (im part ignored / written as 0).  Grid staggering (z index i at
 *     z = zmin + i dz, r_j = j dr, half-integer points stored at the integer
 *     index below them):  E_r (i, j+1/2)  E_phi (i, j)  E_z (i+1/2, j)
 *                         B_r (i+1/2, j)  B_phi (i+1/2, j+1/2)  B_z (i, j+1/2)
 *     J co-located with E.  Rows that lie outside the wall (half-r row nr)
 *     or on the conductor (E_phi, E_z at j = nr) are 0.
 */
#ifndef QPIC_H
#define QPIC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct qpic_ctx qpic_ctx;

typedef enum {
    QPIC_OK = 0,
    QPIC_EINVAL = -1,      /* bad argument or configuration */
    QPIC_ENOMEM = -2,      /* device or host allocation failed */
    QPIC_ECUDA = -3,       /* a CUDA runtime call failed */
    QPIC_ECFL = -4,        /* dt above the stability limit, or no coefficient fit */
    QPIC_EOVERFLOW = -5,   /* fixed-point current accumulator out of range */
    QPIC_ETIMEOUT = -6,    /* a bounded device-side wait gave up */
    QPIC_ENONFINITE = -7,  /* NaN/Inf found by the diagnostics */
    QPIC_ESTATE = -8,      /* call not valid in the current state */
    QPIC_ECAPACITY = -9,   /* particle buffer capacity exceeded */
    QPIC_ECHECK = -10      /* a kernel's invariant check failed (checked build, QPIC_CHECK, only) */
} qpic_status;

enum { QPIC_YEE = 0, QPIC_DUAL = 1 };
enum { QPIC_FP64 = 0, QPIC_FP32_FIXED = 1, QPIC_FP32_FATOMIC = 2 };
enum { QPIC_FIELD_E = 0, QPIC_FIELD_B = 1, QPIC_FIELD_BBAR = 2, QPIC_FIELD_J = 3, QPIC_FIELD_RHO = 4 };
enum { QPIC_COMP_R = 0, QPIC_COMP_PHI = 1, QPIC_COMP_Z = 2 };
enum { QPIC_STAGE_FARADAY = 1, QPIC_STAGE_PARTICLES = 2, QPIC_STAGE_AMPERE = 4,
       QPIC_STAGE_WINDOW = 8, QPIC_STAGE_SORT = 16 };

typedef struct {
    int32_t nz, nr;        /* logical grid: nz cells along z, nr cells in r (wall at nr dr);
                              nz plus the open box's gap below 32768, nr below 65535
                              (QPIC_EINVAL otherwise) */
    int32_t n_modes;       /* M + 1 azimuthal modes (1..4) */
    double dz, dr;
    double dt;             /* <= 0: dt = cfl_frac x the solver's stability limit */
    double cfl_frac;
    int32_t solver;        /* QPIC_YEE or QPIC_DUAL */
    int32_t n_coef;        /* L coefficients per z-operator for QPIC_DUAL (Appendix A: 16) */
    double fit_band;       /* fit range k dz in (0, fit_band*pi] (a reading; default 0.8) */
    int32_t precision;     /* QPIC_FP32_FIXED (default): FP32 push and solve, int64 fixed-point
                              current sums (bit-reproducible; each contribution rounded to
                              units of the largest particle charge / (2^38 (1 - 2^-10)));
                              QPIC_FP32_FATOMIC: the same with the current summed by FP32
                              float atomics in global memory (order-dependent rounding);
                              QPIC_FP64: plain FP64 path, one thread per particle */
    int32_t jz_filter;     /* 1: J_z correction so that Gauss's law holds in the dual form */
    double filter_tol;     /* filter taps kept down to |k_n| >= filter_tol |k_0| */
    int32_t periodic_z;    /* 1: periodic box; 0: open box (zero fields outside) */
    int32_t moving_window; /* 1: window moves at window_v (needs periodic_z = 0) */
    double window_v;
    int32_t tile_z, tile_r;   /* particle tile in cells: 16x8 (default), 32x8, 8x8, 16x16, 32x4 */
    int32_t sort_period;      /* steps between particle sorts (0: default 2; a particle moves
                                 < 1 cell per step, so 2 keeps every one inside its tile halo) */
    int32_t particles_per_thread; /* consecutive particles one thread of the particle kernel
                                 takes in a chunk of 256 x this particles, 1..16 (0: 16).  A
                                 tile's particles are sorted by cell, so about ppc / this many
                                 threads share a cell (the "threads per cell" knob); smaller
                                 values mean more threads per cell and more chunk drains */
    int32_t absorb_cells;     /* absorbing radial layer (an extension; the paper's runs end at a
                                 conducting wall): the cells next to the wall, 0..nr (0: none).
                                 On r0 = R - absorb_cells dr < r <= R, E and B get the
                                 conductivity sigma(r) = absorb_sigma ((r - r0)/(R - r0))^2 with
                                 the centred lossy update F = alpha F + beta dt rhs,
                                 alpha = (1 - sigma dt/2)/(1 + sigma dt/2), beta = 1/(1 + sigma dt/2) */
    double absorb_sigma;      /* peak conductivity (0: 3 ln(1e4) / (2 absorb_cells dr), a round-trip
                                 attenuation of 1e4 in the continuum) */
    int32_t track_work;       /* per-particle work in W0, W1: 0 off; 1 modal (Eq. 16:
                                 W0 from m = 0, W1 from m >= 1); 2 directional (Eq. 17:
                                 W0 = W_z, W1 = W_perp, all modes) */
    uint64_t seed;            /* plasma azimuthal jitter seed */
    int64_t max_particles;    /* capacity (0: sized at the first load, +25%) */
    void *cuda_stream;        /* cudaStream_t to run on, NULL: the legacy default stream */
    /* optional device allocator (e.g. a PyTorch caching allocator); NULL: cudaMalloc */
    void *(*dev_alloc)(size_t bytes, void *user);
    void (*dev_free)(void *ptr, void *user);
    void *alloc_user;
} qpic_config;

/* Fill *cfg with defaults (M = 1, dual solver, L = 16, band 0.8, cfl 0.9,
 * FP32 + int64 fixed point, filter on, tol 1e-16, periodic, 16 x 8 tiles, sort
 * every 2 steps, 8 particles per thread). */
qpic_status qpic_default_config(qpic_config *cfg);

/* Create a context: fit the z-operator coefficients on the host in FP64
 * (Eqs. 11 and 15, Sec. III.A; least squares on the fit band with the exact
 * long-wavelength limit), find dt by bisection of the leapfrog stability
 * bound when cfg->dt <= 0, build the J_z filter taps, allocate zeroed device
 * fields.  *out receives the context; on failure it may still receive one so
 * that qpic_last_error can explain -- destroy it with qpic_destroy.
 * The device current at this call owns every buffer of the context: every
 * later call on the context that touches the device must be made with that
 * device current, else it returns QPIC_ESTATE and launches nothing. */
qpic_status qpic_init(const qpic_config *cfg, qpic_ctx **out);

/* Free everything the context owns.  NULL is allowed. */
void qpic_destroy(qpic_ctx *ctx);

/* Text of the last failure on ctx (static string when ctx is NULL). */
const char *qpic_last_error(const qpic_ctx *ctx);

/* Solver constants chosen at init: dt, L and the coefficients C^E_l, C^B_l
 * (l = 1..L; Eq. 9 operators D f_{i+1/2} = sum_l C_l (f_{i+l} - f_{i+1-l})/dz),
 * and the J_z filter taps k_0..k_{nk-1}.  Arrays may be NULL; caps in entries. */
qpic_status qpic_get_solver(const qpic_ctx *ctx, double *dt, int32_t *L,
                            double *cE, double *cB, int32_t cap_coef,
                            double *taps, int32_t cap_taps, int32_t *n_taps);

/* Host-only numerics, usable without a GPU (same code qpic_init uses).
 * qpic_fit_coefficients: C^E, C^B for `solver` at time step dt (Eqs. 11, 15;
 *   Yee gives L = 1, C = 1); returns L in *L_out; arrays hold >= n_coef entries.
 * qpic_filter_taps: J_z correction taps k_0..k_{n-1} for C^B (symbol
 *   [k]_Yee/[k]_B), truncated below tol |k_0|; *n_out = 0 for Yee.
 * qpic_stability_limit: largest dt with (dt^2/4) lambda_max(curl curl) <= 1
 *   for an nr-cell radial grid and n_modes modes (bisection; the dual
 *   coefficients are refitted at every trial dt). */
qpic_status qpic_fit_coefficients(int32_t solver, double dt, double dz, int32_t n_coef,
                                  double fit_band, double *cE, double *cB, int32_t *L_out);
qpic_status qpic_filter_taps(const double *cB, int32_t L, double tol, double *taps,
                             int32_t cap, int32_t *n_out);
qpic_status qpic_stability_limit(int32_t solver, double dz, double dr, int32_t nr,
                                 int32_t n_modes, int32_t n_coef, double fit_band,
                                 double *dt_max);

/* Host-only, usable without a GPU: the LWFA / DLA split estimated from the
 * directional work of Eq. 17 (a run with track_work = 2), Sec. III.B Eqs. 19-20.
 * For each of n particles (momenta u = p/(m c), work W_z, W_perp in m c^2):
 *   f = -2 sqrt(2 gamma) / (omega0 omega_p w0^2)   (Eq. 19, c = 1, gamma from u),
 *   lwfa[k] = W_z - f W_perp,  dla[k] = (1 + f) W_perp   (Eq. 20).
 * omega_p and omega0 in the units of 1/t (omega0 = 1 in the normalized units),
 * w0 the laser spot size in units of length: the paper takes average values
 * near the electron bunch.  All arrays are caller-owned host arrays of n
 * doubles; lwfa and dla may not alias the inputs.  QPIC_EINVAL for n < 0, a
 * missing array or a non-positive omega_p, omega0 or w0. */
qpic_status qpic_work_f_estimate(int64_t n, const double *ux, const double *uy, const double *uz,
                                 const double *Wz, const double *Wperp, double omega_p, double w0,
                                 double omega0, double *lwfa, double *dla);

/* Reduced model of Sec. II (Eqs. 1-8), independent of any context: n electrons
 * in a spherical bubble wake (Eq. 6) and a channel-guided laser (Eqs. 3-4),
 * moving in the x-z plane, advanced by nsteps fixed steps of dt from time t0
 * with the fifth-order Dormand-Prince Runge-Kutta method, in FP64 on the GPU
 * (one thread per electron).  State per electron: x, zeta = z - t, u_x, u_z
 * (u = gamma v), in/out.  Units c = 1, laser frequency omega0 = 1; omega_p
 * the plasma frequency (the bubble's w_beta^2 = omega_p^2/(2 gamma), Eq. 1),
 * k_perp the laser's transverse wavenumber (Eq. 3; the paper's choice is
 * 2.4/(r_b + c/omega_p)), v_phi its phase velocity (k_z = omega0/v_phi), a0 its
 * normalized amplitude.  bfac multiplies the laser's magnetic terms (those
 * proportional to v sin(k_z xi)): cos(omega0 dt/2) models the time-staggering
 * error of a PIC solver with time step dt (Sec. IV.A; about 0.994 for the
 * paper's Yee runs), 1 gives Eq. 8 as printed.  start_step: NULL, or n int32
 * step indices (host for qpic_reduced_integrate, device for the _device
 * variant): electron i stays at its initial state until step start_step[i]
 * of the grid t0 + k dt and is integrated from there (Appendix A injects the
 * electrons over a time interval); a start at or beyond nsteps leaves it.
 *   qpic_reduced_integrate: caller-owned host arrays of n doubles; the call
 *     copies them to the device and back and returns when done.
 *   qpic_reduced_integrate_device: device arrays, launched on `stream`
 *     (a cudaStream_t, NULL for the default stream); asynchronous.
 * QPIC_EINVAL for n < 0, nsteps < 0, a missing array, dt <= 0, v_phi <= 0,
 * k_perp < 0 or a non-finite parameter; QPIC_ENOMEM / QPIC_ECUDA when device
 * memory or a CUDA call fails.  The paper has no such interface: it integrates
 * Eq. 8 for single electrons. */
qpic_status qpic_reduced_integrate(int64_t n, double *x, double *zeta, double *ux, double *uz,
                                   double a0, double omega_p, double k_perp, double v_phi,
                                   double bfac, double t0, double dt, int32_t nsteps,
                                   const int32_t *start_step);
qpic_status qpic_reduced_integrate_device(int64_t n, double *x, double *zeta, double *ux,
                                          double *uz, double a0, double omega_p, double k_perp,
                                          double v_phi, double bfac, double t0, double dt,
                                          int32_t nsteps, const int32_t *start_step,
                                          void *stream);

/* Stability limit of the configured solver on this grid (leapfrog bound
 * (dt^2/4) lambda_max(curl curl) <= 1, coefficients refitted per trial dt). */
qpic_status qpic_cfl_limit(const qpic_ctx *ctx, double *dt_max);

/* Load the cold plasma lattice into every cell of the current window,
 * replacing all particles: ppc_z x ppc_r x ppc_phi per cell at
 * z = (i + (a+1/2)/ppc_z) dz, r = (j + (b+1/2)/ppc_r) dr,
 * phi = 2 pi (c + jitter)/ppc_phi with one jitter in [0,1) per cell from a
 * SplitMix64 keyed on (seed, absolute z cell, r cell) (0 when phi_jitter = 0);
 * weight w = n(z) 2 pi r (dr/ppc_r)(dz/ppc_z)/ppc_phi, n(z) = n0 times a linear
 * ramp from z_start over ramp_len (lab frame).  The same parameters feed the
 * moving-window injection.  Cells where n = 0 get no particles. */
qpic_status qpic_load_plasma(qpic_ctx *ctx, double n0, double z_start, double ramp_len,
                             int32_t ppc_z, int32_t ppc_r, int32_t ppc_phi, int32_t phi_jitter);

/* Replace all particles with n given ones (host FP64 arrays): lab-frame z,
 * r in [0, nr dr], phi, momenta u = gamma v (Cartesian), weights w >= 0
 * (number of electrons).  Modal work counters start at 0. */
qpic_status qpic_load_particles(qpic_ctx *ctx, int64_t n, const double *z, const double *r,
                                const double *phi, const double *ux, const double *uy,
                                const double *uz, const double *w);

/* Add a linearly polarised Gaussian pulse to the m = 1 fields (Eq. 18 near
 * focus, as a paraxial Gaussian beam): field amplitude a0, waist w0, intensity
 * FWHM duration fwhm, centroid z_centroid and focus z_focus (lab frame),
 * polarisation angle pol_angle from x.  E at t = 0; B at t = -dt/2 with the
 * discrete B/E ratio sqrt([k]_E/[k]_B) at k = 1.  Needs n_modes >= 2. */
qpic_status qpic_add_laser(qpic_ctx *ctx, double a0, double w0, double fwhm,
                           double z_centroid, double z_focus, double pol_angle);

/* Advance nsteps full PIC steps (Faraday -> gather/push/deposit -> J_z filter
 * -> Ampere, then the moving window and the particle sort).  Asynchronous on
 * the context's stream except for a final check of the device error word. */
qpic_status qpic_step(qpic_ctx *ctx, int32_t nsteps);

/* Run only the given stages once (QPIC_STAGE_* bit mask, in step order);
 * for stage-by-stage parity checks and timing. */
qpic_status qpic_run_stages(qpic_ctx *ctx, int32_t stages);

/* Copy one field plane to/from caller-owned host FP64 arrays of
 * (nr+1)*nz entries each (layout above).  which: QPIC_FIELD_*; J is the
 * current of the last step after the J_z correction; RHO (get only) deposits
 * the electron charge density per mode from the current particles. */
qpic_status qpic_get_field(qpic_ctx *ctx, int32_t which, int32_t comp, int32_t mode,
                           double *re, double *im);
qpic_status qpic_set_field(qpic_ctx *ctx, int32_t which, int32_t comp, int32_t mode,
                           const double *re, const double *im);

/* The same with the caller's buffer length: count is the number of doubles
 * each of re and im holds; QPIC_EINVAL (nothing copied) if count is below
 * (nr+1)*nz.  im may be NULL (mode 0, or the imaginary part not wanted/0). */
qpic_status qpic_get_fields(qpic_ctx *ctx, int32_t which, int32_t comp, int32_t mode, double *re,
                            double *im, int64_t count);
qpic_status qpic_set_fields(qpic_ctx *ctx, int32_t which, int32_t comp, int32_t mode,
                            const double *re, const double *im, int64_t count);

/* Charge density per mode like qpic_get_field(ctx, QPIC_FIELD_RHO, ...), but
 * without allocating any device memory.  The paper has no counterpart: this
 * entry point serves callers that cannot allocate -- hosts that hand the
 * library a fixed device-memory budget up front, code running inside a device
 * allocator's own callbacks (which must not re-enter it), and loops that
 * cannot afford the device-wide synchronisation of cudaFree.  The deposit uses a file-scope static device
 * array of 2^21 doubles (16 MiB) that every GPU loading the library holds until
 * exit; grids needing more than n_modes*2*(nr+1)*nz <= 2^21 doubles are
 * rejected with QPIC_EINVAL and a message.  The first call on a device looks
 * up the array's device address (cudaGetSymbolAddress) with that device
 * current, so make that first call before any stream capture.  All calls share
 * the array (each clears what it uses first); calls that overlap on the GPU,
 * from any context or thread, race.  re/im: caller-owned host arrays of
 * (nr+1)*nz doubles in the field-plane layout; im may be NULL.  Synchronises
 * the context's stream.  The context's device (current at qpic_init) must be
 * current; otherwise QPIC_ESTATE and nothing is launched. */
qpic_status qpic_charge_density_noalloc(qpic_ctx *ctx, int32_t mode, double *re, double *im);

/* Checkpoint and resume (the paper has no counterpart; a long run is saved
 * and resumed without changing its result).  A snapshot holds the E, B and
 * Bbar planes, the live particles (sorted, or compacted on the FP64 path),
 * the modal-work counters when tracked, the ion background of the Gauss
 * diagnostic, the step and window counters and the plasma-injection
 * parameters, as raw words after a header.  qpic_state_size gives its size in
 * bytes; qpic_save_state writes it into a caller-owned host buffer of
 * `capacity` bytes (*written = the size; QPIC_ECAPACITY, nothing written, if
 * the buffer is too small); qpic_load_state reads it into a context created
 * with the same configuration (QPIC_EINVAL otherwise) and replaces its state.
 * On the FP32 fixed-point path the current is an integer sum, so the steps
 * after a load are bit-identical to the steps the saved context would have
 * taken.  Saving sorts the particles (FP32) or compacts them (FP64); all three
 * synchronise the context's stream. */
qpic_status qpic_state_size(qpic_ctx *ctx, int64_t *bytes);
qpic_status qpic_save_state(qpic_ctx *ctx, void *buf, int64_t capacity, int64_t *written);
qpic_status qpic_load_state(qpic_ctx *ctx, const void *buf, int64_t size);

/* Number of live particles. */
qpic_status qpic_num_particles(qpic_ctx *ctx, int64_t *n);

/* Copy live particles to a caller-owned host buffer of 9*capacity FP64 in
 * structure-of-arrays order z, r, phi, ux, uy, uz, w, W0, W1 (each block has
 * *n_out entries, packed at stride capacity).  Order is unspecified. */
qpic_status qpic_get_particles(qpic_ctx *ctx, double *out, int64_t capacity, int64_t *n_out);

/* Like qpic_get_particles but in device buffer order without sorting or
 * compaction: slot k of every block is buffer slot k, dead slots have w = 0.
 * Two raw exports with only QPIC_STAGE_FARADAY/PARTICLES/AMPERE stages in
 * between list the same particles in the same order. */
qpic_status qpic_get_particles_raw(qpic_ctx *ctx, double *out, int64_t capacity, int64_t *n_out);

/* FP64 diagnostics into out[0..count): [0] time, [1] steps, [2] window shifts,
 * [3] live particles, [4] total charge, [5] kinetic energy sum w (gamma-1),
 * [6..6+M] field energy per mode (1/2 sum V (|E|^2 + |B|^2), modes m >= 1 counted
 * twice by the Sec. III.B convention F_0 + 2 Re F_m e^{i m phi}), then the
 * fixed-point overflow flag.  Sums are FP64-grade (per-thread double-float
 * partial sums, FP64 block and grid sums in a fixed order).  Synchronises the
 * context's stream once; the first call allocates 512 bytes of pinned host
 * memory for the read-back (freed by qpic_destroy; pageable words are used if
 * pinning fails).  QPIC_ENONFINITE (out still filled) when the charge, the
 * kinetic energy or a field energy is NaN or infinite: a NaN or infinity in
 * any particle or field value reaches these sums. */
qpic_status qpic_get_diag(qpic_ctx *ctx, double *out, int32_t count);

/* Gauss's law residual per mode in the dual form of Eq. 10: out[2m] = L2 norm
 * over nodes of div_B E_m - (rho_e + rho_ion)_m, out[2m+1] = L2 norm of the net
 * charge density (rho_e + rho_ion)_m, where rho_ion = -rho_e at the last particle
 * load (a fixed neutralising background) and div_B uses the finite-volume
 * radial divergence with D^B_z in z.  Conductor nodes and the m >= 1 axis node
 * are left out.  QPIC_ESTATE with a moving window (the background would move). */
qpic_status qpic_gauss_residual(qpic_ctx *ctx, double *out, int32_t count);

/* Energy spectrum of the electrons (the spectra of Sec. IV): weights[k] = sum of w over particles with
 * kinetic energy (gamma - 1) 0.511 MeV in [edges_mev[k], edges_mev[k+1]),
 * k < nbins (edges strictly increasing, nbins <= 4096).  Weights are summed in
 * int64 fixed point, so the result does not depend on particle order. */
qpic_status qpic_spectrum(qpic_ctx *ctx, const double *edges_mev, int32_t nbins, double *weights);

/* Number of CUDA kernels this context has launched so far (bookkeeping; the
 * paper has no counterpart). */
qpic_status qpic_launch_count(const qpic_ctx *ctx, int64_t *n);

/* Per-kernel device time (ms, CUDA events on the context's stream) and launch
 * counts accumulated since the last reset, for n kernel classes; names gives
 * "name" strings (static).  Timing is on only when enabled.  (Measurement
 * support; the paper has no counterpart.) */
qpic_status qpic_profile(qpic_ctx *ctx, int32_t enable, int32_t reset);
qpic_status qpic_kernel_times(qpic_ctx *ctx, int32_t n, double *ms, int64_t *launches,
                              const char **names, int32_t *n_classes);

/* Batches (a systems feature; the paper has no counterpart): many independent
 * runs (for example a parameter scan) advanced by one CUDA graph launch per
 * cycle of steps.  qpic_batch_create captures the cycle once.  Every step of
 * it has three phases: (1) Faraday (Eq. 9) and the step's epoch on each run's
 * own stream, forked from and joined to cuda_stream; (2) one persistent
 * launch per group of up to 64 runs that share the mode count and the tile
 * shape: its blocks (two per SM) take items from a work list -- first the
 * gather, Boris push and charge-conserving deposit (Sec. II.B, Eqs. 10-11) of
 * every (run, tile), then the current reduction of every (run, tile), each of
 * which waits, for at most a bounded number of polls, until the deposits of
 * the 3 x 3 tiles around it have been published; (3) the J filter (Sec. III),
 * Ampere (Eq. 8) and, when due, the sort on the runs' own streams.  A sort
 * swaps the particle buffers, so the cycle is twice the least common multiple
 * of the runs' sort periods (at most 16 steps) and every replay starts from the
 * buffers the graph was recorded with.  cuda_stream NULL: the batch uses a
 * stream of its own (the legacy default stream cannot be captured).  Runs
 * must use the FP32 fixed-point path, a periodic box (no moving window),
 * profiling off, the device current at their creation, and a sort period of
 * at most min(TZ, TR) - 3 (a particle then never deposits outside the 3 x 3
 * tiles around the tile it was sorted into); QPIC_EINVAL otherwise.  Each run
 * is first brought to a cycle boundary with its particles sorted (stepped on
 * its own until then).  A batch is deterministic (the int64 deposit); it
 * agrees with the same runs stepped one by one to FP32 rounding, the batched
 * particle kernel being a separate compilation whose fused multiply-adds may
 * differ.  The contexts stay owned by the caller and must outlive the batch;
 * do not step them individually while it exists.
 * qpic_batch_step: nsteps must be a multiple of qpic_batch_cycle(); it first
 * waits for the runs' own streams, then synchronises cuda_stream and checks
 * every run's error word: QPIC_ETIMEOUT when a wait of the particle phase gave
 * up (that tile's current is left out of the step), QPIC_EOVERFLOW for a
 * fixed-point overflow; qpic_batch_last_error names the run.
 * qpic_batch_set_wait: the number of polls (each about 0.1 us or more) after
 * which a wait gives up (default 2^24, above one second), and an item of the
 * work list (-1: none; 0 .. tiles-1 are the particle items of the first group
 * in run order) whose completion is never published -- a way to exercise the
 * timeout path without a fault; polls >= 0, else QPIC_EINVAL. */
typedef struct qpic_batch qpic_batch;
qpic_status qpic_batch_create(qpic_ctx *const *runs, int32_t n, void *cuda_stream, qpic_batch **out);
qpic_status qpic_batch_step(qpic_batch *batch, int32_t nsteps);
int32_t qpic_batch_cycle(const qpic_batch *batch);
const char *qpic_batch_last_error(const qpic_batch *batch);
qpic_status qpic_batch_set_wait(qpic_batch *batch, int64_t polls, int32_t withheld_item);
void qpic_batch_destroy(qpic_batch *batch);

#ifdef __cplusplus
}
#endif
#endif /* QPIC_H */
