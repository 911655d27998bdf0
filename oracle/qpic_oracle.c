/*
 * qpic_oracle.c -- FP64 CPU reference of one quasi-3D (r-z grid + azimuthal
 * modes) electromagnetic PIC step with the extended-stencil ("dual") Maxwell
 * solver of arXiv:2303.12874, Sec. III.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain oracle that the CUDA
 * library is checked against.  Only tests/, the smoke check and the CPU
 * baseline of the benchmark may load it; the product path never does.  It
 * shares no code, header or table with the CUDA library.
 *
 * Units: c = 1, lengths in c/w0, time in 1/w0, fields in m c w0 / e,
 * momenta u = p/(m c), densities in n_c; electron charge q = -1, mass 1.
 *
 * Representation (Sec. III.B, azimuthal-mode expansion): every field is
 * F(r,phi,z) = F_0 + 2 Re sum_{m>=1} F_m e^{i m phi}; F_0 is real.
 *
 * Grid (Yee staggering in (z,r) per mode; r_j = j dr, j = 0..nr, wall at
 * r = nr dr, z index i at z_i = i dz relative to the window origin):
 *   E_r (i, j+1/2)   E_phi (i, j)       E_z (i+1/2, j)
 *   B_r (i+1/2, j)   B_phi (i+1/2, j+1/2) B_z (i, j+1/2)
 *   J co-located with E; rho at (i, j).
 * Half-integer locations are stored at the integer index below them.
 *
 * Step order (Eq. 12: force at time n from E^n and the time-averaged B):
 *   B^{n-1/2} -> B^{n+1/2}, Bbar^n = (B^{n-1/2}+B^{n+1/2})/2   (Faraday)
 *   gather E^n, Bbar^n; Boris push u^{n-1/2} -> u^{n+1/2}; move x^n -> x^{n+1}
 *   charge-conserving deposit of J^{n+1/2} per mode
 *   J_z <- K * J_z (dual solver only); E^n -> E^{n+1}        (Ampere)
 *
 * Threads: with or_set_partitions(s, P > 1) the particles are split into P
 * fixed contiguous ranges, each pushed and deposited into its own current
 * buffer, and the buffers are summed node by node in range order.  The result
 * then depends on P but not on how many OpenMP threads run the ranges (the
 * current is a sum over particles; the ranges only fix its order).  Field
 * updates are independent per node and match the serial ones bit for bit.
 *
 * Parity pins for each function are in tests/test_oracle_*.py.
 */
#define _USE_MATH_DEFINES
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

typedef double complex cplx;

enum { CR = 0, CP = 1, CZ = 2 };          /* component: r, phi, z */
enum { F_E = 0, F_B = 1, F_BBAR = 2, F_J = 3 };

#define MAXL 64
#define MAXK 512

typedef struct {
    int nz, nr, nm;            /* nm = number of modes (M+1) */
    double dz, dr, dt;
    int L;                     /* taps per z-derivative operator */
    double cE[MAXL], cB[MAXL]; /* Faraday ([k]_E) and Ampere ([k]_B) coefficients */
    int nk;                    /* J_z filter half-length (0: off) */
    double kt[MAXK];           /* symmetric filter taps k_0..k_{nk-1} */
    int periodic;              /* 1: z periodic; 0: open (zero outside) */
    int track_work;
    double zmin;               /* lab z of logical cell 0 */
    int nabs;                  /* absorbing layer: cells next to the wall (0: none) */
    double sigabs;             /* its peak conductivity sigma_max */
    cplx *E, *B, *Bb, *J;      /* [comp][mode][j=0..nr][i=0..nz-1] */
    int nparts;                /* particle ranges deposited separately (1: serial) */
    cplx *Jp;                  /* nparts current buffers when nparts > 1 */
    long np, cap;
    double *z, *x, *y, *ux, *uy, *uz, *w, *W0, *W1;
} ostate;

static size_t fidx(const ostate *s, int c, int m, int j, int i)
{
    return (((size_t)c * s->nm + m) * (size_t)(s->nr + 1) + j) * (size_t)s->nz + i;
}

/* ---------------------------------------------------------------- set-up */

ostate *or_create(int nz, int nr, int nm, double dz, double dr, double dt,
                  int L, const double *cE, const double *cB,
                  int nk, const double *kt, int periodic, int track_work)
{
    if (L < 1 || L > MAXL || nk < 0 || nk > MAXK || nm < 1) return NULL;
    ostate *s = (ostate *)calloc(1, sizeof(ostate));
    s->nz = nz; s->nr = nr; s->nm = nm; s->dz = dz; s->dr = dr; s->dt = dt;
    s->L = L; memcpy(s->cE, cE, L * sizeof(double)); memcpy(s->cB, cB, L * sizeof(double));
    s->nk = nk; if (nk) memcpy(s->kt, kt, nk * sizeof(double));
    s->periodic = periodic; s->track_work = track_work;
    size_t n = (size_t)3 * nm * (nr + 1) * nz;
    s->E = (cplx *)calloc(n, sizeof(cplx)); s->B = (cplx *)calloc(n, sizeof(cplx));
    s->Bb = (cplx *)calloc(n, sizeof(cplx)); s->J = (cplx *)calloc(n, sizeof(cplx));
    s->nparts = 1;
    return s;
}

/* Absorbing radial layer (an extension: the paper's runs end at a conducting
 * wall and it describes no absorbing boundary).  The ncells cells next to the
 * wall, r0 = R - ncells dr < r <= R, get the conductivity
 *     sigma(r) = sigma_max ((r - r0) / (ncells dr))^2
 * on both E and B (equal electric and magnetic conductivity: a layer matched
 * to the vacuum at normal incidence).  In time the loss term -sigma F of
 * dF/dt = rhs - sigma F is centred (the lossy leapfrog update):
 *     F^{new} = alpha F^{old} + beta dt rhs,
 *     alpha = (1 - sigma dt/2) / (1 + sigma dt/2),  beta = 1 / (1 + sigma dt/2),
 * with sigma at the component's own radius (alpha = beta = 1 outside).
 * sigma_max <= 0 takes 3 ln(1e4) / (2 ncells dr), the value at which a wave
 * crossing the layer twice in the continuum is attenuated by 1e4. */
void or_set_absorber(ostate *s, int ncells, double sigma_max)
{
    if (ncells < 0) ncells = 0;
    if (ncells > s->nr) ncells = s->nr;
    s->nabs = ncells;
    s->sigabs = ncells == 0 ? 0.0
              : (sigma_max > 0.0 ? sigma_max : 3.0 * log(1e4) / (2.0 * ncells * s->dr));
}

/* sigma(r) dt / 2 at radius r (0 outside the layer) */
static double half_loss(const ostate *s, double r)
{
    if (s->nabs == 0) return 0.0;
    const double width = s->nabs * s->dr, r0 = s->nr * s->dr - width;
    if (r <= r0) return 0.0;
    const double x = (r - r0) / width;
    return 0.5 * s->sigabs * x * x * s->dt;
}
/* the lossy update F <- alpha F + beta dt rhs at radius r */
static cplx lossy(const ostate *s, double r, cplx f, cplx dt_rhs)
{
    const double h = half_loss(s, r);
    return ((1.0 - h) * f + dt_rhs) / (1.0 + h);
}

/* number of particle ranges deposited separately (1: serial, the default) and,
 * when OpenMP is available, the number of threads (<= 0: leave it) */
void or_set_partitions(ostate *s, int nparts, int nthreads)
{
    if (nparts < 1) nparts = 1;
    if (nparts != s->nparts) { free(s->Jp); s->Jp = NULL; s->nparts = nparts; }
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}

/* 1 when the library was built with OpenMP */
int or_has_openmp(void)
{
#ifdef _OPENMP
    return 1;
#else
    return 0;
#endif
}

void or_destroy(ostate *s)
{
    if (!s) return;
    free(s->E); free(s->B); free(s->Bb); free(s->J); free(s->Jp);
    free(s->z); free(s->x); free(s->y); free(s->ux); free(s->uy); free(s->uz);
    free(s->w); free(s->W0); free(s->W1);
    free(s);
}

static cplx *field_ptr(ostate *s, int which)
{
    switch (which) { case F_E: return s->E; case F_B: return s->B;
                     case F_BBAR: return s->Bb; default: return s->J; }
}

/* copy one (comp, mode) plane, [nr+1][nz], in or out */
void or_set_field(ostate *s, int which, int c, int m, const double *re, const double *im)
{
    if (c < 0 || c > 2 || m < 0 || m >= s->nm) return;     /* no such plane */
    cplx *f = field_ptr(s, which);
    for (int j = 0; j <= s->nr; j++)
        for (int i = 0; i < s->nz; i++) {
            size_t k = (size_t)j * s->nz + i;
            f[fidx(s, c, m, j, i)] = re[k] + I * (im ? im[k] : 0.0);
        }
}

void or_get_field(ostate *s, int which, int c, int m, double *re, double *im)
{
    if (c < 0 || c > 2 || m < 0 || m >= s->nm) return;     /* no such plane */
    cplx *f = field_ptr(s, which);
    for (int j = 0; j <= s->nr; j++)
        for (int i = 0; i < s->nz; i++) {
            size_t k = (size_t)j * s->nz + i;
            re[k] = creal(f[fidx(s, c, m, j, i)]);
            im[k] = cimag(f[fidx(s, c, m, j, i)]);
        }
}

void or_set_zmin(ostate *s, double zmin) { s->zmin = zmin; }

/* particles given as (z, r, phi) with momenta u = gamma v (Cartesian) and weight w */
void or_load_particles(ostate *s, long n, const double *z, const double *r, const double *phi,
                       const double *ux, const double *uy, const double *uz, const double *w)
{
    double **arr[9] = { &s->z, &s->x, &s->y, &s->ux, &s->uy, &s->uz, &s->w, &s->W0, &s->W1 };
    for (int a = 0; a < 9; a++) { free(*arr[a]); *arr[a] = (double *)calloc(n > 0 ? n : 1, sizeof(double)); }
    s->np = n; s->cap = n;
    for (long p = 0; p < n; p++) {
        s->z[p] = z[p]; s->x[p] = r[p] * cos(phi[p]); s->y[p] = r[p] * sin(phi[p]);
        s->ux[p] = ux[p]; s->uy[p] = uy[p]; s->uz[p] = uz[p]; s->w[p] = w[p];
    }
}

long or_num_particles(ostate *s) { return s->np; }

/* out: 9 arrays of np: z, r, phi, ux, uy, uz, w, W0, W1 */
void or_get_particles(ostate *s, double *out)
{
    long n = s->np;
    for (long p = 0; p < n; p++) {
        out[0 * n + p] = s->z[p];
        out[1 * n + p] = hypot(s->x[p], s->y[p]);
        out[2 * n + p] = atan2(s->y[p], s->x[p]);
        out[3 * n + p] = s->ux[p]; out[4 * n + p] = s->uy[p]; out[5 * n + p] = s->uz[p];
        out[6 * n + p] = s->w[p]; out[7 * n + p] = s->W0[p]; out[8 * n + p] = s->W1[p];
    }
}

/* ------------------------------------------------------- finite differences */

/* z index with boundary handling; returns -1 when outside an open box */
static int zwrap(const ostate *s, int i)
{
    if (s->periodic) { i %= s->nz; if (i < 0) i += s->nz; return i; }
    return (i >= 0 && i < s->nz) ? i : -1;
}

static cplx fz(const ostate *s, const cplx *f, int c, int m, int j, int i)
{
    int k = zwrap(s, i);
    return k < 0 ? 0.0 : f[fidx(s, c, m, j, k)];
}

/* Faraday operator D^E_z: from integer-located samples to the half point i+1/2,
 * D f_{i+1/2} = sum_l cE_l (f_{i+l} - f_{i+1-l}) / dz  (Eq. 9, [k]_E) */
static cplx dzE(const ostate *s, const cplx *f, int c, int m, int j, int i)
{
    cplx acc = 0.0;
    for (int l = 1; l <= s->L; l++)
        acc += s->cE[l - 1] * (fz(s, f, c, m, j, i + l) - fz(s, f, c, m, j, i + 1 - l));
    return acc / s->dz;
}

/* Ampere operator D^B_z: from half-located samples (stored at index k for
 * k+1/2) to the integer point i: D f_i = sum_l cB_l (f_{i+l-1/2} - f_{i-l+1/2}) / dz */
static cplx dzB(const ostate *s, const cplx *f, int c, int m, int j, int i)
{
    cplx acc = 0.0;
    for (int l = 1; l <= s->L; l++)
        acc += s->cB[l - 1] * (fz(s, f, c, m, j, i + l - 1) - fz(s, f, c, m, j, i - l));
    return acc / s->dz;
}

/* ----------------------------------------------------------------- Faraday */

/* dB/dt = -curl E per mode:
 *   dB_r/dt   = -(i m / r) E_z + D^E_z E_phi
 *   dB_phi/dt = -D^E_z E_r + d_r E_z
 *   dB_z/dt   = -(1/r) d_r (r E_phi) + (i m / r) E_r
 * Axis (r = 0): m = 0: B_r = 0; m = 1: lim E_z/r = E_z(dr)/dr; m >= 2: 0. */
void or_faraday(ostate *s)
{
    const int nz = s->nz, nr = s->nr;
    const double dt = s->dt, dr = s->dr;
    size_t n = (size_t)3 * s->nm * (nr + 1) * nz;
    cplx *Bn = (cplx *)malloc(n * sizeof(cplx));
    memcpy(Bn, s->B, n * sizeof(cplx));
    #pragma omp parallel for collapse(2) schedule(static)
    for (int m = 0; m < s->nm; m++) {
        for (int j = 0; j <= nr; j++) {
            double rj = j * dr, rh = (j + 0.5) * dr;
            for (int i = 0; i < nz; i++) {
                /* B_r at (i+1/2, j) */
                cplx d;
                if (j == 0) {
                    if (m == 1) d = -I * s->E[fidx(s, CZ, 1, 1, i)] / dr + dzE(s, s->E, CP, 1, 0, i);
                    else d = 0.0;
                } else {
                    d = -I * (double)m / rj * s->E[fidx(s, CZ, m, j, i)] + dzE(s, s->E, CP, m, j, i);
                }
                Bn[fidx(s, CR, m, j, i)] = lossy(s, rj, Bn[fidx(s, CR, m, j, i)], dt * d);
                if (j < nr) {
                    /* B_phi at (i+1/2, j+1/2) */
                    d = -dzE(s, s->E, CR, m, j, i)
                        + (s->E[fidx(s, CZ, m, j + 1, i)] - s->E[fidx(s, CZ, m, j, i)]) / dr;
                    Bn[fidx(s, CP, m, j, i)] = lossy(s, rh, Bn[fidx(s, CP, m, j, i)], dt * d);
                    /* B_z at (i, j+1/2) */
                    d = -((j + 1) * dr * s->E[fidx(s, CP, m, j + 1, i)] - rj * s->E[fidx(s, CP, m, j, i)]) / (rh * dr)
                        + I * (double)m / rh * s->E[fidx(s, CR, m, j, i)];
                    Bn[fidx(s, CZ, m, j, i)] = lossy(s, rh, Bn[fidx(s, CZ, m, j, i)], dt * d);
                }
            }
        }
    }
    for (size_t k = 0; k < n; k++) s->Bb[k] = 0.5 * (s->B[k] + Bn[k]);
    memcpy(s->B, Bn, n * sizeof(cplx));
    free(Bn);
}

/* ------------------------------------------------------------------ Ampere */

/* J_z <- K * J_z along z: the symmetric filter whose symbol is [k]_Yee/[k]_B,
 * so that D^B_z (K*J_z) = D^Yee_z J_z and Gauss's law i[k]_B.E = rho (Eq. 10)
 * is kept by a current that satisfies the two-point continuity equation. */
static void filter_jz(ostate *s)
{
    if (s->nk <= 0) return;
    const int nz = s->nz;
    #pragma omp parallel for collapse(2) schedule(static)
    for (int m = 0; m < s->nm; m++)
        for (int j = 0; j <= s->nr; j++) {
            cplx *tmp = (cplx *)malloc((size_t)nz * sizeof(cplx));
            for (int i = 0; i < nz; i++) {
                cplx acc = s->kt[0] * s->J[fidx(s, CZ, m, j, i)];
                for (int q = 1; q < s->nk; q++)
                    acc += s->kt[q] * (fz(s, s->J, CZ, m, j, i + q) + fz(s, s->J, CZ, m, j, i - q));
                tmp[i] = acc;
            }
            for (int i = 0; i < nz; i++) s->J[fidx(s, CZ, m, j, i)] = tmp[i];
            free(tmp);
        }
}

/* dE/dt = curl B - J per mode:
 *   dE_r/dt   = (i m / r) B_z - D^B_z B_phi - J_r
 *   dE_phi/dt = D^B_z B_r - d_r B_z - J_phi
 *   dE_z/dt   = (1/r) d_r (r B_phi) - (i m / r) B_r - J_z
 * Axis: m = 0: E_phi = 0, E_z advanced with the disk flux 4 B_phi(dr/2)/dr;
 *       m = 1: E_z = 0, d_r B_z(0) = 2 B_z(dr/2)/dr (odd extension); m >= 2: 0.
 * Wall (r = nr dr, conductor): E_phi = E_z = 0. */
void or_ampere(ostate *s)
{
    const int nz = s->nz, nr = s->nr;
    const double dt = s->dt, dr = s->dr;
    filter_jz(s);
    #pragma omp parallel for collapse(2) schedule(static)
    for (int m = 0; m < s->nm; m++) {
        for (int j = 0; j <= nr; j++) {
            double rj = j * dr, rh = (j + 0.5) * dr, rl = (j - 0.5) * dr;
            for (int i = 0; i < nz; i++) {
                if (j < nr) {
                    /* E_r at (i, j+1/2) */
                    cplx d = I * (double)m / rh * s->B[fidx(s, CZ, m, j, i)]
                             - dzB(s, s->B, CP, m, j, i) - s->J[fidx(s, CR, m, j, i)];
                    s->E[fidx(s, CR, m, j, i)] = lossy(s, rh, s->E[fidx(s, CR, m, j, i)], dt * d);
                }
                /* E_phi at (i, j) */
                if (j == nr || (j == 0 && m != 1)) {
                    s->E[fidx(s, CP, m, j, i)] = 0.0;
                } else if (j == 0) {
                    cplx d = dzB(s, s->B, CR, 1, 0, i) - 2.0 * s->B[fidx(s, CZ, 1, 0, i)] / dr
                             - s->J[fidx(s, CP, 1, 0, i)];
                    s->E[fidx(s, CP, 1, 0, i)] = lossy(s, rj, s->E[fidx(s, CP, 1, 0, i)], dt * d);
                } else {
                    cplx d = dzB(s, s->B, CR, m, j, i)
                             - (s->B[fidx(s, CZ, m, j, i)] - s->B[fidx(s, CZ, m, j - 1, i)]) / dr
                             - s->J[fidx(s, CP, m, j, i)];
                    s->E[fidx(s, CP, m, j, i)] = lossy(s, rj, s->E[fidx(s, CP, m, j, i)], dt * d);
                }
                /* E_z at (i+1/2, j) */
                if (j == nr || (j == 0 && m != 0)) {
                    s->E[fidx(s, CZ, m, j, i)] = 0.0;
                } else if (j == 0) {
                    cplx d = 4.0 * s->B[fidx(s, CP, 0, 0, i)] / dr - s->J[fidx(s, CZ, 0, 0, i)];
                    s->E[fidx(s, CZ, 0, 0, i)] = lossy(s, rj, s->E[fidx(s, CZ, 0, 0, i)], dt * d);
                } else {
                    cplx d = ((j + 0.5) * dr * s->B[fidx(s, CP, m, j, i)] - rl * s->B[fidx(s, CP, m, j - 1, i)]) / (rj * dr)
                             - I * (double)m / rj * s->B[fidx(s, CR, m, j, i)] - s->J[fidx(s, CZ, m, j, i)];
                    s->E[fidx(s, CZ, m, j, i)] = lossy(s, rj, s->E[fidx(s, CZ, m, j, i)], dt * d);
                }
            }
        }
    }
}

/* ------------------------------------------------------------------ gather */

static double hat(double t) { double a = fabs(t); return a < 1.0 ? 1.0 - a : 0.0; }

/* sample of a half-r-located component at half index k (r = (k+1/2) dr),
 * continued below the axis by the mode parity (radial/azimuthal components of
 * mode m have parity (-1)^{m+1}, longitudinal ones (-1)^m) and above the wall
 * by the even image of a normal E / tangential B component */
static cplx half_r_sample(const ostate *s, const cplx *f, int c, int m, int k, int i)
{
    if (k < 0) {
        double par = (c == CZ) ? ((m % 2) ? -1.0 : 1.0) : ((m % 2) ? 1.0 : -1.0);
        return par * fz(s, f, c, m, 0, i);
    }
    if (k >= s->nr) k = s->nr - 1;
    return fz(s, f, c, m, k, i);
}

/* bilinear interpolation of mode m of component c at cell coordinates
 * (zc, rc), with the component's stagger (hz, hr in {0, 1/2}) */
static cplx interp(const ostate *s, const cplx *f, int c, int m, double zc, double rc, int hz, int hr)
{
    double tz = zc - 0.5 * hz, tr = rc - 0.5 * hr;
    int i0 = (int)floor(tz), j0 = (int)floor(tr);
    double az = tz - i0, ar = tr - j0;
    cplx v = 0.0;
    for (int a = 0; a < 2; a++)
        for (int b = 0; b < 2; b++) {
            double wgt = (a ? az : 1.0 - az) * (b ? ar : 1.0 - ar);
            if (wgt == 0.0) continue;
            int i = i0 + a, j = j0 + b;
            cplx val;
            if (hr) val = half_r_sample(s, f, c, m, j, i);
            else val = (j >= 0 && j <= s->nr) ? fz(s, f, c, m, j, i) : 0.0;
            v += wgt * val;
        }
    return v;
}

/* E (or Bbar) in Cartesian at a point: modal sum F_0 + 2 Re(F_m e^{i m phi}),
 * then rotation (r, phi) -> (x, y).  out[0..2] = total, out[3..5] = m = 0 part */
static void gather_one(const ostate *s, const cplx *f, int is_b, double zc, double rc,
                       double cph, double sph, double out[6])
{
    /* staggers (hz, hr): E_r (0,1) E_phi (0,0) E_z (1,0); B_r (1,0) B_phi (1,1) B_z (0,1) */
    static const int hzE[3] = { 0, 0, 1 }, hrE[3] = { 1, 0, 0 };
    static const int hzB[3] = { 1, 1, 0 }, hrB[3] = { 0, 1, 1 };
    double comp[3], comp0[3];
    for (int c = 0; c < 3; c++) {
        int hz = is_b ? hzB[c] : hzE[c], hr = is_b ? hrB[c] : hrE[c];
        double tot = creal(interp(s, f, c, 0, zc, rc, hz, hr));
        comp0[c] = tot;
        cplx em = 1.0;                        /* e^{i m phi} */
        cplx e1 = cph + I * sph;
        for (int m = 1; m < s->nm; m++) {
            em *= e1;
            tot += 2.0 * creal(interp(s, f, c, m, zc, rc, hz, hr) * em);
        }
        comp[c] = tot;
    }
    out[0] = comp[CR] * cph - comp[CP] * sph;
    out[1] = comp[CR] * sph + comp[CP] * cph;
    out[2] = comp[CZ];
    out[3] = comp0[CR] * cph - comp0[CP] * sph;
    out[4] = comp0[CR] * sph + comp0[CP] * cph;
    out[5] = comp0[CZ];
}

/* gather E^n and Bbar^n at n given points (z lab, r, phi); out: [n][6] = Ex Ey Ez Bx By Bz */
void or_gather(ostate *s, long n, const double *z, const double *r, const double *phi, double *out)
{
    for (long p = 0; p < n; p++) {
        double e[6], b[6];
        double zc = (z[p] - s->zmin) / s->dz, rc = r[p] / s->dr;
        gather_one(s, s->E, 0, zc, rc, cos(phi[p]), sin(phi[p]), e);
        gather_one(s, s->Bb, 1, zc, rc, cos(phi[p]), sin(phi[p]), b);
        for (int k = 0; k < 3; k++) { out[6 * p + k] = e[k]; out[6 * p + 3 + k] = b[k]; }
    }
}

/* ------------------------------------------------------------------ deposit */

static double cvol(const ostate *s, int j)
{
    const double dr = s->dr, dz = s->dz;
    if (j == 0) return M_PI * 0.25 * dr * dr * dz;
    if (j == s->nr) { double R = s->nr * dr; return M_PI * (R * R - (R - 0.5 * dr) * (R - 0.5 * dr)) * dz; }
    return 2.0 * M_PI * j * dr * dr * dz;
}

static void addJ(const ostate *s, cplx *J, int c, int m, int j, int i, cplx v)
{
    int k = zwrap(s, i);
    if (k < 0 || j < 0 || j > s->nr) return;
    J[fidx(s, c, m, j, k)] += v;
}

/* Charge-conserving deposit of one particle move (z0,r0,phi0) -> (z1,r1,phi1),
 * charge Q, per mode (Sec. III.A "conserves charge"; Sec. III.B modes).
 * The modal charge change Q (S1 e1 - S0 e0), e = e^{-i m phi}, is split as
 *   (S1 - S0) (e0+e1)/2   -> r and z fluxes by the 2D Esirkepov decomposition
 *   (S0 + S1)/2 (e1 - e0)  -> J_phi through (i m / r_j) J_phi V_j = -dQ/dt.
 * For m = 0, J_phi = Q v_phi Sbar / V with v_phi at the mid-point of the move. */
static void deposit_one(const ostate *s, cplx *J, double Q, double zc0, double rc0, double zc1,
                        double rc1, double c0, double s0, double c1, double s1, double vphi)
{
    const double dt = s->dt, dz = s->dz, dr = s->dr;
    int ilo = (int)floor(fmin(zc0, zc1)), jlo = (int)floor(fmin(rc0, rc1));
    int ihi = (int)floor(fmax(zc0, zc1)) + 1, jhi = (int)floor(fmax(rc0, rc1)) + 1;
    int nzs = ihi - ilo + 1, nrs = jhi - jlo + 1;     /* at most 3 x 3 */
    double S0z[4], S1z[4], S0r[4], S1r[4];
    for (int a = 0; a < nzs; a++) { S0z[a] = hat(zc0 - (ilo + a)); S1z[a] = hat(zc1 - (ilo + a)); }
    for (int b = 0; b < nrs; b++) { S0r[b] = hat(rc0 - (jlo + b)); S1r[b] = hat(rc1 - (jlo + b)); }
    double Wz[4][4], Wr[4][4], Sb[4][4];
    for (int a = 0; a < nzs; a++)
        for (int b = 0; b < nrs; b++) {
            double dSz = S1z[a] - S0z[a], dSr = S1r[b] - S0r[b];
            Wz[a][b] = dSz * (S0r[b] + 0.5 * dSr);
            Wr[a][b] = dSr * (S0z[a] + 0.5 * dSz);
            Sb[a][b] = 0.5 * (S0z[a] * S0r[b] + S1z[a] * S1r[b]);
        }
    cplx e0 = c0 - I * s0, e1 = c1 - I * s1;   /* e^{-i phi} */
    cplx em0 = 1.0, em1 = 1.0;
    for (int m = 0; m < s->nm; m++) {
        if (m > 0) { em0 *= e0; em1 *= e1; }
        cplx ebar = 0.5 * (em0 + em1), de = em1 - em0;
        /* z fluxes through faces (i+1/2, j): prefix sums of W^z along z */
        for (int b = 0; b < nrs; b++) {
            int j = jlo + b;
            if (j < 0 || j > s->nr) continue;
            double acc = 0.0;
            for (int a = 0; a < nzs - 1; a++) {
                acc += Wz[a][b];
                cplx flux = -(Q / dt) * acc * ebar;               /* charge per time */
                addJ(s, J, CZ, m, j, ilo + a, flux * dz / cvol(s, j));
            }
        }
        /* r fluxes through faces (i, j+1/2): prefix sums of W^r along r */
        for (int a = 0; a < nzs; a++) {
            double acc = 0.0;
            for (int b = 0; b < nrs - 1; b++) {
                int j = jlo + b;
                acc += Wr[a][b];
                if (j < 0 || j >= s->nr) continue;
                cplx flux = -(Q / dt) * acc * ebar;
                addJ(s, J, CR, m, j, ilo + a, flux / (2.0 * M_PI * (j + 0.5) * dr * dz));
            }
        }
        /* azimuthal current at nodes (i, j) */
        for (int a = 0; a < nzs; a++)
            for (int b = 0; b < nrs; b++) {
                int j = jlo + b;
                if (j < 0 || j > s->nr || Sb[a][b] == 0.0) continue;
                cplx v;
                if (m == 0) v = Q * vphi * Sb[a][b] / cvol(s, j);
                else v = I * (j * dr) * Q * Sb[a][b] * de / ((double)m * cvol(s, j) * dt);
                addJ(s, J, CP, m, j, ilo + a, v);
            }
    }
}

/* charge density per mode, rho_m(i,j) = sum_p Q S_i(z) S_j(r) e^{-i m phi} / V_j;
 * out: [nm][nr+1][nz] re and im */
void or_deposit_rho(ostate *s, double *re, double *im)
{
    size_t plane = (size_t)(s->nr + 1) * s->nz;
    memset(re, 0, s->nm * plane * sizeof(double));
    memset(im, 0, s->nm * plane * sizeof(double));
    for (long p = 0; p < s->np; p++) {
        double Q = -s->w[p];
        double zc = (s->z[p] - s->zmin) / s->dz;
        double r = hypot(s->x[p], s->y[p]), rc = r / s->dr;
        double cph = r > 0 ? s->x[p] / r : 1.0, sph = r > 0 ? s->y[p] / r : 0.0;
        int i0 = (int)floor(zc), j0 = (int)floor(rc);
        cplx e = cph - I * sph, em = 1.0;
        for (int m = 0; m < s->nm; m++) {
            if (m > 0) em *= e;
            for (int a = 0; a < 2; a++)
                for (int b = 0; b < 2; b++) {
                    int i = zwrap(s, i0 + a), j = j0 + b;
                    double wgt = hat(zc - (i0 + a)) * hat(rc - j);
                    if (i < 0 || j > s->nr || wgt == 0.0) continue;
                    cplx v = Q * wgt * em / cvol(s, j);
                    size_t k = (size_t)m * plane + (size_t)j * s->nz + i;
                    re[k] += creal(v); im[k] += cimag(v);
                }
        }
    }
}

/* --------------------------------------------------------------- particles */

/* gather + Boris push + move + deposit for every particle (J is zeroed first).
 * Boris (relativistic): half electric kick, magnetic rotation with
 * t = q dt Bbar / (2 gamma), half electric kick (Eq. 6 time-centred per Eq. 12).
 * Move in Cartesian x, y, then (r, phi) from the new position.  A particle
 * beyond the conducting wall is reflected specularly.  In an open box a
 * particle leaving [0, nz dz) is removed (weight set to 0 after its deposit). */
static void push_one(ostate *s, long p, cplx *J)
{
    const double dt = s->dt, q = -1.0;
    const double R = s->nr * s->dr;
    if (s->w[p] == 0.0) return;
    double z0 = s->z[p], x0 = s->x[p], y0 = s->y[p];
    double r0 = hypot(x0, y0);
    double c0 = r0 > 0 ? x0 / r0 : 1.0, s0 = r0 > 0 ? y0 / r0 : 0.0;
    double zc0 = (z0 - s->zmin) / s->dz, rc0 = r0 / s->dr;
    double e[6], b[6];
    gather_one(s, s->E, 0, zc0, rc0, c0, s0, e);
    gather_one(s, s->Bb, 1, zc0, rc0, c0, s0, b);
    double u[3] = { s->ux[p], s->uy[p], s->uz[p] };
    double g_old = sqrt(1.0 + u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    double um[3], up[3], t[3], sv[3], uprime[3];
    for (int k = 0; k < 3; k++) um[k] = u[k] + 0.5 * q * dt * e[k];
    double gm = sqrt(1.0 + um[0] * um[0] + um[1] * um[1] + um[2] * um[2]);
    for (int k = 0; k < 3; k++) t[k] = 0.5 * q * dt * b[k] / gm;
    double t2 = t[0] * t[0] + t[1] * t[1] + t[2] * t[2];
    for (int k = 0; k < 3; k++) sv[k] = 2.0 * t[k] / (1.0 + t2);
    uprime[0] = um[0] + um[1] * t[2] - um[2] * t[1];
    uprime[1] = um[1] + um[2] * t[0] - um[0] * t[2];
    uprime[2] = um[2] + um[0] * t[1] - um[1] * t[0];
    up[0] = um[0] + uprime[1] * sv[2] - uprime[2] * sv[1];
    up[1] = um[1] + uprime[2] * sv[0] - uprime[0] * sv[2];
    up[2] = um[2] + uprime[0] * sv[1] - uprime[1] * sv[0];
    for (int k = 0; k < 3; k++) up[k] += 0.5 * q * dt * e[k];
    double g = sqrt(1.0 + up[0] * up[0] + up[1] * up[1] + up[2] * up[2]);
    double vx = up[0] / g, vy = up[1] / g, vz = up[2] / g;
    if (s->track_work) {
        /* v at time n: the mean of u/gamma at n -+ 1/2 */
        double vn[3] = { 0.5 * (u[0] / g_old + vx), 0.5 * (u[1] / g_old + vy), 0.5 * (u[2] / g_old + vz) };
        if (s->track_work == 2) {
            /* Eq. 17: W_z += q dt E_z v_z, W_perp += q dt E_perp . v_perp (all modes) */
            s->W0[p] += q * dt * (e[2] * vn[2]);
            s->W1[p] += q * dt * (e[0] * vn[0] + e[1] * vn[1]);
        } else {
            /* Eq. 16: W_m += q dt E^m . v; W0 holds m = 0, W1 the modes m >= 1 */
            double w0 = e[3] * vn[0] + e[4] * vn[1] + e[5] * vn[2];
            double wt = e[0] * vn[0] + e[1] * vn[1] + e[2] * vn[2];
            s->W0[p] += q * dt * w0;
            s->W1[p] += q * dt * (wt - w0);
        }
    }
    double x1 = x0 + dt * vx, y1 = y0 + dt * vy, z1 = z0 + dt * vz;
    double r1 = hypot(x1, y1);
    if (r1 > R) {                       /* specular reflection at the wall */
        double cr = x1 / r1, sr = y1 / r1;
        double urad = up[0] * cr + up[1] * sr;
        up[0] -= 2.0 * urad * cr; up[1] -= 2.0 * urad * sr;
        double rn = 2.0 * R - r1;
        x1 = cr * rn; y1 = sr * rn; r1 = rn;
    }
    double c1 = r1 > 0 ? x1 / r1 : c0, s1 = r1 > 0 ? y1 / r1 : s0;
    /* mid-point azimuthal velocity for the m = 0 J_phi */
    double xm = 0.5 * (x0 + x1), ym = 0.5 * (y0 + y1), rm = hypot(xm, ym);
    double vphi = rm > 0 ? (xm * (y1 - y0) - ym * (x1 - x0)) / (rm * dt) : 0.0;
    double zc1 = (z1 - s->zmin) / s->dz, rc1 = r1 / s->dr;
    deposit_one(s, J, q * s->w[p], zc0, rc0, zc1, rc1, c0, s0, c1, s1, vphi);
    s->z[p] = z1; s->x[p] = x1; s->y[p] = y1;
    s->ux[p] = up[0]; s->uy[p] = up[1]; s->uz[p] = up[2];
    if (s->periodic) {
        double Lz = s->nz * s->dz;
        double zrel = s->z[p] - s->zmin;
        if (zrel < 0) s->z[p] += Lz; else if (zrel >= Lz) s->z[p] -= Lz;
    } else if (zc1 < 0.0 || zc1 >= s->nz) {
        s->w[p] = 0.0;                  /* left the open box */
    }
}

void or_push_deposit(ostate *s)
{
    const size_t n = (size_t)3 * s->nm * (s->nr + 1) * s->nz;
    memset(s->J, 0, n * sizeof(cplx));
    if (s->nparts <= 1) {
        for (long p = 0; p < s->np; p++) push_one(s, p, s->J);
        return;
    }
    const int P = s->nparts;
    if (!s->Jp) s->Jp = (cplx *)malloc((size_t)P * n * sizeof(cplx));
    /* range k: particles [k np / P, (k+1) np / P) into buffer k */
    #pragma omp parallel for schedule(dynamic, 1)
    for (int k = 0; k < P; k++) {
        cplx *Jk = s->Jp + (size_t)k * n;
        memset(Jk, 0, n * sizeof(cplx));
        const long p0 = (long)((long long)s->np * k / P), p1 = (long)((long long)s->np * (k + 1) / P);
        for (long p = p0; p < p1; p++) push_one(s, p, Jk);
    }
    /* node by node, in range order */
    #pragma omp parallel for schedule(static)
    for (long long q = 0; q < (long long)n; q++) {
        cplx acc = s->Jp[q];
        for (int k = 1; k < P; k++) acc += s->Jp[(size_t)k * n + q];
        s->J[q] = acc;
    }
}

/* one full step (Faraday, particles, Ampere) repeated nsteps times */
void or_step(ostate *s, int nsteps)
{
    for (int k = 0; k < nsteps; k++) {
        or_faraday(s);
        or_push_deposit(s);
        or_ampere(s);
    }
}

/* moving window: shift the box by one cell towards +z.  The field columns move
 * back by one index and the new front column is zeroed; particles now behind
 * the box are removed (weight 0).  New plasma is added by the caller. */
void or_shift_window(ostate *s)
{
    const int nz = s->nz;
    cplx *f[4] = { s->E, s->B, s->Bb, s->J };
    for (int a = 0; a < 4; a++)
        for (int c = 0; c < 3; c++)
            for (int m = 0; m < s->nm; m++)
                for (int j = 0; j <= s->nr; j++) {
                    cplx *row = f[a] + fidx(s, c, m, j, 0);
                    memmove(row, row + 1, (size_t)(nz - 1) * sizeof(cplx));
                    row[nz - 1] = 0.0;
                }
    s->zmin += s->dz;
    for (long p = 0; p < s->np; p++)
        if (s->z[p] < s->zmin) s->w[p] = 0.0;
}

/* append particles (e.g. plasma injected into the new front column) */
void or_append_particles(ostate *s, long n, const double *z, const double *r, const double *phi,
                         const double *ux, const double *uy, const double *uz, const double *w)
{
    long np = s->np + n;
    double **arr[9] = { &s->z, &s->x, &s->y, &s->ux, &s->uy, &s->uz, &s->w, &s->W0, &s->W1 };
    for (int a = 0; a < 9; a++) {
        *arr[a] = (double *)realloc(*arr[a], (np > 0 ? np : 1) * sizeof(double));
    }
    for (long k = 0; k < n; k++) {
        long p = s->np + k;
        s->z[p] = z[k]; s->x[p] = r[k] * cos(phi[k]); s->y[p] = r[k] * sin(phi[k]);
        s->ux[p] = ux[k]; s->uy[p] = uy[k]; s->uz[p] = uz[k]; s->w[p] = w[k];
        s->W0[p] = 0.0; s->W1[p] = 0.0;
    }
    s->np = np; s->cap = np;
}

/* drop particles of zero weight, keeping the order of the rest */
void or_compact(ostate *s)
{
    long k = 0;
    for (long p = 0; p < s->np; p++) {
        if (s->w[p] == 0.0) continue;
        s->z[k] = s->z[p]; s->x[k] = s->x[p]; s->y[k] = s->y[p];
        s->ux[k] = s->ux[p]; s->uy[k] = s->uy[p]; s->uz[k] = s->uz[p];
        s->w[k] = s->w[p]; s->W0[k] = s->W0[p]; s->W1[k] = s->W1[p];
        k++;
    }
    s->np = k;
}
