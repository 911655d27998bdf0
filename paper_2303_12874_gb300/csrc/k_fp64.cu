// k_fp64.cu -- the plain FP64 GPU path: the same quasi-3D PIC step done the
// straightforward way, as the baseline the FP32 + int64 fixed-point path is
// measured against.  Double-precision lab-frame z and Cartesian x, y per
// particle, one thread per particle, fields gathered straight from global
// memory, charge-conserving deposit with FP64 global atomics (no tiles, no
// sort, no shared memory).  Field kernels are the templated ones of
// k_fields.cu instantiated for double.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "qpic_internal.h"

namespace qpic {

struct DArgs {
    int nz, nr, nzp, nparts, nm, periodic, track_work;
    int zoff;
    size_t plane;
    double dz, dr, dt, R, zmin;
};

static DArgs dargs(const qpic_ctx *c)
{
    DArgs a;
    a.nz = c->g.nz; a.nr = c->g.nr; a.nzp = c->g.nzp; a.nparts = c->g.nparts; a.nm = c->g.nm;
    a.periodic = c->g.periodic; a.track_work = c->cfg.track_work;
    a.zoff = (int)(c->g.zoff % c->g.nzp); a.plane = c->g.plane;
    a.dz = c->dz; a.dr = c->dr; a.dt = c->dt; a.R = c->g.nr * c->dr; a.zmin = c->shifts * c->dz;
    return a;
}

__device__ __forceinline__ int dwrap(int i, int n)
{
    int r = i % n;
    return r < 0 ? r + n : r;
}

// physical column of logical column il, or -1 outside an open box
__device__ __forceinline__ int dcol(int il, const DArgs &a)
{
    if (a.periodic) return dwrap(il, a.nz);
    if (il < 0 || il >= a.nz) return -1;
    return dwrap(il + a.zoff, a.nzp);
}

// field sample with the boundary images of the half-r components (mode parity
// below the axis, even image beyond the wall); fb: 0 = E, 1 = Bbar
__device__ double dsample(const double *E, const double *Bb, const DArgs &a, int fb, int c, int p,
                          int j, int il)
{
    const double *F = fb == 0 ? E : Bb;
    const int hr = fb == 0 ? (c == 0) : (c != 0);
    double sgn = 1.0;
    if (hr) {
        if (j < 0) {
            int m = (p + 1) >> 1;
            bool longitudinal = (fb == 1 && c == 2);
            bool odd = ((m & 1) != 0) != !longitudinal;
            sgn = odd ? -1.0 : 1.0;
            j = -1 - j;
        }
        if (j >= a.nr) j = 2 * a.nr - 1 - j;
        if (j < 0 || j >= a.nr) return 0.0;
    } else if (j < 0 || j > a.nr) {
        return 0.0;
    }
    int col = dcol(il, a);
    if (col < 0) return 0.0;
    return sgn * F[(size_t)(c * a.nparts + p) * a.plane + (size_t)j * a.nzp + col];
}

__device__ __forceinline__ double dhat(double t)
{
    double x = fabs(t);
    return x < 1.0 ? 1.0 - x : 0.0;
}

__device__ double dcvol(const DArgs &a, int j)
{
    const double PI = 3.14159265358979323846;
    if (j == 0) return PI * 0.25 * a.dr * a.dr * a.dz;
    if (j == a.nr) return PI * (a.R * a.R - (a.R - 0.5 * a.dr) * (a.R - 0.5 * a.dr)) * a.dz;
    return 2.0 * PI * j * a.dr * a.dr * a.dz;
}

__device__ __forceinline__ void jadd64(double *J, const DArgs &a, int c, int p, int j, int il,
                                       double v)
{
    if (v == 0.0 || j < 0 || j > a.nr) return;
    int col = dcol(il, a);
    if (col < 0) return;
    atomicAdd(&J[(size_t)(c * a.nparts + p) * a.plane + (size_t)j * a.nzp + col], v);
}

__global__ void k_push64(Particles64 P, long long np, const double *E, const double *Bb, double *J,
                         DArgs a)
{
    const double PI = 3.14159265358979323846;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < np;
         i += (long long)gridDim.x * blockDim.x) {
        const double w = P.w[i];
        if (w == 0.0) continue;
        const double z0 = P.z[i], x0 = P.x[i], y0 = P.y[i];
        const double r0 = sqrt(x0 * x0 + y0 * y0);
        const double c0 = r0 > 0 ? x0 / r0 : 1.0, s0 = r0 > 0 ? y0 / r0 : 0.0;
        double zc = (z0 - a.zmin) / a.dz;
        if (!a.periodic && (zc < 0.0 || zc >= a.nz)) { P.w[i] = 0.0; continue; }
        const double rc = r0 / a.dr;
        // ---- gather E and Bbar (bilinear at each component's stagger, modal sum)
        double Fc[2][3], F0[3];
        for (int fb = 0; fb < 2; fb++)
            for (int c = 0; c < 3; c++) {
                const int hz = fb == 0 ? (c == 2) : (c != 2);
                const int hr = fb == 0 ? (c == 0) : (c != 0);
                const double tz = zc - 0.5 * hz, tr = rc - 0.5 * hr;
                const int i0 = (int)floor(tz), j0 = (int)floor(tr);
                const double az = tz - i0, ar = tr - j0;
                double tot = 0.0;
                double ecr = 1.0, eci = 0.0;
                for (int m = 0; m < a.nm; m++) {
                    if (m) { double t = ecr * c0 - eci * s0; eci = ecr * s0 + eci * c0; ecr = t; }
                    double vr = 0.0, vi = 0.0;
                    for (int q = 0; q < (m ? 2 : 1); q++) {
                        const int p = m ? 2 * m - 1 + q : 0;
                        double v = (1 - az) * (1 - ar) * dsample(E, Bb, a, fb, c, p, j0, i0) +
                                   az * (1 - ar) * dsample(E, Bb, a, fb, c, p, j0, i0 + 1) +
                                   (1 - az) * ar * dsample(E, Bb, a, fb, c, p, j0 + 1, i0) +
                                   az * ar * dsample(E, Bb, a, fb, c, p, j0 + 1, i0 + 1);
                        if (q == 0) vr = v; else vi = v;
                    }
                    if (m == 0) { tot = vr; if (fb == 0) F0[c] = vr; }
                    else tot += 2.0 * (vr * ecr - vi * eci);
                }
                Fc[fb][c] = tot;
            }
        const double e[3] = {Fc[0][0] * c0 - Fc[0][1] * s0, Fc[0][0] * s0 + Fc[0][1] * c0, Fc[0][2]};
        const double b[3] = {Fc[1][0] * c0 - Fc[1][1] * s0, Fc[1][0] * s0 + Fc[1][1] * c0, Fc[1][2]};
        // ---- Boris push, q = -1
        const double h = -0.5 * a.dt;
        const double u0x = P.ux[i], u0y = P.uy[i], u0z = P.uz[i];
        const double gold = sqrt(1.0 + u0x * u0x + u0y * u0y + u0z * u0z);
        double um[3] = {u0x + h * e[0], u0y + h * e[1], u0z + h * e[2]};
        const double gm = sqrt(1.0 + um[0] * um[0] + um[1] * um[1] + um[2] * um[2]);
        double t[3] = {h * b[0] / gm, h * b[1] / gm, h * b[2] / gm};
        const double t2 = t[0] * t[0] + t[1] * t[1] + t[2] * t[2];
        double sv[3] = {2 * t[0] / (1 + t2), 2 * t[1] / (1 + t2), 2 * t[2] / (1 + t2)};
        double upr[3] = {um[0] + um[1] * t[2] - um[2] * t[1], um[1] + um[2] * t[0] - um[0] * t[2],
                         um[2] + um[0] * t[1] - um[1] * t[0]};
        double un[3] = {um[0] + upr[1] * sv[2] - upr[2] * sv[1] + h * e[0],
                        um[1] + upr[2] * sv[0] - upr[0] * sv[2] + h * e[1],
                        um[2] + upr[0] * sv[1] - upr[1] * sv[0] + h * e[2]};
        const double g = sqrt(1.0 + un[0] * un[0] + un[1] * un[1] + un[2] * un[2]);
        const double vx = un[0] / g, vy = un[1] / g, vz = un[2] / g;
        if (a.track_work == 2) {
            // Eq. 17: W_z and W_perp, v at time n the mean of u/gamma at n -+ 1/2
            const double wx = 0.5 * (u0x / gold + vx), wy = 0.5 * (u0y / gold + vy),
                         wz = 0.5 * (u0z / gold + vz);
            P.W0[i] -= a.dt * (e[2] * wz);
            P.W1[i] -= a.dt * (e[0] * wx + e[1] * wy);
        } else if (a.track_work) {
            // Eq. 16: W0 from the m = 0 field, W1 from the modes m >= 1
            const double wx = 0.5 * (u0x / gold + vx), wy = 0.5 * (u0y / gold + vy),
                         wz = 0.5 * (u0z / gold + vz);
            const double e0x = F0[0] * c0 - F0[1] * s0, e0y = F0[0] * s0 + F0[1] * c0;
            const double p0 = e0x * wx + e0y * wy + F0[2] * wz;
            const double pt = e[0] * wx + e[1] * wy + e[2] * wz;
            P.W0[i] -= a.dt * p0;
            P.W1[i] -= a.dt * (pt - p0);
        }
        // ---- move, wall reflection
        double x1 = x0 + a.dt * vx, y1 = y0 + a.dt * vy, z1 = z0 + a.dt * vz;
        double r1 = sqrt(x1 * x1 + y1 * y1);
        if (r1 > a.R) {
            const double cr = x1 / r1, sr = y1 / r1;
            const double urad = un[0] * cr + un[1] * sr;
            un[0] -= 2.0 * urad * cr; un[1] -= 2.0 * urad * sr;
            const double rn = 2.0 * a.R - r1;
            x1 = cr * rn; y1 = sr * rn; r1 = rn;
        }
        const double c1 = r1 > 0 ? x1 / r1 : c0, s1 = r1 > 0 ? y1 / r1 : s0;
        const double xm = 0.5 * (x0 + x1), ym = 0.5 * (y0 + y1), rm = sqrt(xm * xm + ym * ym);
        const double vphi = rm > 0 ? (xm * (y1 - y0) - ym * (x1 - x0)) / (rm * a.dt) : 0.0;
        // ---- charge-conserving deposit per mode (2D Esirkepov x (e0+e1)/2, J_phi)
        const double Q = -w;
        const double zc1 = (z1 - a.zmin) / a.dz, rc1 = r1 / a.dr;
        const int ilo = (int)floor(fmin(zc, zc1)), jlo = (int)floor(fmin(rc, rc1));
        const int nzs = (int)floor(fmax(zc, zc1)) + 2 - ilo, nrs = (int)floor(fmax(rc, rc1)) + 2 - jlo;
        double S0z[3], S1z[3], S0r[3], S1r[3];
        for (int k = 0; k < 3; k++) {
            S0z[k] = k < nzs ? dhat(zc - (ilo + k)) : 0.0;
            S1z[k] = k < nzs ? dhat(zc1 - (ilo + k)) : 0.0;
            S0r[k] = k < nrs ? dhat(rc - (jlo + k)) : 0.0;
            S1r[k] = k < nrs ? dhat(rc1 - (jlo + k)) : 0.0;
        }
        const int nzu = nzs < 3 ? nzs : 3, nru = nrs < 3 ? nrs : 3;
        double er0 = 1.0, ei0 = 0.0, er1 = 1.0, ei1 = 0.0;
        for (int m = 0; m < a.nm; m++) {
            if (m) {
                double t0 = er0 * c0 + ei0 * s0; ei0 = ei0 * c0 - er0 * s0; er0 = t0;   // *e^{-i phi0}
                double t1 = er1 * c1 + ei1 * s1; ei1 = ei1 * c1 - er1 * s1; er1 = t1;   // *e^{-i phi1}
            }
            const double ebr = 0.5 * (er0 + er1), ebi = 0.5 * (ei0 + ei1);
            const double der = er1 - er0, dei = ei1 - ei0;
            const int pr = m ? 2 * m - 1 : 0;
            for (int bb = 0; bb < nru; bb++) {                    // z fluxes
                const int j = jlo + bb;
                if (j < 0 || j > a.nr) continue;
                double acc = 0.0;
                for (int aa = 0; aa < nzu - 1; aa++) {
                    const double dSz = S1z[aa] - S0z[aa], dSr = S1r[bb] - S0r[bb];
                    acc += dSz * (S0r[bb] + 0.5 * dSr);
                    const double f = -(Q / a.dt) * acc * a.dz / dcvol(a, j);
                    jadd64(J, a, 2, pr, j, ilo + aa, f * ebr);
                    if (m) jadd64(J, a, 2, pr + 1, j, ilo + aa, f * ebi);
                }
            }
            for (int aa = 0; aa < nzu; aa++) {                    // r fluxes
                double acc = 0.0;
                for (int bb = 0; bb < nru - 1; bb++) {
                    const int j = jlo + bb;
                    const double dSz = S1z[aa] - S0z[aa], dSr = S1r[bb] - S0r[bb];
                    acc += dSr * (S0z[aa] + 0.5 * dSz);
                    if (j < 0 || j >= a.nr) continue;
                    const double f = -(Q / a.dt) * acc / (2.0 * PI * (j + 0.5) * a.dr * a.dz);
                    jadd64(J, a, 0, pr, j, ilo + aa, f * ebr);
                    if (m) jadd64(J, a, 0, pr + 1, j, ilo + aa, f * ebi);
                }
            }
            for (int aa = 0; aa < nzu; aa++)                      // J_phi
                for (int bb = 0; bb < nru; bb++) {
                    const int j = jlo + bb;
                    const double sb = 0.5 * (S0z[aa] * S0r[bb] + S1z[aa] * S1r[bb]);
                    if (j < 0 || j > a.nr || sb == 0.0) continue;
                    if (m == 0) {
                        jadd64(J, a, 1, 0, j, ilo + aa, Q * vphi * sb / dcvol(a, j));
                    } else {
                        // i r_j Q Sbar (e1 - e0) / (m V_j dt)
                        const double f = (j * a.dr) * Q * sb / ((double)m * dcvol(a, j) * a.dt);
                        jadd64(J, a, 1, pr, j, ilo + aa, -f * dei);
                        jadd64(J, a, 1, pr + 1, j, ilo + aa, f * der);
                    }
                }
        }
        // ---- new state
        P.x[i] = x1; P.y[i] = y1; P.ux[i] = un[0]; P.uy[i] = un[1]; P.uz[i] = un[2];
        if (a.periodic) {
            const double Lz = a.nz * a.dz, zr = z1 - a.zmin;
            P.z[i] = zr < 0 ? z1 + Lz : (zr >= Lz ? z1 - Lz : z1);
        } else {
            P.z[i] = z1;
            if (zc1 < 0.0 || zc1 >= a.nz) P.w[i] = 0.0;
        }
    }
}

void fp64_push_deposit(qpic_ctx *c)
{
    DArgs a = dargs(c);
    cudaMemsetAsync(c->J64, 0, (size_t)3 * a.nparts * a.plane * sizeof(double), c->stream);
    const long long n = c->np;
    int nblk = (int)std::min<long long>((n + 255) / 256, 152LL * 32);
    if (nblk < 1) nblk = 1;
    prof_begin(c);
    if (n > 0) k_push64<<<nblk, 256, 0, c->stream>>>(c->p64, n, c->E64, c->Bb64, c->J64, a);
    prof_end(c, KC_GPD, n > 0 ? 1 : 0);
}

// ---------------------------------------------------------------- plasma, load, export
__device__ __forceinline__ unsigned long long splitmix64_d(unsigned long long x)
{
    unsigned long long z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

struct PlasmaArgs64 {
    double n0, z_start, ramp_len, dz, dr;
    unsigned long long seed;
    int pz, pr, pp, jitter, nr, track;
    long long first_col, shifts, base;
};

__global__ void k_load_plasma64(Particles64 P, PlasmaArgs64 L, long long ntot)
{
    const double PI = 3.14159265358979323846;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < ntot;
         t += (long long)gridDim.x * blockDim.x) {
        long long q = t;
        int c = (int)(q % L.pp); q /= L.pp;
        int b = (int)(q % L.pr); q /= L.pr;
        int a = (int)(q % L.pz); q /= L.pz;
        int jr = (int)(q % L.nr); q /= L.nr;
        long long iz_abs = L.first_col + q + L.shifts;
        double z = ((double)iz_abs + (a + 0.5) / L.pz) * L.dz;
        double r = (jr + (b + 0.5) / L.pr) * L.dr;
        double jit = 0.0;
        if (L.jitter) {
            unsigned long long key = (L.seed << 40) ^ ((unsigned long long)iz_abs << 20) ^
                                     (unsigned long long)jr;
            jit = (double)(splitmix64_d(key) >> 11) * (1.0 / 9007199254740992.0);
        }
        double phi = 2.0 * PI * (c + jit) / L.pp;
        double n = L.ramp_len <= 0.0 ? (z >= L.z_start ? L.n0 : 0.0)
                                     : L.n0 * fmin(fmax((z - L.z_start) / L.ramp_len, 0.0), 1.0);
        long long d = L.base + t;
        P.z[d] = z; P.x[d] = r * cos(phi); P.y[d] = r * sin(phi);
        P.ux[d] = 0.0; P.uy[d] = 0.0; P.uz[d] = 0.0;
        P.w[d] = n * 2.0 * PI * r * (L.dr / L.pr) * (L.dz / L.pz) / L.pp;
        if (L.track) { P.W0[d] = 0.0; P.W1[d] = 0.0; }
    }
}

int fp64_load_plasma(qpic_ctx *c, long long first_col, int ncols, bool append)
{
    PlasmaArgs64 L;
    L.n0 = c->n0; L.z_start = c->z_start; L.ramp_len = c->ramp_len; L.dz = c->dz; L.dr = c->dr;
    L.seed = c->cfg.seed; L.pz = c->ppc_z; L.pr = c->ppc_r; L.pp = c->ppc_phi; L.jitter = c->jitter;
    L.nr = c->g.nr; L.track = c->cfg.track_work; L.first_col = first_col; L.shifts = c->shifts;
    long long ntot = (long long)ncols * c->g.nr * L.pz * L.pr * L.pp;
    L.base = append ? c->np : 0;
    if (L.base + ntot > c->cap) return 0;
    int nblk = (int)std::min<long long>((ntot + 255) / 256, 152LL * 16);
    if (nblk < 1) nblk = 1;
    prof_begin(c);
    k_load_plasma64<<<nblk, 256, 0, c->stream>>>(c->p64, L, ntot);
    prof_end(c, KC_INJECT);
    c->np = L.base + ntot;
    return 1;
}

__global__ void k_load64(Particles64 P, long long n, const double *z, const double *r,
                         const double *phi, const double *ux, const double *uy, const double *uz,
                         const double *w, int track)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        P.z[i] = z[i]; P.x[i] = r[i] * cos(phi[i]); P.y[i] = r[i] * sin(phi[i]);
        P.ux[i] = ux[i]; P.uy[i] = uy[i]; P.uz[i] = uz[i]; P.w[i] = w[i] > 0 ? w[i] : 0.0;
        if (track) { P.W0[i] = 0.0; P.W1[i] = 0.0; }
    }
}

void fp64_load_particles(qpic_ctx *c, long long n, const double *z, const double *r,
                         const double *phi, const double *ux, const double *uy, const double *uz,
                         const double *w)
{
    int nblk = (int)std::min<long long>((n + 255) / 256, 152LL * 16);
    if (nblk < 1) nblk = 1;
    prof_begin(c);
    if (n > 0) k_load64<<<nblk, 256, 0, c->stream>>>(c->p64, n, z, r, phi, ux, uy, uz, w,
                                                     c->cfg.track_work);
    prof_end(c, KC_OTHER, n > 0 ? 1 : 0);
    c->np = n;
}

// compaction of live particles (w > 0) into the front of the buffers
__global__ void k_flag64(const double *w, long long n, int32_t *flag)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        flag[i] = w[i] > 0.0 ? 1 : 0;
}

__global__ void k_move64(Particles64 src, Particles64 dst, long long n, const int32_t *flag,
                         const int32_t *pos, int track)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        if (!flag[i]) continue;
        long long d = pos[i];
        dst.z[d] = src.z[i]; dst.x[d] = src.x[i]; dst.y[d] = src.y[i];
        dst.ux[d] = src.ux[i]; dst.uy[d] = src.uy[i]; dst.uz[d] = src.uz[i]; dst.w[d] = src.w[i];
        if (track) { dst.W0[d] = src.W0[i]; dst.W1[d] = src.W1[i]; }
    }
}

void fp64_compact(qpic_ctx *c)
{
    const long long n = c->np;
    if (n <= 0) return;
    int32_t *flag = c->scan_flag, *pos = c->scan_pos;
    int nblk = (int)std::min<long long>((n + 255) / 256, 152LL * 16);
    cudaMemsetAsync(flag + n, 0, sizeof(int32_t), c->stream);
    prof_begin(c);
    k_flag64<<<nblk, 256, 0, c->stream>>>(c->p64.w, n, flag);
    exclusive_scan(c, flag, pos, c->scan_tmp64, n + 1);
    k_move64<<<nblk, 256, 0, c->stream>>>(c->p64, c->ps64, n, flag, pos, c->cfg.track_work);
    prof_end(c, KC_SORT, 5);
    int32_t live = 0;
    cudaMemcpyAsync(&live, pos + n, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream);
    cudaStreamSynchronize(c->stream);
    Particles64 t = c->p64; c->p64 = c->ps64; c->ps64 = t;
    c->np = live;
}

__global__ void k_export64(Particles64 P, long long n, double *out, long long stride, int track)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        out[0 * stride + i] = P.z[i];
        out[1 * stride + i] = sqrt(P.x[i] * P.x[i] + P.y[i] * P.y[i]);
        out[2 * stride + i] = atan2(P.y[i], P.x[i]);
        out[3 * stride + i] = P.ux[i]; out[4 * stride + i] = P.uy[i]; out[5 * stride + i] = P.uz[i];
        out[6 * stride + i] = P.w[i];
        out[7 * stride + i] = track ? P.W0[i] : 0.0;
        out[8 * stride + i] = track ? P.W1[i] : 0.0;
    }
}

void fp64_export_particles(qpic_ctx *c, double *dout, long long stride)
{
    const long long n = c->np;
    int nblk = (int)std::min<long long>((n + 255) / 256, 152LL * 16);
    if (nblk < 1) nblk = 1;
    if (n > 0) k_export64<<<nblk, 256, 0, c->stream>>>(c->p64, n, dout, stride, c->cfg.track_work);
}

// rho_m(i,j) = sum_p Q S_i S_j e^{-i m phi} / V_j, logical order, [nm][2][nr+1][nz]
__global__ void k_rho64(Particles64 P, long long n, double *out, DArgs a)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const double w = P.w[i];
        if (w == 0.0) continue;
        const double zc = (P.z[i] - a.zmin) / a.dz;
        const double r = sqrt(P.x[i] * P.x[i] + P.y[i] * P.y[i]), rc = r / a.dr;
        const double c1 = r > 0 ? P.x[i] / r : 1.0, s1 = r > 0 ? -P.y[i] / r : 0.0;
        const int i0 = (int)floor(zc), j0 = (int)floor(rc);
        for (int aa = 0; aa < 2; aa++)
            for (int bb = 0; bb < 2; bb++) {
                int ic = i0 + aa;
                if (a.periodic) ic = dwrap(ic, a.nz);
                else if (ic < 0 || ic >= a.nz) continue;
                const int j = j0 + bb;
                const double wgt = dhat(zc - (i0 + aa)) * dhat(rc - j);
                if (j > a.nr || wgt == 0.0) continue;
                double er = 1.0, ei = 0.0;
                for (int m = 0; m < a.nm; m++) {
                    if (m) { double t = er * c1 - ei * s1; ei = er * s1 + ei * c1; er = t; }
                    const double v = -w * wgt / dcvol(a, j);
                    atomicAdd(&out[((size_t)(2 * m) * (a.nr + 1) + j) * a.nz + ic], v * er);
                    atomicAdd(&out[((size_t)(2 * m + 1) * (a.nr + 1) + j) * a.nz + ic], v * ei);
                }
            }
    }
}

void fp64_rho(qpic_ctx *c, double *dplanes)
{
    DArgs a = dargs(c);
    const long long n = c->np;
    cudaMemsetAsync(dplanes, 0, (size_t)c->g.nm * 2 * (c->g.nr + 1) * c->g.nz * sizeof(double),
                    c->stream);
    int nblk = (int)std::min<long long>((n + 255) / 256, 152LL * 16);
    if (nblk < 1) nblk = 1;
    if (n > 0) k_rho64<<<nblk, 256, 0, c->stream>>>(c->p64, n, dplanes, a);
}

__global__ void k_spectrum64(Particles64 P, long long n, const double *edges, int nb, double wscale,
                             unsigned long long *out)
{
    extern __shared__ unsigned long long hist[];
    for (int k = threadIdx.x; k < nb; k += blockDim.x) hist[k] = 0ull;
    __syncthreads();
    const double mec2 = 0.51099895;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const double w = P.w[i];
        if (w == 0.0) continue;
        const double u2 = P.ux[i] * P.ux[i] + P.uy[i] * P.uy[i] + P.uz[i] * P.uz[i];
        const double e = u2 / (1.0 + sqrt(1.0 + u2)) * mec2;
        if (e < edges[0] || e >= edges[nb]) continue;
        int lo = 0, hi = nb;
        while (hi - lo > 1) { const int mid = (lo + hi) >> 1; if (e >= edges[mid]) lo = mid; else hi = mid; }
        atomicAdd(&hist[lo], (unsigned long long)__double2ll_rn(w * wscale));
    }
    __syncthreads();
    for (int k = threadIdx.x; k < nb; k += blockDim.x)
        if (hist[k]) atomicAdd(&out[k], hist[k]);
}

void fp64_spectrum(qpic_ctx *c, const double *edges, int nb, double wscale, unsigned long long *out)
{
    cudaMemsetAsync(out, 0, nb * sizeof(unsigned long long), c->stream);
    if (c->np > 0)
        k_spectrum64<<<152 * 2, 256, nb * sizeof(unsigned long long), c->stream>>>(c->p64, c->np, edges,
                                                                                   nb, wscale, out);
}

__global__ void k_psums64(Particles64 P, long long n, double *part)
{
    __shared__ double s0[256], s1[256], s2[256];
    double cnt = 0, chg = 0, ke = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const double w = P.w[i];
        if (w == 0.0) continue;
        const double u2 = P.ux[i] * P.ux[i] + P.uy[i] * P.uy[i] + P.uz[i] * P.uz[i];
        cnt += 1.0; chg -= w; ke += w * u2 / (1.0 + sqrt(1.0 + u2));
    }
    s0[threadIdx.x] = cnt; s1[threadIdx.x] = chg; s2[threadIdx.x] = ke;
    __syncthreads();
    for (int k = 128; k > 0; k >>= 1) {
        if (threadIdx.x < k) {
            s0[threadIdx.x] += s0[threadIdx.x + k];
            s1[threadIdx.x] += s1[threadIdx.x + k];
            s2[threadIdx.x] += s2[threadIdx.x + k];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) { part[3 * blockIdx.x] = s0[0]; part[3 * blockIdx.x + 1] = s1[0]; part[3 * blockIdx.x + 2] = s2[0]; }
}

__global__ void k_psums64_final(const double *part, int nb, double *out)
{
    if (threadIdx.x >= 3) return;
    double s = 0.0;
    for (int b = 0; b < nb; b++) s += part[3 * b + threadIdx.x];
    out[threadIdx.x] = s;
}

void fp64_particle_sums(qpic_ctx *c, double *out3)
{
    const int nb = 304;
    double *part = c->d_red + 8;
    prof_begin(c);
    k_psums64<<<nb, 256, 0, c->stream>>>(c->p64, c->np, part);
    k_psums64_final<<<1, 32, 0, c->stream>>>(part, nb, part + 3 * nb);
    prof_end(c, KC_DIAG, 2);
    cudaMemcpyAsync(out3, part + 3 * nb, 3 * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    cudaStreamSynchronize(c->stream);
}

}  // namespace qpic
