// gpd.cuh -- the particle half of the quasi-3D PIC step (FP32 path): kernel
// templates, instantiated per mode count and deposit variant in gpd_inst.cu.
//
// k_gpd: one CTA per particle tile (TZ x TR cells, particles sorted by tile).
//   1. E^n and Bbar^n of the tile plus a halo are staged in shared memory by
//      asynchronous copies, all in flight at once (mode-parity images below the
//      axis, even images beyond the wall, zeros in the gap of an open box), so
//      the gather never branches on boundaries.
//   2. per particle: bilinear gather of every mode at each component's own
//      staggered point, modal sum F_0 + 2 Re(F_m e^{i m phi}) (Sec. III.B),
//      rotation to x, y; relativistic Boris push with E^n and Bbar^n
//      (Eq. 6 time-centred as in Eq. 12); Cartesian move and an update of
//      (r, cos phi, sin phi) written with cancellation-free differences;
//      optional modal work (Eq. 16).
//   3. charge-conserving deposit per mode into fixed-point shared
//      accumulators: each integer contribution v is added as two 32-bit parts,
//      hi 2^20 + lo with 0 <= lo < 2^20, to two 32-bit planes (32-bit shared
//      atomics are several times faster than 64-bit ones); after every chunk of
//      at most 4096 particles but the last the planes are drained into an int64
//      plane, so their sums never leave the 32-bit range (FX_SHIFT, FX_SCALE).  The modal
//      charge change Q (S1 e1 - S0 e0), e = e^{-i m phi},
//      splits into (S1 - S0)(e0 + e1)/2, carried by 2D Esirkepov r/z fluxes,
//      and (S0 + S1)/2 (e1 - e0), carried by J_phi through (i m / r) J_phi.
//      Each thread takes runs of consecutive particles of the tile (sorted by
//      cell), so its moves inside one cell are summed in registers (FastSum)
//      and added once per cell; moves across cells are queued and deposited
//      once per tile.
//   4. the tile's accumulators are stored to its own block of global memory
//      as int64 (hi 2^20 + lo);
//      k_jreduce sums the blocks that cover each node.  Integer addition makes
//      the step independent of particle order (bit-reproducible).
//   Particles beyond the staged halo (drift between sorts, or injected by the
//   moving window) run the same code against global memory (int64 atomics).
//   The FA variant adds every contribution to a global FP32 current with float
//   atomics instead (precision QPIC_FP32_FATOMIC).
//
// k_jreduce: per node, the sum of the tile blocks that cover it, decoded to
// FP32 current.
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <type_traits>

#include "qpic_internal.h"

namespace qpic {

struct PArgs {
    int nz, nr, nzp, nparts, nm;
    long long zoff;
    size_t plane;
    float dz, dr, dt, inv_dz, inv_dr, R;
    int periodic;
    int TZ, TR, ntz, ntr, H, lTZ, lTR;
    float qscale;
    int track_work;
    int chunk;       // particles per chunk of a tile: 256 x (particles per thread) (<= 4096)
};

static PArgs pargs(const qpic_ctx *c)
{
    PArgs a;
    a.nz = c->g.nz; a.nr = c->g.nr; a.nzp = c->g.nzp; a.nparts = c->g.nparts; a.nm = c->g.nm;
    a.zoff = c->g.zoff % c->g.nzp; a.plane = c->g.plane;
    a.dz = (float)c->dz; a.dr = (float)c->dr; a.dt = (float)c->dt;
    a.inv_dz = (float)(1.0 / c->dz); a.inv_dr = (float)(1.0 / c->dr);
    a.R = (float)(c->g.nr * c->dr);
    a.periodic = c->g.periodic;
    a.TZ = c->TZ; a.TR = c->TR; a.ntz = c->ntz; a.ntr = c->ntr; a.H = c->halo;
    a.lTZ = __builtin_ctz(c->TZ); a.lTR = __builtin_ctz(c->TR);
    a.qscale = c->qscale;
    a.track_work = c->cfg.track_work;
    a.chunk = 256 * c->ppt;
    return a;
}

__host__ __device__ __forceinline__ int imin(int x, int y) { return x < y ? x : y; }

__device__ __forceinline__ int pwrap(int i, int n)
{
    int r = i % n;
    return r < 0 ? r + n : r;
}

// staggering: E_r (0,1) E_phi (0,0) E_z (1,0); B_r (1,0) B_phi (1,1) B_z (0,1)
__host__ __device__ __forceinline__ int hz_of(int fb, int c) { return fb == 0 ? (c == 2) : (c != 2); }
__host__ __device__ __forceinline__ int hr_of(int fb, int c) { return fb == 0 ? (c == 0) : (c != 0); }

// sample of plane (fb: 0 = E, 1 = Bbar; comp c; part p) at physical column col
// (any integer, wrapped) and row j (any integer).  Half-r components continue
// below the axis with the mode parity (radial/azimuthal (-1)^(m+1), B_z (-1)^m)
// and beyond the wall with their even image; integer-r components are 0 outside.
__device__ __forceinline__ float gsample_at(const float *E, const float *Bb, const PArgs &a, int fb,
                                            int c, int p, int j, int ic);

__device__ __forceinline__ float gsample(const float *E, const float *Bb, const PArgs &a, int fb,
                                         int c, int p, int j, int col)
{
    return gsample_at(E, Bb, a, fb, c, p, j, pwrap(col, a.nzp));
}

// as gsample, for a column ic already in [0, nzp)
__device__ __forceinline__ float gsample_at(const float *E, const float *Bb, const PArgs &a, int fb,
                                            int c, int p, int j, int ic)
{
    const float *F = fb == 0 ? E : Bb;
    float sgn = 1.f;
    if (hr_of(fb, c)) {
        if (j < 0) {
            int m = (p + 1) >> 1;
            bool longitudinal = (fb == 1 && c == 2);
            bool odd = ((m & 1) != 0) != !longitudinal;   // radial: (-1)^(m+1); z: (-1)^m
            sgn = odd ? -1.f : 1.f;
            j = -1 - j;
        }
        if (j >= a.nr) j = 2 * a.nr - 1 - j;
        if (j < 0 || j >= a.nr) return 0.f;
    } else {
        if (j < 0 || j > a.nr) return 0.f;
    }
    return sgn * F[(size_t)(c * a.nparts + p) * a.plane + (size_t)j * a.nzp + ic];
}

// Fixed point of the current: a contribution x becomes v = round(x qscale)
// with qscale = FX_SCALE / (largest particle charge), so |v| < 2^39 - 2^29
// (the largest factor of a charge in the deposit is 2).  v is rounded as
// hi 2^20 + lo with |hi| <= 2^19 - 511 and |lo| <= 2^19; when the parts are
// added to the shared planes, lo is carried into hi so that it lies in
// [0, 2^20): the hi plane (signed) and the lo plane (unsigned) then hold the
// sums of 4096 contributions of the largest size without wrapping.  A particle
// contributes at most once to a node, so the planes are drained into int64
// after every chunk of at most 4096 particles (GPD_C) but the last; the queued
// moves go to the int64 plane directly.
constexpr float FX_DOWN = 1.0f / (float)(1 << FX_SHIFT);   // 2^-20
constexpr float FX_UP = (float)(1 << FX_SHIFT);            // 2^20
constexpr unsigned FX_LOMASK = (1u << FX_SHIFT) - 1u;

// ------------------------------------------------------------ accessors
// Staged tile of E and Bbar: per (field, component, row, column) node the NP
// mode parts are packed in V = ceil(NP/4) float4 words, so a gather corner is
// one (or two) 16-byte shared loads.  Current accumulators: int64 per
// (component, part, row, column).
template <int NP, int TZ, int TR>
struct TileGeom {
    static constexpr int H = 1;                    // halo of cells around the tile
    static constexpr int FW = TZ + 2 * H + 2, FR = TR + 2 * H + 2;   // staged fields
    static constexpr int JW = FW + 1, JR = FR + 1;                   // accumulators
    static constexpr int V = (NP + 3) / 4;
    static constexpr int JWORDS = 3 * NP * JW * JR;                   // accumulated values (int64 each)
    static constexpr int JPAD = (JWORDS + 3) & ~3;                    // per 32-bit plane; keeps the float4 tile 16-B aligned
    static constexpr int FVEC = 2 * 3 * FR * FW * V;                  // float4 words
    static constexpr int NM = (NP + 1) / 2;
    static constexpr int QW = 8 + 4 * (NM - 1);                       // words per queued move
    static constexpr int QCAP = 256;                                  // queued cell-crossing moves
    static constexpr int PB = 9 * 256;      // prefetched words per buffer: 256 cells, 2 x 256 float4
    static constexpr size_t SMEM = (size_t)JPAD * 8 /* hi, lo 32-bit planes */ + (size_t)JPAD * 8 /* int64 plane */ +
                                   (size_t)FVEC * 16 + (size_t)QCAP * QW * 4 + (size_t)2 * PB * 4 + 16;
    static_assert((JPAD * 8) % 16 == 0, "float4 tile alignment");
};

template <int NP, int TZ, int TR>
struct SmemAcc {
    using G = TileGeom<NP, TZ, TR>;
    const float4 *sf;            // [2][3][FR][FW][V]
    unsigned *sJh, *sJl;         // hi and lo planes, each [3][NP][JR][JW]
    __device__ __forceinline__ void node(int fb, int c, int lj, int li, float out[NP]) const
    {
        const float4 *q = sf + ((size_t)((fb * 3 + c) * G::FR + lj) * G::FW + li) * G::V;
#pragma unroll
        for (int v = 0; v < G::V; v++) {
            const float4 t = q[v];
            if (4 * v + 0 < NP) out[4 * v + 0] = t.x;
            if (4 * v + 1 < NP) out[4 * v + 1] = t.y;
            if (4 * v + 2 < NP) out[4 * v + 2] = t.z;
            if (4 * v + 3 < NP) out[4 * v + 3] = t.w;
        }
    }
    float qs;                    // fixed-point scale
    __device__ __forceinline__ void jadd2(int c, int p, int lj, int li, int hi, int lo) const
    {
        const int k = ((c * NP + p) * G::JR + lj) * G::JW + li;
        const int h = hi + (lo >> FX_SHIFT);              // lo < 0 borrows one from hi
        const unsigned l = (unsigned)lo & FX_LOMASK;
        if (h) atomicAdd(&sJh[k], (unsigned)h);
        if (l) atomicAdd(&sJl[k], l);
    }
    __device__ __forceinline__ void put(int c, int p, int lj, int li, float x) const;
};

template <int NP>
struct GlobAcc {
    const float *E, *Bb;
    unsigned long long *J;
    int *dirty;                  // per tile: epoch of the last global-path deposit into its core
    const int *epoch;            // this step's epoch (read on this rare path only)
    PArgs a;
    __device__ __forceinline__ void node(int fb, int c, int j, int i, float out[NP]) const
    {
#pragma unroll
        for (int p = 0; p < NP; p++) out[p] = gsample(E, Bb, a, fb, c, p, j, i);
    }
    __device__ __forceinline__ void jadd(int c, int p, int j, int i, long long v) const
    {
        if (!v || j < 0 || j > a.nr) return;
        int ic = pwrap(i, a.nzp);
        atomicAdd(&J[(size_t)(c * a.nparts + p) * a.plane + (size_t)j * a.nzp + ic],
                  (unsigned long long)v);
        const int tr = imin(j >> a.lTR, a.ntr - 1);
        dirty[(ic >> a.lTZ) * a.ntr + tr] = *epoch;
    }
    __device__ __forceinline__ void put(int c, int p, int j, int i, float x) const;
};

// FP32 variant of the deposit: contributions are added to a global FP32
// current with float atomics (no fixed point; the sum depends on the order of
// the additions, so results are not bit-reproducible)
struct FloatAcc {
    float *J;
    PArgs a;
    __device__ __forceinline__ void put(int c, int p, int j, int i, float x) const
    {
        if (x == 0.f || j < 0 || j > a.nr) return;
        int ic = pwrap(i, a.nzp);
        atomicAdd(&J[(size_t)(c * a.nparts + p) * a.plane + (size_t)j * a.nzp + ic], x);
    }
};


// Exact round-to-nearest of a scaled contribution |v| < 2^41 into hi 2^20 + lo
// using only FP32 adds: t + 1.5*2^23 has unit spacing, so its bit pattern minus
// that of 1.5*2^23 is round(t).  (A float->int64 conversion would run on the
// FP64 pipe, which is narrow on this part.)
__device__ __forceinline__ void fx_split(float v, int &hi, int &lo)
{
    const float M = 12582912.0f;                       // 1.5 * 2^23
    const float t = __fmul_rn(v, FX_DOWN);              // v 2^-20 (exact)
    const float tm = __fadd_rn(t, M);
    hi = __float_as_int(tm) - 0x4B400000;
    const float hf = __fsub_rn(tm, M);                  // round(t), exact
    const float r = __fmaf_rn(-hf, FX_UP, v);           // v - hi 2^20, exact
    lo = __float_as_int(__fadd_rn(r, M)) - 0x4B400000;
}

__device__ __forceinline__ long long fx(float x, float qs)
{
    int hi, lo;
    fx_split(x * qs, hi, lo);
    return ((long long)hi << FX_SHIFT) + lo;
}

template <int NP, int TZ, int TR>
__device__ __forceinline__ void SmemAcc<NP, TZ, TR>::put(int c, int p, int lj, int li, float x) const
{
    int hi, lo;
    fx_split(x * qs, hi, lo);
    jadd2(c, p, lj, li, hi, lo);
}

template <int NP>
__device__ __forceinline__ void GlobAcc<NP>::put(int c, int p, int j, int i, float x) const
{
    jadd(c, p, j, i, fx(x, a.qscale));
}

// The tile's int64 shared plane, for the queued cell-crossing moves deposited
// after the last chunk (64-bit shared atomics: at most QCAP moves per tile)
template <int NP, int TZ, int TR>
struct SmemAcc64 {
    using G = TileGeom<NP, TZ, TR>;
    unsigned long long *sJ64;    // [3][NP][JR][JW]
    float qs;
    __device__ __forceinline__ void put(int c, int p, int lj, int li, float x) const
    {
        const long long v = fx(x, qs);
        if (v) atomicAdd(&sJ64[((c * NP + p) * G::JR + lj) * G::JW + li], (unsigned long long)v);
    }
};

__device__ __forceinline__ int wrapn(int i, int n)      // for i in [-n, 2n)
{
    i = i < 0 ? i + n : i;
    return i >= n ? i - n : i;
}

// Linear-shape values S0 and differences dS = S1 - S0 at nodes k = -1..2 (index
// k+1) for a move x0 -> x0 + d in old-cell coordinates (x0 in [0,1), |d| < 1).
// A move inside the cell gives dS = (-d, +d) exactly, without cancellation.
__device__ __forceinline__ void shape_delta(float x0, float d, float S0[4], float dS[4], int &lo,
                                            int &hi)
{
    float x1 = x0 + d;
    S0[0] = 0.f; S0[1] = 1.f - x0; S0[2] = x0; S0[3] = 0.f;
    if (x1 >= 1.f) {
        dS[0] = 0.f; dS[1] = x0 - 1.f; dS[2] = (2.f - 2.f * x0) - d; dS[3] = (x0 - 1.f) + d;
        lo = 1; hi = 3;
    } else if (x1 < 0.f) {
        dS[0] = -(x0 + d); dS[1] = 2.f * x0 + d; dS[2] = -x0; dS[3] = 0.f;
        lo = 0; hi = 2;
    } else {
        dS[0] = 0.f; dS[1] = -d; dS[2] = d; dS[3] = 0.f;
        lo = 1; hi = 2;
    }
}

// approximate square root (PTX sqrt.approx, relative error ~2^-23); the move
// needs no IEEE rounding (charge conservation uses the displacement as computed)
__device__ __forceinline__ float sqrt_fast(float x)
{
    float y;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

struct PState {
    float oz, orr, cph, sph, ux, uy, uz, w, W0, W1;
    int jr;          // r cell (absolute)
    int diz, djr;    // cell change of the move
};

// what the deposit needs from the move: old offsets, displacement in cells,
// charge, e^{-i m phi} at the start and its change, and the m = 0 azimuthal
// displacement (x0 dy - y0 dx)/(r_mid dr)
template <int NM>
struct DepIn {
    float oz0, or0, dzc, drc, Q, aphi;
    float e0r[NM], e0i[NM], der[NM], dei[NM];
};

// Gather, push and move one particle.  (bi, bj): accessor coordinates of its
// cell.  On return s holds the new state and d the deposit inputs.
template <int NP, class Acc>
__device__ __forceinline__ void push_move(const Acc &acc, const PArgs &a, int bi, int bj, PState &s,
                                          DepIn<(NP + 1) / 2> &d)
{
    constexpr int NM = (NP + 1) / 2;
    const float oz = s.oz, orr = s.orr, cph = s.cph, sph = s.sph;
    // ---- interpolation weights on the integer and half grids
    const int ozh = oz >= 0.5f ? 0 : -1, orh = orr >= 0.5f ? 0 : -1;
    const float wzH = oz >= 0.5f ? oz - 0.5f : oz + 0.5f;
    const float wrH = orr >= 0.5f ? orr - 0.5f : orr + 0.5f;
    // bilinear weights of the four staggering classes (half z?, half r?)
    const float tzs[2] = {oz, wzH}, trs[2] = {orr, wrH};
    float W[2][2][4];
#pragma unroll
    for (int hz = 0; hz < 2; hz++)
#pragma unroll
        for (int hr = 0; hr < 2; hr++) {
            const float tz = tzs[hz], tr = trs[hr], uz = 1.f - tz, ur = 1.f - tr;
            W[hz][hr][0] = uz * ur; W[hz][hr][1] = tz * ur;
            W[hz][hr][2] = uz * tr; W[hz][hr][3] = tz * tr;
        }
    float F[2][3][NP];
#pragma unroll
    for (int fb = 0; fb < 2; fb++)
#pragma unroll
        for (int c = 0; c < 3; c++) {
            const int hz = hz_of(fb, c), hr = hr_of(fb, c);
            const int i0 = bi + (hz ? ozh : 0), j0 = bj + (hr ? orh : 0);
            const float *w = W[hz][hr];
            float v00[NP], v01[NP], v10[NP], v11[NP];
            acc.node(fb, c, j0, i0, v00);
            acc.node(fb, c, j0, i0 + 1, v01);
            acc.node(fb, c, j0 + 1, i0, v10);
            acc.node(fb, c, j0 + 1, i0 + 1, v11);
#pragma unroll
            for (int p = 0; p < NP; p++)
                F[fb][c][p] = w[0] * v00[p] + w[1] * v01[p] + w[2] * v10[p] + w[3] * v11[p];
        }
    // ---- modal sum, rotation to Cartesian
    float cm[NM], sm[NM];
    cm[0] = 1.f; sm[0] = 0.f;
#pragma unroll
    for (int m = 1; m < NM; m++) {
        cm[m] = cm[m - 1] * cph - sm[m - 1] * sph;
        sm[m] = sm[m - 1] * cph + cm[m - 1] * sph;
    }
    float Ec[3], Bc[3];
#pragma unroll
    for (int c = 0; c < 3; c++) {
        float e = F[0][c][0], b = F[1][c][0];
#pragma unroll
        for (int m = 1; m < NM; m++) {
            e += 2.f * (F[0][c][2 * m - 1] * cm[m] - F[0][c][2 * m] * sm[m]);
            b += 2.f * (F[1][c][2 * m - 1] * cm[m] - F[1][c][2 * m] * sm[m]);
        }
        Ec[c] = e; Bc[c] = b;
    }
    const float Ex = Ec[0] * cph - Ec[1] * sph, Ey = Ec[0] * sph + Ec[1] * cph, Ez = Ec[2];
    const float Bx = Bc[0] * cph - Bc[1] * sph, By = Bc[0] * sph + Bc[1] * cph, Bz = Bc[2];
    // ---- relativistic Boris push, q = -1
    const float h = -0.5f * a.dt;
    const float ux = s.ux, uy = s.uy, uz = s.uz;
    float umx = ux + h * Ex, umy = uy + h * Ey, umz = uz + h * Ez;
    float igm = rsqrtf(1.f + umx * umx + umy * umy + umz * umz);
    float tx = h * Bx * igm, ty = h * By * igm, tz = h * Bz * igm;
    float t2 = tx * tx + ty * ty + tz * tz;
    float f2 = __fdividef(2.f, 1.f + t2);
    float sx = f2 * tx, sy = f2 * ty, sz = f2 * tz;
    float upx = umx + (umy * tz - umz * ty);
    float upy = umy + (umz * tx - umx * tz);
    float upz = umz + (umx * ty - umy * tx);
    float unx = umx + (upy * sz - upz * sy) + h * Ex;
    float uny = umy + (upz * sx - upx * sz) + h * Ey;
    float unz = umz + (upx * sy - upy * sx) + h * Ez;
    const float ig = rsqrtf(1.f + unx * unx + uny * uny + unz * unz);
    const float vx = unx * ig, vy = uny * ig, vz = unz * ig;
    if (a.track_work) {
        // v at time n: the mean of u/gamma at n -+ 1/2
        const float igo = rsqrtf(1.f + ux * ux + uy * uy + uz * uz);
        float wx = 0.5f * (ux * igo + vx), wy = 0.5f * (uy * igo + vy), wz = 0.5f * (uz * igo + vz);
        if (a.track_work == 2) {
            // Eq. 17: W_z += q dt E_z v_z, W_perp += q dt E_perp . v_perp (all modes)
            s.W0 -= a.dt * (Ez * wz);
            s.W1 -= a.dt * (Ex * wx + Ey * wy);
        } else {
            // Eq. 16: W_m += q dt E^m . v; W0 holds m = 0, W1 the modes m >= 1
            float E0x = F[0][0][0] * cph - F[0][1][0] * sph, E0y = F[0][0][0] * sph + F[0][1][0] * cph;
            float p0 = E0x * wx + E0y * wy + F[0][2][0] * wz;
            float pt = Ex * wx + Ey * wy + Ez * wz;
            s.W0 -= a.dt * p0;
            s.W1 -= a.dt * (pt - p0);
        }
    }
    // ---- move in Cartesian x, y; r and angle with cancellation-free differences
    const float ddz = a.dt * vz;
    float ddx = a.dt * vx, ddy = a.dt * vy;
    const float r0 = ((float)s.jr + orr) * a.dr;
    const float x0 = r0 * cph, y0 = r0 * sph;
    float x1 = x0 + ddx, y1 = y0 + ddy;
    float r1 = sqrt_fast(x1 * x1 + y1 * y1);
    float drr, c1, s1, dc, ds;
    if (r1 <= a.R) {
        float den = r0 + r1;
        drr = den > 0.f ? __fdividef(ddx * (2.f * x0 + ddx) + ddy * (2.f * y0 + ddy), den) : 0.f;
        if (r1 > 0.f) {
            float ir = __fdividef(1.f, r1);
            c1 = x1 * ir; s1 = y1 * ir;
            dc = (ddx - cph * drr) * ir; ds = (ddy - sph * drr) * ir;
        } else {
            c1 = cph; s1 = sph; dc = 0.f; ds = 0.f;
        }
    } else {                               // specular reflection at the wall
        float cr = x1 / r1, sr = y1 / r1;
        float urad = unx * cr + uny * sr;
        unx -= 2.f * urad * cr; uny -= 2.f * urad * sr;
        float rn = 2.f * a.R - r1;
        x1 = cr * rn; y1 = sr * rn; r1 = rn;
        ddx = x1 - x0; ddy = y1 - y0;
        drr = r1 - r0; c1 = cr; s1 = sr; dc = c1 - cph; ds = s1 - sph;
    }
    const float dzc = ddz * a.inv_dz, drc = drr * a.inv_dr;
    // ---- deposit inputs
    d.oz0 = oz; d.or0 = orr; d.dzc = dzc; d.drc = drc; d.Q = -s.w;
    d.e0r[0] = 1.f; d.e0i[0] = 0.f; d.der[0] = 0.f; d.dei[0] = 0.f;
    if (NM > 1) {
        const float a0r = cph, a0i = -sph, adr = dc, adi = -ds;     // e0_1, de_1
        const float a1r = a0r + adr, a1i = a0i + adi;                // e1_1
        d.e0r[1] = a0r; d.e0i[1] = a0i; d.der[1] = adr; d.dei[1] = adi;
#pragma unroll
        for (int m = 2; m < NM; m++) {
            // e0_m = e0_{m-1} e0_1 ; de_m = de_{m-1} e1_1 + e0_{m-1} de_1
            d.e0r[m] = d.e0r[m - 1] * a0r - d.e0i[m - 1] * a0i;
            d.e0i[m] = d.e0r[m - 1] * a0i + d.e0i[m - 1] * a0r;
            d.der[m] = d.der[m - 1] * a1r - d.dei[m - 1] * a1i + d.e0r[m - 1] * adr - d.e0i[m - 1] * adi;
            d.dei[m] = d.der[m - 1] * a1i + d.dei[m - 1] * a1r + d.e0r[m - 1] * adi + d.e0i[m - 1] * adr;
        }
    }
    const float xm = x0 + 0.5f * ddx, ym = y0 + 0.5f * ddy;
    const float rm = sqrt_fast(xm * xm + ym * ym);
    d.aphi = rm > 0.f ? __fdividef(x0 * ddy - y0 * ddx, rm * a.dr) : 0.f;
    // ---- new state: offsets renormalised into the cell
    float nz_ = oz + dzc, nr_ = orr + drc;
    int diz = 0, djr = 0;
    if (nz_ >= 1.f) { nz_ -= 1.f; diz = 1; } else if (nz_ < 0.f) { nz_ += 1.f; diz = -1; }
    if (nz_ >= 1.f) nz_ = 0.99999994f;          // rounding guard
    if (nr_ >= 1.f) { nr_ -= 1.f; djr = 1; } else if (nr_ < 0.f) { nr_ += 1.f; djr = -1; }
    if (nr_ >= 1.f) nr_ = 0.99999994f;
    if (s.jr + djr >= a.nr) { djr = a.nr - 1 - s.jr; nr_ = 0.99999994f; }   // r = R exactly
    if (s.jr + djr < 0) { djr = -s.jr; nr_ = 0.f; }
    s.oz = nz_; s.orr = nr_; s.cph = c1; s.sph = s1;
    s.ux = unx; s.uy = uny; s.uz = unz;
    s.diz = diz; s.djr = djr;
}

// True when the move stays inside its cell in z and r (the common case).
template <int NM>
__device__ __forceinline__ bool same_cell(const DepIn<NM> &d)
{
    const float xz = d.oz0 + d.dzc, xr = d.or0 + d.drc;
    return xz >= 0.f && xz < 1.f && xr >= 0.f && xr < 1.f;
}

// Charge-conserving deposit of one move, any cell crossing (2D Esirkepov fluxes
// times (e0+e1)/2 per mode, J_phi from the phase change), direct atomics.
template <int NP, class Acc>
__device__ __forceinline__ void deposit_general(const Acc &acc, const PArgs &a, int bi, int bj,
                                                const DepIn<(NP + 1) / 2> &d)
{
    constexpr int NM = (NP + 1) / 2;
    float S0z[4], dSz[4], S0r[4], dSr[4];
    int zlo, zhi, rlo, rhi;
    shape_delta(d.oz0, d.dzc, S0z, dSz, zlo, zhi);
    shape_delta(d.or0, d.drc, S0r, dSr, rlo, rhi);
    const float Q = d.Q;
    // z fluxes through faces (i0+k+1/2, j0+kr): prefix sums of W^z along z
#pragma unroll
    for (int b = 0; b < 4; b++) {
        if (b < rlo || b > rhi) continue;
        const float srb = S0r[b] + 0.5f * dSr[b];
        float accw = 0.f;
#pragma unroll
        for (int a2 = 0; a2 < 3; a2++) {
            if (a2 < zlo || a2 >= zhi) continue;
            accw += dSz[a2] * srb;
            const float X = -Q * accw;
            const int lj = bj + b - 1, li = bi + a2 - 1;
            acc.put(2, 0, lj, li, X);
#pragma unroll
            for (int m = 1; m < NM; m++) {
                float ebr = d.e0r[m] + 0.5f * d.der[m], ebi = d.e0i[m] + 0.5f * d.dei[m];
                acc.put(2, 2 * m - 1, lj, li, X * ebr);
                acc.put(2, 2 * m, lj, li, X * ebi);
            }
        }
    }
    // r fluxes through faces (i0+k, j0+kr+1/2): prefix sums of W^r along r
#pragma unroll
    for (int a2 = 0; a2 < 4; a2++) {
        if (a2 < zlo || a2 > zhi) continue;
        const float sza = S0z[a2] + 0.5f * dSz[a2];
        float accw = 0.f;
#pragma unroll
        for (int b = 0; b < 3; b++) {
            if (b < rlo || b >= rhi) continue;
            accw += dSr[b] * sza;
            const float X = -Q * accw;
            const int lj = bj + b - 1, li = bi + a2 - 1;
            acc.put(0, 0, lj, li, X);
#pragma unroll
            for (int m = 1; m < NM; m++) {
                float ebr = d.e0r[m] + 0.5f * d.der[m], ebi = d.e0i[m] + 0.5f * d.dei[m];
                acc.put(0, 2 * m - 1, lj, li, X * ebr);
                acc.put(0, 2 * m, lj, li, X * ebi);
            }
        }
    }
    // azimuthal current at nodes: m = 0 from the mid-point azimuthal displacement,
    // m >= 1 from i Q Sbar (e1 - e0) / m
#pragma unroll
    for (int a2 = 0; a2 < 4; a2++) {
        if (a2 < zlo || a2 > zhi) continue;
#pragma unroll
        for (int b = 0; b < 4; b++) {
            if (b < rlo || b > rhi) continue;
            const float sb = S0z[a2] * S0r[b] +
                             0.5f * (S0z[a2] * dSr[b] + dSz[a2] * S0r[b] + dSz[a2] * dSr[b]);
            const int lj = bj + b - 1, li = bi + a2 - 1;
            const float QS = Q * sb;
            acc.put(1, 0, lj, li, QS * d.aphi);
#pragma unroll
            for (int m = 1; m < NM; m++) {
                const float im = 1.f / (float)m;
                acc.put(1, 2 * m - 1, lj, li, -QS * d.dei[m] * im);
                acc.put(1, 2 * m, lj, li, QS * d.der[m] * im);
            }
        }
    }
}

// Same-cell deposits summed in registers.  A thread takes consecutive particles
// of its tile (see chunk_slot), so successive moves mostly stay in one cell and
// go to the same 8*NP accumulator words (J_z at 2 faces, J_r at 2 faces, J_phi
// at 4 nodes, each per part).  Each contribution is rounded to the int64 fixed
// point exactly as fx() does, kept as hi 2^20 + lo, and the two halves are
// summed in 32-bit registers; the biased bit patterns of the rounding sums
// (1.5*2^23 + hi) are added directly and the bias is removed once per flush.
// Integer sums make the result independent of particle order.  A flush adds
// the int64 totals to the tile's shared accumulators when the cell changes and
// at the end of each chunk.  Tile geometry is compile-time, so every
// accumulator offset is an immediate.
template <int NP, int TZ, int TR>
struct FastSum {
    using G = TileGeom<NP, TZ, TR>;
    static constexpr int NV = 8 * NP;
    static constexpr int PL = G::JR * G::JW;           // words per accumulator plane
    unsigned hs[NV], ls[NV];
    unsigned n;                                         // moves summed since the last flush
    int key;                                            // (lj << 12) | li of those moves

    __device__ __forceinline__ void clear()
    {
#pragma unroll
        for (int i = 0; i < NV; i++) { hs[i] = 0u; ls[i] = 0u; }
        n = 0u;
        key = -1;
    }
    // accumulator word of value i relative to the cell's (lj, li)
    static __device__ __forceinline__ constexpr int off(int i)
    {
        const int p = i >> 3, e = i & 7;
        return e == 0 ? (2 * NP + p) * PL
             : e == 1 ? (2 * NP + p) * PL + G::JW
             : e == 2 ? p * PL
             : e == 3 ? p * PL + 1
                      : (NP + p) * PL + ((e - 4) & 1) + ((e - 4) >> 1) * G::JW;
    }
    // two contributions t = value * qscale * 2^-20 (|t| < 2^19) at once, on the
    // paired FP32 units: the same roundings as fx() for each lane
    __device__ __forceinline__ void put2(int i, float2 t)
    {
        const float2 M2 = make_float2(12582912.0f, 12582912.0f);     // 1.5 * 2^23
        const float2 nM2 = make_float2(-12582912.0f, -12582912.0f);
        const float2 tm = __fadd2_rn(t, M2);                          // bits: 0x4B400000 + round(t)
        hs[i] += __float_as_uint(tm.x);
        hs[i + 1] += __float_as_uint(tm.y);
        const float2 hf = __fadd2_rn(tm, nM2);                        // round(t), exact
        const float2 r = __ffma2_rn(hf, make_float2(-1.f, -1.f), t);  // t - round(t), exact
        const float2 lm = __ffma2_rn(r, make_float2(FX_UP, FX_UP), M2);
        ls[i] += __float_as_uint(lm.x);
        ls[i + 1] += __float_as_uint(lm.y);
    }
    static __device__ __forceinline__ float2 mul2(float2 a, float b) { return __fmul2_rn(a, make_float2(b, b)); }
    __device__ __forceinline__ void add(const DepIn<(NP + 1) / 2> &d, float q20)
    {
        constexpr int NM = (NP + 1) / 2;
        const float dz_ = d.dzc, dr_ = d.drc;
        const float Sz0 = (1.f - d.oz0) - 0.5f * dz_, Sz1 = d.oz0 + 0.5f * dz_;
        const float Sr0 = (1.f - d.or0) - 0.5f * dr_, Sr1 = d.or0 + 0.5f * dr_;
        const float c4 = 0.25f * dz_ * dr_;
        const float2 Xz = mul2(make_float2(Sr0, Sr1), q20 * dz_);   // J_z at (i0+1/2, j0+b)
        const float2 Xr = mul2(make_float2(Sz0, Sz1), q20 * dr_);   // J_r at (i0+a, j0+1/2)
        // J_phi at (i0+a, j0+b): Sbar_ab = Sz_a Sr_b + (dSz_a dSr_b)/4
        const float2 Q01 = mul2(make_float2(Sz0 * Sr0 + c4, Sz1 * Sr0 - c4), q20);
        const float2 Q23 = mul2(make_float2(Sz0 * Sr1 - c4, Sz1 * Sr1 + c4), q20);
        put2(0, Xz); put2(2, Xr);
        put2(4, mul2(Q01, d.aphi)); put2(6, mul2(Q23, d.aphi));   // m = 0: azimuthal displacement
#pragma unroll
        for (int m = 1; m < NM; m++) {
            const float ebr = d.e0r[m] + 0.5f * d.der[m], ebi = d.e0i[m] + 0.5f * d.dei[m];
            const float im = 1.f / (float)m;
            const int pr = 8 * (2 * m - 1), pi = 8 * (2 * m);
            put2(pr + 0, mul2(Xz, ebr)); put2(pr + 2, mul2(Xr, ebr));
            put2(pi + 0, mul2(Xz, ebi)); put2(pi + 2, mul2(Xr, ebi));
            const float wr = -d.dei[m] * im, wi = d.der[m] * im;     // m >= 1: i Q Sbar (e1 - e0)/m
            put2(pr + 4, mul2(Q01, wr)); put2(pr + 6, mul2(Q23, wr));
            put2(pi + 4, mul2(Q01, wi)); put2(pi + 6, mul2(Q23, wi));
        }
        n += 1u;
    }
    // the sums go to the hi and lo planes with 32-bit shared atomics, the lo
    // sum L (|L| <= 16 2^19) carried into hi so that the lo plane receives
    // L mod 2^20 (the planes hold their sums exactly: see FX_SCALE)
    __device__ __forceinline__ void flush(unsigned *sJh, unsigned *sJl)
    {
        if (n == 0u) return;
        const int base = (key >> 12) * G::JW + (key & 0xFFF);
        const unsigned bias = 0x4B400000u * n;
#pragma unroll
        for (int i = 0; i < NV; i++) {
            const int L = (int)(ls[i] - bias);
            atomicAdd(sJh + base + off(i), hs[i] - bias + (unsigned)(L >> FX_SHIFT));
            atomicAdd(sJl + base + off(i), (unsigned)L & FX_LOMASK);
            hs[i] = 0u; ls[i] = 0u;
        }
        n = 0u;
    }
};

// ------------------------------------------------------------ the GPD kernel
// Particle order inside a tile.  The n particles of a tile (sorted by cell) are
// taken in chunks of at most C = 256 p particles, p the particles per thread
// (1..16, so C <= GPD_C = 4096: the 32-bit accumulator planes are drained into
// int64 after each chunk, FX_SCALE).  In a chunk of rc particles every
// thread takes kc = ceil(rc / GPD_T) <= p consecutive particles (nt = rc / kc
// threads take kc, thread nt the rem = rc - nt kc left), so one thread's moves
// mostly share a cell (FastSum) and about ppc / kc threads work on one cell.
// Thread t's k-th particle of a chunk is q0 + t kc + k.
constexpr int GPD_T = 256, GPD_C = GPD_PPT_MAX * GPD_T;
static_assert(GPD_T == 256 && GPD_C == 4096 && FX_SHIFT == 20, "chunk sizes assume 256 threads and the 2^20 split");

struct Chunk { int q0, rc, kc, nt, rem; };

__host__ __device__ __forceinline__ int tile_nchunks(int n, int chunk) { return (n + chunk - 1) / chunk; }

__host__ __device__ __forceinline__ Chunk tile_chunk(int n, int c, int chunk)
{
    Chunk k;
    k.q0 = c * chunk;
    k.rc = n - k.q0 < chunk ? n - k.q0 : chunk;
    k.kc = (k.rc + GPD_T - 1) / GPD_T;
    k.nt = k.rc / k.kc;
    k.rem = k.rc - k.nt * k.kc;
    return k;
}

// Storage slot, inside its chunk, of thread t's k-th particle.  The sort
// stores each chunk column by column: the k-th particles of all threads that
// have one lie in consecutive slots (k (nt + 1) + t while every thread up to
// nt has a k-th particle, rem (nt + 1) + (k - rem) nt + t after), so at every
// iteration the block's threads read and write consecutive records
// (coalesced), while each thread still walks consecutive particles of the
// cell-sorted order (u = t kc + k).
__host__ __device__ __forceinline__ int chunk_slot(const Chunk &C, int t, int k)
{
    return k < C.rem ? k * (C.nt + 1) + t : C.rem * (C.nt + 1) + (k - C.rem) * C.nt + t;
}

// Ampere-style asynchronous 4-byte global -> shared copies (one per thread and
// word); a thread waits only for its own groups
__device__ __forceinline__ void cp_async4(void *smem, const void *gmem)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
// 4-byte copy that reads src_bytes (4 or 0) from global memory and zero-fills the rest
__device__ __forceinline__ void cp_async4_zfill(void *smem, const void *gmem, int src_bytes)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(sa), "l"(gmem), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
// one particle record (two float4 words, 32-byte aligned) in a single 256-bit access
__device__ __forceinline__ void ld_rec(const float4 *p, float4 &a, float4 &b)
{
    asm volatile("ld.global.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w), "=f"(b.x), "=f"(b.y), "=f"(b.z), "=f"(b.w)
                 : "l"(p));
}
__device__ __forceinline__ void st_rec(float4 *p, const float4 &a, const float4 &b)
{
    asm volatile("st.global.v8.f32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"l"(p), "f"(a.x), "f"(a.y),
                 "f"(a.z), "f"(a.w), "f"(b.x), "f"(b.y), "f"(b.z), "f"(b.w)
                 : "memory");
}
__device__ __forceinline__ void cp_async_wait_prev() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// cell index of a particle: (iz_phys << 16) | jr
__host__ __device__ __forceinline__ int cell_iz(int cell) { return cell >> 16; }
__host__ __device__ __forceinline__ int cell_jr(int cell) { return cell & 0xFFFF; }
__host__ __device__ __forceinline__ int make_cell(int iz, int jr) { return (iz << 16) | jr; }

// queued cell-crossing move: local cell, offsets, displacement, charge,
// azimuthal displacement, then e0/de per mode m >= 1
template <int NM>
__device__ __forceinline__ void queue_put(float *q, int li, int lj, const DepIn<NM> &d)
{
    q[0] = __int_as_float(li); q[1] = __int_as_float(lj);
    q[2] = d.oz0; q[3] = d.or0; q[4] = d.dzc; q[5] = d.drc; q[6] = d.Q; q[7] = d.aphi;
#pragma unroll
    for (int m = 1; m < NM; m++) {
        q[8 + 4 * (m - 1)] = d.e0r[m]; q[9 + 4 * (m - 1)] = d.e0i[m];
        q[10 + 4 * (m - 1)] = d.der[m]; q[11 + 4 * (m - 1)] = d.dei[m];
    }
}

template <int NM>
__device__ __forceinline__ void queue_get(const float *q, int &li, int &lj, DepIn<NM> &d)
{
    li = __float_as_int(q[0]); lj = __float_as_int(q[1]);
    d.oz0 = q[2]; d.or0 = q[3]; d.dzc = q[4]; d.drc = q[5]; d.Q = q[6]; d.aphi = q[7];
    d.e0r[0] = 1.f; d.e0i[0] = 0.f; d.der[0] = 0.f; d.dei[0] = 0.f;
#pragma unroll
    for (int m = 1; m < NM; m++) {
        d.e0r[m] = q[8 + 4 * (m - 1)]; d.e0i[m] = q[9 + 4 * (m - 1)];
        d.der[m] = q[10 + 4 * (m - 1)]; d.dei[m] = q[11 + 4 * (m - 1)];
    }
}

// One particle through global memory: for particles appended since the last
// sort, particles that drifted beyond the staged halo (sort period above 2) and
// boxes too short for a staged tile.
template <int NP, bool FA>
__device__ __forceinline__ void gpd_global_one(const Particles &P, long long idx, int cell, const PArgs &a,
                                               const GlobAcc<NP> &gacc, const FloatAcc &facc)
{
    constexpr int NM = (NP + 1) / 2;
    const int zoff = (int)a.zoff;
    const int iz = cell_iz(cell), jr = cell_jr(cell);
    if (!a.periodic && wrapn(iz - zoff, a.nzp) >= a.nz) { P.cell[idx] = -1; return; }
    PState s;
    DepIn<NM> d;
    float4 ra, rb;
    ld_rec(P.rec + 2 * idx, ra, rb);
    s.oz = ra.x; s.orr = ra.y; s.cph = ra.z; s.sph = ra.w;
    s.ux = rb.x; s.uy = rb.y; s.uz = rb.z; s.w = rb.w;
    s.W0 = a.track_work ? P.W0[idx] : 0.f;
    s.W1 = a.track_work ? P.W1[idx] : 0.f;
    s.jr = jr;
    push_move<NP>(gacc, a, iz, jr, s, d);
    if constexpr (FA) deposit_general<NP>(facc, a, iz, jr, d);
    else deposit_general<NP>(gacc, a, iz, jr, d);
    const int niz = wrapn(iz + s.diz, a.nzp);
    const bool dead = !a.periodic && wrapn(niz - zoff, a.nzp) >= a.nz;
    P.cell[idx] = dead ? -1 : make_cell(niz, jr + s.djr);
    st_rec(P.rec + 2 * idx, make_float4(s.oz, s.orr, s.cph, s.sph), make_float4(s.ux, s.uy, s.uz, s.w));
    if (a.track_work) { P.W0[idx] = s.W0; P.W1[idx] = s.W1; }
}

// FA: the FP32 float-atomic variant (every deposit goes to the global FP32
// current Jfa with float atomics; the fixed-point accumulators are unused)
// everything one run's particle kernel reads and writes
struct GpdArgs {
    Particles P;
    const float *E, *Bb;
    unsigned long long *J;
    float *Jfa;
    unsigned long long *Jtile;
    int *tstamp, *jdirty;
    const int *d_epoch;
    const int32_t *offsets;
    const long long *dcount;
    PArgs a;
    int *err;        // the run's error word (the checked build's invariant checks)
};

// One block of the particle kernel: tile bid (bid < ntiles) or a chunk of the
// particles appended since the last sort (bid >= ntiles).  sraw: the block's
// dynamic shared memory (TileGeom::SMEM bytes).
template <int NP, int TZ, int TR, bool FA>
__device__ __forceinline__ void gpd_block(const GpdArgs g, int bid, int ntiles, int tail_chunk,
                                          unsigned long long *sraw)
{
    using G = TileGeom<NP, TZ, TR>;
    constexpr int NM = (NP + 1) / 2;
    const Particles P = g.P;
    const float *__restrict__ E = g.E;
    const float *__restrict__ Bb = g.Bb;
    const PArgs a = g.a;
    const int32_t *__restrict__ offsets = g.offsets;
    long long begin, end;
    const bool tile_mode = bid < ntiles;
    int tz0 = 0, tr0 = 0;
    if (tile_mode) {
        const int t = bid;
        begin = offsets[(size_t)t * (TZ * TR)];
        end = offsets[(size_t)(t + 1) * (TZ * TR)];
        if (begin == end) return;
        tz0 = (t / a.ntr) * TZ;
        tr0 = (t % a.ntr) * TR;
    } else {
        const long long nsorted = g.dcount[1], np = g.dcount[0];
        begin = nsorted + (long long)(bid - ntiles) * tail_chunk;
        end = min(begin + tail_chunk, np);
        if (begin >= end) return;
    }
    const GlobAcc<NP> gacc{E, Bb, g.J, g.jdirty, g.d_epoch, a};
    const FloatAcc facc{g.Jfa, a};
    if (!tile_mode || a.nzp < 2 * G::JW) {
        // particles appended since the last sort, or a box too short for the
        // staged tile: every access goes to global memory
        for (long long idx = begin + threadIdx.x; idx < end; idx += blockDim.x) {
            const int cell = P.cell[idx];
            if (cell >= 0) gpd_global_one<NP, FA>(P, idx, cell, a, gacc, facc);
        }
        return;
    }
    const int zoff = (int)a.zoff;
    // ---- shared memory: accumulator planes, staged fields, crossing queue, particle buffers
    unsigned long long *sJ64 = sraw;                          // int64 sums of drained chunks
    unsigned *sJh = reinterpret_cast<unsigned *>(sraw + G::JPAD);   // 32-bit hi, lo planes of the chunk
    unsigned *sJl = sJh + G::JPAD;
    float4 *sf = reinterpret_cast<float4 *>(sJh + 2 * G::JPAD);
    float *queue = reinterpret_cast<float *>(sf + G::FVEC);
    int *qcount = reinterpret_cast<int *>(queue + G::QCAP * G::QW);
    float *pbuf = reinterpret_cast<float *>(qcount + 4);
    const int n = (int)(end - begin);
    const int tid = threadIdx.x;
    int32_t *const cellp = P.cell + begin;          // the tile's particles, tile-relative index
    float4 *const recp = P.rec + 2 * begin;
    // ---- each thread pushes a run of consecutive particles; the next
    // particle's words are copied to shared memory while one is pushed (the
    // first copy overlaps the staging of the fields)
    auto prefetch = [&](int b, int qi) {
        if (qi >= 0) {
            float *pb = pbuf + b * G::PB;
            float4 *pr = reinterpret_cast<float4 *>(pb + GPD_T);
            cp_async4(pb + tid, cellp + qi);
            cp_async16(pr + tid, recp + 2 * qi);
            cp_async16(pr + GPD_T + tid, recp + 2 * qi + 1);
        }
        cp_async_commit();
    };
    const int chunk = a.chunk;
    const int nch = tile_nchunks(n, chunk);
    Chunk C = tile_chunk(n, 0, chunk);
    int cnt = tid < C.nt ? C.kc : (tid == C.nt ? C.rem : 0);
    prefetch(0, cnt > 0 ? C.q0 + chunk_slot(C, tid, 0) : -1);
    // ---- stage E and Bbar of the tile and its halo; clear the accumulators
    const int col0 = tz0 - G::H - 1;
    const int row0 = tr0 - G::H - 1;
    for (int k = tid; k < G::JPAD; k += blockDim.x)               // int64 plane and both 32-bit planes
        reinterpret_cast<uint4 *>(sJ64)[k] = make_uint4(0u, 0u, 0u, 0u);
    if (tid == 0) *qcount = 0;
    // one float4 word (up to 4 mode parts of one node) per thread and pass, each
    // part copied asynchronously from its plane (zero-filled outside the grid),
    // so that all the block's copies are in flight at once (compile-time trip
    // count).  Half-r rows below the axis are copied from their mirror rows and
    // take the mode parity's sign afterwards; rows beyond the wall are copied
    // from their even image.
#pragma unroll
    for (int it = 0; it < (G::FVEC + GPD_T - 1) / GPD_T; it++) {
        const int k = it * GPD_T + (int)threadIdx.x;
        if (k >= G::FVEC) break;
        const int v = k % G::V, t1 = k / G::V;
        const int li = t1 % G::FW, t2 = t1 / G::FW, lj = t2 % G::FR, fc = t2 / G::FR;
        const int c = fc % 3, fb = fc / 3;
        int col = col0 + li;
        col = col < 0 ? col + a.nzp : (col >= a.nzp ? col - a.nzp : col);
        int j = row0 + lj;
        const bool half = hr_of(fb, c);
        if (half) {
            if (j < 0) j = -1 - j;
            if (j >= a.nr) j = 2 * a.nr - 1 - j;
        }
        const bool inside = j >= 0 && (half ? j < a.nr : j <= a.nr);
        const float *F = (fb == 0 ? E : Bb) + (size_t)(c * a.nparts + 4 * v) * a.plane +
                         (size_t)(inside ? j : 0) * a.nzp + col;
        float *dst = reinterpret_cast<float *>(sf + k);
#pragma unroll
        for (int e = 0; e < 4; e++) {
            if (4 * v + e < NP) cp_async4_zfill(dst + e, F + (size_t)e * a.plane, inside ? 4 : 0);
            else dst[e] = 0.f;
        }
    }
    cp_async_wait_all();
    if (row0 < 0) {
        // a tile on the axis: each thread signs its own words of the rows below it
#pragma unroll
        for (int it = 0; it < (G::FVEC + GPD_T - 1) / GPD_T; it++) {
            const int k = it * GPD_T + (int)threadIdx.x;
            if (k >= G::FVEC) break;
            const int v = k % G::V, t1 = k / G::V;
            const int t2 = t1 / G::FW, lj = t2 % G::FR, fc = t2 / G::FR;
            const int c = fc % 3, fb = fc / 3;
            if (row0 + lj >= 0 || !hr_of(fb, c)) continue;
            const bool longitudinal = (fb == 1 && c == 2);
            float *dst = reinterpret_cast<float *>(sf + k);
#pragma unroll
            for (int e = 0; e < 4; e++) {
                const int p = 4 * v + e, m = (p + 1) >> 1;
                if (p < NP && (((m & 1) != 0) != !longitudinal)) dst[e] = -dst[e];   // radial: (-1)^(m+1); z: (-1)^m
            }
        }
    }
    __syncthreads();
    const SmemAcc<NP, TZ, TR> sacc{sf, sJh, sJl, a.qscale};
    // can a particle of this tile be, or move, behind the moving window?  The
    // tile's staged columns are logical L0 ... L0 + FW - 1 (mod nzp); they avoid
    // the gap [nz, nzp) when L0 + FW - 1 < nz
    const bool near_gap = !a.periodic && pwrap(col0 - zoff, a.nzp) + G::FW - 1 >= a.nz;
    // the tile's staged columns do not cross the end of the circular z buffer:
    // column offsets need no wrap
    const bool flat = col0 >= 0 && col0 + G::FW <= a.nzp;
    const float q20 = a.qscale * FX_DOWN;                         // qscale 2^-20
    FastSum<NP, TZ, TR> fs;
    fs.clear();
    for (int ch = 0; ch < nch; ch++) {
        if (ch > 0) {                                              // chunks beyond the first
            C = tile_chunk(n, ch, chunk);
            cnt = tid < C.nt ? C.kc : (tid == C.nt ? C.rem : 0);
            prefetch(0, cnt > 0 ? C.q0 + chunk_slot(C, tid, 0) : -1);
        }
        int buf = 0;
        int qi = C.q0 + chunk_slot(C, tid, 0);                     // slot of this thread's k-th particle
        for (int k = 0; k < C.kc; k++) {                           // block-uniform trip count
            const int qn = qi + C.nt + (k < C.rem ? 1 : 0);         // chunk_slot(C, tid, k + 1)
            prefetch(buf ^ 1, k + 1 < cnt ? qn : -1);
            cp_async_wait_prev();                                  // this particle's words have landed
            if (k < cnt) {
                const float *pb = pbuf + buf * G::PB;
                const float4 *pr = reinterpret_cast<const float4 *>(pb + GPD_T);
                const int cell = __float_as_int(pb[tid]);
                const int iz = cell_iz(cell), jr = cell_jr(cell);
                bool act = cell >= 0;
                const int li = flat ? iz - col0 : wrapn(iz - col0, a.nzp), lj = jr - row0;
                if (act && !(li >= 1 && li <= G::FW - 2 && lj >= 1 && lj <= G::FR - 2)) {
                    gpd_global_one<NP, FA>(P, begin + qi, cell, a, gacc, facc);   // drifted beyond the halo
                    act = false;
                } else if (act && near_gap && wrapn(iz - zoff, a.nzp) >= a.nz) {
                    cellp[qi] = -1;                    // behind the moving window
                    act = false;
                }
                if (act) {
                    PState s;
                    DepIn<NM> d;
                    const float4 ra = pr[tid], rb = pr[GPD_T + tid];
                    s.oz = ra.x; s.orr = ra.y; s.cph = ra.z; s.sph = ra.w;
                    s.ux = rb.x; s.uy = rb.y; s.uz = rb.z; s.w = rb.w;
                    s.W0 = a.track_work ? P.W0[begin + qi] : 0.f;
                    s.W1 = a.track_work ? P.W1[begin + qi] : 0.f;
                    s.jr = jr;
                    push_move<NP>(sacc, a, li, lj, s, d);
                    if constexpr (FA) {
                        deposit_general<NP>(facc, a, iz, jr, d);
                    } else if (same_cell(d)) {
                        const int key = (lj << 12) | li;
                        if (key != fs.key) { fs.flush(sJh, sJl); fs.key = key; }
                        fs.add(d, d.Q * q20);
                    } else {
                        // a move across a cell boundary waits in the queue (deposited
                        // directly when the queue is full)
                        const int slot = atomicAdd(qcount, 1);
                        if (slot < G::QCAP) queue_put<NM>(queue + G::QW * slot, li, lj, d);
                        else deposit_general<NP>(sacc, a, li, lj, d);
                    }
                    const int niz = flat ? iz + s.diz : wrapn(iz + s.diz, a.nzp);
                    const bool dead = near_gap && wrapn(niz - zoff, a.nzp) >= a.nz;
                    const int ncell = dead ? -1 : make_cell(niz, jr + s.djr);
                    // at most one cell per step (the stability limit), a cell inside the
                    // grid, a slot inside the tile
                    QPIC_DCHECK(fabsf(d.dzc) < 1.f && fabsf(d.drc) < 1.f && s.diz >= -1 && s.diz <= 1 &&
                                    s.djr >= -1 && s.djr <= 1 && niz >= 0 && niz < a.nzp && jr + s.djr >= 0 &&
                                    jr + s.djr < a.nr && qi >= 0 && qi < n && li + 1 < G::JW && lj + 1 < G::JR,
                                g.err);
                    if (ncell != cell) cellp[qi] = ncell;   // most particles keep their cell
                    st_rec(recp + 2 * qi, make_float4(s.oz, s.orr, s.cph, s.sph),
                           make_float4(s.ux, s.uy, s.uz, s.w));
                    if (a.track_work) { P.W0[begin + qi] = s.W0; P.W1[begin + qi] = s.W1; }
                }
            }
            buf ^= 1;
            qi = qn;
        }
        if constexpr (!FA) {
            fs.flush(sJh, sJl);
            fs.key = -1;
            if (ch + 1 == nch) break;                              // the last chunk stays in its planes
            // drain the chunk's 32-bit planes into the int64 plane (each thread its
            // own words: no atomics), so the next chunk starts from zero
            __syncthreads();
            for (int w = tid; w < G::JWORDS; w += blockDim.x) {
                sJ64[w] += (unsigned long long)(((long long)(int)sJh[w] << FX_SHIFT) + (long long)sJl[w]);
                sJh[w] = 0u;
                sJl[w] = 0u;
            }
            __syncthreads();
        }
    }
    if constexpr (FA) return;
    // the queued cell-crossing moves, spread over all threads, into the int64
    // plane (the last chunk's sums stay in the 32-bit planes)
    __syncthreads();
    const int nq = imin(*qcount, G::QCAP);
    const SmemAcc64<NP, TZ, TR> sacc64{sJ64, a.qscale};
    for (int qq = tid; qq < nq; qq += blockDim.x) {
        int qi, qj;
        DepIn<NM> dq;
        queue_get<NM>(queue + G::QW * qq, qi, qj, dq);
        deposit_general<NP>(sacc64, a, qi, qj, dq);
    }
    __syncthreads();
    // the tile's accumulators (the int64 plane plus the last chunk's 32-bit
    // parts) go to its own scratch block with plain stores; the reduction
    // kernel sums the tiles that cover each node
    unsigned long long *dst = g.Jtile + (size_t)bid * G::JWORDS;
    for (int k = tid; k < G::JWORDS; k += blockDim.x)
        dst[k] = sJ64[k] + (unsigned long long)(((long long)(int)sJh[k] << FX_SHIFT) + (long long)sJl[k]);
    if (tid == 0) g.tstamp[bid] = *g.d_epoch;
}

template <int NP, int TZ, int TR, bool FA>
__global__ void __launch_bounds__(GPD_T, 2) k_gpd(GpdArgs g, int ntiles, int tail_chunk)
{
    extern __shared__ __align__(16) unsigned long long sraw[];
    gpd_block<NP, TZ, TR, FA>(g, blockIdx.x, ntiles, tail_chunk, sraw);
}

template <int NP, int TZ, int TR, bool FA>
static void gpd_launch2(qpic_ctx *c, const PArgs &a, int grid, int ntiles, int chunk)
{
    const size_t sm = TileGeom<NP, TZ, TR>::SMEM;
    cudaFuncSetAttribute(k_gpd<NP, TZ, TR, FA>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    const GpdArgs g{c->p, c->E, c->Bb, c->Jacc, c->Jfa, c->Jtile, c->tstamp, c->jdirty, c->d_epoch,
                    c->offsets, c->d_count, a, c->d_err};
    k_gpd<NP, TZ, TR, FA><<<grid, GPD_T, sm, c->stream>>>(g, ntiles, chunk);
}


// ------------------------------------------------------------ current reduction + decode
// One thread per node of a tile's core (its TZ x TR cells; the last tile row
// also owns the wall row j = nr) and current component, all NP parts of that
// component unrolled.  A node's current is the word of every neighbouring
// tile block (3 x 3 candidates, written this step, whose staged region covers
// the node) plus, in tiles that received global-path deposits this step (their
// mark equals the step's epoch), the global accumulator (then cleared), summed
// in a fixed order in int64 and turned into FP32 current with the per-row
// finite-volume factor.

// everything one run's current reduction reads and writes
struct JredArgs {
    const unsigned long long *Jtile;
    const int *tstamp, *d_epoch;
    unsigned long long *Jacc;
    const int *jdirty;
    float *Jf;
    const float *rowf;
    PArgs a;
    long long tile_words;
    float inv_qscale;
    int tiles_ok;
    int *err;
};

// a load of a word that another block of the same launch may have stored
// (COH: from L2, never through the non-coherent read-only path)
template <bool COH, typename T>
__device__ __forceinline__ T ld_maybe_cg(const T *p)
{
    if constexpr (COH) return __ldcg(p);
    else return *p;
}

// Work item w of tile t of the reduction: component w / (TZ TR) of node
// w % (TZ TR) of the tile's core, every row of it that the tile owns.  COH:
// the tile blocks and stamps were stored by other blocks of the same launch
// (the batched particle phase), so they are read coherently.
template <int NP, int TZ, int TR, bool COH = false>
__device__ __forceinline__ void jreduce_work(const JredArgs g, int t, int w)
{
    const unsigned long long *__restrict__ Jtile = g.Jtile;
    const int *__restrict__ tstamp = g.tstamp;
    unsigned long long *__restrict__ Jacc = g.Jacc;
    float *__restrict__ Jf = g.Jf;
    const float *__restrict__ rowf = g.rowf;
    const PArgs a = g.a;
    const long long tile_words = g.tile_words;
    const float inv_qscale = g.inv_qscale;
    const int tiles_ok = g.tiles_ok;
    int *err = g.err;
    constexpr int H = 1, JW = TZ + 2 * H + 3, JR = TR + 2 * H + 3, NN = TZ * TR;
    const int tzi = t / a.ntr, tri = t - tzi * a.ntr;
    const int tz0 = tzi * TZ, tr0 = tri * TR;
    const int comp = w / NN, node = w - comp * NN;
    const int c = node % TZ, r0 = node / TZ;
    if (c >= a.nzp - tz0) return;                          // past the last (partial) column
    const int CR = (tri == a.ntr - 1) ? a.nr + 1 - tr0 : TR;
    const int i = tz0 + c;
    const int epoch = *g.d_epoch;
    const bool dirty = ld_maybe_cg<COH>(g.jdirty + t) == epoch;
    // candidate blocks: geometry first, per z neighbour and per r neighbour
    // (3 + 3), then combined into bit masks (geo: the node lies in the
    // candidate's staged block; ok: the block was written this step); the
    // words are loaded together with the stamps (no wait between).  Offsets
    // stay 32-bit inside a block; the block's base is formed per load.
    int ztile[3], zli[3];
    unsigned zok = 0u;
#pragma unroll
    for (int e = 0; e < 3; e++) {
        int kz = tzi + e - 1;
        kz = kz < 0 ? kz + a.ntz : (kz >= a.ntz ? kz - a.ntz : kz);
        zli[e] = wrapn(i - (kz * TZ - H - 1), a.nzp);
        ztile[e] = kz * a.ntr;
        if (tiles_ok && zli[e] < JW) zok |= 1u << e;
    }
    unsigned geo = 0u, ok = 0u;
#pragma unroll
    for (int d = 0; d < 9; d++) {
        const int ez = d / 3, er = d % 3, kr = tri + er - 1;
        if (((zok >> ez) & 1u) && kr >= 0 && kr < a.ntr) {
            geo |= 1u << d;
            if (ld_maybe_cg<COH>(tstamp + ztile[ez] + kr) == epoch) ok |= 1u << d;
        }
    }
    const int cbase = comp * NP * (JR * JW);
    int l = i - (int)a.zoff;
    l = l < 0 ? l + a.nzp : l;
    const bool gap = l >= a.nz;
    for (int r = r0; r < CR; r += TR) {
        const int j = tr0 + r;
        const size_t q0 = (size_t)j * a.nzp + i;
        long long v[NP];
#pragma unroll
        for (int p = 0; p < NP; p++) v[p] = 0;
        if (dirty) {
#pragma unroll
            for (int p = 0; p < NP; p++) {
                const size_t q = (size_t)(comp * NP + p) * a.plane + q0;
                v[p] = (long long)ld_maybe_cg<COH>(Jacc + q);
                Jacc[q] = 0ull;
            }
        }
#pragma unroll
        for (int d = 0; d < 9; d++) {
            const int ez = d / 3, er = d % 3;
            const int lj = r + (1 - er) * TR + H + 1;          // row of the node in candidate d's block
            if (((geo >> d) & 1u) && lj >= 0 && lj < JR) {
                QPIC_DCHECK(cbase + lj * JW + zli[ez] + (NP - 1) * (JR * JW) < tile_words &&
                                ztile[ez] + tri + er - 1 < a.ntz * a.ntr, err);
                const unsigned long long *src = Jtile + (size_t)(ztile[ez] + tri + er - 1) * tile_words +
                                                (cbase + lj * JW + zli[ez]);
                unsigned long long w[NP];
#pragma unroll
                for (int p = 0; p < NP; p++) w[p] = ld_maybe_cg<COH>(src + p * (JR * JW));
                if ((ok >> d) & 1u) {
#pragma unroll
                    for (int p = 0; p < NP; p++) v[p] += (long long)w[p];
                }
            }
        }
        const float f0 = comp == 2 ? rowf[j] : (comp == 0 ? rowf[(a.nr + 1) + j] : rowf[3 * (a.nr + 1) + j]);
        const float f1 = comp == 1 ? rowf[2 * (a.nr + 1) + j] : f0;   // J_phi, modes m >= 1
#pragma unroll
        for (int p = 0; p < NP; p++) {
            if (v[p] > (1ll << 62) || v[p] < -(1ll << 62)) atomicOr(err, 1);   // fixed-point headroom gone
            // int64 -> float from two 32-bit halves (integer conversions stay off the FP64 pipe)
            const float fv = __int2float_rn((int)(v[p] >> 32)) * 4294967296.f +
                             __uint2float_rn((unsigned)v[p]);
            Jf[(size_t)(comp * NP + p) * a.plane + q0] = gap ? 0.f : fv * inv_qscale * (p == 0 ? f0 : f1);
        }
    }
}

// as many blocks per SM as its 2048 threads allow: the kernel is latency
// bound, and occupancy matters more than the few registers it then spills
template <int NP, int TZ, int TR>
__global__ void __launch_bounds__(3 * TZ * TR, 2048 / (3 * TZ * TR)) k_jreduce(JredArgs g)
{
    jreduce_work<NP, TZ, TR>(g, blockIdx.x, threadIdx.x);
}

// ------------------------------------------------------------ batched particle phase
// One launch advances the particle phase of every run of a batch that shares
// this mode count and tile shape.  Its work list holds first one particle
// item per (run, tile) -- gather, push and deposit of the tile -- and then one
// reduction item per (run, tile).  The blocks stay resident and take items in
// list order from a counter.  A reduction item waits until the particle items
// of the 3 x 3 tiles around it have published this step's epoch; every item
// it waits on was taken earlier by a running block and waits on nothing, so
// the waits end.  A wait gives up after ctl->spins polls: the run's error
// word gets bit 2 (reported as QPIC_ETIMEOUT) and the item is skipped.
struct BatchRun {
    GpdArgs g;
    JredArgs j;
    int *gdone;      // per tile: epoch of its last stored deposit
    int ntiles;
};

using BatchCtl = BatchCtlHost;     // spins: polls before a wait gives up; hold: item that publishes nothing

template <int TZ, int TR>
__device__ bool batch_wait(const BatchRun *R, int t, long long cap)
{
    const int ntr = R->g.a.ntr, ntz = R->g.a.ntz;
    const int tzi = t / ntr, tri = t - (t / ntr) * ntr;
    const int epoch = *R->g.d_epoch;
    long long polls = 0;
    for (int ez = -1; ez <= 1; ez++) {
        int kz = tzi + ez;
        kz = kz < 0 ? kz + ntz : (kz >= ntz ? kz - ntz : kz);
        for (int er = -1; er <= 1; er++) {
            const int kr = tri + er;
            if (kr < 0 || kr >= ntr) continue;
            const volatile int *f = R->gdone + kz * ntr + kr;
            while (*f != epoch) {
                if (++polls > cap) return false;
                __nanosleep(100);
            }
        }
    }
    return true;
}

// the run table of the launch in flight, in constant memory so that the
// kernel reads its fields like kernel parameters (copied in from a device
// table by the launching stream right before the launch)
constexpr int BATCH_MAX_RUNS = 64;
static __constant__ __align__(16) unsigned char c_batch_runs[BATCH_MAX_RUNS * sizeof(BatchRun)];

template <int NP, int TZ, int TR>
__global__ void __launch_bounds__(GPD_T, 2) k_batch_particles(const int *__restrict__ tprefix, int nruns,
                                                              int *__restrict__ head,
                                                              const BatchCtl *__restrict__ ctl)
{
    const BatchRun *runs = reinterpret_cast<const BatchRun *>(c_batch_runs);
    extern __shared__ __align__(16) unsigned long long sraw[];
    __shared__ int s_item, s_ok;
    const int total = tprefix[nruns];
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(head, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= 2 * total) return;
        const bool reduce = it >= total;
        const int k = reduce ? it - total : it;
        int lo = 0, hi = nruns;                    // tprefix[lo] <= k < tprefix[hi]
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (tprefix[mid] <= k) lo = mid; else hi = mid;
        }
        const BatchRun *R = runs + lo;
        const int t = k - tprefix[lo];
        if (!reduce) {
            gpd_block<NP, TZ, TR, false>(R->g, t, R->ntiles, 0, sraw);
            __syncthreads();                        // every store of the tile is issued
            if (threadIdx.x == 0 && it != ctl->hold) {
                __threadfence();
                atomicExch(R->gdone + t, *R->g.d_epoch);
            }
        } else {
            if (threadIdx.x == 0) s_ok = batch_wait<TZ, TR>(R, t, ctl->spins);
            __syncthreads();
            if (s_ok) {
                __threadfence();
                for (int w = threadIdx.x; w < 3 * TZ * TR; w += blockDim.x)
                    jreduce_work<NP, TZ, TR, true>(R->j, t, w);
            } else if (threadIdx.x == 0) {
                atomicOr(R->j.err, 4);
            }
        }
        __syncthreads();                            // s_item and s_ok are reused
    }
}

template <int NP, int TZ, int TR>
static void batch_particles_launch2(const BatchRun *runs, const int *tprefix, int nruns, int *head,
                                    const BatchCtl *ctl, int blocks, cudaStream_t st)
{
    const size_t sm = TileGeom<NP, TZ, TR>::SMEM;
    cudaFuncSetAttribute(k_batch_particles<NP, TZ, TR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    cudaMemcpyToSymbolAsync(c_batch_runs, runs, (size_t)nruns * sizeof(BatchRun), 0, cudaMemcpyDeviceToDevice, st);
    k_batch_particles<NP, TZ, TR><<<blocks, GPD_T, sm, st>>>(tprefix, nruns, head, ctl);
}


template <int NP, int TZ, int TR>
static void jreduce_launch(qpic_ctx *c, const PArgs &a, int tiles_ok)
{
    const JredArgs g{c->Jtile, c->tstamp, c->d_epoch, c->Jacc, c->jdirty, c->Jf, c->rowf, a,
                     (long long)gpd_tile_words(c->g.nparts, TZ, TR), 1.0f / c->qscale, tiles_ok, c->d_err};
    k_jreduce<NP, TZ, TR><<<c->ntz * c->ntr, 3 * TZ * TR, 0, c->stream>>>(g);
}


// One launch per (mode parts, tile shape): defined and explicitly
// instantiated in gpd_inst.cu, which the build compiles once per group of
// instantiations so that they compile in parallel.
template <int NP, int TZ, int TR, bool FA>
void gpd_shape(qpic_ctx *c, const PArgs &a, int grid, int ntiles, int chunk);
template <int NP, int TZ, int TR>
void jreduce_shape(qpic_ctx *c, const PArgs &a, int tiles_ok);
template <int NP, int TZ, int TR>
void batch_shape(const BatchRun *runs, const int *tprefix, int nruns, int *head, const BatchCtl *ctl,
                 int blocks, cudaStream_t st);

// the supported tile shapes (TZ x TR): 16x8, 32x8, 8x8, 16x16, 32x4
template <typename F>
inline bool tile_dispatch(int tz, int tr, F &&f)
{
    if (tz == 16 && tr == 8) f(std::integral_constant<int, 16>(), std::integral_constant<int, 8>());
    else if (tz == 32 && tr == 8) f(std::integral_constant<int, 32>(), std::integral_constant<int, 8>());
    else if (tz == 8 && tr == 8) f(std::integral_constant<int, 8>(), std::integral_constant<int, 8>());
    else if (tz == 16 && tr == 16) f(std::integral_constant<int, 16>(), std::integral_constant<int, 16>());
    else if (tz == 32 && tr == 4) f(std::integral_constant<int, 32>(), std::integral_constant<int, 4>());
    else return false;
    return true;
}

template <int NP, bool FA>
inline bool gpd_run(qpic_ctx *c, const PArgs &a, int grid, int ntiles, int chunk)
{
    return tile_dispatch(c->TZ, c->TR, [&](auto tz, auto tr) {
        gpd_shape<NP, decltype(tz)::value, decltype(tr)::value, FA>(c, a, grid, ntiles, chunk);
    });
}
template <int NP>
inline bool jreduce_run(qpic_ctx *c, const PArgs &a, int tiles_ok)
{
    return tile_dispatch(c->TZ, c->TR, [&](auto tz, auto tr) {
        jreduce_shape<NP, decltype(tz)::value, decltype(tr)::value>(c, a, tiles_ok);
    });
}
template <int NP>
inline bool batch_particles_run(int tz, int tr, const BatchRun *runs, const int *tprefix, int nruns, int *head,
                                const BatchCtl *ctl, int blocks, cudaStream_t st)
{
    return tile_dispatch(tz, tr, [&](auto z, auto r) {
        batch_shape<NP, decltype(z)::value, decltype(r)::value>(runs, tprefix, nruns, head, ctl, blocks, st);
    });
}

}  // namespace qpic
