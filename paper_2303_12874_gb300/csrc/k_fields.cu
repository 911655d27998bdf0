// k_fields.cu -- FP32 field kernels of the quasi-3D dual solver (Sec. III.A-B).
//
// Faraday and Ampere per azimuthal mode on the (z, r) Yee grid, with the
// extended z-stencils D^E_z (Faraday) and D^B_z (Ampere) of Eq. 9 and the
// cylindrical radial operators; axis rules per mode; conducting wall.
// Each block owns one r row and 128 z columns; the rows that need a z
// derivative are staged in shared memory with an L-column halo on each side
// (the z-stencil reaches L columns), every other operand is a coalesced
// global read.  These kernels are bandwidth bound (about 18 floats read and
// written per cell and part); the tensor cores have no role here.
#include <cuda_runtime.h>
#include <math.h>

#include "qpic_internal.h"

namespace qpic {

static const int FTILE = 128;     // z columns per solver block

// Coefficients live in a per-context device array [cE (MAX_L) | cB (MAX_L) |
// taps (MAX_TAPS)] (FP32 copies of the FP64 host values); blocks stage what
// they use in shared memory, so several contexts can coexist in a process.
void set_solver_constants(qpic_ctx *c)
{
    static_assert(MAX_L * 2 + MAX_TAPS <= 1024, "coefficient block size");
    float h[2 * MAX_L + MAX_TAPS] = {0};
    for (int l = 0; l < c->L; l++) { h[l] = (float)c->cE[l]; h[MAX_L + l] = (float)c->cB[l]; }
    for (size_t q = 0; q < c->taps.size(); q++) h[2 * MAX_L + q] = (float)c->taps[q];
    cudaMemcpyAsync(c->coef, h, sizeof(h), cudaMemcpyHostToDevice, c->stream);
    double h64[2 * MAX_L + MAX_TAPS];
    for (int k = 0; k < 2 * MAX_L + MAX_TAPS; k++) h64[k] = 0.0;
    for (int l = 0; l < c->L; l++) { h64[l] = c->cE[l]; h64[MAX_L + l] = c->cB[l]; }
    for (size_t q = 0; q < c->taps.size(); q++) h64[2 * MAX_L + q] = c->taps[q];
    cudaMemcpy(c->coef64, h64, sizeof(h64), cudaMemcpyHostToDevice);
}

struct GridArgs {
    int nz, nr, nzp, nparts, L;
    long long zoff;
    size_t plane;
    float dz, dr, dt, idz, idr;
    double dz64, dr64, dt64, idz64, idr64;
    const float *coef;     // [cE | cB | taps] FP32
    const double *coef64;  // the same in FP64 (plain FP64 path)
    // absorbing layer: rows j >= loss_row0 take F = alpha F + beta dt rhs with
    // [alpha(r_j), beta(r_j), alpha(r_{j+1/2}), beta(r_{j+1/2})] at
    // loss[k (nr + 1) + j] (FP32) and loss64 (FP64); loss_row0 > nr: no layer
    int loss_row0;
    const float *loss;
    const double *loss64;
};

static GridArgs grid_args(const qpic_ctx *c)
{
    GridArgs a;
    a.nz = c->g.nz; a.nr = c->g.nr; a.nzp = c->g.nzp; a.nparts = c->g.nparts; a.L = c->L;
    a.zoff = c->g.zoff % c->g.nzp; a.plane = c->g.plane;
    a.dz = (float)c->dz; a.dr = (float)c->dr; a.dt = (float)c->dt;
    a.dz64 = c->dz; a.dr64 = c->dr; a.dt64 = c->dt;
    a.idz64 = 1.0 / c->dz; a.idr64 = 1.0 / c->dr;
    a.idz = (float)a.idz64; a.idr = (float)a.idr64;
    a.coef = c->coef;
    a.coef64 = c->coef64;
    a.loss_row0 = c->nabs > 0 ? c->g.nr - c->nabs : c->g.nr + 1;
    a.loss = c->lossf;
    a.loss64 = c->loss64;
    return a;
}

// factor k (0, 1: alpha, beta at r_j; 2, 3: at r_{j+1/2}) of row j of the layer
template <typename T>
__device__ __forceinline__ T loss_at(const GridArgs &a, int k, int j)
{
    if constexpr (sizeof(T) == 8) return a.loss64[k * (a.nr + 1) + j];
    else return a.loss[k * (a.nr + 1) + j];
}

__device__ __forceinline__ int wrapz(int i, int nzp)
{
    int r = i % nzp;
    return r < 0 ? r + nzp : r;
}

// column index for i in [-nzp, 2 nzp): one wrap (staging uses it when the box
// is at least a block plus both halos wide, else wrapz)
__device__ __forceinline__ int wrap1(int i, int nzp)
{
    return i < 0 ? i + nzp : (i >= nzp ? i - nzp : i);
}

// a grid parameter in the kernel's precision (the FP32 kernels take the FP32
// copies: no conversions from FP64 on the device)
template <typename T>
__device__ __forceinline__ T gparam(float f, double d)
{
    if constexpr (sizeof(T) == 4) return f;
    else return d;
}

// true when the physical column lies in the gap of an open box
__device__ __forceinline__ bool in_gap(int col, const GridArgs &a)
{
    int l = col - (int)a.zoff;          // col, zoff in [0, nzp)
    l = l < 0 ? l + a.nzp : l;
    return l >= a.nz;
}

// mode number of a part and the (i m / r) coupling: returns the value of part p
// of (i m / r) F given both parts of F (re = F[pr], im = F[pi])
__host__ __device__ __forceinline__ int part_mode(int p) { return (p + 1) >> 1; }
__host__ __device__ __forceinline__ constexpr int imin_f(int x, int y) { return x < y ? x : y; }

// The two staged components of a solver row are interleaved per column, so one
// stencil tap reads both with one shared load; zstep adds c (hi - lo) to both
// sums (for FP32 as paired operations, same rounding as two scalar FMAs).
template <typename T> struct Pair2;
template <> struct Pair2<float> { using t = float2; };
template <> struct Pair2<double> { using t = double2; };

__device__ __forceinline__ void zstep(float2 &acc, float c, float2 hi, float2 lo)
{
    acc = __ffma2_rn(make_float2(c, c), __fadd2_rn(hi, make_float2(-lo.x, -lo.y)), acc);
}
__device__ __forceinline__ void zstep(double2 &acc, double c, double2 hi, double2 lo)
{
    acc.x = fma(c, hi.x - lo.x, acc.x);
    acc.y = fma(c, hi.y - lo.y, acc.y);
}

// sum_{l=1..L} C_l (f[l] - f[1 - l]) for both components of the pairs at f;
// LT > 0 fixes L at compile time (the stencil unrolls), LT = 0 reads it from L
template <int LT, typename T, typename V>
__device__ __forceinline__ V zdiff(const V *f, const T *C, int L)
{
    V acc;
    acc.x = 0; acc.y = 0;
    const int n = LT > 0 ? LT : L;
#pragma unroll
    for (int l = 1; l <= n; l++) zstep(acc, C[l - 1], f[l], f[1 - l]);
    return acc;
}

// The same difference in FP64 from FP32 samples and FP64 coefficients: the
// axis (r = 0) rows of the FP32 path are advanced in FP64 (their mode terms
// carry the 1/r limits), then rounded to the stored FP32 fields.
template <typename V>
__device__ __forceinline__ double2 zdiff64(const V *f, const double *C, int L)
{
    double2 acc = make_double2(0.0, 0.0);
    for (int l = 1; l <= L; l++) {
        acc.x = fma(C[l - 1], (double)f[l].x - (double)f[1 - l].x, acc.x);
        acc.y = fma(C[l - 1], (double)f[l].y - (double)f[1 - l].y, acc.y);
    }
    return acc;
}

// ---------------------------------------------------------------- Faraday
// dB/dt = -curl E:  B_r: -(i m/r) E_z + D^E_z E_phi;  B_phi: -D^E_z E_r + d_r E_z;
// B_z: -(1/r) d_r(r E_phi) + (i m/r) E_r.  Writes B^{n+1/2} and Bbar^n.  One
// block per row segment; E_phi and E_r of the row are staged with the stencil
// halo.  Each thread loads its other operands (B, E_z, row j+1) before the
// staging barrier, so both loads overlap.  P: parts (2M+1), compile time.
template <typename T, int P, int LT>
__global__ void __launch_bounds__(FTILE, sizeof(T) == 4 && P <= 3 ? 6 : 1) k_faraday(const T *__restrict__ E, T *__restrict__ B,
                                                  T *__restrict__ Bb, GridArgs a)
{
    using V = typename Pair2<T>::t;
    extern __shared__ __align__(16) unsigned char shraw[];
    T *sh = reinterpret_cast<T *>(shraw);
    const int j = blockIdx.y;
    const int i0 = blockIdx.x * FTILE;
    const int W = FTILE + 2 * a.L;
    T *sC = sh;                                    // [L] C^E
    V *sE2 = reinterpret_cast<V *>(sh + MAX_L);    // [P][W] (E_phi, E_r)
    const int i = i0 + threadIdx.x;
    const bool live = i < a.nzp;
    const bool up = j < a.nr;        // row j + 1 exists
    const size_t base = (size_t)j * a.nzp + (live ? i : 0);
    T br[P], bp[P], bz[P], ez[P], ez1[P], ep1[P];
#pragma unroll
    for (int p = 0; p < P; p++) {
        br[p] = B[(size_t)(0 * P + p) * a.plane + base];
        bp[p] = B[(size_t)(1 * P + p) * a.plane + base];
        bz[p] = B[(size_t)(2 * P + p) * a.plane + base];
        ez[p] = E[(size_t)(2 * P + p) * a.plane + base];
        ez1[p] = up ? E[(size_t)(2 * P + p) * a.plane + base + a.nzp] : (T)0;
        ep1[p] = up ? E[(size_t)(1 * P + p) * a.plane + base + a.nzp] : (T)0;
    }
    for (int k = threadIdx.x; k < a.L; k += FTILE)
        sC[k] = sizeof(T) == 8 ? (T)a.coef64[k] : (T)a.coef[k];
    const bool wide = a.nzp >= W;
    for (int k = threadIdx.x; k < W; k += FTILE) {
        const int col = wide ? wrap1(i0 - a.L + k, a.nzp) : wrapz(i0 - a.L + k, a.nzp);
#pragma unroll
        for (int p = 0; p < P; p++) {
            V v;
            v.x = E[(size_t)(1 * P + p) * a.plane + (size_t)j * a.nzp + col];
            v.y = E[(size_t)(0 * P + p) * a.plane + (size_t)j * a.nzp + col];
            sE2[p * W + k] = v;
        }
    }
    __syncthreads();
    if (!live) return;
    const bool gap = in_gap(i, a);
    const T dr = gparam<T>(a.dr, a.dr64), dt = gparam<T>(a.dt, a.dt64);
    const T idz = gparam<T>(a.idz, a.idz64), idr = gparam<T>(a.idr, a.idr64);
    const T rj = j * dr, rh = (j + (T)0.5) * dr, rj1 = (j + 1) * dr;
    // the row's reciprocals, once per thread (divisions are long sequences)
    const T irh = (T)1 / rh, irj = j > 0 ? (T)1 / rj : (T)0, irhdr = irh * idr;
    const int s = threadIdx.x + a.L;   // smem index of column i
    // absorbing layer (block-uniform): lossy update factors at r_j and r_{j+1/2}
    const bool lossy = j >= a.loss_row0;
    T aI = 1, bI = 1, aH = 1, bH = 1;
    if (lossy) { aI = loss_at<T>(a, 0, j); bI = loss_at<T>(a, 1, j); aH = loss_at<T>(a, 2, j); bH = loss_at<T>(a, 3, j); }
#pragma unroll
    for (int p = 0; p < P; p++) {
        const int m = part_mode(p);
        const bool isim = (p > 0) && !(p & 1);
        const int pr = isim ? p - 1 : p, pim = isim ? p : imin_f(p + 1, P - 1);   // re / im partner
        // D^E_z of E_phi and E_r at i + 1/2: sum_l C_l (f_{i+l} - f_{i+1-l})
        const V dE = zdiff<LT>(sE2 + p * W + s, sC, a.L);
        const T dEphi = dE.x * idz, dEr = dE.y * idz;
        // B_r at (i+1/2, j)
        T d;
        if (j == 0) {
            // m = 1: -(i/r) E_z -> -i E_z^1(dr)/dr on the axis; m != 1: 0
            d = m == 1 ? (isim ? -ez1[pr] : ez1[pim]) * idr + dEphi : (T)0;
        } else {
            const T imr = m > 0 ? (isim ? ez[pr] : -ez[pim]) * ((T)m * irj) : (T)0;   // (i m / r) E_z
            d = -imr + dEphi;
        }
        {
            const size_t q = (size_t)(0 * P + p) * a.plane + base;
            if (sizeof(T) == 4 && j == 0 && m == 1) {
                // the axis term in FP64 on the FP32 path (dE_phi again from the staged row)
                const double d64 = (double)(isim ? -ez1[pr] : ez1[pim]) * a.idr64 +
                                   zdiff64(sE2 + p * W + s, a.coef64, a.L).x * a.idz64;
                const double b64 = lossy ? a.loss64[j] * (double)br[p] + a.loss64[(a.nr + 1) + j] * (a.dt64 * d64)
                                         : (double)br[p] + a.dt64 * d64;
                B[q] = gap ? (T)0 : (T)b64;
                Bb[q] = gap ? (T)0 : (T)(0.5 * ((double)br[p] + b64));
            } else {
                const T bn = gap ? (T)0 : (lossy ? aI * br[p] + bI * (dt * d) : br[p] + dt * d);
                B[q] = bn; Bb[q] = gap ? (T)0 : (T)0.5 * (br[p] + bn);
            }
        }
        if (up) {
            // B_phi at (i+1/2, j+1/2)
            d = -dEr + (ez1[p] - ez[p]) * idr;
            size_t q = (size_t)(1 * P + p) * a.plane + base;
            T bn = gap ? (T)0 : (lossy ? aH * bp[p] + bH * (dt * d) : bp[p] + dt * d);
            B[q] = bn; Bb[q] = gap ? (T)0 : (T)0.5 * (bp[p] + bn);
            // B_z at (i, j+1/2); E_phi(j) and E_r(j) from the staged row
            const T imr = m > 0 ? (isim ? sE2[pr * W + s].y : -sE2[pim * W + s].y) * ((T)m * irh) : (T)0;
            d = -(rj1 * ep1[p] - rj * sE2[p * W + s].x) * irhdr + imr;
            q = (size_t)(2 * P + p) * a.plane + base;
            bn = gap ? (T)0 : (lossy ? aH * bz[p] + bH * (dt * d) : bz[p] + dt * d);
            B[q] = bn; Bb[q] = gap ? (T)0 : (T)0.5 * (bz[p] + bn);
        } else {
            // half-r row beyond the wall: not advanced; its average is the value itself
            Bb[(size_t)(1 * P + p) * a.plane + base] = gap ? (T)0 : bp[p];
            Bb[(size_t)(2 * P + p) * a.plane + base] = gap ? (T)0 : bz[p];
        }
    }
}

// the dual solver's 16 coefficients get an unrolled FP32 stencil; other L
// (and the plain FP64 path) the generic loop
template <typename T, int P>
static void faraday_launch(const GridArgs &a, dim3 grid, size_t sm, cudaStream_t st, const T *E, T *B, T *Bb)
{
    if constexpr (sizeof(T) == 4) {
        if (a.L == 16) {
            k_faraday<T, P, 16><<<grid, FTILE, sm, st>>>(E, B, Bb, a);
            return;
        }
    }
    k_faraday<T, P, 0><<<grid, FTILE, sm, st>>>(E, B, Bb, a);
}

template <typename T>
static void faraday_dispatch(const GridArgs &a, dim3 grid, size_t sm, cudaStream_t st, const T *E, T *B, T *Bb)
{
    switch (a.nparts) {
    case 1: faraday_launch<T, 1>(a, grid, sm, st, E, B, Bb); break;
    case 3: faraday_launch<T, 3>(a, grid, sm, st, E, B, Bb); break;
    case 5: faraday_launch<T, 5>(a, grid, sm, st, E, B, Bb); break;
    default: faraday_launch<T, 7>(a, grid, sm, st, E, B, Bb); break;
    }
}

void launch_faraday(qpic_ctx *c)
{
    GridArgs a = grid_args(c);
    dim3 grid((a.nzp + FTILE - 1) / FTILE, a.nr + 1);
    prof_begin(c);
    if (c->fp64) {
        size_t sm = (MAX_L + (size_t)2 * a.nparts * (FTILE + 2 * a.L)) * sizeof(double);
        faraday_dispatch<double>(a, grid, sm, c->stream, c->E64, c->B64, c->Bb64);
    } else {
        size_t sm = (MAX_L + (size_t)2 * a.nparts * (FTILE + 2 * a.L)) * sizeof(float);
        faraday_dispatch<float>(a, grid, sm, c->stream, c->E, c->B, c->Bb);
    }
    prof_end(c, KC_FARADAY);
}

// ---------------------------------------------------------------- J_z filter
// J_z <- K * J_z along z (symbol [k]_Yee/[k]_B): keeps Gauss's law in the dual
// form when the deposit satisfies the two-point continuity equation.
// Each thread filters JF_R = 8 consecutive columns.  The taps beyond the centre
// are taken 8 at a time: the 16 columns on each side that 8 outputs x 8 taps
// touch are read into registers with aligned vector loads and the products are
// added in tap order, right + left side first (the symmetric stencil).  The
// halo is rounded up to whole blocks of 8 taps, with 0 for the taps past the
// last.  A block covers JF_T * JF_R columns of one row and part.
static const int JF_T = 128;     // threads per filter block
static const int JF_R = 8;       // columns per thread, taps per block

__device__ __forceinline__ void ld8(const float *p, float x[8])
{
    const float4 *v = reinterpret_cast<const float4 *>(p);
#pragma unroll
    for (int k = 0; k < 2; k++) {
        const float4 t = v[k];
        x[4 * k] = t.x; x[4 * k + 1] = t.y; x[4 * k + 2] = t.z; x[4 * k + 3] = t.w;
    }
}
__device__ __forceinline__ void ld8(const double *p, double x[8])
{
    const double2 *v = reinterpret_cast<const double2 *>(p);
#pragma unroll
    for (int k = 0; k < 4; k++) {
        const double2 t = v[k];
        x[2 * k] = t.x; x[2 * k + 1] = t.y;
    }
}

template <typename T>
__global__ void __launch_bounds__(JF_T) k_jfilter(const T *__restrict__ Jf, T *__restrict__ Jzf,
                                                 GridArgs a, int nk)
{
    extern __shared__ __align__(16) unsigned char shraw2[];
    T *sh2 = reinterpret_cast<T *>(shraw2);
    const int j = blockIdx.y, p = blockIdx.z;
    const int i0 = blockIdx.x * (JF_T * JF_R);
    const int nb = (nk - 1 + JF_R - 1) / JF_R;          // blocks of 8 taps beyond the centre
    const int H = nb * JF_R, W = JF_T * JF_R + 2 * H;
    T *sT = sh2, *sh = sh2 + MAX_TAPS;                  // sT[k]: tap k + 1, 0 past the last
    for (int k = threadIdx.x; k < H; k += JF_T)
        sT[k] = k + 1 < nk ? (sizeof(T) == 8 ? (T)a.coef64[2 * MAX_L + k + 1] : (T)a.coef[2 * MAX_L + k + 1])
                           : (T)0;
    const T c0 = sizeof(T) == 8 ? (T)a.coef64[2 * MAX_L] : (T)a.coef[2 * MAX_L];
    const T *src = Jf + (size_t)(2 * a.nparts + p) * a.plane + (size_t)j * a.nzp;
    const bool wide = a.nzp >= W;
    for (int k = threadIdx.x; k < W; k += JF_T)
        sh[k] = src[wide ? wrap1(i0 - H + k, a.nzp) : wrapz(i0 - H + k, a.nzp)];
    __syncthreads();
    const int ib = i0 + threadIdx.x * JF_R;
    if (ib >= a.nzp) return;
    const int s = threadIdx.x * JF_R + H;               // smem index of column ib, a multiple of 8
    T acc[JF_R];
    {
        T x[8];
        ld8(sh + s, x);
#pragma unroll
        for (int r = 0; r < JF_R; r++) acc[r] = c0 * x[r];
    }
    for (int b = 0; b < nb; b++) {
        const int q0 = b * JF_R;                         // taps q0 + 1 .. q0 + 8
        T X[16], Y[16], c[8];
        ld8(sh + s + q0, X); ld8(sh + s + q0 + 8, X + 8);    // X[k]: column ib + q0 + k
        ld8(sh + s - q0 - 8, Y); ld8(sh + s - q0, Y + 8);    // Y[k]: column ib - q0 - 8 + k
        ld8(sT + q0, c);
#pragma unroll
        for (int t = 0; t < JF_R; t++)                   // tap q = q0 + 1 + t
#pragma unroll
            for (int r = 0; r < JF_R; r++) acc[r] += c[t] * (X[r + t + 1] + Y[r - t + 7]);
    }
    T *dst = Jzf + (size_t)p * a.plane + (size_t)j * a.nzp;
#pragma unroll
    for (int r = 0; r < JF_R; r++) {
        const int i = ib + r;
        if (i < a.nzp) dst[i] = in_gap(i, a) ? (T)0 : acc[r];
    }
}

void launch_jfilter(qpic_ctx *c)
{
    GridArgs a = grid_args(c);
    int nk = (int)c->taps.size();
    const int H = (nk - 1 + JF_R - 1) / JF_R * JF_R;
    dim3 grid((a.nzp + JF_T * JF_R - 1) / (JF_T * JF_R), a.nr + 1, a.nparts);
    prof_begin(c);
    if (c->fp64) {
        size_t sm = (size_t)(MAX_TAPS + JF_T * JF_R + 2 * H) * sizeof(double);
        k_jfilter<double><<<grid, JF_T, sm, c->stream>>>(c->J64, c->Jz64, a, nk);
    } else {
        size_t sm = (size_t)(MAX_TAPS + JF_T * JF_R + 2 * H) * sizeof(float);
        k_jfilter<float><<<grid, JF_T, sm, c->stream>>>(c->Jf, c->Jzf, a, nk);
    }
    prof_end(c, KC_JFILTER);
}

// ---------------------------------------------------------------- Ampere
// dE/dt = curl B - J:  E_r: (i m/r) B_z - D^B_z B_phi - J_r;
// E_phi: D^B_z B_r - d_r B_z - J_phi;  E_z: (1/r) d_r(r B_phi) - (i m/r) B_r - J_z.
// Axis: m = 0: E_phi = 0, E_z uses 4 B_phi(dr/2)/dr; m = 1: E_z = 0,
// d_r B_z(0) = 2 B_z(dr/2)/dr; m >= 2: 0.  Wall: E_phi = E_z = 0.
// B_phi and B_r of the row are staged with the stencil halo; each thread loads
// its other operands (E, J, B_z, row j - 1) before the staging barrier.
template <typename T, int P, int LT>
__global__ void __launch_bounds__(FTILE, sizeof(T) == 4 && P <= 3 ? 6 : 1) k_ampere(T *__restrict__ E, const T *__restrict__ B,
                                                 const T *__restrict__ Jf,
                                                 const T *__restrict__ Jz, GridArgs a)
{
    using V = typename Pair2<T>::t;
    extern __shared__ __align__(16) unsigned char shraw[];
    T *sh = reinterpret_cast<T *>(shraw);
    const int j = blockIdx.y;
    const int i0 = blockIdx.x * FTILE;
    const int W = FTILE + 2 * a.L;
    T *sC = sh;                                    // [L] C^B
    V *sB2 = reinterpret_cast<V *>(sh + MAX_L);    // [P][W] (B_phi, B_r)
    const int i = i0 + threadIdx.x;
    const bool live = i < a.nzp;
    const bool down = j > 0;             // row j - 1 exists
    const size_t base = (size_t)j * a.nzp + (live ? i : 0);
    T er[P], ep[P], ez[P], jr[P], jp[P], jz[P], bz[P], bzm[P], bpm[P];
#pragma unroll
    for (int p = 0; p < P; p++) {
        er[p] = E[(size_t)(0 * P + p) * a.plane + base];
        ep[p] = E[(size_t)(1 * P + p) * a.plane + base];
        ez[p] = E[(size_t)(2 * P + p) * a.plane + base];
        jr[p] = Jf[(size_t)(0 * P + p) * a.plane + base];
        jp[p] = Jf[(size_t)(1 * P + p) * a.plane + base];
        jz[p] = Jz[(size_t)p * a.plane + base];
        bz[p] = B[(size_t)(2 * P + p) * a.plane + base];
        bzm[p] = down ? B[(size_t)(2 * P + p) * a.plane + base - a.nzp] : (T)0;
        bpm[p] = down ? B[(size_t)(1 * P + p) * a.plane + base - a.nzp] : (T)0;
    }
    for (int k = threadIdx.x; k < a.L; k += FTILE)
        sC[k] = sizeof(T) == 8 ? (T)a.coef64[MAX_L + k] : (T)a.coef[MAX_L + k];
    const bool wide = a.nzp >= W;
    for (int k = threadIdx.x; k < W; k += FTILE) {
        const int col = wide ? wrap1(i0 - a.L + k, a.nzp) : wrapz(i0 - a.L + k, a.nzp);
#pragma unroll
        for (int p = 0; p < P; p++) {
            V v;
            v.x = B[(size_t)(1 * P + p) * a.plane + (size_t)j * a.nzp + col];
            v.y = B[(size_t)(0 * P + p) * a.plane + (size_t)j * a.nzp + col];
            sB2[p * W + k] = v;
        }
    }
    __syncthreads();
    if (!live) return;
    const bool gap = in_gap(i, a);
    const T dr = gparam<T>(a.dr, a.dr64), dt = gparam<T>(a.dt, a.dt64);
    const T idz = gparam<T>(a.idz, a.idz64), idr = gparam<T>(a.idr, a.idr64);
    const T rj = j * dr, rh = (j + (T)0.5) * dr, rl = (j - (T)0.5) * dr;
    const T irh = (T)1 / rh, irj = j > 0 ? (T)1 / rj : (T)0, irjdr = irj * idr;
    const int s = threadIdx.x + a.L;
    const bool lossy = j >= a.loss_row0;           // absorbing layer (block-uniform)
    T aI = 1, bI = 1, aH = 1, bH = 1;
    if (lossy) { aI = loss_at<T>(a, 0, j); bI = loss_at<T>(a, 1, j); aH = loss_at<T>(a, 2, j); bH = loss_at<T>(a, 3, j); }
    // the lossy update of an FP64 axis term on the FP32 path
    const double aI64 = lossy ? a.loss64[j] : 1.0, bI64 = lossy ? a.loss64[(a.nr + 1) + j] : 1.0;
#pragma unroll
    for (int p = 0; p < P; p++) {
        const int m = part_mode(p);
        const bool isim = (p > 0) && !(p & 1);
        const int pr = isim ? p - 1 : p, pim = isim ? p : imin_f(p + 1, P - 1);
        // D^B_z of B_phi and B_r at integer i: sum_l C_l (f_{i+l-1/2} - f_{i-l+1/2})
        const V dB = zdiff<LT>(sB2 + p * W + s - 1, sC, a.L);
        const T dBphi = dB.x * idz, dBr = dB.y * idz;
        // E_r at (i, j+1/2)
        if (j < a.nr) {
            const T imr = m > 0 ? (isim ? bz[pr] : -bz[pim]) * ((T)m * irh) : (T)0;
            const T d = imr - dBphi - jr[p];
            E[(size_t)(0 * P + p) * a.plane + base] = gap ? (T)0 : (lossy ? aH * er[p] + bH * (dt * d) : er[p] + dt * d);
        }
        // E_phi at (i, j)
        {
            T v;
            if (j == a.nr || (j == 0 && m != 1)) v = 0;
            else if (j == 0 && sizeof(T) == 4) {        // the axis term in FP64
                const double dtd = a.dt64 * (zdiff64(sB2 + p * W + s - 1, a.coef64 + MAX_L, a.L).y * a.idz64 -
                                             2.0 * (double)bz[p] * a.idr64 - (double)jp[p]);
                v = (T)(lossy ? aI64 * (double)ep[p] + bI64 * dtd : (double)ep[p] + dtd);
            } else if (j == 0) {
                const T d = dBr - (T)2 * bz[p] * idr - jp[p];
                v = lossy ? aI * ep[p] + bI * (dt * d) : ep[p] + dt * d;
            } else {
                const T d = dBr - (bz[p] - bzm[p]) * idr - jp[p];
                v = lossy ? aI * ep[p] + bI * (dt * d) : ep[p] + dt * d;
            }
            E[(size_t)(1 * P + p) * a.plane + base] = gap ? (T)0 : v;
        }
        // E_z at (i+1/2, j); B_phi(j) and B_r(j) from the staged row
        {
            const T bp0 = sB2[p * W + s].x;
            T v;
            if (j == a.nr || (j == 0 && m != 0)) {
                v = 0;
            } else if (j == 0) {                       // the axis term in FP64 on the FP32 path
                if (sizeof(T) == 4) {
                    const double dtd = a.dt64 * (4.0 * (double)bp0 * a.idr64 - (double)jz[p]);
                    v = (T)(lossy ? aI64 * (double)ez[p] + bI64 * dtd : (double)ez[p] + dtd);
                } else {
                    const T d = (T)4 * bp0 * idr - jz[p];
                    v = lossy ? aI * ez[p] + bI * (dt * d) : ez[p] + dt * d;
                }
            } else {
                const T imr = m > 0 ? (isim ? sB2[pr * W + s].y : -sB2[pim * W + s].y) * ((T)m * irj) : (T)0;
                const T d = (rh * bp0 - rl * bpm[p]) * irjdr - imr - jz[p];
                v = lossy ? aI * ez[p] + bI * (dt * d) : ez[p] + dt * d;
            }
            E[(size_t)(2 * P + p) * a.plane + base] = gap ? (T)0 : v;
        }
    }
}

template <typename T, int P>
static void ampere_launch(const GridArgs &a, dim3 grid, size_t sm, cudaStream_t st, T *E, const T *B,
                          const T *J, const T *Jz)
{
    if constexpr (sizeof(T) == 4) {
        if (a.L == 16) {
            k_ampere<T, P, 16><<<grid, FTILE, sm, st>>>(E, B, J, Jz, a);
            return;
        }
    }
    k_ampere<T, P, 0><<<grid, FTILE, sm, st>>>(E, B, J, Jz, a);
}

template <typename T>
static void ampere_dispatch(const GridArgs &a, dim3 grid, size_t sm, cudaStream_t st, T *E, const T *B,
                            const T *J, const T *Jz)
{
    switch (a.nparts) {
    case 1: ampere_launch<T, 1>(a, grid, sm, st, E, B, J, Jz); break;
    case 3: ampere_launch<T, 3>(a, grid, sm, st, E, B, J, Jz); break;
    case 5: ampere_launch<T, 5>(a, grid, sm, st, E, B, J, Jz); break;
    default: ampere_launch<T, 7>(a, grid, sm, st, E, B, J, Jz); break;
    }
}

void launch_ampere(qpic_ctx *c)
{
    GridArgs a = grid_args(c);
    dim3 grid((a.nzp + FTILE - 1) / FTILE, a.nr + 1);
    prof_begin(c);
    if (c->fp64) {
        size_t sm = (MAX_L + (size_t)2 * a.nparts * (FTILE + 2 * a.L)) * sizeof(double);
        const double *jz = c->taps.empty() ? c->J64 + (size_t)2 * a.nparts * a.plane : c->Jz64;
        ampere_dispatch<double>(a, grid, sm, c->stream, c->E64, c->B64, c->J64, jz);
    } else {
        size_t sm = (MAX_L + (size_t)2 * a.nparts * (FTILE + 2 * a.L)) * sizeof(float);
        const float *jz = c->taps.empty() ? c->Jf + (size_t)2 * a.nparts * a.plane : c->Jzf;
        ampere_dispatch<float>(a, grid, sm, c->stream, c->E, c->B, c->Jf, jz);
    }
    prof_end(c, KC_AMPERE);
}

// ---------------------------------------------------------------- window column
template <typename T>
__global__ void k_zero_column(T *E, T *B, T *Bb, T *Jf, T *Jzf, int col, GridArgs a, int nplanes,
                              int nzf)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int pl = blockIdx.y;
    if (j > a.nr) return;
    size_t q = (size_t)pl * a.plane + (size_t)j * a.nzp + col;
    E[q] = 0; B[q] = 0; Bb[q] = 0; Jf[q] = 0;
    if (pl < nzf) Jzf[q] = 0;
}

void launch_zero_column(qpic_ctx *c, long long phys_col)
{
    GridArgs a = grid_args(c);
    int np = 3 * a.nparts;
    dim3 grid((a.nr + 1 + 127) / 128, np);
    prof_begin(c);
    if (c->fp64)
        k_zero_column<double><<<grid, 128, 0, c->stream>>>(c->E64, c->B64, c->Bb64, c->J64, c->Jz64,
                                                           (int)(phys_col % a.nzp), a, np, a.nparts);
    else
        k_zero_column<float><<<grid, 128, 0, c->stream>>>(c->E, c->B, c->Bb, c->Jf, c->Jzf,
                                                          (int)(phys_col % a.nzp), a, np, a.nparts);
    prof_end(c, KC_WINDOW);
}

// ---------------------------------------------------------------- laser
// Paraxial Gaussian beam (Eq. 18 near focus), evaluated in FP64 per grid point:
// q = (z - z_f) - i zR, zR = w0^2/2, A = (-i zR/q) exp(i r^2/(2q)),
// Ex_c = a0 env(xi) (-i) A e^{i(xi + (1-omega) t)}, xi = z - z_c - t,
// env = exp(-2 ln2 xi^2/fwhm^2); E_x = Re Ex_c, E_z = Re(-(x/q) Ex_c),
// B_y = E_x, B_z = Re(-(y/q) Ex_c).  m = 1 amplitudes (polarisation psi):
// E_r = Ex/2, E_phi = i Ex/2, E_z = r h/2, B_r = -i By/2, B_phi = By/2,
// B_z = -i r h/2 with h = Re(-Ex_c/q), all times e^{-i psi}.
struct LaserArgs {
    double a0, w0, fwhm, zc, zf, psi, omega, ratio, zmin, Lz, dz, dr, dt;
    int periodic;
};

__device__ void laser_core(const LaserArgs &L, double z, double r, double t, double *exr,
                           double *hr)
{
    double xi = z - L.zc - t;
    if (L.periodic) {
        xi = fmod(xi + 0.5 * L.Lz, L.Lz);
        if (xi < 0) xi += L.Lz;
        xi -= 0.5 * L.Lz;
    }
    double env = exp(-2.0 * 0.69314718055994530942 * xi * xi / (L.fwhm * L.fwhm));
    double zR = 0.5 * L.w0 * L.w0;
    double qr = z - L.zf, qi = -zR;                      // q = qr + i qi
    double qq = qr * qr + qi * qi;
    // 1/q = (qr - i qi)/|q|^2 ; i r^2 / (2q) = i r^2 (qr - i qi) / (2|q|^2)
    double er = r * r * qi / (2.0 * qq);                  // real part of i r^2/(2q)
    double ei = r * r * qr / (2.0 * qq);                  // imag part
    double mag = exp(er);
    double cr = mag * cos(ei), ci = mag * sin(ei);        // exp(i r^2/(2q))
    // -i zR / q = -i zR (qr - i qi)/qq = (-zR qi - i zR qr)/qq
    double pr_ = -zR * qi / qq, pi_ = -zR * qr / qq;
    double Ar = pr_ * cr - pi_ * ci, Ai = pr_ * ci + pi_ * cr;
    // (-i) A = Ai - i Ar
    double Br_ = Ai, Bi_ = -Ar;
    double ph = xi + (1.0 - L.omega) * t;
    double sr = cos(ph), si = sin(ph);
    double exc_r = L.a0 * env * (Br_ * sr - Bi_ * si);
    double exc_i = L.a0 * env * (Br_ * si + Bi_ * sr);
    *exr = exc_r;
    // h = Re(-Ex_c / q) = -Re(Ex_c (qr - i qi))/qq = -(exc_r qr + exc_i qi)/qq
    *hr = -(exc_r * qr + exc_i * qi) / qq;
}

template <typename T>
__global__ void k_laser(T *E, T *B, GridArgs a, LaserArgs L)
{
    const int il = blockIdx.x * blockDim.x + threadIdx.x;     // logical column
    const int j = blockIdx.y;
    if (il >= a.nz) return;
    const int col = wrapz(il + (int)a.zoff, a.nzp);
    const size_t base = (size_t)j * a.nzp + col;
    const int P = a.nparts;
    const double cp = cos(L.psi), sp = -sin(L.psi);           // e^{-i psi}
    const double zi = L.zmin + il * L.dz, zh = zi + 0.5 * L.dz;
    const double ri = j * L.dr, rh = (j + 0.5) * L.dr;
    double ex, h;
    // value (vr + i vi) * e^{-i psi} added to mode-1 planes of component comp
    auto add = [&](T *F, int comp, double vr, double vi, bool zero) {
        if (zero) return;
        double wr = vr * cp - vi * sp, wi = vr * sp + vi * cp;
        F[(size_t)(comp * P + 1) * a.plane + base] += (T)wr;
        F[(size_t)(comp * P + 2) * a.plane + base] += (T)wi;
    };
    const bool wall = (j == a.nr);
    // E at t = 0
    laser_core(L, zi, rh, 0.0, &ex, &h);
    add(E, 0, 0.5 * ex, 0.0, wall);                           // E_r (i, j+1/2)
    laser_core(L, zi, ri, 0.0, &ex, &h);
    add(E, 1, 0.0, 0.5 * ex, wall);                           // E_phi (i, j)
    laser_core(L, zh, ri, 0.0, &ex, &h);
    add(E, 2, 0.5 * ri * h, 0.0, wall || j == 0);             // E_z (i+1/2, j)
    // B at t = -dt/2, times the discrete B/E ratio
    const double t = -0.5 * L.dt, R = L.ratio;
    laser_core(L, zh, ri, t, &ex, &h);
    add(B, 0, 0.0, -0.5 * ex * R, wall);                      // B_r (i+1/2, j)
    laser_core(L, zh, rh, t, &ex, &h);
    add(B, 1, 0.5 * ex * R, 0.0, wall);                       // B_phi (i+1/2, j+1/2)
    laser_core(L, zi, rh, t, &ex, &h);
    add(B, 2, 0.0, -0.5 * rh * h * R, wall);                  // B_z (i, j+1/2)
}

void launch_laser(qpic_ctx *c, double a0, double w0, double fwhm, double zc, double zf, double psi)
{
    GridArgs a = grid_args(c);
    LaserArgs L;
    L.a0 = a0; L.w0 = w0; L.fwhm = fwhm; L.zc = zc; L.zf = zf; L.psi = psi;
    L.omega = 2.0 / c->dt * asin(0.5 * c->dt * sqrt(c->kE1 * c->kB1));
    L.ratio = sqrt(c->kE1 / c->kB1);
    L.zmin = c->shifts * c->dz; L.Lz = c->g.nz * c->dz; L.dz = c->dz; L.dr = c->dr; L.dt = c->dt;
    L.periodic = c->g.periodic;
    dim3 grid((a.nz + 127) / 128, a.nr + 1);
    prof_begin(c);
    if (c->fp64) k_laser<double><<<grid, 128, 0, c->stream>>>(c->E64, c->B64, a, L);
    else k_laser<float><<<grid, 128, 0, c->stream>>>(c->E, c->B, a, L);
    prof_end(c, KC_OTHER);
}

// ---------------------------------------------------------------- field energy (FP64)
// 1/2 sum V(r_loc) (|E|^2 + |B|^2) per mode, each component at its own radius,
// modes m >= 1 counted twice.  Deterministic two-pass reduction.
template <typename T>
__global__ void k_energy_partial(const T *E, const T *B, GridArgs a, double *part)
{
    __shared__ double red[256];
    const int j = blockIdx.y, m = blockIdx.z;
    const double PI = 3.14159265358979323846;
    const double dr = a.dr64, dz = a.dz64, R = a.nr * dr;
    double Vi, Vh;
    if (j == 0) Vi = PI * 0.25 * dr * dr * dz;
    else if (j == a.nr) Vi = PI * (R * R - (R - 0.5 * dr) * (R - 0.5 * dr)) * dz;
    else Vi = 2.0 * PI * j * dr * dr * dz;
    Vh = (j < a.nr) ? 2.0 * PI * (j + 0.5) * dr * dr * dz : 0.0;
    double s = 0.0;
    if constexpr (sizeof(T) == 8) {
        for (int il = blockIdx.x * blockDim.x + threadIdx.x; il < a.nz; il += gridDim.x * blockDim.x) {
            int col = wrapz(il + (int)a.zoff, a.nzp);
            size_t base = (size_t)j * a.nzp + col;
            for (int k = 0; k < (m ? 2 : 1); k++) {
                int p = m ? 2 * m - 1 + k : 0;
                auto v2 = [&](const T *F, int comp) {
                    double x = F[(size_t)(comp * a.nparts + p) * a.plane + base];
                    return x * x;
                };
                s += Vh * (v2(E, 0) + v2(B, 1) + v2(B, 2)) + Vi * (v2(E, 1) + v2(E, 2) + v2(B, 0));
            }
        }
    } else {
        // FP32 fields: squares summed per row class in double-float (FP64-grade,
        // on the FP32 pipe), weighted by the row's volumes in FP64 at the end
        DFAcc sh_, si_;
        for (int il = blockIdx.x * blockDim.x + threadIdx.x; il < a.nz; il += gridDim.x * blockDim.x) {
            const int col = wrapz(il + (int)a.zoff, a.nzp);
            const size_t base = (size_t)j * a.nzp + col;
            for (int k = 0; k < (m ? 2 : 1); k++) {
                const int p = m ? 2 * m - 1 + k : 0;
                auto f = [&](const T *F, int comp) { return (float)F[(size_t)(comp * a.nparts + p) * a.plane + base]; };
                const float er = f(E, 0), bp = f(B, 1), bz = f(B, 2);
                const float ep = f(E, 1), ez = f(E, 2), br = f(B, 0);
                sh_.add_prod(er, er); sh_.add_prod(bp, bp); sh_.add_prod(bz, bz);
                si_.add_prod(ep, ep); si_.add_prod(ez, ez); si_.add_prod(br, br);
            }
        }
        s = Vh * sh_.value() + Vi * si_.value();
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        part[((size_t)m * gridDim.y + j) * gridDim.x + blockIdx.x] = red[0] * (m ? 1.0 : 0.5);
}

// one block per segment: each thread sums a fixed strided subset, then a
// fixed-shape tree (the order of every addition is fixed: deterministic)
__global__ void k_sum_ordered(const double *part, int n_per, int nseg, double *out)
{
    __shared__ double red[256];
    const int sgm = blockIdx.x;
    double s = 0.0;
    for (int k = threadIdx.x; k < n_per; k += 256) s += part[(size_t)sgm * n_per + k];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[sgm] = red[0];
}

void launch_field_energy(qpic_ctx *c, double *out_modes)
{
    GridArgs a = grid_args(c);
    const int nm = c->g.nm, nbx = 4;
    dim3 grid(nbx, a.nr + 1, nm);
    size_t need = (size_t)nbx * (a.nr + 1) * nm + nm;
    if ((size_t)c->red_cap < need) return;
    prof_begin(c);
    if (c->fp64) k_energy_partial<double><<<grid, 256, 0, c->stream>>>(c->E64, c->B64, a, c->d_red);
    else k_energy_partial<float><<<grid, 256, 0, c->stream>>>(c->E, c->B, a, c->d_red);
    k_sum_ordered<<<nm, 256, 0, c->stream>>>(c->d_red, nbx * (a.nr + 1), nm, c->d_red + need - nm);
    prof_end(c, KC_DIAG, 2);
    // out_modes holds the energies once the stream has passed the copy (the
    // caller synchronises)
    cudaMemcpyAsync(out_modes, c->d_red + need - nm, nm * sizeof(double), cudaMemcpyDeviceToHost,
                    c->stream);
}

}  // namespace qpic

namespace qpic {

// ---------------------------------------------------------------- Gauss residual
// R_m(i,j) = div_B E_m - (rho_e + rho_ion)_m with the finite-volume divergence
// (r_{j+1/2} E_r(j+1/2) - r_{j-1/2} E_r(j-1/2))/(r_j dr) + (i m/r_j) E_phi + D^B_z E_z
// (4 E_r(dr/2)/dr on the axis for m = 0).  Nodes on the conductor and the
// m >= 1 axis node are excluded.  Per mode: sum |R|^2 and sum |rho_net|^2.
// rho planes: [nm][2][nr+1][nz] in logical order.
template <typename T>
__global__ void k_gauss_partial(const T *E, const double *rho_e, const double *rho_ion, GridArgs a,
                                int nm, double *part)
{
    __shared__ double s0[256], s1[256];
    const int j = blockIdx.y, m = blockIdx.z;
    const int nz = a.nz;
    double sr = 0.0, sq = 0.0;
    const double dr = a.dr64, dz = a.dz64;
    for (int il = blockIdx.x * blockDim.x + threadIdx.x; il < nz; il += gridDim.x * blockDim.x) {
        if (j >= a.nr || (j == 0 && m > 0)) break;
        const int col = wrapz(il + (int)a.zoff, a.nzp);
        double dre = 0.0, dim = 0.0;
        for (int q = 0; q < (m ? 2 : 1); q++) {
            const int p = m ? 2 * m - 1 + q : 0;
            const T *Er = E + (size_t)(0 * a.nparts + p) * a.plane;
            const T *Ez = E + (size_t)(2 * a.nparts + p) * a.plane;
            double v;
            if (j == 0) {
                v = 4.0 * (double)Er[col] / dr;
            } else {
                const double rp = (j + 0.5) * dr, rm = (j - 0.5) * dr, rj = j * dr;
                v = (rp * (double)Er[(size_t)j * a.nzp + col] - rm * (double)Er[(size_t)(j - 1) * a.nzp + col]) /
                    (rj * dr);
            }
            double dzv = 0.0;
            for (int l = 1; l <= a.L; l++) {
                const double cl = a.coef64[MAX_L + l - 1];
                dzv += cl * ((double)Ez[(size_t)j * a.nzp + wrapz(col + l - 1, a.nzp)] -
                             (double)Ez[(size_t)j * a.nzp + wrapz(col - l, a.nzp)]);
            }
            v += dzv / dz;
            if (q == 0) dre = v; else dim = v;
        }
        if (m > 0 && j > 0) {
            // (i m / r_j) E_phi
            const T *Epr = E + (size_t)(1 * a.nparts + 2 * m - 1) * a.plane;
            const T *Epi = E + (size_t)(1 * a.nparts + 2 * m) * a.plane;
            const double rj = j * dr;
            dre += -m * (double)Epi[(size_t)j * a.nzp + col] / rj;
            dim += m * (double)Epr[(size_t)j * a.nzp + col] / rj;
        }
        const size_t qr = ((size_t)(2 * m) * (a.nr + 1) + j) * nz + il;
        const size_t qi = ((size_t)(2 * m + 1) * (a.nr + 1) + j) * nz + il;
        const double nre = rho_e[qr] + rho_ion[qr], nim = rho_e[qi] + rho_ion[qi];
        const double rre = dre - nre, rim = dim - nim;
        sr += rre * rre + rim * rim;
        sq += nre * nre + nim * nim;
    }
    s0[threadIdx.x] = sr; s1[threadIdx.x] = sq;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) { s0[threadIdx.x] += s0[threadIdx.x + w]; s1[threadIdx.x] += s1[threadIdx.x + w]; }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const size_t k = ((size_t)m * gridDim.y + j) * gridDim.x + blockIdx.x;
        part[2 * k] = s0[0];
        part[2 * k + 1] = s1[0];
    }
}

__global__ void k_gauss_final(const double *part, int per_mode, int nm, double *out)
{
    const int m = threadIdx.x;
    if (m >= nm) return;
    double a0 = 0.0, a1 = 0.0;
    for (int k = 0; k < per_mode; k++) {
        a0 += part[2 * ((size_t)m * per_mode + k)];
        a1 += part[2 * ((size_t)m * per_mode + k) + 1];
    }
    out[2 * m] = a0;
    out[2 * m + 1] = a1;
}

// out[2m] = sum |R_m|^2, out[2m+1] = sum |rho_net,m|^2 (host); scratch >= 2*4*(nr+1)*nm + 2*nm doubles
void launch_gauss(qpic_ctx *c, const double *rho_e, const double *rho_ion, double *scratch,
                  double *out_host)
{
    GridArgs a = grid_args(c);
    const int nm = c->g.nm, nbx = 4;
    dim3 grid(nbx, a.nr + 1, nm);
    prof_begin(c);
    if (c->fp64) k_gauss_partial<double><<<grid, 256, 0, c->stream>>>(c->E64, rho_e, rho_ion, a, nm, scratch);
    else k_gauss_partial<float><<<grid, 256, 0, c->stream>>>(c->E, rho_e, rho_ion, a, nm, scratch);
    const int per = nbx * (a.nr + 1);
    k_gauss_final<<<1, 32, 0, c->stream>>>(scratch, per, nm, scratch + (size_t)2 * per * nm);
    prof_end(c, KC_DIAG, 2);
    cudaMemcpyAsync(out_host, scratch + (size_t)2 * per * nm, 2 * nm * sizeof(double),
                    cudaMemcpyDeviceToHost, c->stream);
    cudaStreamSynchronize(c->stream);
}

}  // namespace qpic
