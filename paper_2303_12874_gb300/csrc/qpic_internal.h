// qpic_internal.h -- context layout and kernel entry points of libqpic.
//
// Device data layout (FP32 path)
//   Fields: planes of (nr+1) rows x nzp columns, z fastest.  A component c in
//   {r, phi, z} has nparts = 2*n_modes - 1 planes: part 0 = mode 0 (real),
//   part 2m-1 = Re F_m, part 2m = Im F_m; plane index = c*nparts + part.
//   The z axis is a circular buffer of nzp = nz + gap physical columns: logical
//   column i lives at physical (i + zoff) mod nzp.  An open box keeps a gap of
//   zero columns wider than every stencil, so stencils that reach past either
//   end read zeros; a periodic box has gap = 0 and wraps.  A moving window only
//   advances zoff, zeroes the column that left and fills the new front one.
//   Particles: structure of arrays, 36 B each: cell = (iz_phys << 16) | jr (int32,
//   -1 = dead), oz, or in [0,1) (offsets in the cell), cos phi, sin phi,
//   ux, uy, uz, w (float); optional W0, W1 (modal work, Eq. 16).
//   Current: int64 fixed point per plane, value = round(X * qscale) where X is
//   the per-particle "charge" quantity of the deposit; J = X * row factor.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/qpic.h"

namespace qpic {

constexpr int MAX_L = 64;      // max coefficients per z-operator
constexpr int MAX_TAPS = 512;  // max J_z filter half-length
constexpr int MAX_MODES = 4;

// Fixed point of the current (FP32 path).  A deposit contribution X (at most
// 2 qref in magnitude, qref the largest particle charge) becomes the integer
// v = round(X qscale), qscale = FX_SCALE / qref, so |v| < 2^39 - 2^29.  Inside
// the particle kernel v is carried as hi 2^FX_SHIFT + lo in two 32-bit shared
// planes (hi signed, |hi| <= 2^19 - 511 per contribution; lo made non-negative,
// below 2^FX_SHIFT, by a carry into hi when it is added), so a chunk of up to
// GPD_PPT_MAX x 256 = 4096 particles, each adding at most once to a node, keeps
// both planes inside 32 bits.  The resolution, 2^-38 qref, is far below the
// FP32 rounding of the contributions themselves.
constexpr int FX_SHIFT = 20;
constexpr double FX_SCALE = 274877906944.0 * (1023.0 / 1024.0);   // 2^38 (1 - 2^-10)
constexpr int GPD_PPT_MAX = 16;
// the bounds above: a contribution of 2 qref (times 1 + 2^-20 for its FP32
// rounding) gives a high part of at most 2^19 - 511; with the carry of the
// low part (at most 1 per contribution) a chunk's hi sums stay below 2^31, and
// its non-negative lo sums (each below 2^FX_SHIFT) below 2^32
constexpr double FX_HI_MAX = 2.0 * FX_SCALE * (1.0 + 1.0 / 1048576.0) / (double)(1 << FX_SHIFT) + 0.5;
static_assert((double)(GPD_PPT_MAX * 256) * (FX_HI_MAX + 1.0) < 2147483648.0, "hi plane of a chunk");
static_assert((double)(GPD_PPT_MAX * 256) * (double)((1 << FX_SHIFT) - 1) < 4294967296.0, "lo plane of a chunk");

struct FieldGeom {
    int nz, nr, nzp, gap, nparts, nm;
    long long zoff;            // physical column of logical 0 (mod nzp)
    size_t plane;              // (nr+1)*nzp
    float dz, dr, dt;
    int periodic;
};

// FP32 particles: the cell index (iz << 16 | jr, -1 = dead) in its own array and
// the eight floats of a particle as one 32-byte record of two float4 words,
// (oz, orr, cos phi, sin phi) and (ux, uy, uz, w), so that moving a particle
// writes whole 32-byte sectors
struct Particles {
    int32_t *cell = nullptr;
    float4 *rec = nullptr;                 // [2 * capacity]
    float *W0 = nullptr, *W1 = nullptr;    // modal work (when tracked)
};

struct Particles64 {  // plain FP64 path: lab z, Cartesian x, y
    double *z = nullptr, *x = nullptr, *y = nullptr, *ux = nullptr, *uy = nullptr,
           *uz = nullptr, *w = nullptr, *W0 = nullptr, *W1 = nullptr;
};

enum KernelClass {
    KC_FARADAY = 0, KC_GPD, KC_JDECODE, KC_JFILTER, KC_AMPERE, KC_SORT, KC_WINDOW,
    KC_INJECT, KC_DIAG, KC_OTHER, KC_COUNT
};

#ifdef __CUDACC__
// Double-float accumulator for FP64-grade sums of FP32 terms on the FP32 pipe
// (FP64 arithmetic is slow on this part): hi + lo, each addition exact through
// TwoSum (Knuth), products split exactly with an FMA.  Relative error of a sum
// of n terms about n * 2^-48; read out in FP64.
struct DFAcc {
    float hi = 0.f, lo = 0.f;
    __device__ __forceinline__ void add(float x)
    {
        const float s = __fadd_rn(hi, x);
        const float bb = __fsub_rn(s, hi);
        const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(x, bb));
        hi = s;
        lo = __fadd_rn(lo, err);
    }
    __device__ __forceinline__ void add_prod(float a, float b)
    {
        const float p = __fmul_rn(a, b);
        const float e = __fmaf_rn(a, b, -p);       // a b - p, exact
        add(p);
        lo = __fadd_rn(lo, e);
    }
    __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};
#endif

}  // namespace qpic

struct qpic_ctx {
    qpic_config cfg;
    std::string err;
    cudaStream_t stream = nullptr;
    int device = -1;                      // the device current at qpic_init (owns every buffer)
    bool fp64 = false;
    bool fatomic = false;                 // FP32 path with float-atomic deposit (precision variant)

    // grid and solver
    qpic::FieldGeom g;
    double dz, dr, dt;
    int L = 1;
    double cE[qpic::MAX_L], cB[qpic::MAX_L];
    std::vector<double> taps;     // k_0..k_{nk-1}; empty = no filter
    double kE1, kB1;              // symbols at k = 1 (laser set-up)

    // window / time
    long long shifts = 0, nstep = 0;

    // FP32 fields
    float *E = nullptr, *B = nullptr, *Bb = nullptr, *Jf = nullptr, *Jzf = nullptr;
    unsigned long long *Jacc = nullptr;   // global-path deposits (int64 atomics)
    float *Jfa = nullptr;                 // float-atomic variant: FP32 current sums
    unsigned long long *Jtile = nullptr;  // per-tile accumulator blocks
    int *tstamp = nullptr;                // epoch at which each tile block was written
    int *jdirty = nullptr;                // per tile: Jacc holds global-path deposits in its core
    int *d_epoch = nullptr;               // device counter stamping tile blocks
    float *rowf = nullptr;        // [4][nr+1]: J_z, J_r, J_phi(m>=1), J_phi(m=0)
    float *coef = nullptr;        // [cE (MAX_L) | cB (MAX_L) | taps (MAX_TAPS)] FP32
    double *coef64 = nullptr;     // the same in FP64
    bool j_filtered = false;      // J_z of the last deposit has been filtered

    // FP64 fields (plain path)
    double *E64 = nullptr, *B64 = nullptr, *Bb64 = nullptr, *J64 = nullptr, *Jz64 = nullptr;

    // particles
    long long np = 0, cap = 0;    // np: host upper bound of the device count d_count[0]
    long long n_tail = 0;         // particles appended since the last sort (unsorted tail)
    long long *d_count = nullptr; // device: [0] particles in the buffer, [1] of them sorted
    qpic::Particles p, ps;        // live buffers and the sort's second buffer
    qpic::Particles64 p64, ps64;  // plain FP64 path: live buffers and compaction target
    int32_t *scan_flag = nullptr, *scan_pos = nullptr, *scan_tmp64 = nullptr;
    double qref = 0.0;            // max |charge| of a particle
    float qscale = 0.f;           // fixed-point scale FX_SCALE / qref

    // plasma (for the moving-window injection)
    bool have_plasma = false;
    double n0 = 0, z_start = 0, ramp_len = 0;
    int ppc_z = 0, ppc_r = 0, ppc_phi = 0, jitter = 0;

    // tiles and sort
    int TZ = 16, TR = 8, ntz = 0, ntr = 0, halo = 1;
    int ppt = 16;                // consecutive particles per thread in the particle kernel
    int nabs = 0;                // absorbing radial layer: cells next to the wall (0: none)
    double sigabs = 0;           // its peak conductivity
    float *lossf = nullptr;      // lossy update factors per row (4 (nr + 1)), FP32 and FP64
    double *loss64 = nullptr;
    long long nkeys = 0;
    int32_t *counts = nullptr, *offsets = nullptr, *scan_tmp = nullptr;
    int sort_period = 1;

    // device scratch
    int *d_err = nullptr;         // error word: bit 0 overflow, bit 1 capacity
    double *h_diag = nullptr;     // pinned host words: diagnostics read back with one synchronisation
    double *rho_ion = nullptr;    // fixed ion background -rho_e at plasma load, [nm][2][nr+1][nz]
    double *d_red = nullptr;      // reduction scratch
    int red_cap = 0;

    // profiling
    bool profile = false;
    double kms[qpic::KC_COUNT] = {0};
    long long klaunch[qpic::KC_COUNT] = {0};
    long long n_kernels = 0;                   // kernels launched by this context
    std::vector<cudaEvent_t> ev_pool;          // recorded pairs, resolved on demand
    std::vector<int> ev_class;
    size_t ev_used = 0;

    // allocations made through the allocator hooks
    std::vector<void *> allocs;
};

namespace qpic {

// ---- host numerics (host_numerics.cpp) ----
int fit_coefficients(int solver, double dt, double dz, int L, double band, double *cE, double *cB,
                     std::string &err);
double symbol(const double *C, int L, double theta);       // [k] dz of an operator
int filter_taps_host(const double *cB, int L, double tol, std::vector<double> &taps,
                     std::string &err);
double radial_lambda_max(int nr, double dr, int m);
int cfl_limit(int solver, double dz, double dr, int nr, int n_modes, int L, double band,
              double *dt_out, std::string &err);

// ---- kernel launchers (k_fields.cu) ----
void set_solver_constants(qpic_ctx *c);
void launch_faraday(qpic_ctx *c);
void launch_jdecode(qpic_ctx *c);
void launch_jfilter(qpic_ctx *c);
void launch_ampere(qpic_ctx *c);
void launch_zero_column(qpic_ctx *c, long long phys_col);
void launch_laser(qpic_ctx *c, double a0, double w0, double fwhm, double zc, double zf,
                  double psi);
void launch_field_energy(qpic_ctx *c, double *out_modes);   // host out[n_modes]
void launch_gauss(qpic_ctx *c, const double *rho_e, const double *rho_ion, double *scratch,
                  double *out_host);
void launch_spectrum(qpic_ctx *c, const double *edges, int nb, double wscale,
                     unsigned long long *out);

// ---- kernel launchers (k_particles.cu) ----
void launch_gpd(qpic_ctx *c);
bool gpd_tile_supported(int tile_z, int tile_r);
size_t gpd_tile_words(int nparts, int tile_z, int tile_r);   // accumulator words per tile
size_t gpd_tile_smem(int nparts, int tile_z, int tile_r);    // shared memory of one particle-kernel block
double launch_absmax(qpic_ctx *c, const double *w, long long n);  // max |w[i]| (device array; syncs)
void launch_sort(qpic_ctx *c);
int launch_load_plasma(qpic_ctx *c, long long first_logical_col, int ncols, bool append);
void launch_load_particles(qpic_ctx *c, long long n, const double *dz_, const double *dr_,
                           const double *dphi, const double *dux, const double *duy,
                           const double *duz, const double *dw);
void launch_export_particles(qpic_ctx *c, double *dout, long long stride);
void launch_rho(qpic_ctx *c, double *dplanes);               // nm*2 planes (nr+1)*nz logical
void launch_particle_sums(qpic_ctx *c, double *out3);        // count, charge, kinetic
void exclusive_scan(qpic_ctx *c, const int32_t *in, int32_t *out, int32_t *tmp, long long n);

// ---- plain FP64 path (k_fp64.cu) ----
void fp64_faraday(qpic_ctx *c);
void fp64_push_deposit(qpic_ctx *c);
void fp64_ampere(qpic_ctx *c);
void fp64_zero_column(qpic_ctx *c, long long phys_col);
void fp64_laser(qpic_ctx *c, double a0, double w0, double fwhm, double zc, double zf, double psi);
int fp64_load_plasma(qpic_ctx *c, long long first_logical_col, int ncols, bool append);
void fp64_load_particles(qpic_ctx *c, long long n, const double *dz_, const double *dr_,
                         const double *dphi, const double *dux, const double *duy,
                         const double *duz, const double *dw);
void fp64_export_particles(qpic_ctx *c, double *dout, long long stride);
void fp64_compact(qpic_ctx *c);
void fp64_rho(qpic_ctx *c, double *dplanes);
void fp64_particle_sums(qpic_ctx *c, double *out3);
void fp64_spectrum(qpic_ctx *c, const double *edges, int nb, double wscale, unsigned long long *out);
void scale_buffer(qpic_ctx *c, double *buf, size_t n, double s);
void fp64_field_energy(qpic_ctx *c, double *out_modes);

// ---- batched particle phase (k_particles.cu): one persistent launch over the
// (run, tile) work list of the runs of a batch that share mode count and tile
// shape.  Table entries are opaque here (batch_run_bytes each).
struct BatchCtlHost {
    long long spins;   // polls of one dependency wait before it gives up (QPIC_ETIMEOUT)
    int hold;          // particle item that publishes nothing (-1: none; tests of the bounded wait)
    int pad;
};
size_t batch_run_bytes();
BatchCtlHost batch_ctl_default();
void batch_fill_run(qpic_ctx *c, const Particles &p_cur, int *gdone, void *out);
void launch_epoch(qpic_ctx *c);
bool launch_batch_particles(int nparts, int tz, int tr, const void *d_table, const int *d_prefix, int nruns,
                            int *d_head, const void *d_ctl, int blocks, cudaStream_t st);

// QPIC_OK when the context's device is the current one, else QPIC_ESTATE (or
// QPIC_ECUDA) with the context's error text set (api.cu)
qpic_status check_device(qpic_ctx *c);

// profiling helpers (api.cu)
void prof_begin(qpic_ctx *c);
void prof_end(qpic_ctx *c, int kclass, int nkernels = 1);

}  // namespace qpic

// return early from an entry point whose context belongs to another device
// Device-side invariant checks of the checked build (QPIC_CHECK defined):
// a violation sets bit 3 of the error word (reported as QPIC_ECHECK); no trap.
#ifdef QPIC_CHECK
#define QPIC_DCHECK(cond, errp)                                    \
    do {                                                           \
        if (!(cond)) atomicOr((errp), 8);                          \
    } while (0)
#else
#define QPIC_DCHECK(cond, errp) \
    do {                        \
    } while (0)
#endif

#define QPIC_REQUIRE_DEVICE(c)                                                         \
    do {                                                                               \
        qpic_status _s = qpic::check_device(c);                                        \
        if (_s != QPIC_OK) return _s;                                                  \
    } while (0)

#define QPIC_CUDA_OK(c, call)                                                          \
    do {                                                                               \
        cudaError_t _e = (call);                                                       \
        if (_e != cudaSuccess) {                                                       \
            (c)->err = std::string(#call) + ": " + cudaGetErrorString(_e);            \
            return QPIC_ECUDA;                                                         \
        }                                                                              \
    } while (0)
