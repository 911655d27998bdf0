// api.cu -- the C ABI of libqpic (declared in include/qpic.h): context set-up,
// particle and field I/O, the step loop, diagnostics and kernel timing.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "qpic_internal.h"

using namespace qpic;

namespace {

const double kPi = 3.14159265358979323846;

void *dalloc(qpic_ctx *c, size_t bytes)
{
    if (bytes == 0) bytes = 16;
    void *p = nullptr;
    if (c->cfg.dev_alloc) {
        p = c->cfg.dev_alloc(bytes, c->cfg.alloc_user);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    if (p) c->allocs.push_back(p);
    return p;
}

void dfree(qpic_ctx *c, void *p)
{
    if (!p) return;
    auto it = std::find(c->allocs.begin(), c->allocs.end(), p);
    if (it != c->allocs.end()) c->allocs.erase(it);
    if (c->cfg.dev_free) c->cfg.dev_free(p, c->cfg.alloc_user);
    else cudaFree(p);
}

template <class T>
bool alloc_arr(qpic_ctx *c, T **out, size_t n)
{
    *out = static_cast<T *>(dalloc(c, n * sizeof(T)));
    return *out != nullptr;
}

qpic_status fail(qpic_ctx *c, qpic_status s, const std::string &msg)
{
    if (c) c->err = msg;
    return s;
}

qpic_status cuda_check(qpic_ctx *c, const char *where)
{
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(c, QPIC_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
    return QPIC_OK;
}

bool alloc_particles(qpic_ctx *c, qpic::Particles &p, long long cap)
{
    bool ok = alloc_arr(c, &p.cell, cap) && alloc_arr(c, &p.rec, 2 * (size_t)cap);
    if (ok && c->cfg.track_work) ok = alloc_arr(c, &p.W0, cap) && alloc_arr(c, &p.W1, cap);
    return ok;
}

void free_particles(qpic_ctx *c, qpic::Particles &p)
{
    void *arr[4] = {p.cell, p.rec, p.W0, p.W1};
    for (void *a : arr) dfree(c, a);
    p = qpic::Particles();
}

bool alloc_particles64(qpic_ctx *c, qpic::Particles64 &p, long long cap)
{
    bool ok = alloc_arr(c, &p.z, cap) && alloc_arr(c, &p.x, cap) && alloc_arr(c, &p.y, cap) &&
              alloc_arr(c, &p.ux, cap) && alloc_arr(c, &p.uy, cap) && alloc_arr(c, &p.uz, cap) &&
              alloc_arr(c, &p.w, cap);
    if (ok && c->cfg.track_work) ok = alloc_arr(c, &p.W0, cap) && alloc_arr(c, &p.W1, cap);
    return ok;
}

void free_particles64(qpic_ctx *c, qpic::Particles64 &p)
{
    void *arr[9] = {p.z, p.x, p.y, p.ux, p.uy, p.uz, p.w, p.W0, p.W1};
    for (void *a : arr) dfree(c, a);
    p = qpic::Particles64();
}

qpic_status ensure_capacity(qpic_ctx *c, long long need)
{
    if (need <= c->cap) return QPIC_OK;
    long long cap = c->cfg.max_particles > 0 ? c->cfg.max_particles
                                             : std::max(need + need / 4 + 4096, c->cap);
    if (cap < need) return fail(c, QPIC_ECAPACITY, "particle capacity (max_particles) exceeded");
    cudaStreamSynchronize(c->stream);
    if (c->fp64) {
        free_particles64(c, c->p64);
        free_particles64(c, c->ps64);
        dfree(c, c->scan_flag); dfree(c, c->scan_pos); dfree(c, c->scan_tmp64);
        c->cap = 0;
        if (!alloc_particles64(c, c->p64, cap) || !alloc_particles64(c, c->ps64, cap) ||
            !alloc_arr(c, &c->scan_flag, (size_t)cap + 1) || !alloc_arr(c, &c->scan_pos, (size_t)cap + 1) ||
            !alloc_arr(c, &c->scan_tmp64, (size_t)(cap + 1) / 4096 + 4))
            return fail(c, QPIC_ENOMEM, "particle buffers: device allocation failed");
        c->cap = cap;
        return QPIC_OK;
    }
    free_particles(c, c->p);
    free_particles(c, c->ps);
    c->cap = 0;
    if (!alloc_particles(c, c->p, cap) || !alloc_particles(c, c->ps, cap))
        return fail(c, QPIC_ENOMEM, "particle buffers: device allocation failed");
    c->cap = cap;
    return QPIC_OK;
}

// logical column <-> physical column
long long phys_col(const qpic_ctx *c, long long il)
{
    long long p = (il + c->g.zoff) % c->g.nzp;
    return p < 0 ? p + c->g.nzp : p;
}

// logical columns [0, nz) map onto physical columns by a rotation: columns
// [0, split) start at physical column c0, the rest at column 0
struct ColMap { long long c0, split; };
ColMap col_map(const qpic_ctx *c)
{
    const long long c0 = phys_col(c, 0);
    return {c0, std::min<long long>(c->g.nz, c->g.nzp - c0)};
}

double *field_base64(qpic_ctx *c, int which)
{
    switch (which) {
    case QPIC_FIELD_E: return c->E64;
    case QPIC_FIELD_B: return c->B64;
    case QPIC_FIELD_BBAR: return c->Bb64;
    default: return c->J64;
    }
}

float *field_base(qpic_ctx *c, int which)
{
    switch (which) {
    case QPIC_FIELD_E: return c->E;
    case QPIC_FIELD_B: return c->B;
    case QPIC_FIELD_BBAR: return c->Bb;
    default: return c->Jf;
    }
}

void set_qscale(qpic_ctx *c, double qmax)
{
    c->qref = qmax > 0 ? qmax : 1.0;
    // per-particle contributions stay below 2 qref, i.e. 2^39 - 2^29 units: the
    // particle kernel's 32-bit planes hold chunks of 4096 of them (FX_SCALE),
    // and int64 keeps 2^24 contributions of the largest size per accumulator
    c->qscale = (float)(FX_SCALE / c->qref);
}

void do_shift(qpic_ctx *c)
{
    long long back = phys_col(c, 0);
    launch_zero_column(c, back);
    c->g.zoff = (c->g.zoff + 1) % c->g.nzp;
    c->shifts++;
    if (c->have_plasma && c->fp64) {
        if (c->np + (long long)c->g.nr * c->ppc_z * c->ppc_r * c->ppc_phi > c->cap) fp64_compact(c);
        fp64_load_plasma(c, c->g.nz - 1, 1, true);
    } else if (c->have_plasma) {
        if (c->np + (long long)c->g.nr * c->ppc_z * c->ppc_r * c->ppc_phi > c->cap) {
            // host bound is loose after sorts dropped particles: refresh it
            long long n = 0;
            cudaMemcpyAsync(&n, c->d_count, sizeof(long long), cudaMemcpyDeviceToHost, c->stream);
            cudaStreamSynchronize(c->stream);
            c->np = n;
        }
        launch_load_plasma(c, c->g.nz - 1, 1, true);
    }
}

// an NVTX range for the phases of a step (a no-op unless a profiler is attached)
struct PhaseRange {
    explicit PhaseRange(const char *name) { nvtxRangePushA(name); }
    ~PhaseRange() { nvtxRangePop(); }
};

qpic_status run_one_step(qpic_ctx *c, int stages)
{
    PhaseRange step_range("qpic step");
    if (stages & QPIC_STAGE_FARADAY) {
        PhaseRange r("faraday");
        launch_faraday(c);
    }
    if (stages & QPIC_STAGE_PARTICLES) {
        PhaseRange r("gather push deposit");
        if (c->fp64) {
            fp64_push_deposit(c);
        } else {
            launch_gpd(c);
            launch_jdecode(c);
        }
        c->j_filtered = false;
    }
    if (stages & QPIC_STAGE_AMPERE) {
        PhaseRange r("filter ampere");
        if (!c->taps.empty()) launch_jfilter(c);
        c->j_filtered = !c->taps.empty();
        launch_ampere(c);
    }
    bool full = (stages & (QPIC_STAGE_FARADAY | QPIC_STAGE_PARTICLES | QPIC_STAGE_AMPERE)) ==
                (QPIC_STAGE_FARADAY | QPIC_STAGE_PARTICLES | QPIC_STAGE_AMPERE);
    if (full) c->nstep++;
    if ((stages & QPIC_STAGE_WINDOW) && c->cfg.moving_window) {
        PhaseRange r("window");
        while (c->cfg.window_v * ((double)c->nstep * c->dt) >= (double)(c->shifts + 1) * c->dz)
            do_shift(c);
    }
    if ((stages & QPIC_STAGE_SORT) && c->fp64) return QPIC_OK;    // plain path: no sort
    if (stages & QPIC_STAGE_SORT) {
        bool due = c->sort_period <= 1 || (c->nstep % c->sort_period) == 0 ||
                   c->n_tail > c->cap / 64;
        if (due) {
            PhaseRange r("sort");
            launch_sort(c);
        }
    }
    return QPIC_OK;
}

qpic_status check_device_error(qpic_ctx *c)
{
    int e = 0;
    cudaMemcpyAsync(&e, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    cudaError_t ce = cudaStreamSynchronize(c->stream);
    if (ce != cudaSuccess) return fail(c, QPIC_ECUDA, std::string("step: ") + cudaGetErrorString(ce));
    if (e & 1) return fail(c, QPIC_EOVERFLOW, "fixed-point current accumulator overflow");
    if (e & 2) return fail(c, QPIC_ECAPACITY, "particle capacity exceeded during injection");
    if (e & 8) return fail(c, QPIC_ECHECK, "a kernel invariant check failed (checked build)");
    return QPIC_OK;
}

long long live_count(qpic_ctx *c)
{
    long long n = 0;
    cudaMemcpyAsync(&n, c->d_count, sizeof(long long), cudaMemcpyDeviceToHost, c->stream);
    cudaStreamSynchronize(c->stream);
    c->np = n;
    return n;
}

// fixed ion background: minus the electron density at load time
void record_ions(qpic_ctx *c)
{
    const size_t n = (size_t)c->g.nm * 2 * (c->g.nr + 1) * c->g.nz;
    if (!c->rho_ion && !alloc_arr(c, &c->rho_ion, n)) return;
    launch_rho(c, c->rho_ion);
    scale_buffer(c, c->rho_ion, n, -1.0);
}

}  // namespace

namespace qpic {

qpic_status check_device(qpic_ctx *c)
{
    int dev = -1;
    const cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(c, QPIC_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev != c->device)
        return fail(c, QPIC_ESTATE, "the context was created on device " + std::to_string(c->device) +
                                        " but device " + std::to_string(dev) + " is current");
    return QPIC_OK;
}

void prof_begin(qpic_ctx *c)
{
    if (!c->profile) return;
    if (c->ev_used + 2 > c->ev_pool.size()) {
        for (int k = 0; k < 256; k++) {
            cudaEvent_t e;
            cudaEventCreate(&e);
            c->ev_pool.push_back(e);
        }
    }
    cudaEventRecord(c->ev_pool[c->ev_used], c->stream);
}

void prof_end(qpic_ctx *c, int kclass, int nkernels)
{
    c->n_kernels += nkernels;
    if (!c->profile) return;
    cudaEventRecord(c->ev_pool[c->ev_used + 1], c->stream);
    c->ev_class.push_back(kclass);
    c->ev_used += 2;
}

}  // namespace qpic

static void resolve_events(qpic_ctx *c)
{
    if (c->ev_used == 0) return;
    cudaStreamSynchronize(c->stream);
    for (size_t k = 0; k < c->ev_class.size(); k++) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, c->ev_pool[2 * k], c->ev_pool[2 * k + 1]);
        c->kms[c->ev_class[k]] += ms;
        c->klaunch[c->ev_class[k]] += 1;
    }
    c->ev_class.clear();
    c->ev_used = 0;
}

extern "C" {

qpic_status qpic_default_config(qpic_config *cfg)
{
    if (!cfg) return QPIC_EINVAL;
    std::memset(cfg, 0, sizeof(*cfg));
    cfg->n_modes = 2;
    cfg->cfl_frac = 0.9;
    cfg->solver = QPIC_DUAL;
    cfg->n_coef = 16;
    cfg->fit_band = 0.8;
    cfg->precision = QPIC_FP32_FIXED;
    cfg->jz_filter = 1;
    cfg->filter_tol = 1e-16;
    cfg->periodic_z = 1;
    cfg->window_v = 1.0;
    cfg->tile_z = 16;
    cfg->tile_r = 8;
    cfg->sort_period = 2;
    cfg->particles_per_thread = 16;
    cfg->absorb_cells = 0;
    cfg->absorb_sigma = 0.0;
    cfg->seed = 1;
    return QPIC_OK;
}

const char *qpic_last_error(const qpic_ctx *ctx)
{
    if (!ctx) return "no context";
    return ctx->err.c_str();
}

void qpic_destroy(qpic_ctx *ctx)
{
    if (!ctx) return;
    cudaStreamSynchronize(ctx->stream);
    if (ctx->h_diag) cudaFreeHost(ctx->h_diag);
    for (cudaEvent_t e : ctx->ev_pool) cudaEventDestroy(e);
    std::vector<void *> all = ctx->allocs;
    for (void *p : all) dfree(ctx, p);
    delete ctx;
}

qpic_status qpic_init(const qpic_config *cfg, qpic_ctx **out)
{
    if (!out) return QPIC_EINVAL;
    *out = nullptr;
    if (!cfg) return QPIC_EINVAL;
    qpic_ctx *c = new (std::nothrow) qpic_ctx();
    if (!c) return QPIC_ENOMEM;
    c->cfg = *cfg;
    auto bad = [&](qpic_status s, const std::string &m) {
        c->err = m;
        *out = c;          // returned so that qpic_last_error can explain; caller destroys
        return s;
    };
    if (cfg->nz < 4 || cfg->nr < 2 || cfg->n_modes < 1 || cfg->n_modes > MAX_MODES)
        return bad(QPIC_EINVAL, "grid: need nz >= 4, nr >= 2, 1 <= n_modes <= 4");
    if (!(cfg->dz > 0) || !(cfg->dr > 0)) return bad(QPIC_EINVAL, "dz, dr must be positive");
    if (cfg->track_work < 0 || cfg->track_work > 2)
        return bad(QPIC_EINVAL, "track_work: 0, 1 (modal work, Eq. 16) or 2 (directional work, Eq. 17)");
    if (cfg->solver != QPIC_YEE && cfg->solver != QPIC_DUAL) return bad(QPIC_EINVAL, "solver");
    if (cfg->precision != QPIC_FP32_FIXED && cfg->precision != QPIC_FP64 &&
        cfg->precision != QPIC_FP32_FATOMIC)
        return bad(QPIC_EINVAL, "precision: QPIC_FP32_FIXED, QPIC_FP32_FATOMIC or QPIC_FP64");
    c->fp64 = cfg->precision == QPIC_FP64;
    c->fatomic = cfg->precision == QPIC_FP32_FATOMIC;
    if (cfg->moving_window && cfg->periodic_z) return bad(QPIC_EINVAL, "moving window needs periodic_z = 0");
    {
        const cudaError_t e = cudaGetDevice(&c->device);
        if (e != cudaSuccess) return bad(QPIC_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    }
    c->stream = static_cast<cudaStream_t>(cfg->cuda_stream);
    c->dz = cfg->dz;
    c->dr = cfg->dr;
    const int L = cfg->solver == QPIC_YEE ? 1 : (cfg->n_coef > 0 ? cfg->n_coef : 16);
    const double band = cfg->fit_band > 0 ? cfg->fit_band : 0.8;
    double dtmax = 0.0;
    if (!cfl_limit(cfg->solver, cfg->dz, cfg->dr, cfg->nr, cfg->n_modes, L, band, &dtmax, c->err))
        return bad(QPIC_ECFL, c->err);
    c->dt = cfg->dt > 0 ? cfg->dt : (cfg->cfl_frac > 0 ? cfg->cfl_frac : 0.9) * dtmax;
    if (c->dt > dtmax * (1.0 + 1e-9)) return bad(QPIC_ECFL, "dt above the stability limit");
    c->L = fit_coefficients(cfg->solver, c->dt, cfg->dz, L, band, c->cE, c->cB, c->err);
    if (!c->L) return bad(QPIC_ECFL, c->err);
    if (cfg->solver == QPIC_DUAL && cfg->jz_filter) {
        double tol = cfg->filter_tol > 0 ? cfg->filter_tol : 1e-16;
        if (!filter_taps_host(c->cB, c->L, tol, c->taps, c->err)) return bad(QPIC_ECFL, c->err);
    }
    c->kE1 = symbol(c->cE, c->L, cfg->dz) / cfg->dz;
    c->kB1 = symbol(c->cB, c->L, cfg->dz) / cfg->dz;
    // geometry: circular z buffer, gap wider than the widest stencil for open boxes
    c->TZ = cfg->tile_z > 0 ? cfg->tile_z : 16;
    c->TR = cfg->tile_r > 0 ? cfg->tile_r : 8;
    if (!gpd_tile_supported(c->TZ, c->TR))
        return bad(QPIC_EINVAL, "tile_z x tile_r: one of 16x8, 32x8, 8x8, 16x16, 32x4");
    c->halo = 1;
    if (cfg->sort_period < 0) return bad(QPIC_EINVAL, "sort_period: >= 1 (0: 2)");
    c->sort_period = cfg->sort_period > 0 ? cfg->sort_period : 2;
    if (cfg->particles_per_thread < 0 || cfg->particles_per_thread > GPD_PPT_MAX)
        return bad(QPIC_EINVAL, "particles_per_thread: 1..16 (0: 16)");
    c->ppt = cfg->particles_per_thread > 0 ? cfg->particles_per_thread : 16;
    if (cfg->absorb_cells < 0 || cfg->absorb_cells > cfg->nr || !(cfg->absorb_sigma >= 0.0) ||
        !std::isfinite(cfg->absorb_sigma))
        return bad(QPIC_EINVAL, "absorb_cells: 0..nr; absorb_sigma: finite, >= 0");
    c->nabs = cfg->absorb_cells;
    c->sigabs = c->nabs == 0 ? 0.0
              : (cfg->absorb_sigma > 0 ? cfg->absorb_sigma : 3.0 * std::log(1e4) / (2.0 * c->nabs * cfg->dr));
    if (cfg->precision != QPIC_FP64) {
        // the tile's staged fields and accumulators must fit one block's shared memory
        int dev = 0, optin = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        const size_t need = gpd_tile_smem(2 * cfg->n_modes - 1, c->TZ, c->TR);
        if (optin > 0 && need > (size_t)optin)
            return bad(QPIC_EINVAL, "tile_z x tile_r too large for n_modes: the particle kernel needs " +
                                        std::to_string(need) + " B of shared memory per block, the device has " +
                                        std::to_string(optin) + " B (take a smaller tile)");
    }
    FieldGeom &g = c->g;
    g.nz = cfg->nz; g.nr = cfg->nr; g.nm = cfg->n_modes; g.nparts = 2 * cfg->n_modes - 1;
    g.periodic = cfg->periodic_z ? 1 : 0;
    int reach = std::max({2 * c->L + 2, (int)c->taps.size() + 2, 2 * (c->TZ + 2 * c->halo + 3)});
    g.gap = g.periodic ? 0 : ((reach + c->TZ - 1) / c->TZ) * c->TZ;
    g.nzp = g.nz + g.gap;
    if (g.nzp >= 32768 || g.nr >= 65535)
        return bad(QPIC_EINVAL, "grid too large: nz + gap < 32768 (packed cell index), nr < 65535 "
                                "(packed cell index; one block row per grid row, nr + 1 <= 65535)");
    g.zoff = 0;
    g.plane = (size_t)(g.nr + 1) * g.nzp;
    g.dz = (float)c->dz; g.dr = (float)c->dr; g.dt = (float)c->dt;
    const size_t nplanes = (size_t)3 * g.nparts;
    if (c->fp64) {
        if (!alloc_arr(c, &c->E64, nplanes * g.plane) || !alloc_arr(c, &c->B64, nplanes * g.plane) ||
            !alloc_arr(c, &c->Bb64, nplanes * g.plane) || !alloc_arr(c, &c->J64, nplanes * g.plane) ||
            !alloc_arr(c, &c->Jz64, (size_t)g.nparts * g.plane))
            return bad(QPIC_ENOMEM, "field buffers: device allocation failed");
        cudaMemsetAsync(c->E64, 0, nplanes * g.plane * 8, c->stream);
        cudaMemsetAsync(c->B64, 0, nplanes * g.plane * 8, c->stream);
        cudaMemsetAsync(c->Bb64, 0, nplanes * g.plane * 8, c->stream);
        cudaMemsetAsync(c->J64, 0, nplanes * g.plane * 8, c->stream);
        cudaMemsetAsync(c->Jz64, 0, (size_t)g.nparts * g.plane * 8, c->stream);
    } else if (!alloc_arr(c, &c->E, nplanes * g.plane) || !alloc_arr(c, &c->B, nplanes * g.plane) ||
               !alloc_arr(c, &c->Bb, nplanes * g.plane) || !alloc_arr(c, &c->Jf, nplanes * g.plane) ||
               !alloc_arr(c, &c->Jzf, (size_t)g.nparts * g.plane) ||
               !alloc_arr(c, &c->Jacc, nplanes * g.plane) ||
               (c->fatomic && !alloc_arr(c, &c->Jfa, nplanes * g.plane))) {
        return bad(QPIC_ENOMEM, "field buffers: device allocation failed");
    }
    if (c->fatomic) cudaMemsetAsync(c->Jfa, 0, nplanes * g.plane * sizeof(float), c->stream);
    if (!alloc_arr(c, &c->rowf, (size_t)4 * (g.nr + 1)) ||
        !alloc_arr(c, &c->coef, (size_t)2 * MAX_L + MAX_TAPS) ||
        !alloc_arr(c, &c->coef64, (size_t)2 * MAX_L + MAX_TAPS) || !alloc_arr(c, &c->d_err, 4) ||
        !alloc_arr(c, &c->d_count, 4))
        return bad(QPIC_ENOMEM, "field buffers: device allocation failed");
    c->ntz = (g.nzp + c->TZ - 1) / c->TZ;
    c->ntr = (g.nr + c->TR - 1) / c->TR;
    c->nkeys = (long long)c->ntz * c->ntr * c->TZ * c->TR;
    const int nb = (int)((c->nkeys + 1 + 4095) / 4096);
    c->red_cap = std::max(4 * (g.nr + 1) * g.nm + 64, 8 + 3 * 609);
    if (!c->fp64) {
        const size_t tw = gpd_tile_words(g.nparts, c->TZ, c->TR) * (size_t)c->ntz * c->ntr;
        if (!alloc_arr(c, &c->Jtile, tw) || !alloc_arr(c, &c->tstamp, (size_t)c->ntz * c->ntr) ||
            !alloc_arr(c, &c->jdirty, (size_t)c->ntz * c->ntr) || !alloc_arr(c, &c->d_epoch, 4))
            return bad(QPIC_ENOMEM, "tile accumulators: device allocation failed");
        cudaMemsetAsync(c->tstamp, 0xff, (size_t)c->ntz * c->ntr * sizeof(int), c->stream);
        cudaMemsetAsync(c->jdirty, 0, (size_t)c->ntz * c->ntr * sizeof(int), c->stream);
        cudaMemsetAsync(c->d_epoch, 0, 4 * sizeof(int), c->stream);
    }
    if (!alloc_arr(c, &c->counts, (size_t)c->nkeys + 1) ||
        !alloc_arr(c, &c->offsets, (size_t)c->nkeys + 1) || !alloc_arr(c, &c->scan_tmp, (size_t)nb + 2) ||
        !alloc_arr(c, &c->d_red, (size_t)c->red_cap))
        return bad(QPIC_ENOMEM, "sort buffers: device allocation failed");
    if (!c->fp64) {
        cudaMemsetAsync(c->E, 0, nplanes * g.plane * sizeof(float), c->stream);
        cudaMemsetAsync(c->B, 0, nplanes * g.plane * sizeof(float), c->stream);
        cudaMemsetAsync(c->Bb, 0, nplanes * g.plane * sizeof(float), c->stream);
        cudaMemsetAsync(c->Jf, 0, nplanes * g.plane * sizeof(float), c->stream);
        cudaMemsetAsync(c->Jzf, 0, (size_t)g.nparts * g.plane * sizeof(float), c->stream);
        cudaMemsetAsync(c->Jacc, 0, nplanes * g.plane * 8, c->stream);
    }
    cudaMemsetAsync(c->d_err, 0, 4 * sizeof(int), c->stream);
    cudaMemsetAsync(c->d_count, 0, 4 * sizeof(long long), c->stream);
    cudaMemsetAsync(c->offsets, 0, ((size_t)c->nkeys + 1) * sizeof(int32_t), c->stream);
    // row factors turning the deposit's charge quantities into current densities:
    // J_z = X dz/(V_j dt), J_r = X/(2 pi r_{j+1/2} dz dt), J_phi^{m>=1} = X r_j/(V_j dt),
    // J_phi^0 = X dr/(V_j dt); V_j the control volume of node j
    std::vector<float> rf((size_t)4 * (g.nr + 1));
    const double dz = c->dz, dr = c->dr, dt = c->dt, R = g.nr * dr;
    for (int j = 0; j <= g.nr; j++) {
        double V = j == 0 ? kPi * 0.25 * dr * dr * dz
                 : j == g.nr ? kPi * (R * R - (R - 0.5 * dr) * (R - 0.5 * dr)) * dz
                             : 2.0 * kPi * j * dr * dr * dz;
        rf[j] = (float)(dz / (V * dt));
        rf[(g.nr + 1) + j] = j < g.nr ? (float)(1.0 / (2.0 * kPi * (j + 0.5) * dr * dz * dt)) : 0.f;
        rf[2 * (g.nr + 1) + j] = (float)(j * dr / (V * dt));
        rf[3 * (g.nr + 1) + j] = (float)(dr / (V * dt));
    }
    cudaMemcpy(c->rowf, rf.data(), rf.size() * sizeof(float), cudaMemcpyHostToDevice);
    // absorbing radial layer: sigma(r) = sigma_max ((r - r0) / (n_abs dr))^2 on
    // r0 < r <= R, and the lossy leapfrog update F = alpha F + beta dt rhs with
    // alpha = (1 - sigma dt/2) / (1 + sigma dt/2), beta = 1 / (1 + sigma dt/2),
    // per row at r_j and r_{j+1/2}
    if (c->nabs > 0) {
        const size_t nl = (size_t)4 * (g.nr + 1);
        if (!alloc_arr(c, &c->lossf, nl) || !alloc_arr(c, &c->loss64, nl))
            return bad(QPIC_ENOMEM, "absorbing layer: device allocation failed");
        std::vector<double> l64(nl);
        std::vector<float> l32(nl);
        const double width = c->nabs * dr, r0 = R - width;
        for (int j = 0; j <= g.nr; j++) {
            for (int k = 0; k < 2; k++) {
                const double r = (j + 0.5 * k) * dr;
                const double x = r > r0 ? (r - r0) / width : 0.0;
                const double h = 0.5 * c->sigabs * x * x * dt;
                l64[(size_t)(2 * k) * (g.nr + 1) + j] = (1.0 - h) / (1.0 + h);
                l64[(size_t)(2 * k + 1) * (g.nr + 1) + j] = 1.0 / (1.0 + h);
            }
        }
        for (size_t k = 0; k < nl; k++) l32[k] = (float)l64[k];
        cudaMemcpy(c->loss64, l64.data(), nl * sizeof(double), cudaMemcpyHostToDevice);
        cudaMemcpy(c->lossf, l32.data(), nl * sizeof(float), cudaMemcpyHostToDevice);
    }
    set_solver_constants(c);
    set_qscale(c, 1.0);
    qpic_status st = cuda_check(c, "init");
    if (st != QPIC_OK) { *out = c; return st; }
    cudaStreamSynchronize(c->stream);
    *out = c;
    return QPIC_OK;
}

qpic_status qpic_get_solver(const qpic_ctx *ctx, double *dt, int32_t *L, double *cE, double *cB,
                            int32_t cap_coef, double *taps, int32_t cap_taps, int32_t *n_taps)
{
    if (!ctx) return QPIC_EINVAL;
    if (dt) *dt = ctx->dt;
    if (L) *L = ctx->L;
    for (int l = 0; l < ctx->L && l < cap_coef; l++) {
        if (cE) cE[l] = ctx->cE[l];
        if (cB) cB[l] = ctx->cB[l];
    }
    if (n_taps) *n_taps = (int32_t)ctx->taps.size();
    for (int q = 0; q < (int)ctx->taps.size() && q < cap_taps; q++)
        if (taps) taps[q] = ctx->taps[q];
    return QPIC_OK;
}

qpic_status qpic_fit_coefficients(int32_t solver, double dt, double dz, int32_t n_coef,
                                  double fit_band, double *cE, double *cB, int32_t *L_out)
{
    if (!cE || !cB || !L_out || (solver != QPIC_YEE && solver != QPIC_DUAL)) return QPIC_EINVAL;
    std::string err;
    int L = fit_coefficients(solver, dt, dz, solver == QPIC_YEE ? 1 : n_coef,
                             fit_band > 0 ? fit_band : 0.8, cE, cB, err);
    if (!L) return QPIC_ECFL;
    *L_out = L;
    return QPIC_OK;
}

qpic_status qpic_filter_taps(const double *cB, int32_t L, double tol, double *taps, int32_t cap,
                             int32_t *n_out)
{
    if (!cB || !n_out || L < 1 || L > MAX_L) return QPIC_EINVAL;
    std::string err;
    std::vector<double> t;
    if (!filter_taps_host(cB, L, tol > 0 ? tol : 1e-16, t, err)) return QPIC_ECFL;
    *n_out = (int32_t)t.size();
    for (int q = 0; q < (int)t.size() && q < cap; q++)
        if (taps) taps[q] = t[q];
    return QPIC_OK;
}

qpic_status qpic_stability_limit(int32_t solver, double dz, double dr, int32_t nr, int32_t n_modes,
                                 int32_t n_coef, double fit_band, double *dt_max)
{
    if (!dt_max || nr < 1 || n_modes < 1 || !(dz > 0) || !(dr > 0)) return QPIC_EINVAL;
    std::string err;
    if (!cfl_limit(solver, dz, dr, nr, n_modes, solver == QPIC_YEE ? 1 : n_coef,
                   fit_band > 0 ? fit_band : 0.8, dt_max, err))
        return QPIC_ECFL;
    return QPIC_OK;
}

qpic_status qpic_cfl_limit(const qpic_ctx *ctx, double *dt_max)
{
    if (!ctx || !dt_max) return QPIC_EINVAL;
    std::string err;
    const int L = ctx->cfg.solver == QPIC_YEE ? 1 : ctx->L;
    if (!cfl_limit(ctx->cfg.solver, ctx->dz, ctx->dr, ctx->g.nr, ctx->g.nm, L,
                   ctx->cfg.fit_band > 0 ? ctx->cfg.fit_band : 0.8, dt_max, err))
        return QPIC_ECFL;
    return QPIC_OK;
}

qpic_status qpic_load_plasma(qpic_ctx *c, double n0, double z_start, double ramp_len,
                             int32_t ppc_z, int32_t ppc_r, int32_t ppc_phi, int32_t phi_jitter)
{
    if (!c) return QPIC_EINVAL;
    if (ppc_z < 1 || ppc_r < 1 || ppc_phi < 1 || !(n0 >= 0)) return fail(c, QPIC_EINVAL, "plasma parameters");
    QPIC_REQUIRE_DEVICE(c);
    long long n = (long long)c->g.nz * c->g.nr * ppc_z * ppc_r * ppc_phi;
    long long per_col = (long long)c->g.nr * ppc_z * ppc_r * ppc_phi;
    qpic_status s = ensure_capacity(c, n + (c->cfg.moving_window ? 64 * per_col : 0));
    if (s != QPIC_OK) return s;           // refused: the context keeps its previous state
    c->have_plasma = true;
    c->n0 = n0; c->z_start = z_start; c->ramp_len = ramp_len;
    c->ppc_z = ppc_z; c->ppc_r = ppc_r; c->ppc_phi = ppc_phi; c->jitter = phi_jitter ? 1 : 0;
    // largest weight: density n0 at the outermost sub-particle radius
    double rmax = (c->g.nr - 1 + (ppc_r - 0.5) / ppc_r) * c->dr;
    set_qscale(c, n0 * 2.0 * kPi * rmax * (c->dr / ppc_r) * (c->dz / ppc_z) / ppc_phi);
    cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream);
    if (c->fp64) {
        if (!fp64_load_plasma(c, 0, c->g.nz, false)) return fail(c, QPIC_ECAPACITY, "capacity");
        fp64_compact(c);
        record_ions(c);
        return cuda_check(c, "load_plasma");
    }
    if (!launch_load_plasma(c, 0, c->g.nz, false)) return fail(c, QPIC_ECAPACITY, "capacity");
    launch_sort(c);
    live_count(c);
    record_ions(c);
    return cuda_check(c, "load_plasma");
}

qpic_status qpic_load_particles(qpic_ctx *c, int64_t n, const double *z, const double *r,
                                const double *phi, const double *ux, const double *uy,
                                const double *uz, const double *w)
{
    if (!c || n < 0 || (n > 0 && (!z || !r || !phi || !ux || !uy || !uz || !w)))
        return fail(c, QPIC_EINVAL, "load_particles arguments");
    QPIC_REQUIRE_DEVICE(c);
    qpic_status s = ensure_capacity(c, n);
    if (s != QPIC_OK) return s;
    double *tmp = nullptr;
    if (n > 0) {
        if (!alloc_arr(c, &tmp, (size_t)7 * n)) return fail(c, QPIC_ENOMEM, "staging buffer");
        const double *src[7] = {z, r, phi, ux, uy, uz, w};
        for (int k = 0; k < 7; k++)
            cudaMemcpyAsync(tmp + (size_t)k * n, src[k], n * sizeof(double), cudaMemcpyHostToDevice,
                            c->stream);
    }
    // fixed-point scale from the largest weight (a device reduction over the copy)
    set_qscale(c, n > 0 ? launch_absmax(c, tmp + (size_t)6 * n, n) : 0.0);
    if (c->fp64) {
        fp64_load_particles(c, n, tmp, tmp + n, tmp + 2 * n, tmp + 3 * n, tmp + 4 * n, tmp + 5 * n,
                            tmp + 6 * n);
        cudaStreamSynchronize(c->stream);
        if (tmp) dfree(c, tmp);
        record_ions(c);
        return cuda_check(c, "load_particles");
    }
    launch_load_particles(c, n, tmp, tmp + n, tmp + 2 * n, tmp + 3 * n, tmp + 4 * n, tmp + 5 * n,
                          tmp + 6 * n);
    launch_sort(c);
    cudaStreamSynchronize(c->stream);
    if (tmp) dfree(c, tmp);
    live_count(c);
    record_ions(c);
    return cuda_check(c, "load_particles");
}

qpic_status qpic_add_laser(qpic_ctx *c, double a0, double w0, double fwhm, double z_centroid,
                           double z_focus, double pol_angle)
{
    if (!c) return QPIC_EINVAL;
    if (c->g.nm < 2) return fail(c, QPIC_EINVAL, "a laser needs n_modes >= 2");
    if (!(w0 > 0) || !(fwhm > 0)) return fail(c, QPIC_EINVAL, "laser parameters");
    QPIC_REQUIRE_DEVICE(c);
    launch_laser(c, a0, w0, fwhm, z_centroid, z_focus, pol_angle);
    return cuda_check(c, "add_laser");
}

qpic_status qpic_run_stages(qpic_ctx *c, int32_t stages)
{
    if (!c) return QPIC_EINVAL;
    QPIC_REQUIRE_DEVICE(c);
    cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream);
    run_one_step(c, stages);
    qpic_status s = cuda_check(c, "run_stages");
    if (s != QPIC_OK) return s;
    return check_device_error(c);
}

qpic_status qpic_step(qpic_ctx *c, int32_t nsteps)
{
    if (!c || nsteps < 0) return QPIC_EINVAL;
    QPIC_REQUIRE_DEVICE(c);
    cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream);
    const int all = QPIC_STAGE_FARADAY | QPIC_STAGE_PARTICLES | QPIC_STAGE_AMPERE |
                    QPIC_STAGE_WINDOW | QPIC_STAGE_SORT;
    for (int s = 0; s < nsteps; s++) run_one_step(c, all);
    qpic_status st = cuda_check(c, "step");
    if (st != QPIC_OK) return st;
    return check_device_error(c);
}

qpic_status qpic_get_field(qpic_ctx *c, int32_t which, int32_t comp, int32_t mode, double *re,
                           double *im)
{
    if (!c || !re || comp < 0 || comp > 2 || mode < 0 || mode >= c->g.nm || which < 0 || which > 4)
        return fail(c, QPIC_EINVAL, "get_field arguments");
    QPIC_REQUIRE_DEVICE(c);
    const FieldGeom &g = c->g;
    const size_t nout = (size_t)(g.nr + 1) * g.nz;
    const ColMap cm = col_map(c);
    if (which == QPIC_FIELD_RHO) {
        double *d = nullptr;
        size_t sz = (size_t)g.nm * 2 * nout;
        if (!alloc_arr(c, &d, sz)) return fail(c, QPIC_ENOMEM, "rho buffer");
        launch_rho(c, d);
        cudaMemcpyAsync(re, d + (size_t)(2 * mode) * nout, nout * sizeof(double),
                        cudaMemcpyDeviceToHost, c->stream);
        if (im)
            cudaMemcpyAsync(im, d + (size_t)(2 * mode + 1) * nout, nout * sizeof(double),
                            cudaMemcpyDeviceToHost, c->stream);
        cudaStreamSynchronize(c->stream);
        dfree(c, d);
        return cuda_check(c, "get_field rho");
    }
    if (c->fp64) {
        std::vector<double> dre(g.plane), dim(g.plane, 0.0);
        const double *base = field_base64(c, which);
        int pre = mode == 0 ? 0 : 2 * mode - 1;
        const double *sr = base + (size_t)(comp * g.nparts + pre) * g.plane;
        const double *si = mode ? base + (size_t)(comp * g.nparts + pre + 1) * g.plane : nullptr;
        if (which == QPIC_FIELD_J && comp == QPIC_COMP_Z && c->j_filtered) {
            sr = c->Jz64 + (size_t)pre * g.plane;
            si = mode ? c->Jz64 + (size_t)(pre + 1) * g.plane : nullptr;
        }
        cudaMemcpyAsync(dre.data(), sr, g.plane * 8, cudaMemcpyDeviceToHost, c->stream);
        if (si) cudaMemcpyAsync(dim.data(), si, g.plane * 8, cudaMemcpyDeviceToHost, c->stream);
        if (cudaStreamSynchronize(c->stream) != cudaSuccess) return cuda_check(c, "get_field");
        for (int j = 0; j <= g.nr; j++)
            for (int il = 0; il < g.nz; il++) {
                size_t q = (size_t)j * g.nzp + (il < cm.split ? cm.c0 + il : il - cm.split);
                re[(size_t)j * g.nz + il] = dre[q];
                if (im) im[(size_t)j * g.nz + il] = dim[q];
            }
        return QPIC_OK;
    }
    std::vector<float> hre(g.plane), him(g.plane, 0.f);
    const float *base = field_base(c, which);
    int pre = mode == 0 ? 0 : 2 * mode - 1;
    const float *src_re = base + (size_t)(comp * g.nparts + pre) * g.plane;
    const float *src_im = mode ? base + (size_t)(comp * g.nparts + pre + 1) * g.plane : nullptr;
    if (which == QPIC_FIELD_J && comp == QPIC_COMP_Z && c->j_filtered) {
        src_re = c->Jzf + (size_t)pre * g.plane;
        src_im = mode ? c->Jzf + (size_t)(pre + 1) * g.plane : nullptr;
    }
    cudaMemcpyAsync(hre.data(), src_re, g.plane * sizeof(float), cudaMemcpyDeviceToHost, c->stream);
    if (src_im)
        cudaMemcpyAsync(him.data(), src_im, g.plane * sizeof(float), cudaMemcpyDeviceToHost, c->stream);
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return cuda_check(c, "get_field");
    for (int j = 0; j <= g.nr; j++)
        for (int il = 0; il < g.nz; il++) {
            size_t q = (size_t)j * g.nzp + (il < cm.split ? cm.c0 + il : il - cm.split);
            re[(size_t)j * g.nz + il] = hre[q];
            if (im) im[(size_t)j * g.nz + il] = him[q];
        }
    return QPIC_OK;
}

qpic_status qpic_set_field(qpic_ctx *c, int32_t which, int32_t comp, int32_t mode, const double *re,
                           const double *im)
{
    if (!c || !re || comp < 0 || comp > 2 || mode < 0 || mode >= c->g.nm ||
        (which != QPIC_FIELD_E && which != QPIC_FIELD_B && which != QPIC_FIELD_BBAR))
        return fail(c, QPIC_EINVAL, "set_field arguments");
    QPIC_REQUIRE_DEVICE(c);
    const FieldGeom &g = c->g;
    const ColMap cm = col_map(c);
    if (c->fp64) {
        std::vector<double> dre(g.plane, 0.0), dim(g.plane, 0.0);
        for (int j = 0; j <= g.nr; j++)
            for (int il = 0; il < g.nz; il++) {
                size_t q = (size_t)j * g.nzp + (il < cm.split ? cm.c0 + il : il - cm.split);
                dre[q] = re[(size_t)j * g.nz + il];
                dim[q] = im ? im[(size_t)j * g.nz + il] : 0.0;
            }
        double *base = field_base64(c, which);
        int pre = mode == 0 ? 0 : 2 * mode - 1;
        cudaMemcpyAsync(base + (size_t)(comp * g.nparts + pre) * g.plane, dre.data(), g.plane * 8,
                        cudaMemcpyHostToDevice, c->stream);
        if (mode)
            cudaMemcpyAsync(base + (size_t)(comp * g.nparts + pre + 1) * g.plane, dim.data(),
                            g.plane * 8, cudaMemcpyHostToDevice, c->stream);
        cudaStreamSynchronize(c->stream);
        return cuda_check(c, "set_field");
    }
    std::vector<float> hre(g.plane, 0.f), him(mode ? g.plane : 0, 0.f);
    for (int j = 0; j <= g.nr; j++) {
        const double *rr = re + (size_t)j * g.nz;
        float *dr_ = hre.data() + (size_t)j * g.nzp;
        for (long long il = 0; il < cm.split; il++) dr_[cm.c0 + il] = (float)rr[il];
        for (long long il = cm.split; il < g.nz; il++) dr_[il - cm.split] = (float)rr[il];
        if (mode && im) {
            const double *ri = im + (size_t)j * g.nz;
            float *di = him.data() + (size_t)j * g.nzp;
            for (long long il = 0; il < cm.split; il++) di[cm.c0 + il] = (float)ri[il];
            for (long long il = cm.split; il < g.nz; il++) di[il - cm.split] = (float)ri[il];
        }
    }
    float *base = field_base(c, which);
    int pre = mode == 0 ? 0 : 2 * mode - 1;
    cudaMemcpyAsync(base + (size_t)(comp * g.nparts + pre) * g.plane, hre.data(),
                    g.plane * sizeof(float), cudaMemcpyHostToDevice, c->stream);
    if (mode)
        cudaMemcpyAsync(base + (size_t)(comp * g.nparts + pre + 1) * g.plane, him.data(),
                        g.plane * sizeof(float), cudaMemcpyHostToDevice, c->stream);
    cudaStreamSynchronize(c->stream);
    return cuda_check(c, "set_field");
}

qpic_status qpic_get_fields(qpic_ctx *c, int32_t which, int32_t comp, int32_t mode, double *re,
                            double *im, int64_t count)
{
    if (!c) return QPIC_EINVAL;
    if (count < (int64_t)(c->g.nr + 1) * c->g.nz)
        return fail(c, QPIC_EINVAL, "get_fields: buffer shorter than (nr+1)*nz");
    return qpic_get_field(c, which, comp, mode, re, im);
}

qpic_status qpic_set_fields(qpic_ctx *c, int32_t which, int32_t comp, int32_t mode, const double *re,
                            const double *im, int64_t count)
{
    if (!c) return QPIC_EINVAL;
    if (count < (int64_t)(c->g.nr + 1) * c->g.nz)
        return fail(c, QPIC_EINVAL, "set_fields: buffer shorter than (nr+1)*nz");
    return qpic_set_field(c, which, comp, mode, re, im);
}

// ---------------------------------------------------------------- snapshots
// A snapshot is a header followed by raw device words: the E, B and Bbar
// planes in their physical (circular z) layout, the live particles (sorted,
// dead ones dropped), the modal-work counters when tracked and the ion
// background of the Gauss diagnostic.  Loading it into a context of the same
// configuration resumes the run: the current is an integer sum over particles
// (FP32 path), so the steps after a load are bit-identical to the steps the
// saved context would have taken.
namespace {

const unsigned long long kSnapMagic = 0x50414e5343495051ull;   // "QPICSNAP"

struct SnapHeader {
    unsigned long long magic;
    int32_t version, nz, nr, nm, precision, track_work, periodic, solver, L, nzp;
    double dz, dr, dt, qref;
    long long nstep, shifts, zoff, np;
    int32_t have_plasma, ppc_z, ppc_r, ppc_phi, jitter, has_ions;
    double n0, z_start, ramp_len;
    unsigned long long seed;
    long long field_bytes, particle_bytes, ion_bytes;
};

size_t snap_field_words(const qpic_ctx *c) { return (size_t)3 * c->g.nparts * c->g.plane; }
size_t snap_ion_doubles(const qpic_ctx *c) { return (size_t)c->g.nm * 2 * (c->g.nr + 1) * c->g.nz; }

// live particles in buffer order, sorted (FP32) or compacted (FP64); returns the count
long long snap_prepare(qpic_ctx *c)
{
    if (c->fp64) {
        fp64_compact(c);
        cudaStreamSynchronize(c->stream);
        return c->np;
    }
    launch_sort(c);
    return live_count(c);
}

SnapHeader snap_header(const qpic_ctx *c, long long np)
{
    SnapHeader h;
    std::memset(&h, 0, sizeof(h));
    h.magic = kSnapMagic; h.version = 1;
    h.nz = c->g.nz; h.nr = c->g.nr; h.nm = c->g.nm; h.precision = c->cfg.precision;
    h.track_work = c->cfg.track_work; h.periodic = c->g.periodic; h.solver = c->cfg.solver; h.L = c->L;
    h.nzp = c->g.nzp;
    h.dz = c->dz; h.dr = c->dr; h.dt = c->dt; h.qref = c->qref;
    h.nstep = c->nstep; h.shifts = c->shifts; h.zoff = c->g.zoff; h.np = np;
    h.have_plasma = c->have_plasma; h.ppc_z = c->ppc_z; h.ppc_r = c->ppc_r; h.ppc_phi = c->ppc_phi;
    h.jitter = c->jitter; h.has_ions = c->rho_ion != nullptr;
    h.n0 = c->n0; h.z_start = c->z_start; h.ramp_len = c->ramp_len; h.seed = c->cfg.seed;
    const size_t fw = c->fp64 ? sizeof(double) : sizeof(float);
    h.field_bytes = (long long)(3 * snap_field_words(c) * fw);
    const long long per = c->fp64 ? (7 + (c->cfg.track_work ? 2 : 0)) * 8
                                  : 4 + 32 + (c->cfg.track_work ? 8 : 0);
    h.particle_bytes = np * per;
    h.ion_bytes = h.has_ions ? (long long)(snap_ion_doubles(c) * sizeof(double)) : 0;
    return h;
}

long long snap_bytes(const SnapHeader &h)
{
    return (long long)sizeof(SnapHeader) + h.field_bytes + h.particle_bytes + h.ion_bytes;
}

// the device arrays of a snapshot, in order, with their byte sizes
std::vector<std::pair<void *, size_t>> snap_arrays(qpic_ctx *c, long long np)
{
    std::vector<std::pair<void *, size_t>> v;
    const size_t fwords = snap_field_words(c);
    if (c->fp64) {
        v.push_back({c->E64, fwords * 8}); v.push_back({c->B64, fwords * 8}); v.push_back({c->Bb64, fwords * 8});
        double *a[7] = {c->p64.z, c->p64.x, c->p64.y, c->p64.ux, c->p64.uy, c->p64.uz, c->p64.w};
        for (double *x : a) v.push_back({x, (size_t)np * 8});
        if (c->cfg.track_work) { v.push_back({c->p64.W0, (size_t)np * 8}); v.push_back({c->p64.W1, (size_t)np * 8}); }
    } else {
        v.push_back({c->E, fwords * 4}); v.push_back({c->B, fwords * 4}); v.push_back({c->Bb, fwords * 4});
        v.push_back({c->p.cell, (size_t)np * 4});
        v.push_back({c->p.rec, (size_t)np * 32});
        if (c->cfg.track_work) { v.push_back({c->p.W0, (size_t)np * 4}); v.push_back({c->p.W1, (size_t)np * 4}); }
    }
    if (c->rho_ion) v.push_back({c->rho_ion, snap_ion_doubles(c) * 8});
    return v;
}

}  // namespace

qpic_status qpic_state_size(qpic_ctx *c, int64_t *bytes)
{
    if (!c || !bytes) return QPIC_EINVAL;
    QPIC_REQUIRE_DEVICE(c);
    const long long np = snap_prepare(c);
    *bytes = snap_bytes(snap_header(c, np));
    return cuda_check(c, "state_size");
}

qpic_status qpic_save_state(qpic_ctx *c, void *buf, int64_t capacity, int64_t *written)
{
    if (!c || !buf) return QPIC_EINVAL;
    QPIC_REQUIRE_DEVICE(c);
    const long long np = snap_prepare(c);
    const SnapHeader h = snap_header(c, np);
    const long long need = snap_bytes(h);
    if (written) *written = need;
    if (need > capacity) return fail(c, QPIC_ECAPACITY, "save_state: buffer holds " + std::to_string(capacity) +
                                                            " bytes, the snapshot needs " + std::to_string(need));
    char *out = static_cast<char *>(buf);
    std::memcpy(out, &h, sizeof(h));
    size_t off = sizeof(h);
    for (const auto &a : snap_arrays(c, np)) {
        if (a.second) cudaMemcpyAsync(out + off, a.first, a.second, cudaMemcpyDeviceToHost, c->stream);
        off += a.second;
    }
    cudaStreamSynchronize(c->stream);
    return cuda_check(c, "save_state");
}

qpic_status qpic_load_state(qpic_ctx *c, const void *buf, int64_t size)
{
    if (!c || !buf || size < (int64_t)sizeof(SnapHeader)) return fail(c, QPIC_EINVAL, "load_state arguments");
    QPIC_REQUIRE_DEVICE(c);
    SnapHeader h;
    std::memcpy(&h, buf, sizeof(h));
    if (h.magic != kSnapMagic || h.version != 1) return fail(c, QPIC_EINVAL, "load_state: not a snapshot");
    if (h.nz != c->g.nz || h.nr != c->g.nr || h.nm != c->g.nm || h.precision != c->cfg.precision ||
        h.track_work != c->cfg.track_work || h.periodic != c->g.periodic || h.solver != c->cfg.solver ||
        h.L != c->L || h.nzp != c->g.nzp || h.dz != c->dz || h.dr != c->dr || h.dt != c->dt)
        return fail(c, QPIC_EINVAL, "load_state: the snapshot was taken with another configuration");
    if (snap_bytes(h) != size) return fail(c, QPIC_EINVAL, "load_state: size does not match the header");
    qpic_status st = ensure_capacity(c, h.np);
    if (st != QPIC_OK) return st;
    if (h.has_ions && !c->rho_ion && !alloc_arr(c, &c->rho_ion, snap_ion_doubles(c)))
        return fail(c, QPIC_ENOMEM, "load_state: ion background");
    c->nstep = h.nstep; c->shifts = h.shifts; c->g.zoff = h.zoff;
    c->have_plasma = h.have_plasma != 0; c->n0 = h.n0; c->z_start = h.z_start; c->ramp_len = h.ramp_len;
    c->ppc_z = h.ppc_z; c->ppc_r = h.ppc_r; c->ppc_phi = h.ppc_phi; c->jitter = h.jitter;
    c->cfg.seed = h.seed;
    set_qscale(c, h.qref);
    const char *in = static_cast<const char *>(buf);
    size_t off = sizeof(h);
    for (const auto &a : snap_arrays(c, h.np)) {
        if (a.second) cudaMemcpyAsync(a.first, in + off, a.second, cudaMemcpyHostToDevice, c->stream);
        off += a.second;
    }
    c->np = h.np;
    c->n_tail = 0;
    c->j_filtered = false;
    cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream);
    if (c->fp64) {
        cudaStreamSynchronize(c->stream);
        return cuda_check(c, "load_state");
    }
    // the saved particles are sorted: set the counts and rebuild the tile offsets
    const long long counts[2] = {h.np, h.np};
    cudaMemcpyAsync(c->d_count, counts, sizeof(counts), cudaMemcpyHostToDevice, c->stream);
    cudaMemsetAsync(c->tstamp, 0xff, (size_t)c->ntz * c->ntr * sizeof(int), c->stream);
    cudaMemsetAsync(c->jdirty, 0, (size_t)c->ntz * c->ntr * sizeof(int), c->stream);
    cudaMemsetAsync(c->d_epoch, 0, 4 * sizeof(int), c->stream);
    launch_sort(c);
    cudaStreamSynchronize(c->stream);
    return cuda_check(c, "load_state");
}

qpic_status qpic_num_particles(qpic_ctx *c, int64_t *n)
{
    if (!c || !n) return QPIC_EINVAL;
    QPIC_REQUIRE_DEVICE(c);
    if (c->fp64) {
        fp64_compact(c);
        *n = c->np;
        return cuda_check(c, "num_particles");
    }
    launch_sort(c);
    *n = live_count(c);
    return cuda_check(c, "num_particles");
}

qpic_status qpic_get_particles(qpic_ctx *c, double *out, int64_t capacity, int64_t *n_out)
{
    if (!c || !out || !n_out) return QPIC_EINVAL;
    QPIC_REQUIRE_DEVICE(c);
    long long n;
    if (c->fp64) {
        fp64_compact(c);
        n = c->np;
    } else {
        launch_sort(c);
        n = live_count(c);
    }
    *n_out = n;
    if (n > capacity) return fail(c, QPIC_ECAPACITY, "get_particles: capacity too small");
    double *d = nullptr;
    if (n > 0) {
        if (!alloc_arr(c, &d, (size_t)9 * n)) return fail(c, QPIC_ENOMEM, "export buffer");
        if (c->fp64) fp64_export_particles(c, d, n);
        else launch_export_particles(c, d, n);
        for (int k = 0; k < 9; k++)
            cudaMemcpyAsync(out + (size_t)k * capacity, d + (size_t)k * n, n * sizeof(double),
                            cudaMemcpyDeviceToHost, c->stream);
        cudaStreamSynchronize(c->stream);
        dfree(c, d);
    }
    return cuda_check(c, "get_particles");
}

qpic_status qpic_get_particles_raw(qpic_ctx *c, double *out, int64_t capacity, int64_t *n_out)
{
    if (!c || !out || !n_out) return QPIC_EINVAL;
    QPIC_REQUIRE_DEVICE(c);
    long long n = c->fp64 ? c->np : live_count(c);   // buffer slots in use
    *n_out = n;
    if (n > capacity) return fail(c, QPIC_ECAPACITY, "get_particles_raw: capacity too small");
    double *d = nullptr;
    if (n > 0) {
        if (!alloc_arr(c, &d, (size_t)9 * n)) return fail(c, QPIC_ENOMEM, "export buffer");
        if (c->fp64) fp64_export_particles(c, d, n);
        else launch_export_particles(c, d, n);
        for (int k = 0; k < 9; k++)
            cudaMemcpyAsync(out + (size_t)k * capacity, d + (size_t)k * n, n * sizeof(double),
                            cudaMemcpyDeviceToHost, c->stream);
        cudaStreamSynchronize(c->stream);
        dfree(c, d);
    }
    return cuda_check(c, "get_particles_raw");
}

qpic_status qpic_work_f_estimate(int64_t n, const double *ux, const double *uy, const double *uz,
                                 const double *Wz, const double *Wperp, double omega_p, double w0,
                                 double omega0, double *lwfa, double *dla)
{
    if (n < 0 || !(omega_p > 0) || !(w0 > 0) || !(omega0 > 0)) return QPIC_EINVAL;
    if (n > 0 && (!ux || !uy || !uz || !Wz || !Wperp || !lwfa || !dla)) return QPIC_EINVAL;
    const double k = -2.0 / (omega0 * omega_p * w0 * w0);
    for (int64_t p = 0; p < n; p++) {
        const double gamma = std::sqrt(1.0 + ux[p] * ux[p] + uy[p] * uy[p] + uz[p] * uz[p]);
        const double f = k * std::sqrt(2.0 * gamma);          // Eq. 19
        lwfa[p] = Wz[p] - f * Wperp[p];                        // Eq. 20
        dla[p] = (1.0 + f) * Wperp[p];
    }
    return QPIC_OK;
}

qpic_status qpic_get_diag(qpic_ctx *c, double *out, int32_t count)
{
    if (!c || !out) return QPIC_EINVAL;
    QPIC_REQUIRE_DEVICE(c);
    const int nm = c->g.nm;
    std::vector<double> v(7 + nm, 0.0);
    v[0] = c->nstep * c->dt;
    v[1] = (double)c->nstep;
    v[2] = (double)c->shifts;
    // all reductions and the error word are copied into pinned host words and
    // read after one synchronisation (pageable words when pinning failed)
    if (!c->h_diag && cudaMallocHost(&c->h_diag, 64 * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        c->h_diag = nullptr;
    }
    double hv[64];
    double *hb = c->h_diag ? c->h_diag : hv;
    int *he = reinterpret_cast<int *>(hb + 32);
    for (int m = 0; m < nm; m++) hb[3 + m] = 0.0;       // (no copy when the reduction buffer is short)
    if (c->fp64) fp64_particle_sums(c, hb);
    else launch_particle_sums(c, hb);
    launch_field_energy(c, hb + 3);
    cudaMemcpyAsync(he, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    cudaStreamSynchronize(c->stream);
    v[3] = hb[0]; v[4] = hb[1]; v[5] = hb[2];
    for (int m = 0; m < nm; m++) v[6 + m] = hb[3 + m];
    v[6 + nm] = (*he & 1) ? 1.0 : 0.0;
    for (int k = 0; k < count && k < (int)v.size(); k++) out[k] = v[k];
    qpic_status st = cuda_check(c, "get_diag");
    if (st != QPIC_OK) return st;
    // a NaN or infinity anywhere in the fields or the particles reaches these sums
    for (int k = 4; k < 6 + nm; k++)
        if (!std::isfinite(v[k]))
            return fail(c, QPIC_ENONFINITE, "get_diag: non-finite charge, kinetic or field energy "
                                            "(NaN or infinity in the particles or fields)");
    return QPIC_OK;
}

qpic_status qpic_gauss_residual(qpic_ctx *c, double *out, int32_t count)
{
    if (!c || !out) return QPIC_EINVAL;
    QPIC_REQUIRE_DEVICE(c);
    if (c->cfg.moving_window) return fail(c, QPIC_ESTATE, "gauss_residual: ion background moves with the window");
    if (!c->rho_ion) return fail(c, QPIC_ESTATE, "gauss_residual: no particles loaded");
    const int nm = c->g.nm;
    const size_t n = (size_t)nm * 2 * (c->g.nr + 1) * c->g.nz;
    double *rho = nullptr, *scr = nullptr;
    const size_t nscr = (size_t)2 * 4 * (c->g.nr + 1) * nm + 2 * nm;
    if (!alloc_arr(c, &rho, n) || !alloc_arr(c, &scr, nscr)) {
        dfree(c, rho);
        return fail(c, QPIC_ENOMEM, "gauss_residual buffers");
    }
    launch_rho(c, rho);
    std::vector<double> h(2 * nm);
    launch_gauss(c, rho, c->rho_ion, scr, h.data());
    dfree(c, rho);
    dfree(c, scr);
    for (int k = 0; k < 2 * nm && k < count; k++) out[k] = std::sqrt(h[k]);
    return cuda_check(c, "gauss_residual");
}

qpic_status qpic_spectrum(qpic_ctx *c, const double *edges_mev, int32_t nbins, double *weights)
{
    if (!c || !edges_mev || !weights || nbins < 1 || nbins > 4096) return fail(c, QPIC_EINVAL, "spectrum arguments");
    for (int k = 0; k < nbins; k++)
        if (!(edges_mev[k + 1] > edges_mev[k])) return fail(c, QPIC_EINVAL, "spectrum: edges must increase");
    QPIC_REQUIRE_DEVICE(c);
    const double wmax = c->fp64 ? 0.0 : c->qref;
    double *de = nullptr;
    unsigned long long *dh = nullptr;
    if (!alloc_arr(c, &de, (size_t)nbins + 1) || !alloc_arr(c, &dh, (size_t)nbins)) {
        dfree(c, de);
        return fail(c, QPIC_ENOMEM, "spectrum buffers");
    }
    cudaMemcpyAsync(de, edges_mev, (nbins + 1) * sizeof(double), cudaMemcpyHostToDevice, c->stream);
    // weights in int64 fixed point at 2^32 per largest weight
    double wref = wmax;
    if (c->fp64 || !(wref > 0)) {
        double s3[3];
        if (c->fp64) fp64_particle_sums(c, s3); else launch_particle_sums(c, s3);
        cudaStreamSynchronize(c->stream);
        wref = s3[0] > 0 ? std::fabs(s3[1]) / s3[0] * 64.0 : 1.0;    // mean weight x 64
    }
    const double wscale = 4294967296.0 / wref;
    if (c->fp64) fp64_spectrum(c, de, nbins, wscale, dh);
    else launch_spectrum(c, de, nbins, wscale, dh);
    std::vector<unsigned long long> h(nbins);
    cudaMemcpyAsync(h.data(), dh, nbins * sizeof(unsigned long long), cudaMemcpyDeviceToHost, c->stream);
    cudaStreamSynchronize(c->stream);
    dfree(c, de);
    dfree(c, dh);
    for (int k = 0; k < nbins; k++) weights[k] = (double)h[k] / wscale;
    return cuda_check(c, "spectrum");
}

qpic_status qpic_profile(qpic_ctx *c, int32_t enable, int32_t reset)
{
    if (!c) return QPIC_EINVAL;
    resolve_events(c);
    c->profile = enable != 0;
    // events are created up front: creating them between launches would hold
    // the host back and leave gaps on the GPU inside the timed pairs
    while (c->profile && c->ev_pool.size() < 4096) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) { cudaGetLastError(); break; }
        c->ev_pool.push_back(e);
    }
    if (reset) {
        for (int k = 0; k < KC_COUNT; k++) { c->kms[k] = 0.0; c->klaunch[k] = 0; }
    }
    return QPIC_OK;
}

qpic_status qpic_launch_count(const qpic_ctx *c, int64_t *n)
{
    if (!c || !n) return QPIC_EINVAL;
    *n = c->n_kernels;
    return QPIC_OK;
}

qpic_status qpic_kernel_times(qpic_ctx *c, int32_t n, double *ms, int64_t *launches,
                              const char **names, int32_t *n_classes)
{
    static const char *kNames[KC_COUNT] = {"faraday", "gather_push_deposit", "j_decode",
                                           "jz_filter", "ampere", "sort", "window",
                                           "inject", "diag", "other"};
    if (!c) return QPIC_EINVAL;
    resolve_events(c);
    if (n_classes) *n_classes = KC_COUNT;
    for (int k = 0; k < n && k < KC_COUNT; k++) {
        if (ms) ms[k] = c->kms[k];
        if (launches) launches[k] = c->klaunch[k];
        if (names) names[k] = kNames[k];
    }
    return QPIC_OK;
}

// ---------------------------------------------------------------- batches
// A batch advances many independent runs with one graph launch per cycle of
// steps.  At creation the cycle is captured once.  Each step has three
// phases: Faraday and the step's epoch on each run's own stream (parallel
// branches of the graph); then one persistent launch per group of runs with
// the same mode count and tile shape, walking the (run, tile) work list of
// the particle phase -- gather, push and deposit, then the current
// reduction, with bounded waits between them (k_batch_particles); then the
// J_z filter, Ampere and the sort again on the runs' own streams.

}  // extern "C"

struct qpic_batch {
    std::vector<qpic_ctx *> runs;
    cudaStream_t main = nullptr;
    std::vector<cudaStream_t> side;
    std::vector<cudaEvent_t> ev_join;
    cudaEvent_t ev_fork = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int period = 2;
    bool own_main = false;
    std::vector<long long> kernels_per_cycle;
    long long batch_kernels_per_cycle = 0;
    // the batched particle phase: runs grouped by (mode parts, tile shape), at
    // most BATCH_GROUP runs per group; per group the tile prefix over its runs,
    // its work-list counter and one device run table per step of the cycle
    struct Group {
        int nparts = 0, tz = 0, tr = 0;
        std::vector<int> members;      // indices into runs
        int *d_prefix = nullptr, *d_head = nullptr;
        std::vector<void *> d_tables;
    };
    std::vector<Group> groups;
    std::vector<int *> gdone;          // per run: per tile, epoch of its last stored deposit
    qpic::BatchCtlHost *d_ctl = nullptr;
    int blocks = 304;
    std::string err;
};

static const int BATCH_GROUP = 64;   // runs per persistent launch (its constant-memory run table)

static qpic_status batch_fail(qpic_batch *b, qpic_status s, const std::string &m)
{
    b->err = m;
    return s;
}

extern "C" {

void qpic_batch_destroy(qpic_batch *b)
{
    if (!b) return;
    if (b->main) cudaStreamSynchronize(b->main);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (cudaStream_t s : b->side) cudaStreamDestroy(s);
    for (cudaEvent_t e : b->ev_join) cudaEventDestroy(e);
    if (b->ev_fork) cudaEventDestroy(b->ev_fork);
    for (auto &g : b->groups) {
        cudaFree(g.d_prefix);
        cudaFree(g.d_head);
        for (void *t : g.d_tables) cudaFree(t);
    }
    for (int *p : b->gdone) cudaFree(p);
    cudaFree(b->d_ctl);
    if (b->own_main && b->main) cudaStreamDestroy(b->main);
    delete b;
}

int32_t qpic_batch_cycle(const qpic_batch *b)
{
    return b ? b->period : 0;
}

const char *qpic_batch_last_error(const qpic_batch *b) { return b ? b->err.c_str() : "no batch"; }

qpic_status qpic_batch_set_wait(qpic_batch *b, int64_t polls, int32_t withheld_item)
{
    if (!b || !b->d_ctl || polls < 0) return QPIC_EINVAL;
    const qpic::BatchCtlHost h{(long long)polls, withheld_item < 0 ? -1 : (int)withheld_item, 0};
    cudaStreamSynchronize(b->main);
    return cudaMemcpy(b->d_ctl, &h, sizeof(h), cudaMemcpyHostToDevice) == cudaSuccess ? QPIC_OK : QPIC_ECUDA;
}

qpic_status qpic_batch_create(qpic_ctx *const *runs, int32_t n, void *cuda_stream, qpic_batch **out)
{
    if (!out) return QPIC_EINVAL;
    *out = nullptr;
    if (!runs || n < 1) return QPIC_EINVAL;
    qpic_batch *b = new (std::nothrow) qpic_batch();
    if (!b) return QPIC_ENOMEM;
    *out = b;
    b->main = static_cast<cudaStream_t>(cuda_stream);
    if (!b->main) {                    // the legacy default stream cannot be captured
        if (cudaStreamCreateWithFlags(&b->main, cudaStreamNonBlocking) != cudaSuccess)
            return batch_fail(b, QPIC_ECUDA, "batch stream creation failed");
        b->own_main = true;
    }
    // a sort swaps the particle buffers on the host; a captured cycle must hold
    // an even number of sorts of every run, so that each replay starts from the
    // buffers the graph was recorded with: the cycle is twice the least common
    // multiple of the runs' sort periods
    long long lcm = 1;
    for (int k = 0; k < n; k++) {
        qpic_ctx *c = runs[k];
        if (!c) return batch_fail(b, QPIC_EINVAL, "null run");
        if (c->fp64 || c->fatomic || c->cfg.moving_window || c->profile)
            return batch_fail(b, QPIC_EINVAL, "batch runs: FP32 fixed-point path, periodic box, profiling off");
        if (check_device(c) != QPIC_OK) return batch_fail(b, QPIC_ESTATE, "batch runs: " + c->err);
        const long long sp = c->sort_period > 1 ? c->sort_period : 1;
        // a particle drifts at most one cell per step from the tile it was
        // sorted into, and its deposit reaches two nodes further: the current
        // reduction of a tile then needs the particle items of the 3 x 3 tiles
        // around it only while the sort period is below the tile size minus 2
        if (sp + 3 > std::min(c->TZ, c->TR))
            return batch_fail(b, QPIC_EINVAL, "batch runs: sort period must be at most min(TZ, TR) - 3");
        long long a = lcm, bb = sp;
        while (bb) { const long long t = a % bb; a = bb; bb = t; }
        lcm = lcm / a * sp;
        if (lcm > 8) return batch_fail(b, QPIC_EINVAL, "batch runs: sort periods whose cycle exceeds 16 steps");
        b->runs.push_back(c);
    }
    b->period = (int)(2 * lcm);
    const int all = QPIC_STAGE_FARADAY | QPIC_STAGE_PARTICLES | QPIC_STAGE_AMPERE |
                    QPIC_STAGE_WINDOW | QPIC_STAGE_SORT;
    // bring every run to a cycle boundary with its particles sorted (a run
    // stepped on its own does the same steps: a sort falls on every cycle
    // boundary), then drain all work
    for (qpic_ctx *c : b->runs) {
        for (int guard = 0; c->nstep % b->period || c->n_tail > 0; guard++) {
            if (guard > 2 * b->period) return batch_fail(b, QPIC_ESTATE, "batch runs: particles stay unsorted");
            run_one_step(c, all);
        }
        cudaStreamSynchronize(c->stream);
    }
    // groups of the particle phase, per-tile publication flags, control word
    int nsm = 152;
    {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    }
    b->blocks = 2 * nsm;                          // resident blocks: two per SM
    b->gdone.assign(n, nullptr);
    for (int k = 0; k < n; k++) {
        qpic_ctx *c = b->runs[k];
        const size_t nt = (size_t)c->ntz * c->ntr;
        if (cudaMalloc(&b->gdone[k], nt * sizeof(int)) != cudaSuccess)
            return batch_fail(b, QPIC_ENOMEM, "batch flags");
        cudaMemset(b->gdone[k], 0xff, nt * sizeof(int));
        bool placed = false;
        for (auto &g : b->groups)
            if (g.nparts == c->g.nparts && g.tz == c->TZ && g.tr == c->TR && (int)g.members.size() < BATCH_GROUP) {
                g.members.push_back(k);
                placed = true;
                break;
            }
        if (!placed) {
            qpic_batch::Group g;
            g.nparts = c->g.nparts; g.tz = c->TZ; g.tr = c->TR;
            g.members.push_back(k);
            b->groups.push_back(g);
        }
    }
    if (cudaMalloc(&b->d_ctl, sizeof(qpic::BatchCtlHost)) != cudaSuccess)
        return batch_fail(b, QPIC_ENOMEM, "batch control word");
    const qpic::BatchCtlHost ctl = qpic::batch_ctl_default();
    cudaMemcpy(b->d_ctl, &ctl, sizeof(ctl), cudaMemcpyHostToDevice);
    // the run tables hold each run's particle buffers at each step of the
    // cycle: the buffers swap after every sort, which is due after step s
    // when (nstep + s + 1) is a multiple of the run's period
    const size_t rb = qpic::batch_run_bytes();
    for (auto &g : b->groups) {
        const int m = (int)g.members.size();
        std::vector<int> prefix(m + 1, 0);
        for (int i = 0; i < m; i++) {
            qpic_ctx *c = b->runs[g.members[i]];
            prefix[i + 1] = prefix[i] + c->ntz * c->ntr;
        }
        if (cudaMalloc(&g.d_prefix, (m + 1) * sizeof(int)) != cudaSuccess ||
            cudaMalloc(&g.d_head, sizeof(int)) != cudaSuccess)
            return batch_fail(b, QPIC_ENOMEM, "batch work list");
        cudaMemcpy(g.d_prefix, prefix.data(), (m + 1) * sizeof(int), cudaMemcpyHostToDevice);
        std::vector<char> host((size_t)m * rb);
        for (int s2 = 0; s2 < b->period; s2++) {
            for (int i = 0; i < m; i++) {
                const int k = g.members[i];
                qpic_ctx *c = b->runs[k];
                const long long sp = c->sort_period > 1 ? c->sort_period : 1;
                long long sorts = 0;                  // sorts of this run before step s2 of the cycle
                for (int q = 0; q < s2; q++)
                    if ((c->nstep + q + 1) % sp == 0) sorts++;
                qpic::batch_fill_run(c, (sorts & 1) ? c->ps : c->p, b->gdone[k], host.data() + (size_t)i * rb);
            }
            void *t = nullptr;
            if (cudaMalloc(&t, (size_t)m * rb) != cudaSuccess) return batch_fail(b, QPIC_ENOMEM, "batch tables");
            cudaMemcpy(t, host.data(), (size_t)m * rb, cudaMemcpyHostToDevice);
            g.d_tables.push_back(t);
        }
    }
    b->side.resize(n);
    b->ev_join.resize(n);
    for (int k = 0; k < n; k++) {
        if (cudaStreamCreateWithFlags(&b->side[k], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&b->ev_join[k], cudaEventDisableTiming) != cudaSuccess)
            return batch_fail(b, QPIC_ECUDA, "stream/event creation failed");
    }
    if (cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming) != cudaSuccess)
        return batch_fail(b, QPIC_ECUDA, "event creation failed");
    cudaError_t e = cudaStreamBeginCapture(b->main, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) return batch_fail(b, QPIC_ECUDA, std::string("capture: ") + cudaGetErrorString(e));
    b->kernels_per_cycle.assign(n, 0);
    std::vector<long long> nk0(n), ns0(n);
    std::vector<Particles> p0(n);
    std::vector<cudaStream_t> old(n);
    for (int k = 0; k < n; k++) {
        qpic_ctx *c = b->runs[k];
        nk0[k] = c->n_kernels; ns0[k] = c->nstep; p0[k] = c->p; old[k] = c->stream;
        c->stream = b->side[k];
    }
    // fork the runs' branches off the batch stream, then join them back
    auto fork = [&]() {
        cudaEventRecord(b->ev_fork, b->main);
        for (int k = 0; k < n; k++) cudaStreamWaitEvent(b->side[k], b->ev_fork, 0);
    };
    auto join = [&]() {
        for (int k = 0; k < n; k++) {
            cudaEventRecord(b->ev_join[k], b->side[k]);
            cudaStreamWaitEvent(b->main, b->ev_join[k], 0);
        }
    };
    bool shape_ok = true;
    for (int s2 = 0; s2 < b->period; s2++) {
        fork();
        for (qpic_ctx *c : b->runs) {
            launch_faraday(c);
            qpic::launch_epoch(c);
        }
        join();
        for (auto &g : b->groups) {
            cudaMemsetAsync(g.d_head, 0, sizeof(int), b->main);
            if (!qpic::launch_batch_particles(g.nparts, g.tz, g.tr, g.d_tables[s2], g.d_prefix,
                                              (int)g.members.size(), g.d_head, b->d_ctl, b->blocks, b->main))
                shape_ok = false;
        }
        fork();
        for (qpic_ctx *c : b->runs) {
            c->j_filtered = false;
            if (!c->taps.empty()) launch_jfilter(c);
            c->j_filtered = !c->taps.empty();
            launch_ampere(c);
            c->nstep++;
            const long long sp = c->sort_period > 1 ? c->sort_period : 1;
            if (c->nstep % sp == 0) launch_sort(c);
        }
        join();
    }
    b->batch_kernels_per_cycle = (long long)b->period * (long long)b->groups.size();
    bool odd = false;
    for (int k = 0; k < n; k++) {
        qpic_ctx *c = b->runs[k];
        b->kernels_per_cycle[k] = c->n_kernels - nk0[k];
        c->n_kernels = nk0[k];                  // captured, not executed
        c->nstep = ns0[k];
        c->stream = old[k];
        if (c->p.cell != p0[k].cell) odd = true;
    }
    e = cudaStreamEndCapture(b->main, &b->graph);
    if (odd) {
        for (int k = 0; k < n; k++) {
            qpic_ctx *c = b->runs[k];
            if (c->p.cell != p0[k].cell) { Particles t = c->p; c->p = c->ps; c->ps = t; }
        }
        return batch_fail(b, QPIC_EINVAL, "captured cycle holds an odd number of sorts");
    }
    if (e != cudaSuccess) return batch_fail(b, QPIC_ECUDA, std::string("end capture: ") + cudaGetErrorString(e));
    if (!shape_ok) return batch_fail(b, QPIC_EINVAL, "batch runs: tile shape without a batched particle kernel");
    e = cudaGraphInstantiate(&b->exec, b->graph, 0);
    if (e != cudaSuccess) return batch_fail(b, QPIC_ECUDA, std::string("instantiate: ") + cudaGetErrorString(e));
    return QPIC_OK;
}

qpic_status qpic_batch_step(qpic_batch *b, int32_t nsteps)
{
    if (!b || !b->exec || nsteps < 0) return QPIC_EINVAL;
    if (nsteps % b->period) { b->err = "nsteps must be a multiple of the cycle (qpic_batch_cycle)"; return QPIC_EINVAL; }
    for (qpic_ctx *c : b->runs) cudaStreamSynchronize(c->stream);   // earlier work of the runs
    for (qpic_ctx *c : b->runs) cudaMemsetAsync(c->d_err, 0, sizeof(int), b->main);
    for (int r = 0; r < nsteps / b->period; r++) {
        cudaError_t e = cudaGraphLaunch(b->exec, b->main);
        if (e != cudaSuccess) return batch_fail(b, QPIC_ECUDA, std::string("graph launch: ") + cudaGetErrorString(e));
    }
    cudaError_t e = cudaStreamSynchronize(b->main);
    if (e != cudaSuccess) return batch_fail(b, QPIC_ECUDA, std::string("batch step: ") + cudaGetErrorString(e));
    qpic_status st = QPIC_OK;
    for (size_t k = 0; k < b->runs.size(); k++) {
        qpic_ctx *c = b->runs[k];
        c->nstep += nsteps;
        c->n_kernels += b->kernels_per_cycle[k] * (nsteps / b->period);
        if (k == 0) c->n_kernels += b->batch_kernels_per_cycle * (nsteps / b->period);
        int err = 0;
        cudaMemcpy(&err, c->d_err, sizeof(int), cudaMemcpyDeviceToHost);
        if ((err & 4) && st == QPIC_OK) {
            b->err = "run " + std::to_string(k) + ": a dependency wait of the particle phase gave up";
            st = QPIC_ETIMEOUT;
        }
        if ((err & 1) && st == QPIC_OK) { b->err = "fixed-point overflow in run " + std::to_string(k); st = QPIC_EOVERFLOW; }
    }
    return st;
}

}  // extern "C"
