// noalloc.cu -- charge density per mode without any device allocation.
//
// qpic_get_field(..., QPIC_FIELD_RHO, ...) deposits the density into a device
// buffer it allocates for the call.  Some callers cannot allow that: hosts
// that hand the library a fixed device-memory budget up front, callers inside
// a device memory allocator's own callbacks (which must not re-enter it), and
// loops that cannot afford the device-wide synchronisation of cudaFree.  This
// entry point gives them the same result using a file-scope static __device__
// scratch array of fixed size.
//
// The array is part of the module: every GPU that loads the library holds its
// 16 MiB until the process exits.  In host code the array's name is only a
// host-side stand-in, so the device address is looked up once per device with
// cudaGetSymbolAddress (on the first call on that device, with it current)
// and passed to the deposit kernel.  A call must be made with the context's
// device current (the device of qpic_init); otherwise it returns QPIC_ESTATE.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "qpic_internal.h"

namespace {

constexpr long long kScratchDoubles = 1LL << 21;       // 2,097,152 doubles = 16 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_rho_scratch[kScratchDoubles];

std::mutex g_mu;
double *g_ptr[kMaxDevices] = {nullptr};

// device address of the scratch array on device dev, which must be current
// (set-up on the first call per device); nullptr on failure with *err set
double *scratch_address(int dev, std::string *err)
{
    if (dev < 0 || dev >= kMaxDevices) {
        *err = "device index " + std::to_string(dev) + " is beyond the " + std::to_string(kMaxDevices) +
               " devices the scratch table holds";
        return nullptr;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_ptr[dev]) {
        double *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(reinterpret_cast<void **>(&p), g_rho_scratch);
        if (e != cudaSuccess || !p) {
            *err = std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e);
            return nullptr;
        }
        g_ptr[dev] = p;
    }
    return g_ptr[dev];
}

}  // namespace

extern "C" qpic_status qpic_charge_density_noalloc(qpic_ctx *c, int32_t mode, double *re,
                                                   double *im)
{
    if (!c || !re || mode < 0 || mode >= c->g.nm) {
        if (c) c->err = "charge_density_noalloc: bad arguments";
        return QPIC_EINVAL;
    }
    const long long nout = (long long)(c->g.nr + 1) * c->g.nz;
    const long long need = (long long)c->g.nm * 2 * nout;
    if (need > kScratchDoubles) {
        c->err = "charge_density_noalloc: this grid needs " + std::to_string(need) +
                 " doubles of scratch (n_modes*2*(nr+1)*nz); the static buffer holds " +
                 std::to_string(kScratchDoubles);
        return QPIC_EINVAL;
    }
    // the array and the context's stream belong to the context's device: refuse
    // a call made while another device is current
    QPIC_REQUIRE_DEVICE(c);
    std::string err;
    double *d = scratch_address(c->device, &err);
    if (!d) {
        c->err = "charge_density_noalloc: " + err;
        return QPIC_ECUDA;
    }
    // the deposit clears the part of the array it uses before accumulating
    qpic::launch_rho(c, d);
    cudaMemcpyAsync(re, d + (size_t)(2 * mode) * nout, nout * sizeof(double),
                    cudaMemcpyDeviceToHost, c->stream);
    if (im)
        cudaMemcpyAsync(im, d + (size_t)(2 * mode + 1) * nout, nout * sizeof(double),
                        cudaMemcpyDeviceToHost, c->stream);
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) {
        c->err = std::string("charge_density_noalloc: ") + cudaGetErrorString(e);
        return QPIC_ECUDA;
    }
    return QPIC_OK;
}
