// k_reduced.cu -- the reduced model of Sec. II (Eqs. 1-8): electrons in a
// spherical bubble wake (Eq. 6) and a channel-guided laser (Eqs. 3-4), motion
// in the x-z plane, integrated in FP64 with one thread per electron.
//
// Units: c = 1, laser frequency omega0 = 1; u = gamma v.  Eq. 8 written for
// the state (x, zeta = z - t, u_x, u_z) is explicit:
//   dx/dt = u_x/gamma,  dzeta/dt = u_z/gamma - 1,
//   du_x/dt = gamma F_x - (w_p^2/4)(1 + z') x,
//   du_z/dt = gamma F_z - (w_p^2/2)(zeta - x x'/2),
// with gamma F_x = a0 [(1 - k_z z') J0(s) - (k_perp^2/k_z) z' J1'(s)] sin(k_z xi),
//      gamma F_z = -a0 {(k_perp/k_z) J1(s) cos(k_z xi) - k_z x' [J0(s) + (k_perp/k_z)^2 J1'(s)] sin(k_z xi)},
// s = k_perp x, xi = z - v_phi t, k_z = omega0 / v_phi, J1'(s) = J0(s) - J1(s)/s.
// Time-staggering factor (Sec. IV.A): the laser's magnetic terms, those
// proportional to v sin(k_z xi), are multiplied by b = cos(omega0 dt_PIC/2)
// (b = 1: no staggering).  Injection (Appendix A): electron i stays at its
// initial state until step start[i] of the grid t0 + k dt.
// (Eq. 8's x'' + (gamma'/gamma) x' is d(gamma x')/dt / gamma, and
// zeta'' + (gamma'/gamma)(zeta' + 1) is d(gamma z')/dt / gamma.)
//
// Integrator: an explicit fifth-order Runge-Kutta method (Appendix A), here
// Dormand-Prince (Dormand & Prince 1980) at a fixed step.  Each electron is independent: the kernel
// reads its four words once, keeps the state in registers for all the steps
// and writes it back; it is bound by FP64 arithmetic and the Bessel functions.
#include <cuda_runtime.h>
#include <math.h>

#include <cmath>

#include "qpic_internal.h"

namespace {

struct RedPar {
    double a0, wp, kperp, vphi, kz, bfac;
};

__device__ __forceinline__ void red_rhs(double t, const double y[4], double dy[4], const RedPar &p)
{
    const double x = y[0], zeta = y[1], ux = y[2], uz = y[3];
    const double gamma = sqrt(1.0 + ux * ux + uz * uz);
    const double vx = ux / gamma, vz = uz / gamma;
    const double xi = zeta + t - p.vphi * t;
    const double s = p.kperp * x;
    const double J0 = j0(s), J1 = j1(s);
    const double J1p = s != 0.0 ? J0 - J1 / s : 0.5;
    double sn, cs;
    sincos(p.kz * xi, &sn, &cs);
    const double gFx =
        p.a0 * ((1.0 - p.bfac * p.kz * vz) * J0 - p.bfac * (p.kperp * p.kperp / p.kz) * vz * J1p) * sn;
    const double gFz = -p.a0 * ((p.kperp / p.kz) * J1 * cs -
                                p.bfac * p.kz * vx * (J0 + (p.kperp * p.kperp) / (p.kz * p.kz) * J1p) * sn);
    dy[0] = vx;
    dy[1] = vz - 1.0;
    dy[2] = gFx - 0.25 * p.wp * p.wp * (1.0 + vz) * x;
    dy[3] = gFz - 0.5 * p.wp * p.wp * (zeta - 0.5 * x * vx);
}

__global__ void __launch_bounds__(128) k_reduced_dp5(double *__restrict__ X, double *__restrict__ Z,
                                                     double *__restrict__ UX, double *__restrict__ UZ,
                                                     long long n, RedPar p, double t0, double dt,
                                                     int nsteps, const int *__restrict__ start)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int k0 = start ? max(start[i], 0) : 0;
    if (k0 >= nsteps) return;                  // not injected within these steps
    double y[4] = {X[i], Z[i], UX[i], UZ[i]};
    // Dormand-Prince 5(4) nodes, stage coefficients and fifth-order weights
    const double c2 = 1.0 / 5, c3 = 3.0 / 10, c4 = 4.0 / 5, c5 = 8.0 / 9;
    const double a21 = 1.0 / 5;
    const double a31 = 3.0 / 40, a32 = 9.0 / 40;
    const double a41 = 44.0 / 45, a42 = -56.0 / 15, a43 = 32.0 / 9;
    const double a51 = 19372.0 / 6561, a52 = -25360.0 / 2187, a53 = 64448.0 / 6561, a54 = -212.0 / 729;
    const double a61 = 9017.0 / 3168, a62 = -355.0 / 33, a63 = 46732.0 / 5247, a64 = 49.0 / 176,
                 a65 = -5103.0 / 18656;
    const double b1 = 35.0 / 384, b3 = 500.0 / 1113, b4 = 125.0 / 192, b5 = -2187.0 / 6784, b6 = 11.0 / 84;
    for (int k = k0; k < nsteps; k++) {
        const double t = t0 + k * dt;
        double k1[4], k2[4], k3[4], k4[4], k5[4], k6[4], yt[4];
        red_rhs(t, y, k1, p);
#pragma unroll
        for (int q = 0; q < 4; q++) yt[q] = y[q] + dt * (a21 * k1[q]);
        red_rhs(t + c2 * dt, yt, k2, p);
#pragma unroll
        for (int q = 0; q < 4; q++) yt[q] = y[q] + dt * (a31 * k1[q] + a32 * k2[q]);
        red_rhs(t + c3 * dt, yt, k3, p);
#pragma unroll
        for (int q = 0; q < 4; q++) yt[q] = y[q] + dt * (a41 * k1[q] + a42 * k2[q] + a43 * k3[q]);
        red_rhs(t + c4 * dt, yt, k4, p);
#pragma unroll
        for (int q = 0; q < 4; q++)
            yt[q] = y[q] + dt * (a51 * k1[q] + a52 * k2[q] + a53 * k3[q] + a54 * k4[q]);
        red_rhs(t + c5 * dt, yt, k5, p);
#pragma unroll
        for (int q = 0; q < 4; q++)
            yt[q] = y[q] + dt * (a61 * k1[q] + a62 * k2[q] + a63 * k3[q] + a64 * k4[q] + a65 * k5[q]);
        red_rhs(t + dt, yt, k6, p);
#pragma unroll
        for (int q = 0; q < 4; q++)
            y[q] = y[q] + dt * (b1 * k1[q] + b3 * k3[q] + b4 * k4[q] + b5 * k5[q] + b6 * k6[q]);
    }
    X[i] = y[0]; Z[i] = y[1]; UX[i] = y[2]; UZ[i] = y[3];
}

bool red_args_ok(long long n, double dt, int nsteps, double vphi, double kperp, double wp, double a0,
                 double bfac, double t0)
{
    return n >= 0 && nsteps >= 0 && std::isfinite(dt) && dt > 0 && vphi > 0 && std::isfinite(vphi) &&
           kperp >= 0 && std::isfinite(kperp) && std::isfinite(wp) && std::isfinite(a0) &&
           std::isfinite(bfac) && std::isfinite(t0);
}

qpic_status red_launch(long long n, double *x, double *zeta, double *ux, double *uz, double a0,
                       double wp, double kperp, double vphi, double bfac, double t0, double dt,
                       int nsteps, const int32_t *start, cudaStream_t st)
{
    if (n == 0 || nsteps == 0) return QPIC_OK;
    const RedPar p{a0, wp, kperp, vphi, 1.0 / vphi, bfac};
    const long long blocks = (n + 127) / 128;
    k_reduced_dp5<<<(unsigned)blocks, 128, 0, st>>>(x, zeta, ux, uz, n, p, t0, dt, nsteps, start);
    return cudaGetLastError() == cudaSuccess ? QPIC_OK : QPIC_ECUDA;
}

}  // namespace

extern "C" qpic_status qpic_reduced_integrate_device(int64_t n, double *x, double *zeta, double *ux,
                                                     double *uz, double a0, double omega_p,
                                                     double k_perp, double v_phi, double bfac,
                                                     double t0, double dt, int32_t nsteps,
                                                     const int32_t *start_step, void *stream)
{
    if (!red_args_ok(n, dt, nsteps, v_phi, k_perp, omega_p, a0, bfac, t0)) return QPIC_EINVAL;
    if (n > 0 && (!x || !zeta || !ux || !uz)) return QPIC_EINVAL;
    if (n > (long long)(1u << 31) * 127) return QPIC_EINVAL;
    return red_launch(n, x, zeta, ux, uz, a0, omega_p, k_perp, v_phi, bfac, t0, dt, nsteps, start_step,
                      (cudaStream_t)stream);
}

extern "C" qpic_status qpic_reduced_integrate(int64_t n, double *x, double *zeta, double *ux, double *uz,
                                              double a0, double omega_p, double k_perp, double v_phi,
                                              double bfac, double t0, double dt, int32_t nsteps,
                                              const int32_t *start_step)
{
    if (!red_args_ok(n, dt, nsteps, v_phi, k_perp, omega_p, a0, bfac, t0)) return QPIC_EINVAL;
    if (n > 0 && (!x || !zeta || !ux || !uz)) return QPIC_EINVAL;
    if (n == 0) return QPIC_OK;
    double *d = nullptr;
    const size_t bytes = (size_t)n * sizeof(double);
    // state and, when given, the start steps in one allocation
    const size_t sbytes = start_step ? (size_t)n * sizeof(int32_t) : 0;
    const cudaError_t e = cudaMalloc(&d, 4 * bytes + sbytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? QPIC_ENOMEM : QPIC_ECUDA;
    }
    int32_t *dstart = start_step ? reinterpret_cast<int32_t *>(d + 4 * (size_t)n) : nullptr;
    double *h[4] = {x, zeta, ux, uz};
    bool ok = true;
    for (int k = 0; k < 4 && ok; k++)
        ok = cudaMemcpy(d + (size_t)k * n, h[k], bytes, cudaMemcpyHostToDevice) == cudaSuccess;
    if (ok && dstart) ok = cudaMemcpy(dstart, start_step, sbytes, cudaMemcpyHostToDevice) == cudaSuccess;
    qpic_status s = ok ? qpic_reduced_integrate_device(n, d, d + n, d + 2 * (size_t)n, d + 3 * (size_t)n, a0,
                                                       omega_p, k_perp, v_phi, bfac, t0, dt, nsteps,
                                                       dstart, nullptr)
                       : QPIC_ECUDA;
    if (s == QPIC_OK)
        for (int k = 0; k < 4 && ok; k++)
            ok = cudaMemcpy(h[k], d + (size_t)k * n, bytes, cudaMemcpyDeviceToHost) == cudaSuccess;
    cudaFree(d);
    if (s == QPIC_OK && !ok) s = QPIC_ECUDA;
    if (s != QPIC_OK) cudaGetLastError();
    return s;
}
