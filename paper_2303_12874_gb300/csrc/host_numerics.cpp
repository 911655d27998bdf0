// host_numerics.cpp -- FP64 host numerics of the dual solver (Sec. III.A).
//
//  * z-operator coefficients.  A staggered derivative with L coefficients,
//      D f_{i+1/2} = sum_{l=1..L} C_l (f_{i+l} - f_{i+1-l}) / dz,
//    has the symbol [k] dz = 2 sum_l C_l sin((l-1/2) k dz).  Eq. 11
//    ([k]_B [k]_E = (sin(k dt/2)/(dt/2))^2) and Eq. 15
//    (sqrt([k]_E/[k]_B) cos(k dt/2) = 1) are solved exactly by
//    [k]_E = (2/dt) tan(k dt/2) and [k]_B = sin(k dt)/dt; C^E and C^B are the
//    least-squares fits of those symbols on the samples
//    theta_k = band*pi*k/4000 (k = 1..4000), uniform weight, subject to the
//    exact long-wavelength limit sum_l (2l-1) C_l = 1.  Here the constraint is
//    used to eliminate C_1 and the reduced problem is solved by Householder QR.
//  * J_z correction filter: Fourier-cosine coefficients of
//    sin(theta/2) / sum_l C^B_l sin((l-1/2) theta) by the midpoint rule.
//  * stability limit: leapfrog is stable while (dt^2/4) lambda_max <= 1 with
//    lambda_max = max_theta [k]_E[k]_B + max_m mu_m; mu_m is the top of the
//    radial curl curl spectrum of mode m, which splits into a TM operator on E_z
//    and a TE operator on B_z, each a tridiagonal matrix made symmetric by the
//    finite-volume weights; its top eigenvalue comes from Sturm bisection.
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "qpic_internal.h"

namespace qpic {

static const double kPi = 3.14159265358979323846;
static const int kFitSamples = 4000;
static const int kThetaScan = 8192;

double symbol(const double *C, int L, double theta)
{
    double s = 0.0;
    for (int l = 1; l <= L; l++) s += C[l - 1] * std::sin((l - 0.5) * theta);
    return 2.0 * s;
}

// min |A x - b| for a column-major m x n A (m >= n) by Householder QR; A, b overwritten
static bool lsq_householder(std::vector<double> &A, std::vector<double> &b, int m, int n,
                            std::vector<double> &x)
{
    for (int k = 0; k < n; k++) {
        double *a = &A[(size_t)k * m];
        double norm = 0.0;
        for (int i = k; i < m; i++) norm += a[i] * a[i];
        norm = std::sqrt(norm);
        if (norm == 0.0) return false;
        double alpha = a[k] > 0 ? -norm : norm;
        std::vector<double> v(m - k);
        v[0] = a[k] - alpha;
        for (int i = k + 1; i < m; i++) v[i - k] = a[i];
        double vv = 0.0;
        for (double t : v) vv += t * t;
        if (vv == 0.0) continue;
        for (int j = k; j < n; j++) {
            double *c = &A[(size_t)j * m];
            double d = 0.0;
            for (int i = k; i < m; i++) d += v[i - k] * c[i];
            d = 2.0 * d / vv;
            for (int i = k; i < m; i++) c[i] -= d * v[i - k];
        }
        double d = 0.0;
        for (int i = k; i < m; i++) d += v[i - k] * b[i];
        d = 2.0 * d / vv;
        for (int i = k; i < m; i++) b[i] -= d * v[i - k];
    }
    x.assign(n, 0.0);
    for (int k = n - 1; k >= 0; k--) {
        double s = b[k];
        for (int j = k + 1; j < n; j++) s -= A[(size_t)j * m + k] * x[j];
        double rkk = A[(size_t)k * m + k];
        if (rkk == 0.0) return false;
        x[k] = s / rkk;
    }
    return true;
}

// fit of sum_l C_l sin((l-1/2) theta) to g(theta)/2 with sum (2l-1) C_l = 1
static bool fit_one(int L, double band, double nu, bool is_E, double *C)
{
    if (L == 1) { C[0] = 1.0; return true; }
    const int m = kFitSamples, n = L - 1;
    std::vector<double> A((size_t)m * n), b(m), x;
    for (int k = 0; k < m; k++) {
        double th = band * kPi * (k + 1) / m;
        double g = is_E ? 2.0 * std::tan(0.5 * nu * th) / nu : std::sin(nu * th) / nu;
        double s1 = 2.0 * std::sin(0.5 * th);
        // C_1 = 1 - sum_{l>=2} (2l-1) C_l
        b[k] = g - s1;
        for (int l = 2; l <= L; l++)
            A[(size_t)(l - 2) * m + k] = 2.0 * std::sin((l - 0.5) * th) - (2.0 * l - 1.0) * s1;
    }
    if (!lsq_householder(A, b, m, n, x)) return false;
    double c1 = 1.0;
    for (int l = 2; l <= L; l++) { C[l - 1] = x[l - 2]; c1 -= (2.0 * l - 1.0) * x[l - 2]; }
    C[0] = c1;
    return true;
}

int fit_coefficients(int solver, double dt, double dz, int L, double band, double *cE, double *cB,
                     std::string &err)
{
    if (solver == QPIC_YEE) { cE[0] = cB[0] = 1.0; return 1; }
    if (L < 1 || L > MAX_L) { err = "n_coef out of range"; return 0; }
    double nu = dt / dz;
    if (!(nu > 0.0) || nu * band >= 1.0) { err = "dt/dz outside the range of the dual fit"; return 0; }
    if (!fit_one(L, band, nu, true, cE) || !fit_one(L, band, nu, false, cB)) {
        err = "coefficient fit failed (rank deficient)";
        return 0;
    }
    return L;
}

int filter_taps_host(const double *cB, int L, double tol, std::vector<double> &taps,
                     std::string &err)
{
    taps.clear();
    if (L == 1 && cB[0] == 1.0) return 1;                 // Yee: identity
    const int N = 1 << 14;
    std::vector<double> ratio(N), th(N);
    for (int k = 0; k < N; k++) {
        th[k] = (k + 0.5) * kPi / N;
        double s = 0.5 * symbol(cB, L, th[k]);
        if (std::fabs(s) < 1e-12) { err = "[k]_B vanishes in (0, pi]: no J_z filter"; return 0; }
        ratio[k] = std::sin(0.5 * th[k]) / s;
    }
    // cos(n theta_k) with n theta_k = pi n (2k+1) / (2N) reduced exactly in integers
    std::vector<double> ctab(4 * N);
    for (int q = 0; q < 4 * N; q++) ctab[q] = std::cos(kPi * q / (2.0 * N));
    std::vector<double> k_all(MAX_TAPS);
    for (int n = 0; n < MAX_TAPS; n++) {
        double s = 0.0, comp = 0.0;                       // compensated (Kahan) sum
        for (int k = 0; k < N; k++) {
            long long q = ((long long)n * (2 * k + 1)) % (4 * N);
            double y = ratio[k] * ctab[q] - comp;
            double t = s + y;
            comp = (t - s) - y;
            s = t;
        }
        k_all[n] = s / N;
    }
    int last = 0;
    for (int n = 0; n < MAX_TAPS; n++)
        if (std::fabs(k_all[n]) >= tol * std::fabs(k_all[0])) last = n;
    if (last == MAX_TAPS - 1) { err = "J_z filter taps do not decay"; return 0; }
    taps.assign(k_all.begin(), k_all.begin() + last + 1);
    return 1;
}

// largest eigenvalue of a symmetric tridiagonal (diag d, off-diag e[i] between i, i+1)
static double tridiag_max_eig(const std::vector<double> &d, const std::vector<double> &e)
{
    int n = (int)d.size();
    if (n == 0) return 0.0;
    double lo = 1e300, hi = -1e300;
    for (int i = 0; i < n; i++) {
        double r = (i > 0 ? std::fabs(e[i - 1]) : 0.0) + (i < n - 1 ? std::fabs(e[i]) : 0.0);
        lo = std::min(lo, d[i] - r);
        hi = std::max(hi, d[i] + r);
    }
    auto count_below = [&](double x) {            // Sturm count of eigenvalues < x
        int c = 0;
        double q = d[0] - x;
        if (q < 0) c++;
        for (int i = 1; i < n; i++) {
            double qq = (q == 0.0) ? 1e-300 : q;
            q = d[i] - x - e[i - 1] * e[i - 1] / qq;
            if (q < 0) c++;
        }
        return c;
    };
    for (int it = 0; it < 200 && hi - lo > 1e-15 * std::max(1.0, std::fabs(hi)); it++) {
        double mid = 0.5 * (lo + hi);
        if (count_below(mid) >= n) hi = mid; else lo = mid;
    }
    return hi;
}

double radial_lambda_max(int nr, double dr, int m)
{
    const double m2 = (double)m * m;
    // TM family: E_z(j), j = 0 (m = 0 only) .. nr-1; E_z(nr) = 0 at the conductor
    std::vector<double> d, e;
    int j0 = (m == 0) ? 0 : 1;
    std::vector<double> wts;
    for (int j = j0; j < nr; j++) {
        double rj = j * dr, rp = (j + 0.5) * dr, rm = (j - 0.5) * dr;
        if (j == 0) {
            d.push_back(4.0 / (dr * dr));
            wts.push_back(dr / 8.0);
        } else {
            d.push_back((rp + rm) / (rj * dr * dr) + m2 / (rj * rj));
            wts.push_back(rj);
        }
    }
    for (size_t a = 0; a + 1 < d.size(); a++) {
        int j = j0 + (int)a;
        double rp = (j + 0.5) * dr;
        // M_{j,j+1} M_{j+1,j} with M_{j,j+1} = -(flux coefficient)/weight_j
        double flux = (j == 0) ? 0.5 / dr : rp / (dr * dr);    // symmetric coupling w_j M_{j,j+1}
        e.push_back(-flux / std::sqrt(wts[a] * wts[a + 1]));
    }
    double tm = tridiag_max_eig(d, e);
    // TE family: B_z(j+1/2), j = 0..nr-1; E_phi(nr) = 0 (Neumann-like wall for B_z)
    d.clear(); e.clear(); wts.clear();
    for (int j = 0; j < nr; j++) {
        double rh = (j + 0.5) * dr;
        double up = (j + 1 < nr) ? (j + 1) * dr : 0.0;        // r_{j+1} coupling (0 at the wall)
        double dn = j * dr;                                    // r_j coupling (0 on the axis)
        d.push_back((up + dn) / (rh * dr * dr) + m2 / (rh * rh));
        wts.push_back(rh);
    }
    for (int j = 0; j + 1 < nr; j++) {
        double flux = (j + 1) * dr / (dr * dr);
        e.push_back(-flux / std::sqrt(wts[j] * wts[j + 1]));
    }
    double te = tridiag_max_eig(d, e);
    return std::max(tm, te);
}

int cfl_limit(int solver, double dz, double dr, int nr, int n_modes, int L, double band,
              double *dt_out, std::string &err)
{
    double mu = 0.0;
    for (int m = 0; m < n_modes; m++) mu = std::max(mu, radial_lambda_max(nr, dr, m));
    std::vector<double> cE(MAX_L), cB(MAX_L);
    auto stable = [&](double dt) -> int {
        std::string e2;
        int Lf = fit_coefficients(solver, dt, dz, L, band, cE.data(), cB.data(), e2);
        if (!Lf) return -1;
        double zmax = 0.0;
        for (int k = 1; k <= kThetaScan; k++) {
            double th = kPi * k / kThetaScan;
            zmax = std::max(zmax, symbol(cE.data(), Lf, th) * symbol(cB.data(), Lf, th));
        }
        return 0.25 * dt * dt * (zmax / (dz * dz) + mu) <= 1.0 ? 1 : 0;
    };
    double lo = 0.0, hi = (solver == QPIC_YEE) ? 2.0 * dz : dz;
    while (hi - lo > 1e-10 * hi) {
        double mid = 0.5 * (lo + hi);
        int s = stable(mid);
        if (s > 0) lo = mid; else hi = mid;
    }
    if (lo <= 0.0) { err = "no stable time step found"; return 0; }
    *dt_out = lo;
    return 1;
}

}  // namespace qpic
