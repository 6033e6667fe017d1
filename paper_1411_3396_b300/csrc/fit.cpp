// Host-side binary64 fit of the Gaussian-split long-range force (Sec. 2:
// the long/short split; the polynomial replaces F_long(r)/r inside r_c).
//
//   F_long(r) = (1/r^2) [erf(r/2 sigma) - (r/(sigma sqrt pi)) exp(-r^2/4 sigma^2)]
//   g(s)      = F_long(sqrt s)/sqrt s,   p(s) = sum_k c_k s^k  (degree 5)
//
// Least squares on 4096 midpoints s_k = r_c^2 (k+1/2)/4096, basis t^m with
// t = s/r_c^2.  The constrained mode eliminates a_0 through
// sum_m a_m = (r_c^2+eps^2)^(-3/2) (so f_SR(r_c^2) = 0) and solves the
// reduced 5-column problem.  Solver: Householder QR (column-oriented),
// back substitution.
#include <cmath>
#include <vector>

#include "sr_internal.h"

namespace sr {
namespace {

constexpr int kSamples = 4096;
constexpr int kDeg = 5;

double g_long(double s, double sigma) {
    const double u = std::sqrt(s) / (2.0 * sigma);
    const double two_over_sqrt_pi = 2.0 / std::sqrt(M_PI);
    if (u < 0.25) {
        // sum_{n>=1} (-1)^(n+1) 2n u^(2n-2) / (n! (2n+1)), from the difference
        // of the erf and u exp(-u^2) Taylor series.
        double acc = 0.0, upow = 1.0, fact = 1.0;
        const double u2 = u * u;
        for (int n = 1; n < 16; ++n) {
            fact *= n;
            const double term = (2.0 * n) * upow / (fact * (2 * n + 1));
            acc += (n % 2 == 1) ? term : -term;
            upow *= u2;
        }
        return two_over_sqrt_pi / (8.0 * sigma * sigma * sigma) * acc;
    }
    const double r = std::sqrt(s);
    const double fl = (std::erf(u) - (r / (sigma * std::sqrt(M_PI))) * std::exp(-u * u)) / (r * r);
    return fl / r;
}

// Least squares min |A x - b| for A (m x n, column major), Householder QR.
bool lstsq_qr(std::vector<double> A, std::vector<double> b, int m, int n, double* x) {
    for (int k = 0; k < n; ++k) {
        double* col = &A[(size_t)k * m];
        double norm = 0.0;
        for (int i = k; i < m; ++i) norm += col[i] * col[i];
        norm = std::sqrt(norm);
        if (norm == 0.0) return false;
        const double alpha = col[k] > 0 ? -norm : norm;
        // v = x - alpha e_k, stored in col[k..m)
        col[k] -= alpha;
        double vnorm2 = 0.0;
        for (int i = k; i < m; ++i) vnorm2 += col[i] * col[i];
        for (int j = k + 1; j < n; ++j) {
            double* cj = &A[(size_t)j * m];
            double dot = 0.0;
            for (int i = k; i < m; ++i) dot += col[i] * cj[i];
            const double f = 2.0 * dot / vnorm2;
            for (int i = k; i < m; ++i) cj[i] -= f * col[i];
        }
        double dot = 0.0;
        for (int i = k; i < m; ++i) dot += col[i] * b[i];
        const double f = 2.0 * dot / vnorm2;
        for (int i = k; i < m; ++i) b[i] -= f * col[i];
        // R diagonal entry
        for (int i = k + 1; i < m; ++i) col[i] = 0.0;
        col[k] = alpha;
    }
    for (int k = n - 1; k >= 0; --k) {
        double s = b[k];
        for (int j = k + 1; j < n; ++j) s -= A[(size_t)j * m + k] * x[j];
        x[k] = s / A[(size_t)k * m + k];
    }
    return true;
}

}  // namespace

int fit_poly(double rc, double sigma, double eps, int mode, double c[6]) {
    if (!(rc > 0) || !(sigma > 0) || !(eps >= 0) || !std::isfinite(rc) ||
        !std::isfinite(sigma) || !std::isfinite(eps) ||
        (mode != SR_FIT_CONSTRAINED && mode != SR_FIT_UNCONSTRAINED) || c == nullptr)
        return set_error(SR_ERR_ARG, "sr_fit_poly: bad arguments");
    const int m = kSamples;
    std::vector<double> t(m), g(m);
    for (int k = 0; k < m; ++k) {
        t[k] = (k + 0.5) / m;
        g[k] = g_long(rc * rc * t[k], sigma);
    }
    double a[kDeg + 1];
    if (mode == SR_FIT_UNCONSTRAINED) {
        std::vector<double> A((size_t)m * (kDeg + 1));
        for (int k = 0; k < m; ++k) {
            double p = 1.0;
            for (int j = 0; j <= kDeg; ++j) { A[(size_t)j * m + k] = p; p *= t[k]; }
        }
        if (!lstsq_qr(A, g, m, kDeg + 1, a)) return set_error(SR_ERR_ARG, "sr_fit_poly: singular");
    } else {
        const double target = std::pow(rc * rc + eps * eps, -1.5);
        std::vector<double> A((size_t)m * kDeg), b(m);
        for (int k = 0; k < m; ++k) {
            double p = t[k];
            for (int j = 1; j <= kDeg; ++j) { A[(size_t)(j - 1) * m + k] = p - 1.0; p *= t[k]; }
            b[k] = g[k] - target;
        }
        double rest[kDeg];
        if (!lstsq_qr(A, b, m, kDeg, rest)) return set_error(SR_ERR_ARG, "sr_fit_poly: singular");
        double sum = 0.0;
        for (int j = 0; j < kDeg; ++j) { a[j + 1] = rest[j]; sum += rest[j]; }
        a[0] = target - sum;
    }
    double scale = 1.0;
    for (int j = 0; j <= kDeg; ++j) { c[j] = a[j] / scale; scale *= rc * rc; }
    return SR_OK;
}

}  // namespace sr
