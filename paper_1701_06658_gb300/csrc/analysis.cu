// Size analysis of Sec. 5 on the host: the size distributions the measured
// one is compared with, and the fits the section reports (a few dozen numbers
// per call; the grain statistics themselves come from the device,
// lsgg_grain_statistics).
//
//   Rios' distribution (Eq. (Rios)) of z = R / <R> with H = 3, whose factor
//   printed as nu^(H0/2) is nu^(H/2): the reading under which it integrates
//   to 1.  Hillert's distribution is its nu -> 4 limit with rho = 8/9, here in
//   its own closed form P(u) = (2e)^3 3u / (2 - u)^5 exp(-6 / (2 - u)),
//   u = rho z < 2, so p(z) = rho P(rho z).
//   The kinetic law is printed as <R>^n - <R_0>^n = k t with n = 0.45-0.46,
//   which only makes sense as <R> ~ t^n: the fit takes
//   <R>^(1/n) - <R_0>^(1/n) = k t (n = 1/2: parabolic growth).
#include <cmath>
#include <cstdint>

#include "../../include/lsgg.h"

namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr double kE = 2.71828182845904523536;

// Minimum of f on [a, b] by golden-section search (f unimodal there).
template <class F>
double golden_min(F f, double a, double b, double tol) {
    const double g = 0.5 * (std::sqrt(5.0) - 1.0);
    double c = b - g * (b - a), d = a + g * (b - a);
    double fc = f(c), fd = f(d);
    for (int it = 0; it < 400 && b - a > tol; ++it) {
        if (fc <= fd) {
            b = d; d = c; fd = fc;
            c = b - g * (b - a); fc = f(c);
        } else {
            a = c; c = d; fc = fd;
            d = a + g * (b - a); fd = f(d);
        }
    }
    return 0.5 * (a + b);
}

double rios(double z, double nu, double rho) {
    const double H = 3.0;
    const double s = std::sqrt(4.0 * nu - nu * nu);
    const double base = rho * rho * z * z - nu * rho * z + nu;
    const double ang = std::atan((2.0 * rho * z - nu) / s) + std::atan(nu / s);
    return z * rho * rho * H * std::pow(nu, H / 2.0) / std::pow(base, 1.0 + H / 2.0) * std::exp(-H * nu / s * ang);
}

// Relative squared residual of the kinetic law for exponent n, and its
// least-squares k (through the origin in t - t_0).
double growth_cost(const double* t, const double* r, int n, double e, double* k_out) {
    const double p = 1.0 / e, y0 = std::pow(r[0], p);
    double sty = 0.0, stt = 0.0;
    for (int i = 0; i < n; ++i) {
        const double dt = t[i] - t[0], y = std::pow(r[i], p) - y0;
        sty += dt * y;
        stt += dt * dt;
    }
    const double k = sty / stt;
    double res = 0.0, yy = 0.0;
    for (int i = 0; i < n; ++i) {
        const double dt = t[i] - t[0], y = std::pow(r[i], p) - y0;
        res += (y - k * dt) * (y - k * dt);
        yy += y * y;
    }
    if (k_out) *k_out = k;
    return yy > 0.0 ? res / yy : 0.0;
}

}  // namespace

extern "C" {

double lsgg_rios_pdf(double z, double nu, double rho) {
    if (!(nu > 0.0 && nu < 4.0 && rho > 0.0) || z < 0.0) return NAN;
    return rios(z, nu, rho);
}

double lsgg_hillert_pdf(double z) {
    const double rho = 8.0 / 9.0, u = rho * z;
    if (z < 0.0) return NAN;
    if (u >= 2.0) return 0.0;
    const double P = std::pow(2.0 * kE, 3.0) * 3.0 * u / std::pow(2.0 - u, 5.0) * std::exp(-6.0 / (2.0 - u));
    return rho * P;
}

int lsgg_fit_rios_nu(const double* hist, int32_t n_bins, double r_max_rel, double rho, double* nu) {
    if (!hist || !nu || n_bins < 2 || !(r_max_rel > 0.0) || !(rho > 0.0)) return LSGG_ERR_INVALID_ARG;
    const double w = r_max_rel / n_bins;
    auto cost = [&](double v) {
        double c = 0.0;
        for (int b = 0; b < n_bins; ++b) {
            const double d = rios((b + 0.5) * w, v, rho) - hist[b] / w;
            c += d * d;
        }
        return c;
    };
    *nu = golden_min(cost, 1e-3, 4.0 - 1e-6, 1e-10);
    return LSGG_OK;
}

int lsgg_fit_growth_exponent(const double* t, const double* mean_r, int32_t n, double* n_out, double* k_out) {
    if (!t || !mean_r || !n_out || n < 3) return LSGG_ERR_INVALID_ARG;
    for (int i = 0; i < n; ++i)
        if (!(mean_r[i] > 0.0) || (i > 0 && !(t[i] > t[i - 1]))) return LSGG_ERR_INVALID_ARG;
    const double e = golden_min([&](double x) { return growth_cost(t, mean_r, n, x, nullptr); }, 0.05, 2.0, 1e-12);
    *n_out = e;
    double k = 0.0;
    growth_cost(t, mean_r, n, e, &k);
    if (k_out) *k_out = k;
    return LSGG_OK;
}

}  // extern "C"
