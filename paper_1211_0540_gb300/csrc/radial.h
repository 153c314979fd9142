// Radial integrals of the convolution weights (internal, host only).
//
//   I(a, b) = int_0^L r^(lam+2) sinc(ar) sinc(br) dr,  J(c) = int_0^L r^(lam+2) sinc(cr) dr
// (Sec. 2.2, Eq. GHat_calc, cut off at r0 = L). For lambda = 0, 1 they have
// closed forms (Radial); for other lambda > -3 the series-and-panels rule
// (SeriesRule); RadialRule is the plain panel rule the inelastic weights use
// where a closed form would cancel. Kept in a header of its own so that a host
// program can check them against high-precision quadrature.
#pragma once

#include <cmath>
#include <vector>

namespace bte {
namespace radial {

constexpr double kPi = 3.14159265358979323846;

struct Radial {
    double L, lam;
    double C(double k) const {
        if (k == 0.0) return lam == 0.0 ? L : 0.5 * L * L;
        double sk = std::sin(k * L) / k;
        if (lam == 0.0) return sk;
        double h = std::sin(0.5 * k * L);
        return L * sk - 2.0 * h * h / (k * k);
    }
    double J(double c) const {
        if (c == 0.0) return std::pow(L, lam + 3.0) / (lam + 3.0);
        double x = c * L, s = std::sin(x), co = std::cos(x);
        if (lam == 0.0) return (s - x * co) / (c * c * c);
        return (2.0 * x * s - (x * x - 2.0) * co - 2.0) / (c * c * c * c);
    }
    double I(double a, double b) const {
        if (a == 0.0) return J(b);
        if (b == 0.0) return J(a);
        return (C(a - b) - C(a + b)) / (2.0 * a * b);
    }
};

// Plain panel rule: composite Clenshaw-Curtis on [0, L], uniform panels of at
// most half a period of the highest frequency omega (25 points each); on the
// first panel [0, h] the substitution r = h u^2 (dr = 2 h u du), 33 points. Clenshaw-Curtis
// weights on [-1, 1] for n intervals (n even), nodes cos(j pi / n):
//   w_j = (c_j / n) [1 - sum_{k=1}^{n/2} b_k cos(2 pi j k / n) / (4k^2 - 1)],
//   c_0 = c_n = 1, c_j = 2 otherwise, b_{n/2} = 1, b_k = 2 otherwise.
struct RadialRule {
    std::vector<double> r, w;  // nodes on [0, L] and weights of int_0^L g(r) dr
};

inline void cc_rule(int n, std::vector<double> &x, std::vector<double> &w) {
    x.assign(n + 1, 0.0);
    w.assign(n + 1, 0.0);
    for (int j = 0; j <= n; ++j) {
        x[j] = std::cos(j * kPi / n);
        double s = 0.0;
        for (int k = 1; k <= n / 2; ++k) {
            const double b = (2 * k == n) ? 1.0 : 2.0;
            s += b * std::cos(2.0 * kPi * j * k / n) / (4.0 * k * k - 1.0);
        }
        const double c = (j == 0 || j == n) ? 1.0 : 2.0;
        w[j] = c / n * (1.0 - s);
    }
}

inline RadialRule radial_rule(double L, double omega) {
    const int panels = (int)std::ceil(omega * L / kPi) + 4;
    const double h = L / panels;
    RadialRule R;
    std::vector<double> x, w;
    cc_rule(32, x, w);  // first panel, u in [0, 1]: u = (x + 1) / 2
    for (size_t j = 0; j < x.size(); ++j) {
        const double u = 0.5 * (x[j] + 1.0);
        R.r.push_back(h * u * u);
        R.w.push_back(0.5 * w[j] * 2.0 * h * u);
    }
    cc_rule(24, x, w);
    for (int p = 1; p < panels; ++p)
        for (size_t j = 0; j < x.size(); ++j) {
            R.r.push_back(p * h + 0.5 * h * (x[j] + 1.0));
            R.w.push_back(0.5 * h * w[j]);
        }
    return R;
}

inline double sinc(double x) { return x == 0.0 ? 1.0 : std::sin(x) / x; }

// Radial integrals for any lambda > -3 (Sec. 2.1: hard, Maxwell and variable
// hard or soft potentials, -3 < lambda <= 1; Sec. 2.2: for lambda other than
// 0 and 1 a one-dimensional integral done by quadrature). [0, L] splits at
// h = min(L, 1 / omega), omega >= the largest a + b evaluated:
// - on [0, h] the integrand's power series is integrated term by term, which
//   is exact for the factor r^s, s = lambda + 2 > -1, however singular at 0:
//     sinc(ar) sinc(br) = sum_{i,j} c_i(a) c_j(b) r^(2i+2j),  c_i(a) = (-1)^i a^(2i) / (2i+1)!,
//     int_0^h r^(s+2k) dr = h^(s+1+2k) / (s+1+2k);
//   with a h, b h <= 1 the terms fall below 1e-30 before i = kSeriesTerms;
// - on [h, L], where r^s is smooth, composite Clenshaw-Curtis panels of at most
//   half a period of omega (25 points each), the weights carrying r^s.
constexpr int kSeriesTerms = 16;
struct SeriesRule {
    double L = 0, s = 0, h = 0, hs1 = 0;  // hs1 = h^(s+1)
    double inv[2 * kSeriesTerms] = {};   // 1 / (s + 1 + 2k)
    std::vector<double> r, w;            // [h, L]: nodes, weights times r^s
};

inline SeriesRule series_rule(double lam, double L, double omega) {
    SeriesRule R;
    R.L = L;
    R.s = lam + 2.0;
    R.h = omega > 1.0 / L ? 1.0 / omega : L;
    R.hs1 = std::pow(R.h, R.s + 1.0);
    for (int k = 0; k < 2 * kSeriesTerms; ++k) R.inv[k] = 1.0 / (R.s + 1.0 + 2.0 * k);
    if (R.h < L) {
        const int panels = (int)std::ceil(omega * (L - R.h) / kPi) + 4;
        const double ph = (L - R.h) / panels;
        std::vector<double> x, w;
        cc_rule(24, x, w);
        for (int p = 0; p < panels; ++p)
            for (size_t j = 0; j < x.size(); ++j) {
                const double rr = R.h + p * ph + 0.5 * ph * (x[j] + 1.0);
                R.r.push_back(rr);
                R.w.push_back(0.5 * ph * w[j] * std::pow(rr, R.s));
            }
    }
    return R;
}

// c_i(a) h^(2i) = (-1)^i (a h)^(2i) / (2i+1)!, i < kSeriesTerms
inline void series_coeffs(double a, double h, double (&c)[kSeriesTerms]) {
    const double x2 = (a * h) * (a * h);
    c[0] = 1.0;
    for (int i = 1; i < kSeriesTerms; ++i) c[i] = -c[i - 1] * x2 / ((2.0 * i) * (2.0 * i + 1.0));
}

// I(a, b) = int_0^L r^s sinc(ar) sinc(br) dr with the rule (a + b <= omega of the rule)
inline double I_series(const SeriesRule &R, double a, double b) {
    double ca[kSeriesTerms], cb[kSeriesTerms];
    series_coeffs(a, R.h, ca);
    series_coeffs(b, R.h, cb);
    double first = 0.0;
    for (int i = kSeriesTerms - 1; i >= 0; --i)
        for (int j = kSeriesTerms - 1; j >= 0; --j) first += ca[i] * cb[j] * R.inv[i + j];
    double rest = 0.0;
    for (size_t k = 0; k < R.r.size(); ++k) rest += R.w[k] * sinc(a * R.r[k]) * sinc(b * R.r[k]);
    return R.hs1 * first + rest;
}

// I(a, b) by the plain panel rule (smooth integrand: lambda = 0, 1), for the
// inelastic pairs whose closed form would cancel (b L < 0.25).
inline double I_quad(double lam, double L, double a, double b) {
    const RadialRule Q = radial_rule(L, std::fabs(a) + std::fabs(b));
    double acc = 0.0;
    for (size_t i = 0; i < Q.r.size(); ++i) acc += Q.w[i] * std::pow(Q.r[i], lam + 2.0) * sinc(a * Q.r[i]) * sinc(b * Q.r[i]);
    return acc;
}

}  // namespace radial
}  // namespace bte
