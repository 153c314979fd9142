// Host check of the library's radial integrals (radial.h): prints, for each
// case "lam a b", the closed form and the plain panel rule (lambda = 0, 1;
// else nan) and the series-and-panels rule of the tables (two values of its
// omega) for I(a, b) = int_0^L r^(lam+2) sinc(ar) sinc(br) dr, L = 6, and the
// Clenshaw-Curtis rule's error on x^k over [-1, 1] (exact for k <= n). The
// Python side compares with 30-digit quadrature.
#include <cmath>
#include <cstdio>

#include "../../paper_1211_0540_gb300/csrc/radial.h"

int main() {
    using namespace bte::radial;
    const double L = 6.0;
    const double lams[] = {0.0, 1.0, 0.1, 0.3, 0.5, 0.75, -0.5, -1.0, -1.5, -2.0, -2.5, -2.9};
    const double ab[][2] = {{0.0, 0.0}, {0.26, 0.26}, {1.3, 4.1}, {7.2, 13.9}, {0.0, 5.0}, {3.3, 0.2}, {2.1, 1e-3}, {15.0, 21.0}};
    for (double lam : lams)
        for (const auto &p : ab) {
            double cf = NAN, pq = NAN;
            if (lam == 0.0 || lam == 1.0) {
                cf = Radial{L, lam}.I(p[0], p[1]);
                pq = I_quad(lam, L, p[0], p[1]);
            }
            // the tables' rule, its omega the table's largest a + b (here 40) or this pair's
            const double sr = I_series(series_rule(lam, L, 40.0), p[0], p[1]);
            const double sp = I_series(series_rule(lam, L, p[0] + p[1]), p[0], p[1]);
            std::printf("I %.17g %.17g %.17g %.17g %.17g %.17g %.17g\n", lam, p[0], p[1], cf, pq, sr, sp);
        }
    std::vector<double> x, w;
    cc_rule(24, x, w);
    for (int k = 0; k <= 24; ++k) {
        double s = 0.0;
        for (size_t j = 0; j < x.size(); ++j) s += w[j] * std::pow(x[j], k);
        const double exact = (k % 2) ? 0.0 : 2.0 / (k + 1);
        std::printf("P %d %.3e\n", k, std::fabs(s - exact));
    }
    return 0;
}
