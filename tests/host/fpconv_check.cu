// Host check of the integer-pipe conversions (fpconv.cuh) against the
// compiler's binary32 <-> binary64 conversions (round to nearest even):
// special values, every binary32 exponent with random fractions, binary64
// values around the binary32 range limits (subnormal boundary, overflow,
// halfway cases) and random bit patterns. Prints "mismatches <n> checked <m>".
#include <cmath>
#include <cstdio>
#include <random>

#include "../../paper_1211_0540_gb300/csrc/fpconv.cuh"

using namespace bte::fpc;

static long long bad = 0, total = 0;

static void check_widen(float x) {
    ++total;
    const double a = widen(x), b = (double)x;
    if (std::isnan(b) ? !std::isnan(a) : bits64(a) != bits64(b)) {
        if (bad < 5) std::printf("widen %a -> %a, expected %a\n", (double)x, a, b);
        ++bad;
    }
}
static void check_narrow(double x) {
    ++total;
    const float a = narrow(x), b = (float)x;
    if (std::isnan(b) ? !std::isnan(a) : bits32(a) != bits32(b)) {
        if (bad < 5) std::printf("narrow %a -> %a, expected %a\n", x, (double)a, (double)b);
        ++bad;
    }
    if (finite64(x) != std::isfinite(x)) ++bad;
}

int main() {
    std::mt19937_64 g(11);
    const float fs[] = {0.f, -0.f, 1.f, -1.f, INFINITY, -INFINITY, NAN, 1e-45f, -1e-45f, 1.17549435e-38f,
                        1.17549421e-38f, 3.40282347e38f, 0.1f};
    for (float x : fs) check_widen(x);
    for (uint32_t e = 0; e < 256; ++e)
        for (int k = 0; k < 2000; ++k) {
            const uint32_t u = (uint32_t)(g() & 1) << 31 | e << 23 | (uint32_t)(g() & 0x7fffff);
            check_widen(from32(u));
        }
    const double ds[] = {0.0, -0.0, 1.0, -1.0, INFINITY, -INFINITY, NAN, 1e-310, 3.4028234663852886e38,
                         3.4028235677973366e38, 3.4028235677973362e38, 1.1754943508222875e-38,
                         1.401298464324817e-45, 7.006492321624085e-46, 7.006492321624087e-46,
                         2.1019476964872256e-45, 1e-50, 0.1, 1.0000000596046448, 1.0000001788139343};
    for (double x : ds) check_narrow(x);
    // every binary64 exponent that can reach binary32 and a margin beyond, random fractions
    for (int e = 1023 - 160; e <= 1023 + 130; ++e)
        for (int k = 0; k < 4000; ++k) {
            uint64_t f = g() & 0xfffffffffffffull;
            if (k % 4 == 1) f = (f & ~0x1fffffffull) | 0x10000000ull;       // exact halfway (normal)
            if (k % 4 == 2) f = (f & ~0x1fffffffull) | (g() & 1);           // just off a grid point
            const uint64_t u = (g() & 1) << 63 | (uint64_t)e << 52 | f;
            check_narrow(from64(u));
        }
    // halfway cases in the subnormal range: m has exactly one bit below the kept part
    for (int e = 1023 - 150; e <= 1023 - 126; ++e)
        for (int k = 0; k < 4000; ++k) {
            const int shift = 29 + 1 - (e - 896);
            uint64_t m = (g() & ((1ull << 52) - 1)) | (1ull << 52);
            m = (m >> shift << shift) | (1ull << (shift - 1));
            check_narrow(from64((uint64_t)e << 52 | (m & 0xfffffffffffffull)));
        }
    for (int k = 0; k < 2000000; ++k) {
        check_widen(from32((uint32_t)g()));
        check_narrow(from64(g()));
    }
    std::printf("mismatches %lld checked %lld\n", bad, total);
    return 0;
}
