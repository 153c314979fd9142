// Host check of the register FFT used by the fused transforms: every size the
// library supports, both signs, plain and centred, against the dense sums
// y_k = sum_j x_j exp(2 pi i S j k / N) and exp(2 pi i S (k - N/2)(j - N/2) / N)
// in double precision. Prints one line per case: N S max|error| / max|y|.
#include <cmath>
#include <cstdio>
#include <random>

#include "../../paper_1211_0540_gb300/csrc/fft_reg.cuh"

using namespace bte::fftr;

template <int N, int S, bool CENTRED>
static double check(std::mt19937 &g) {
    const double pi = 3.14159265358979323846;
    float2 rt[N];
    for (int t = 0; t < N; ++t) rt[t] = make_float2((float)std::cos(2 * pi * t / N), (float)std::sin(2 * pi * t / N));
    std::uniform_real_distribution<float> u(-1.f, 1.f);
    float2 x[N], y[N];
    for (int j = 0; j < N; ++j) y[j] = x[j] = make_float2(u(g), u(g));
    if (CENTRED) centred<N, S>(y, rt);
    else fft<N, S, N>(y, rt);
    const int h = CENTRED ? N / 2 : 0;
    double err = 0.0, mag = 0.0;
    for (int k = 0; k < N; ++k) {
        double re = 0.0, im = 0.0;
        for (int j = 0; j < N; ++j) {
            const double a = 2 * pi * S * (double)((k - h) * (j - h)) / N;
            re += x[j].x * std::cos(a) - x[j].y * std::sin(a);
            im += x[j].x * std::sin(a) + x[j].y * std::cos(a);
        }
        err = std::fmax(err, std::hypot(re - y[k].x, im - y[k].y));
        mag = std::fmax(mag, std::hypot(re, im));
    }
    return err / mag;
}

template <int N>
static void all(std::mt19937 &g) {
    std::printf("%d +1 plain %.3e\n", N, check<N, 1, false>(g));
    std::printf("%d -1 plain %.3e\n", N, check<N, -1, false>(g));
    std::printf("%d +1 centred %.3e\n", N, check<N, 1, true>(g));
    std::printf("%d -1 centred %.3e\n", N, check<N, -1, true>(g));
}

int main() {
    std::mt19937 g(7);
    all<8>(g);
    all<12>(g);
    all<16>(g);
    all<24>(g);
    all<32>(g);
    return 0;
}
