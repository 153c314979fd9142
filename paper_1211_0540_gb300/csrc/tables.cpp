// Host FP64 tabulation of the convolution weights Ghat (Sec. 2.2, Eq. GHat_calc)
// and their packing into the layouts the GPU kernels stream.
//
// Ghat(xi, zeta) = sqrt(2/pi) [ I(beta |zeta|/2, |xi - beta zeta/2|) - J(|xi|) ]
// (b = 1/(4 pi), d = 3, radial integral cut off at r0 = L, Sec. 3.1) with
//   I(a, b) = int_0^L r^{lam+2} sinc(ar) sinc(br) dr,  J(c) = int_0^L r^{lam+2} sinc(cr) dr.
// The paper notes that for integer lambda these integrals have closed forms;
// for lambda = 0, 1 they are
//   I(a, b) = [C(a-b) - C(a+b)] / (2ab),   C(k) = int_0^L r^lam cos(kr) dr,
//   C_0(k) = sin(kL)/k,   C_1(k) = L sin(kL)/k - 2 sin^2(kL/2)/k^2,
//   J_0(c) = (sin cL - cL cos cL)/c^3,  J_1(c) = (2cL sin cL - (c^2L^2 - 2) cos cL - 2)/c^4,
// and I(0, b) = J(b). On the grid every argument is (dz/2) sqrt(integer), so the
// integrals are evaluated once per integer invariant:
//   p = |k'|^2 (|zeta| = (dz/2) sqrt p),  q = |2m' - k'|^2 (|xi - zeta/2| = (dz/2) sqrt q),
//   s = |m'|^2 (|xi| = (dz/2) sqrt(4s)),  k' = k - N/2, m' = m - N/2.
// With I(0, b) and J evaluated by the same function at bitwise-equal
// arguments, Ghat(xi, 0) = 0 exactly, as in the continuous weights.
// Non-integer lambda (0 < lambda < 1, variable hard potentials): the same
// tables by quadrature (quadrature_tables). Inelastic collisions (beta < 1,
// restitution parameter of the rule v' = v + (beta/2)(|u| sigma - u)): the gain
// arguments are a = beta hz sqrt(p), b = hz |2m' - beta k'|, no longer on the
// lattice of I, so the gain integral is evaluated per pair (closed form, or
// quadrature where it would cancel); J is unchanged.
//
// FP32 pair-symmetrised layout (the fast path). For a zeta point k the terms m
// and n = k - m + N/2 (zeta - xi_m = xi_n) multiply the same product
// fhat_m fhat_n, so the sum over m is taken over unordered pairs with the
// weight Ghat(k, m) + Ghat(k, n). Pairs are grouped by the first two
// components: for a "pencil" (k1, k2) the kept blocks are the (m1, m2) of the
// valid box with (m1, m2) <= (n1, n2) lexicographically; a block with
// (m1, m2) == (n1, n2) pairs with itself and keeps the plain weight Ghat(k, m)
// over all m3. Inside a block, for a k3 tile [K0, K0 + T), the weights are
// stored in the order the kernel consumes them: m3 ascending, then k3
// ascending, skipping (k3, m3) whose partner n3 = k3 - m3 + N/2 is off the
// grid. Every weight already carries the trapezoid factor dz^3.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "bte_internal.h"
#include "radial.h"

namespace bte {

namespace {

using radial::kPi;
using radial::Radial;
using radial::sinc;

// I[p][q] = int_0^L r^(lam+2) sinc(a_p r) sinc(b_q r) dr and J[s] = I[0][4s]
// (a_p = hz sqrt p, b_q = hz sqrt q) for every p < np, q < nq of the parity of
// p, by one series-and-panels rule for the whole table (radial.h): on [0, h]
// I = h^(s+1) sum_j W_p[j] c_j(b_q), W_p[j] = sum_i c_i(a_p) / (s+1+2(i+j));
// on [h, L] sum_i A_p[i] sinc(b_q r_i), A_p[i] = w_i sinc(a_p r_i). J is read
// off the same sums, so Ghat(xi, 0) = I(0, |xi|) - J(|xi|) is exactly 0.
void quadrature_tables(Table &t, double hz) {
    using radial::kSeriesTerms;
    constexpr int K = kSeriesTerms;
    const int nrow = std::max(t.nq, 4 * (t.ns - 1) + 1);
    const radial::SeriesRule R =
        radial::series_rule(t.lam, t.L, hz * (std::sqrt((double)(t.np - 1)) + std::sqrt((double)(nrow - 1))));
    const size_t nn = R.r.size();
    std::vector<double> S((size_t)nrow * nn), A((size_t)t.np * nn), C((size_t)nrow * K), W((size_t)t.np * K);
#pragma omp parallel for schedule(static)
    for (int q = 0; q < nrow; ++q) {
        const double b = hz * std::sqrt((double)q);
        for (size_t i = 0; i < nn; ++i) S[(size_t)q * nn + i] = sinc(b * R.r[i]);
        double c[K];
        radial::series_coeffs(b, R.h, c);
        for (int j = 0; j < K; ++j) C[(size_t)q * K + j] = c[j];
    }
#pragma omp parallel for schedule(static)
    for (int p = 0; p < t.np; ++p) {
        for (size_t i = 0; i < nn; ++i) A[(size_t)p * nn + i] = R.w[i] * S[(size_t)p * nn + i];
        const double *c = &C[(size_t)p * K];  // c_i(a_p): a_p = b_p on this lattice
        for (int j = 0; j < K; ++j) {
            double acc = 0.0;
            for (int i = K - 1; i >= 0; --i) acc += c[i] * R.inv[i + j];
            W[(size_t)p * K + j] = acc;
        }
    }
    auto value = [&](int p, int q) {
        const double *a = &A[(size_t)p * nn], *b = &S[(size_t)q * nn];
        double rest = 0.0;
        for (size_t i = 0; i < nn; ++i) rest += a[i] * b[i];
        const double *wp = &W[(size_t)p * K], *cq = &C[(size_t)q * K];
        double first = 0.0;
        for (int j = K - 1; j >= 0; --j) first += wp[j] * cq[j];
        return R.hs1 * first + rest;
    };
#pragma omp parallel for schedule(dynamic, 4)
    for (int p = 0; p < t.np; ++p)
        for (int q = (p & 1); q < t.nq; q += 2) t.I[(size_t)p * t.nq + q] = value(p, q);
    for (int s = 0; s < t.ns; ++s) t.J[s] = value(0, 4 * s);
}

inline int box_lo(int k, int N) { return std::max(0, k - N / 2 + 1); }
inline int box_hi(int k, int N) { return std::min(N - 1, k + N / 2); }
inline int box_len(int k, int N) { return box_hi(k, N) - box_lo(k, N) + 1; }

}  // namespace

int first_kind_for_N(int N) {
    switch (N) {
        case 8: return 0;
        case 12: return 1;
        case 16: return 2;
        case 24: return 3;
        case 32: return 5;
        case 48: return 7;
        default: return -1;
    }
}

int tiles_for_N(int N) { return N == 48 ? 3 : ((N == 24 || N == 32) ? 2 : 1); }

double Table::ghat(int k1, int k2, int k3, int m1, int m2, int m3) const {
    const int h = N / 2;
    int k[3] = {k1 - h, k2 - h, k3 - h}, m[3] = {m1 - h, m2 - h, m3 - h};
    int p = 0, q = 0, s = 0;
    for (int d = 0; d < 3; ++d) {
        p += k[d] * k[d];
        q += (2 * m[d] - k[d]) * (2 * m[d] - k[d]);
        s += m[d] * m[d];
    }
    if (beta == 1.0) return std::sqrt(2.0 / kPi) * (I[(size_t)p * nq + q] - J[s]);
    // inelastic: gain arguments a = beta |zeta| / 2, b = |xi - beta zeta / 2| (Eq. GHat_calc)
    const double hz = 0.5 * dz;
    double b2 = 0.0;
    for (int d = 0; d < 3; ++d) {
        const double c = 2.0 * m[d] - beta * k[d];
        b2 += c * c;
    }
    const double a = beta * hz * std::sqrt((double)p), b = hz * std::sqrt(b2);
    return std::sqrt(2.0 / kPi) * (gain_inelastic(a, b) - J[s]);
}

// The closed form loses digits when a b L^2 is small (C(a - b) and C(a + b)
// nearly cancel); such pairs (|xi - beta zeta / 2| near 0, which the elastic
// lattice never produces) take the quadrature rule instead.
double Table::gain_inelastic(double a, double b) const {
    Radial R{L, lam};
    if (a == 0.0 || b == 0.0 || b * L >= 0.25) return R.I(a, b);
    return radial::I_quad(lam, L, a, b);
}

int build_table(Table &t, std::string &err) {
    const int N = t.N;
    if (first_kind_for_N(N) < 0) {
        err = "unsupported N (supported: 8, 12, 16, 24, 32, 48)";
        return BTE_EINVAL;
    }
    if (!(t.L > 0.0) || !std::isfinite(t.L)) {
        err = "L must be finite and > 0";
        return BTE_EINVAL;
    }
    if (!(t.lam > -3.0 && t.lam <= 1.0)) {
        err = "lambda must lie in (-3, 1] (variable soft potentials, Maxwell molecules, variable hard "
              "potentials, hard spheres)";
        return BTE_EINVAL;
    }
    if (!(t.beta > 0.0 && t.beta <= 1.0)) {
        err = "beta must lie in (0, 1] (beta = 1: elastic collisions)";
        return BTE_EINVAL;
    }
    const bool integer_lam = t.lam == 0.0 || t.lam == 1.0;
    if (t.beta != 1.0 && !integer_lam) {
        err = "inelastic weights (beta < 1) need lambda = 0 or 1 (closed forms)";
        return BTE_EINVAL;
    }
    const int h = N / 2;
    t.kind0 = first_kind_for_N(N);
    t.ntiles = tiles_for_N(N);
    t.dv = 2.0 * t.L / N;
    t.dz = kPi / t.L;
    const double hz = 0.5 * t.dz, dz3 = t.dz * t.dz * t.dz;

    // radial integrals on integer invariants
    t.np = 3 * h * h + 1;
    t.nq = 3 * (N - 1) * (N - 1) + 1;
    t.ns = 3 * h * h + 1;
    t.I.assign((size_t)t.np * t.nq, 0.0);
    t.J.assign(t.ns, 0.0);
    if (integer_lam) {
        Radial R{t.L, t.lam};
#pragma omp parallel for schedule(dynamic, 4)
        for (int p = 0; p < t.np; ++p) {
            double a = hz * std::sqrt((double)p);
            for (int q = 0; q < t.nq; ++q) {
                if ((p - q) % 2 != 0) continue;  // q = |2m'-k'|^2 has the parity of |k'|^2
                double b = hz * std::sqrt((double)q);
                t.I[(size_t)p * t.nq + q] = R.I(a, b);
            }
        }
        for (int s = 0; s < t.ns; ++s) t.J[s] = R.J(hz * std::sqrt((double)(4 * s)));
    } else {
        quadrature_tables(t, hz);
    }

    // pencil descriptors: kept (m1, m2) blocks
    std::vector<uint32_t> desc;
    t.desc_off.assign(N * N, 0);
    t.nblocks.assign(N * N, 0);
    for (int k1 = 0; k1 < N; ++k1)
        for (int k2 = 0; k2 < N; ++k2) {
            t.desc_off[k1 * N + k2] = (uint32_t)desc.size();
            uint32_t nb = 0;
            for (int m1 = box_lo(k1, N); m1 <= box_hi(k1, N); ++m1) {
                int n1 = k1 - m1 + h;
                if (m1 > n1) continue;
                for (int m2 = box_lo(k2, N); m2 <= box_hi(k2, N); ++m2) {
                    int n2 = k2 - m2 + h;
                    if (m1 == n1 && m2 > n2) continue;
                    desc.push_back((uint32_t)m1 | ((uint32_t)m2 << 16));
                    ++nb;
                }
            }
            t.nblocks[k1 * N + k2] = nb;
        }
    t.n_desc = desc.size();

    // weight offsets per (tile, k1, k2)
    const int T = conv_kind(t.kind0).T;
    t.wofs.assign((size_t)t.ntiles * N * N, 0);
    size_t total = 0;
    for (int tile = 0; tile < t.ntiles; ++tile) {
        int K0 = tile * T, cnt = 0;
        for (int j = 0; j < T; ++j) cnt += box_len(K0 + j, N);
        t.cpad[tile] = (cnt + 3) & ~3;
        for (int kk = 0; kk < N * N; ++kk) {
            t.wofs[(size_t)tile * N * N + kk] = total;
            total += (size_t)t.nblocks[kk] * t.cpad[tile];
        }
    }
    t.n_w32 = total;
    t.desc_host = desc;

    // projection constants: A = sum_j c_j c_j^T, c_j = (1, v1, v2, v3, |v|^2);
    // inelastic collisions do not conserve energy (Sec. 3.3): the constraint set
    // is then the first four rows, and (C C^T)^{-1} is the 4 x 4 inverse bordered
    // by zeros (so the energy multiplier is 0)
    const int nr = t.beta == 1.0 ? 5 : 4;
    double A[5][5] = {{0}};
    for (int j1 = 0; j1 < N; ++j1)
        for (int j2 = 0; j2 < N; ++j2)
            for (int j3 = 0; j3 < N; ++j3) {
                double v1 = t.dv * (j1 - h), v2 = t.dv * (j2 - h), v3 = t.dv * (j3 - h);
                double c[5] = {1.0, v1, v2, v3, v1 * v1 + v2 * v2 + v3 * v3};
                for (int a = 0; a < 5; ++a)
                    for (int b = 0; b < 5; ++b) A[a][b] += c[a] * c[b];
            }
    // Gauss-Jordan inverse of the leading nr x nr block with partial pivoting
    double Ai[5][10];
    for (int a = 0; a < nr; ++a)
        for (int b = 0; b < 2 * nr; ++b) Ai[a][b] = b < nr ? A[a][b] : (b - nr == a ? 1.0 : 0.0);
    for (int c = 0; c < nr; ++c) {
        int piv = c;
        for (int r = c + 1; r < nr; ++r)
            if (std::fabs(Ai[r][c]) > std::fabs(Ai[piv][c])) piv = r;
        for (int b = 0; b < 2 * nr; ++b) std::swap(Ai[c][b], Ai[piv][b]);
        double d = Ai[c][c];
        for (int b = 0; b < 2 * nr; ++b) Ai[c][b] /= d;
        for (int r = 0; r < nr; ++r)
            if (r != c) {
                double f = Ai[r][c];
                for (int b = 0; b < 2 * nr; ++b) Ai[r][b] -= f * Ai[c][b];
            }
    }
    for (int a = 0; a < 5; ++a)
        for (int b = 0; b < 5; ++b) t.ainv[a * 5 + b] = (a < nr && b < nr) ? Ai[a][b + nr] : 0.0;

    // DFT roots exp(2 pi i t / N)
    std::vector<float2> r32(N);
    std::vector<double2> r64(N);
    for (int s = 0; s < N; ++s) {
        double c = std::cos(2.0 * kPi * s / N), sn = std::sin(2.0 * kPi * s / N);
        r32[s] = make_float2((float)c, (float)sn);
        r64[s] = make_double2(c, sn);
    }

    // one group's work items, costliest first (stable, so ties keep (tile, k1, k2) order)
    std::vector<ConvItem> tmpl;
    std::vector<uint64_t> tcost;
    for (int tile = 0; tile < t.ntiles; ++tile)
        for (int kk = 0; kk < N * N; ++kk) {
            if (t.nblocks[kk] == 0) continue;
            ConvItem ci{};
            ci.fofs = 0;
            ci.wofs = t.wofs[(size_t)tile * N * N + kk];
            ci.desc_off = t.desc_off[kk];
            ci.nblocks = t.nblocks[kk];
            ci.k1 = (uint16_t)(kk / N);
            ci.k2 = (uint16_t)(kk % N);
            ci.kind = (uint16_t)(t.kind0 + tile);
            ci.table = 0;
            tmpl.push_back(ci);
            tcost.push_back((uint64_t)ci.nblocks * t.cpad[tile]);
        }
    {
        std::vector<size_t> ord(tmpl.size());
        for (size_t i = 0; i < ord.size(); ++i) ord[i] = i;
        std::stable_sort(ord.begin(), ord.end(), [&](size_t a, size_t b) { return tcost[a] > tcost[b]; });
        std::vector<ConvItem> sorted(tmpl.size());
        for (size_t i = 0; i < ord.size(); ++i) sorted[i] = tmpl[ord[i]];
        tmpl.swap(sorted);
    }
    t.n_tmpl = (int)tmpl.size();

    // on-the-fly weights (elastic tables): radial integrals in FP32 with the
    // constant factor, and each tile's entry list (m3 ascending, then k3)
    std::vector<float> I32, J32;
    std::vector<uint16_t> etab;
    if (t.beta == 1.0) {
        const double cw = std::sqrt(2.0 / kPi) * dz3;
        I32.resize(t.I.size());
        for (size_t i = 0; i < t.I.size(); ++i) I32[i] = (float)(cw * t.I[i]);
        J32.resize(t.J.size());
        for (size_t i = 0; i < t.J.size(); ++i) J32[i] = (float)(cw * t.J[i]);
        // per entry (m3, k3) of a tile, in the kernel's order: the third
        // components of the invariants, (k3'^2 | (2m3' - k3')^2 << 16,
        // m3'^2 | n3'^2 << 16) with n3' = k3' - m3', as four 16-bit fields
        t.estride = std::max(t.cpad[0], std::max(t.cpad[1], t.cpad[2]));
        etab.assign((size_t)t.ntiles * t.estride * 4, 0);
        for (int tile = 0; tile < t.ntiles; ++tile) {
            int e = 0;
            for (int m3 = 0; m3 < N; ++m3)
                for (int j = 0; j < T; ++j) {
                    const int k3 = tile * T + j, n3 = k3 - m3 + h;
                    if (n3 < 0 || n3 >= N) continue;
                    const int kp = k3 - h, mp = m3 - h, np3 = kp - mp;
                    uint16_t *c = &etab[((size_t)tile * t.estride + e++) * 4];
                    c[0] = (uint16_t)(kp * kp);
                    c[1] = (uint16_t)((2 * mp - kp) * (2 * mp - kp));
                    c[2] = (uint16_t)(mp * mp);
                    c[3] = (uint16_t)(np3 * np3);
                }
        }
    }

    // upload
    cudaError_t e = cudaSuccess;
    e = cudaMalloc(&t.d_tmpl, sizeof(ConvItem) * std::max<size_t>(tmpl.size(), 1));
    if (e == cudaSuccess && !I32.empty()) e = cudaMalloc(&t.d_I32, sizeof(float) * I32.size());
    if (e == cudaSuccess && !J32.empty()) e = cudaMalloc(&t.d_J32, sizeof(float) * J32.size());
    if (e == cudaSuccess && !etab.empty()) e = cudaMalloc(&t.d_etab, sizeof(uint16_t) * etab.size());
    if (e == cudaSuccess) e = cudaMalloc(&t.d_desc, sizeof(uint32_t) * std::max<size_t>(t.n_desc, 1));
    if (e == cudaSuccess) e = cudaMalloc(&t.d_root32, sizeof(float2) * N);
    if (e == cudaSuccess) e = cudaMalloc(&t.d_root64, sizeof(double2) * N);
    if (e != cudaSuccess) {
        err = std::string("cudaMalloc (weight table): ") + cudaGetErrorString(e);
        free_table(t);
        return BTE_ENOMEM;
    }
    if (e == cudaSuccess && !tmpl.empty())
        e = cudaMemcpy(t.d_tmpl, tmpl.data(), sizeof(ConvItem) * tmpl.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !I32.empty())
        e = cudaMemcpy(t.d_I32, I32.data(), sizeof(float) * I32.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !J32.empty())
        e = cudaMemcpy(t.d_J32, J32.data(), sizeof(float) * J32.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !etab.empty())
        e = cudaMemcpy(t.d_etab, etab.data(), sizeof(uint16_t) * etab.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(t.d_desc, desc.data(), sizeof(uint32_t) * t.n_desc, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(t.d_root32, r32.data(), sizeof(float2) * N, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(t.d_root64, r64.data(), sizeof(double2) * N, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        err = std::string("cudaMemcpy (weight table): ") + cudaGetErrorString(e);
        free_table(t);
        return BTE_ECUDA;
    }
    // the stored FP32 weights: built now up to N = 32; at N = 48 (10 GB) only
    // when a variant that streams them runs (weights on the fly need none)
    if (N <= 32) {
        const int r = build_table_fp32(t, err);
        if (r != BTE_OK) {
            free_table(t);
            return r;
        }
    }
    return BTE_OK;
}

// The FP32 pair-symmetrised weights (times dz^3) in the kernel's layout:
// per (tile, k1, k2) its kept blocks, per block m3 ascending then k3.
int build_table_fp32(Table &t, std::string &err) {
    if (t.d_w32) return BTE_OK;
    const int N = t.N, h = N / 2, T = conv_kind(t.kind0).T;
    const double dz3 = t.dz * t.dz * t.dz;
    std::vector<float> w32(t.n_w32, 0.0f);
#pragma omp parallel for collapse(2) schedule(dynamic, 1)
    for (int tile = 0; tile < t.ntiles; ++tile)
        for (int kk = 0; kk < N * N; ++kk) {
            const int k1 = kk / N, k2 = kk % N, K0 = tile * T;
            size_t o = t.wofs[(size_t)tile * N * N + kk];
            for (uint32_t b = 0; b < t.nblocks[kk]; ++b) {
                uint32_t d = t.desc_host[t.desc_off[kk] + b];
                int m1 = d & 0xffff, m2 = d >> 16, n1 = k1 - m1 + h, n2 = k2 - m2 + h;
                bool pair = !(m1 == n1 && m2 == n2);
                size_t wi = o + (size_t)b * t.cpad[tile];
                for (int m3 = 0; m3 < N; ++m3)
                    for (int j = 0; j < T; ++j) {
                        int k3 = K0 + j, n3 = k3 - m3 + h;
                        if (n3 < 0 || n3 >= N) continue;
                        double g = t.ghat(k1, k2, k3, m1, m2, m3);
                        if (pair) g += t.ghat(k1, k2, k3, n1, n2, n3);
                        w32[wi++] = (float)(g * dz3);
                    }
            }
        }
    cudaError_t e = cudaMalloc(&t.d_w32, sizeof(float) * std::max<size_t>(t.n_w32, 4));
    if (e != cudaSuccess) {
        cudaGetLastError();
        t.d_w32 = nullptr;
        err = std::string("cudaMalloc (FP32 weight table): ") + cudaGetErrorString(e);
        return BTE_ENOMEM;
    }
    e = cudaMemcpy(t.d_w32, w32.data(), sizeof(float) * t.n_w32, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        err = std::string("cudaMemcpy (FP32 weight table): ") + cudaGetErrorString(e);
        return BTE_ECUDA;
    }
    return BTE_OK;
}

// FP64 table of the plain operator: for each zeta point k (k1-major, k3
// fastest) the weights Ghat(k, m) dz^3 over its valid box of m (m1-major, m3
// fastest); off[k] is the prefix sum of the box sizes.
int build_table_fp64(Table &t, std::string &err) {
    if (t.d_w64) return BTE_OK;
    const int N = t.N, M = N * N * N;
    const double dz3 = t.dz * t.dz * t.dz;
    std::vector<uint64_t> off(M + 1, 0);
    for (int k = 0; k < M; ++k) {
        int k1 = k / (N * N), k2 = (k / N) % N, k3 = k % N;
        off[k + 1] = off[k] + (uint64_t)box_len(k1, N) * box_len(k2, N) * box_len(k3, N);
    }
    t.n_w64 = off[M];
    std::vector<double> w((size_t)t.n_w64);
#pragma omp parallel for schedule(dynamic, 16)
    for (int k = 0; k < M; ++k) {
        int k1 = k / (N * N), k2 = (k / N) % N, k3 = k % N;
        size_t o = off[k];
        for (int m1 = box_lo(k1, N); m1 <= box_hi(k1, N); ++m1)
            for (int m2 = box_lo(k2, N); m2 <= box_hi(k2, N); ++m2)
                for (int m3 = box_lo(k3, N); m3 <= box_hi(k3, N); ++m3)
                    w[o++] = t.ghat(k1, k2, k3, m1, m2, m3) * dz3;
    }
    cudaError_t e = cudaMalloc(&t.d_w64, sizeof(double) * std::max<uint64_t>(t.n_w64, 1));
    if (e == cudaSuccess) e = cudaMalloc(&t.d_w64_off, sizeof(uint64_t) * (M + 1));
    if (e != cudaSuccess) {
        err = std::string("cudaMalloc (FP64 weight table): ") + cudaGetErrorString(e);
        cudaFree(t.d_w64);
        cudaFree(t.d_w64_off);
        t.d_w64 = nullptr;
        t.d_w64_off = nullptr;
        return BTE_ENOMEM;
    }
    e = cudaMemcpy(t.d_w64, w.data(), sizeof(double) * t.n_w64, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(t.d_w64_off, off.data(), sizeof(uint64_t) * (M + 1), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        err = std::string("cudaMemcpy (FP64 weight table): ") + cudaGetErrorString(e);
        return BTE_ECUDA;
    }
    return BTE_OK;
}

void free_table(Table &t) {
    cudaFree(t.d_w32);
    cudaFree(t.d_tmpl);
    cudaFree(t.d_I32);
    cudaFree(t.d_J32);
    cudaFree(t.d_etab);
    t.d_tmpl = nullptr;
    t.d_I32 = t.d_J32 = nullptr;
    t.d_etab = nullptr;
    cudaFree(t.d_desc);
    cudaFree(t.d_w64);
    cudaFree(t.d_w64_off);
    cudaFree(t.d_root32);
    cudaFree(t.d_root64);
    t.d_w32 = nullptr;
    t.d_desc = nullptr;
    t.d_w64 = nullptr;
    t.d_w64_off = nullptr;
    t.d_root32 = nullptr;
    t.d_root64 = nullptr;
}

}  // namespace bte
