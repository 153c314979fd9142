/*
 * FP64 CPU oracle for the conservative spectral Boltzmann collision operator of
 * Haack & Gamba, "High Performance Computing with a Conservative Spectral
 * Boltzmann Solver" (arXiv:1211.0540).
 *
 * TEST INFRASTRUCTURE. This file is the independent, slow, obviously-correct
 * restatement of what the method computes. Only the tests, the smoke check and
 * the CPU-baseline leg of the benchmark may load it. It shares no code, header,
 * table or constant generator with the CUDA library; the product never calls it.
 *
 * Everything is plain FP64 with direct sums written as in the paper:
 *   - Sec. 2.2, Eq. GHat_calc: the convolution weights Ghat(xi, zeta) as a
 *     radial integral, evaluated here by composite Gauss-Legendre quadrature
 *     (NOT by a closed form; the library uses closed forms).
 *   - Sec. 3.1, Eq. meshpoints: v_k = dv (k - N/2), zeta_k = dz (k - N/2),
 *     dv = 2L/N, dz = pi/L.
 *   - Sec. 3.2: fhat by the discrete Fourier sum, the trapezoid weighted
 *     convolution with zero extension, the inverse sum back to velocity space.
 *   - Sec. 3.3: the constrained L2 projection with the 5 x M integration matrix C,
 *     solved through the 5 x 5 normal equations.
 *   - Sec. 3.1 / 3.4: RK2 time stepping, Strang splitting, second-order upwind
 *     finite-volume transport with the minmod slope (Eq. upwind) and the diffuse
 *     wall of Sec. 2.1 (Eq. BC).
 *
 * Readings where the paper is silent, garbled or ambiguous (each one is also
 * listed in the design notes of the repository):
 *   - projection: the printed "Q = Qt + C (C C^T)^-1 C Qt" is taken as
 *     Q = Qt - C^T (C C^T)^-1 C Qt, the Lagrange solution of the stated
 *     minimisation;
 *   - beta = 1 (elastic), sinc x = sin(x)/x (unnormalised);
 *   - trapezoid weights: uniform dz^3 in Fourier space, dv^3 in velocity space;
 *   - zero extension: fhat(zeta_k - xi_m) is used only when the grid index
 *     n = k - m + N/2 lies in [0, N) in every dimension;
 *   - the inverse transform keeps the real part (its imaginary part is reported);
 *   - RK2 = Heun (SSP-RK2), with the projection applied at each stage;
 *   - Strang ordering T(dt/2) C(dt) T(dt/2), collision sub-step dt/eps;
 *   - diffuse wall sigma_w normalised by the discrete outgoing flux, specular
 *     mirror i -> N - i on the asymmetric v1 grid (i = 0 has no partner: ghost 0);
 *   - non-uniform cells: the reconstruction uses the upwind cell's width, the
 *     minmod slope divided differences over centre distances; ghost widths
 *     mirror the adjacent cells; "no flux for the incoming characteristics":
 *     incoming ghost components 0, outgoing ones copied.
 *
 * Layout: one cell holds M = N^3 values, index (k1*N + k2)*N + k3 (k3 fastest).
 * Complex arrays are interleaved (re, im) pairs.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORA_PI 3.14159265358979323846

void ora_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int ora_get_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Quadrature                                                               */
/* ------------------------------------------------------------------------ */

/* Gauss-Legendre nodes/weights on [-1, 1]: roots of P_n by Newton's method on
 * the three-term recurrence (k P_k = (2k-1) z P_{k-1} - (k-1) P_{k-2}),
 * w = 2 / ((1 - z^2) P_n'(z)^2). */
int ora_gauss_legendre(int n, double *x, double *w) {
    if (n < 1) return -1;
    for (int i = 0; i < (n + 1) / 2; ++i) {
        double z = cos(ORA_PI * (i + 0.75) / (n + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 200; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            if (n == 1) { p1 = z; p0 = 1.0; }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (fabs(dz) < 1e-17) break;
        }
        {   /* derivative at the converged root */
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            if (n == 1) { p1 = z; p0 = 1.0; }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
        }
        x[i] = -z;
        x[n - 1 - i] = z;
        w[i] = w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
    return 0;
}

/* sinc x = sin(x)/x, sinc 0 = 1 (Taylor series near 0 to avoid 0/0). */
double ora_sinc(double x) {
    double ax = fabs(x);
    if (ax < 1e-4) {
        double x2 = x * x;
        return 1.0 - x2 / 6.0 + x2 * x2 / 120.0;
    }
    return sin(x) / x;
}

#define ORA_GL_PER_PANEL 16

/* Composite Gauss-Legendre rule on [0, L] whose panel count resolves the
 * highest angular frequency omega: at least 16 nodes per half period. The
 * first panel [0, h] is graded geometrically towards r = 0 (sub-panels
 * [h s^(j+1), h s^j], j < levels, and [0, h s^levels]): for non-integer
 * lambda the factor r^(lambda+2) is not smooth at 0, and one 16-point panel
 * there leaves errors of ~1e-9 relative; graded, the rule reaches FP64
 * accuracy (checked against 30-digit quadrature in the tests). For
 * lambda >= 0: s = 0.15, 12 levels. For the soft potentials, -3 < lambda < 0
 * (Sec. 2.1), the factor r^(lambda+2) may be singular: s = 0.3 (each graded
 * panel then keeps the singularity a panel width away) and enough levels that
 * the innermost panel's share, (h s^levels)^(lambda+3), falls below 1e-17 of
 * the first panel's. The caller frees *r and *w. Returns the node count. */
static int ora_radial_rule(double L, double omega, double lam, double **r, double **w) {
    const double ratio = lam >= 0.0 ? 0.15 : 0.3;
    const int levels = lam >= 0.0 ? 12 : (int)ceil(17.0 * log(10.0) / ((lam + 3.0) * -log(ratio))) + 4;
    int panels = (int)ceil(omega * L / ORA_PI) + 4;
    int nseg = panels - 1 + levels + 1;
    int n = nseg * ORA_GL_PER_PANEL;
    double gx[ORA_GL_PER_PANEL], gw[ORA_GL_PER_PANEL];
    ora_gauss_legendre(ORA_GL_PER_PANEL, gx, gw);
    *r = (double *)malloc(sizeof(double) * n);
    *w = (double *)malloc(sizeof(double) * n);
    double h = L / panels;
    int k = 0;
    for (int seg = 0; seg < nseg; ++seg) {
        double a, b;
        if (seg < panels - 1) { /* the uniform panels [p h, (p + 1) h], p >= 1 */
            a = (seg + 1) * h;
            b = (seg + 2) * h;
        } else if (seg < panels - 1 + levels) { /* graded sub-panels of [0, h] */
            int j = seg - (panels - 1);
            b = h * pow(ratio, j);
            a = b * ratio;
        } else {
            a = 0.0;
            b = h * pow(ratio, levels);
        }
        for (int q = 0; q < ORA_GL_PER_PANEL; ++q, ++k) {
            (*r)[k] = a + 0.5 * (b - a) * (gx[q] + 1.0);
            (*w)[k] = 0.5 * (b - a) * gw[q];
        }
    }
    return n;
}

/* I_lambda(a, b) = int_0^L r^{lambda+2} sinc(a r) sinc(b r) dr  (Eq. GHat_calc, gain term,
 * radial integral cut off at r0 = L, Sec. 3.1). */
double ora_radial_I(double lam, double L, double a, double b) {
    double *r, *w;
    int n = ora_radial_rule(L, fabs(a) + fabs(b), lam, &r, &w);
    double s = 0.0;
    for (int i = 0; i < n; ++i)
        s += w[i] * pow(r[i], lam + 2.0) * ora_sinc(a * r[i]) * ora_sinc(b * r[i]);
    free(r);
    free(w);
    return s;
}

/* J_lambda(c) = int_0^L r^{lambda+2} sinc(c r) dr  (Eq. GHat_calc, loss term). */
double ora_radial_J(double lam, double L, double c) {
    double *r, *w;
    int n = ora_radial_rule(L, fabs(c), lam, &r, &w);
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += w[i] * pow(r[i], lam + 2.0) * ora_sinc(c * r[i]);
    free(r);
    free(w);
    return s;
}

/* Ghat(xi_m, zeta_k) for one pair, straight from Eq. GHat_calc with beta = 1,
 * b = 1/(4 pi) (isotropic, Eq. cut-off), d = 3:
 *   Ghat = 4 pi / (2 pi)^{3/2} int_0^L r^{lambda+2} [sinc(r|zeta|/2) sinc(r|xi - zeta/2|) - sinc(r|xi|)] dr. */
double ora_ghat_pair(int N, double L, double lam, const int *k, const int *m) {
    double dz = ORA_PI / L;
    double zeta[3], xi[3];
    for (int d = 0; d < 3; ++d) {
        zeta[d] = dz * (k[d] - N / 2);
        xi[d] = dz * (m[d] - N / 2);
    }
    double nz = sqrt(zeta[0] * zeta[0] + zeta[1] * zeta[1] + zeta[2] * zeta[2]);
    double hx[3] = {xi[0] - 0.5 * zeta[0], xi[1] - 0.5 * zeta[1], xi[2] - 0.5 * zeta[2]};
    double nh = sqrt(hx[0] * hx[0] + hx[1] * hx[1] + hx[2] * hx[2]);
    double nx = sqrt(xi[0] * xi[0] + xi[1] * xi[1] + xi[2] * xi[2]);
    double pref = 4.0 * ORA_PI / pow(2.0 * ORA_PI, 1.5);
    return pref * (ora_radial_I(lam, L, 0.5 * nz, nh) - ora_radial_J(lam, L, nx));
}

/* ------------------------------------------------------------------------ */
/* Weight tables on integer invariants                                      */
/* ------------------------------------------------------------------------ */
/* On the grid of Eq. meshpoints every argument of the radial integrals is
 * (dz/2) * sqrt(integer):
 *   |zeta_k|/2        = (dz/2) sqrt(p),  p = |k'|^2,
 *   |xi_m - zeta_k/2| = (dz/2) sqrt(q),  q = |2m' - k'|^2,
 *   |xi_m|            =  dz    sqrt(s),  s = |m'|^2,
 * with k' = k - N/2, m' = m - N/2. So the oracle evaluates the integrals once
 * per integer and looks them up: Itab[p * nq + q] = I(p, q), Jtab[s] = J(s). */

void ora_weights_sizes(int N, int *np, int *nq, int *ns) {
    int h = N / 2;
    *np = 3 * h * h + 1;
    *nq = 3 * (N - 1) * (N - 1) + 1;
    *ns = 3 * h * h + 1;
}

int ora_weights_build(int N, double L, double lam, double *Itab, double *Jtab) {
    if (N < 2 || (N % 2) != 0 || L <= 0.0) return -1;
    int np, nq, ns;
    ora_weights_sizes(N, &np, &nq, &ns);
    double hz = 0.5 * ORA_PI / L; /* dz / 2 */
    /* One quadrature rule resolves the largest frequency of the table; the
     * sinc rows S[t][i] = sinc(hz sqrt(t) r_i) serve both integrals
     * (J(s) uses row t = 4s, since |xi| = hz sqrt(4s)). With the same rule for
     * both, Ghat(xi, 0) = I(0, 4s) - J(s) is exactly 0 as in the continuous form. */
    int nt = nq > 4 * (ns - 1) + 1 ? nq : 4 * (ns - 1) + 1;
    double *r, *w;
    int nn = ora_radial_rule(L, hz * (sqrt((double)(np - 1)) + sqrt((double)(nt - 1))), lam, &r, &w);
    double *S = (double *)malloc(sizeof(double) * (size_t)nt * nn);
    double *wr = (double *)malloc(sizeof(double) * nn); /* w_i r_i^{lambda+2} */
    for (int i = 0; i < nn; ++i) wr[i] = w[i] * pow(r[i], lam + 2.0);
#pragma omp parallel for schedule(static)
    for (int t = 0; t < nt; ++t) {
        double a = hz * sqrt((double)t);
        for (int i = 0; i < nn; ++i) S[(size_t)t * nn + i] = ora_sinc(a * r[i]);
    }
#pragma omp parallel for schedule(dynamic, 4)
    for (int p = 0; p < np; ++p) {
        const double *Sp = S + (size_t)p * nn;
        for (int q = 0; q < nq; ++q) {
            const double *Sq = S + (size_t)q * nn;
            double acc = 0.0;
            for (int i = 0; i < nn; ++i) acc += wr[i] * Sp[i] * Sq[i];
            Itab[(size_t)p * nq + q] = acc;
        }
    }
    for (int t = 0; t < ns; ++t) {
        const double *S0 = S, *St = S + (size_t)(4 * t) * nn;
        double acc = 0.0;
        for (int i = 0; i < nn; ++i) acc += wr[i] * S0[i] * St[i]; /* S0[i] == 1 */
        Jtab[t] = acc;
    }
    free(S);
    free(wr);
    free(r);
    free(w);
    return 0;
}

/* Ghat(xi_m, zeta_k) from the integer-invariant tables. part: 0 = full weight,
 * 1 = loss term only (-sqrt(2/pi) J), 2 = gain term only (sqrt(2/pi) I). */
static double ora_ghat_lookup(int N, int nq, const double *Itab, const double *Jtab, int part,
                              const int *k, const int *m) {
    int h = N / 2;
    int p = 0, q = 0, s = 0;
    for (int d = 0; d < 3; ++d) {
        int kp = k[d] - h, mp = m[d] - h;
        p += kp * kp;
        q += (2 * mp - kp) * (2 * mp - kp);
        s += mp * mp;
    }
    if (q >= nq) return NAN; /* pair outside the zero-extended support: never summed */
    double pref = 4.0 * ORA_PI / pow(2.0 * ORA_PI, 1.5);
    double gain = Itab[(size_t)p * nq + q], loss = Jtab[s];
    if (part == 1) return -pref * loss;
    if (part == 2) return pref * gain;
    return pref * (gain - loss);
}

/* Dense table G[k][m] (M x M, row = zeta index k) for small N. Entries whose
 * partner index n = k - m + N/2 leaves the grid are set to 0: the zero
 * extension of Sec. 3.2 drops those terms, so they never enter the sum. */
void ora_ghat_dense(int N, const double *Itab, const double *Jtab, int part, double *G) {
    int np, nq, ns;
    ora_weights_sizes(N, &np, &nq, &ns);
    int M = N * N * N, h = N / 2;
#pragma omp parallel for schedule(static)
    for (int kk = 0; kk < M; ++kk) {
        int k[3] = {kk / (N * N), (kk / N) % N, kk % N};
        for (int mm = 0; mm < M; ++mm) {
            int m[3] = {mm / (N * N), (mm / N) % N, mm % N};
            int valid = 1;
            for (int d = 0; d < 3; ++d) {
                int n = k[d] - m[d] + h;
                if (n < 0 || n >= N) valid = 0;
            }
            G[(size_t)kk * M + mm] = valid ? ora_ghat_lookup(N, nq, Itab, Jtab, part, k, m) : 0.0;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Discrete Fourier transforms (Sec. 3.2, Eq. meshpoints)                   */
/* ------------------------------------------------------------------------ */
/* zeta_k . v_j = dz dv sum_d k'_d j'_d = (2 pi / N) sum_d k'_d j'_d, so the
 * phase is reduced exactly with integer arithmetic modulo N. */

static void ora_phase_table(int N, double sign, double *c, double *s) {
    for (int t = 0; t < N; ++t) {
        c[t] = cos(2.0 * ORA_PI * t / N);
        s[t] = sign * sin(2.0 * ORA_PI * t / N);
    }
}

static int ora_mod(int a, int n) {
    int r = a % n;
    return r < 0 ? r + n : r;
}

/* fhat(zeta_k) = (2 pi)^{-3/2} dv^3 sum_j f(v_j) exp(-i zeta_k . v_j): the full
 * O(M^2) triple sum, one cell. */
void ora_dft_forward_direct(int N, double L, const double *f, double *fh) {
    int M = N * N * N, h = N / 2;
    double dv = 2.0 * L / N;
    double scale = pow(2.0 * ORA_PI, -1.5) * dv * dv * dv;
    double *c = (double *)malloc(sizeof(double) * N), *s = (double *)malloc(sizeof(double) * N);
    ora_phase_table(N, -1.0, c, s);
#pragma omp parallel for schedule(static)
    for (int kk = 0; kk < M; ++kk) {
        int k1 = kk / (N * N) - h, k2 = (kk / N) % N - h, k3 = kk % N - h;
        double re = 0.0, im = 0.0;
        for (int jj = 0; jj < M; ++jj) {
            int j1 = jj / (N * N) - h, j2 = (jj / N) % N - h, j3 = jj % N - h;
            int t = ora_mod(k1 * j1 + k2 * j2 + k3 * j3, N);
            re += f[jj] * c[t];
            im += f[jj] * s[t];
        }
        fh[2 * kk] = scale * re;
        fh[2 * kk + 1] = scale * im;
    }
    free(c);
    free(s);
}

/* One 1-D pass of exp(sign * i * 2 pi k' j' / N) along dimension `dim` of a
 * complex N^3 array (in -> out). */
static void ora_dft_axis(int N, int dim, double sign, const double *in, double *out) {
    int h = N / 2;
    double *c = (double *)malloc(sizeof(double) * N), *s = (double *)malloc(sizeof(double) * N);
    ora_phase_table(N, sign, c, s);
    int stride = dim == 0 ? N * N : (dim == 1 ? N : 1);
    for (int a = 0; a < N; ++a)
        for (int b = 0; b < N; ++b) {
            int base;
            if (dim == 0) base = a * N + b;
            else if (dim == 1) base = a * N * N + b;
            else base = (a * N + b) * N;
            for (int k = 0; k < N; ++k) {
                double re = 0.0, im = 0.0;
                for (int j = 0; j < N; ++j) {
                    int t = ora_mod((k - h) * (j - h), N);
                    double xr = in[2 * (base + j * stride)], xi = in[2 * (base + j * stride) + 1];
                    re += xr * c[t] - xi * s[t];
                    im += xr * s[t] + xi * c[t];
                }
                out[2 * (base + k * stride)] = re;
                out[2 * (base + k * stride) + 1] = im;
            }
        }
    free(c);
    free(s);
}

/* Forward transform of ncells cells: the same triple sum as
 * ora_dft_forward_direct, evaluated one dimension at a time (the kernel
 * exp(-i zeta.v) is a product over dimensions). */
void ora_dft_forward(int N, double L, int ncells, const double *f, double *fh) {
    int M = N * N * N;
    double dv = 2.0 * L / N;
    double scale = pow(2.0 * ORA_PI, -1.5) * dv * dv * dv;
#pragma omp parallel for schedule(dynamic, 1)
    for (int cidx = 0; cidx < ncells; ++cidx) {
        double *a = (double *)malloc(sizeof(double) * 2 * M), *b = (double *)malloc(sizeof(double) * 2 * M);
        for (int j = 0; j < M; ++j) {
            a[2 * j] = f[(size_t)cidx * M + j];
            a[2 * j + 1] = 0.0;
        }
        ora_dft_axis(N, 2, -1.0, a, b);
        ora_dft_axis(N, 1, -1.0, b, a);
        ora_dft_axis(N, 0, -1.0, a, b);
        for (int j = 0; j < 2 * M; ++j) fh[(size_t)cidx * 2 * M + j] = scale * b[j];
        free(a);
        free(b);
    }
}

/* Inverse transform (Sec. 3.2): Qt(v_j) = Re[(2 pi)^{-3/2} dz^3 sum_k Qhat_k exp(+i zeta_k . v_j)].
 * imag_ratio[c] (optional) receives ||Im|| / ||Re|| of the sum. */
void ora_dft_inverse(int N, double L, int ncells, const double *qh, double *q, double *imag_ratio) {
    int M = N * N * N;
    double dz = ORA_PI / L;
    double scale = pow(2.0 * ORA_PI, -1.5) * dz * dz * dz;
#pragma omp parallel for schedule(dynamic, 1)
    for (int cidx = 0; cidx < ncells; ++cidx) {
        double *a = (double *)malloc(sizeof(double) * 2 * M), *b = (double *)malloc(sizeof(double) * 2 * M);
        memcpy(a, qh + (size_t)cidx * 2 * M, sizeof(double) * 2 * M);
        ora_dft_axis(N, 2, +1.0, a, b);
        ora_dft_axis(N, 1, +1.0, b, a);
        ora_dft_axis(N, 0, +1.0, a, b);
        double nre = 0.0, nim = 0.0;
        for (int j = 0; j < M; ++j) {
            q[(size_t)cidx * M + j] = scale * b[2 * j];
            nre += b[2 * j] * b[2 * j];
            nim += b[2 * j + 1] * b[2 * j + 1];
        }
        if (imag_ratio) imag_ratio[cidx] = nre > 0.0 ? sqrt(nim / nre) : 0.0;
        free(a);
        free(b);
    }
}

/* ------------------------------------------------------------------------ */
/* Weighted convolution (Sec. 3.2, trapezoid rule, zero extension)          */
/* ------------------------------------------------------------------------ */
/* Qhat(zeta_k) = sum_m Ghat(xi_m, zeta_k) fhat(xi_m) fhat(zeta_k - xi_m) dz^3,
 * zeta_k - xi_m = zeta_n with n = k - m + N/2; terms with n outside the grid are
 * dropped (zero extension). Weights from the invariant tables. */
void ora_convolve(int N, double L, int ncells, const double *Itab, const double *Jtab, int part,
                  const double *fh, double *qh) {
    int np, nq, ns;
    ora_weights_sizes(N, &np, &nq, &ns);
    int M = N * N * N, h = N / 2;
    double dz = ORA_PI / L;
    double w = dz * dz * dz;
#pragma omp parallel for collapse(2) schedule(dynamic, 16)
    for (int cidx = 0; cidx < ncells; ++cidx)
        for (int kk = 0; kk < M; ++kk) {
            const double *F = fh + (size_t)cidx * 2 * M;
            int k[3] = {kk / (N * N), (kk / N) % N, kk % N};
            double re = 0.0, im = 0.0;
            for (int mm = 0; mm < M; ++mm) {
                int m[3] = {mm / (N * N), (mm / N) % N, mm % N};
                int n[3] = {k[0] - m[0] + h, k[1] - m[1] + h, k[2] - m[2] + h};
                if (n[0] < 0 || n[0] >= N || n[1] < 0 || n[1] >= N || n[2] < 0 || n[2] >= N) continue;
                int nn = (n[0] * N + n[1]) * N + n[2];
                double g = ora_ghat_lookup(N, nq, Itab, Jtab, part, k, m);
                double ar = F[2 * mm], ai = F[2 * mm + 1], br = F[2 * nn], bi = F[2 * nn + 1];
                re += g * (ar * br - ai * bi);
                im += g * (ar * bi + ai * br);
            }
            qh[(size_t)cidx * 2 * M + 2 * kk] = w * re;
            qh[(size_t)cidx * 2 * M + 2 * kk + 1] = w * im;
        }
}

/* Same sum with an arbitrary dense weight table G[k][m] (M x M), for tests. */
void ora_convolve_dense(int N, double L, int ncells, const double *G, const double *fh, double *qh) {
    int M = N * N * N, h = N / 2;
    double dz = ORA_PI / L;
    double w = dz * dz * dz;
#pragma omp parallel for collapse(2) schedule(static)
    for (int cidx = 0; cidx < ncells; ++cidx)
        for (int kk = 0; kk < M; ++kk) {
            const double *F = fh + (size_t)cidx * 2 * M;
            int k[3] = {kk / (N * N), (kk / N) % N, kk % N};
            double re = 0.0, im = 0.0;
            for (int mm = 0; mm < M; ++mm) {
                int m[3] = {mm / (N * N), (mm / N) % N, mm % N};
                int n[3] = {k[0] - m[0] + h, k[1] - m[1] + h, k[2] - m[2] + h};
                if (n[0] < 0 || n[0] >= N || n[1] < 0 || n[1] >= N || n[2] < 0 || n[2] >= N) continue;
                int nn = (n[0] * N + n[1]) * N + n[2];
                double g = G[(size_t)kk * M + mm];
                double ar = F[2 * mm], ai = F[2 * mm + 1], br = F[2 * nn], bi = F[2 * nn + 1];
                re += g * (ar * br - ai * bi);
                im += g * (ar * bi + ai * br);
            }
            qh[(size_t)cidx * 2 * M + 2 * kk] = w * re;
            qh[(size_t)cidx * 2 * M + 2 * kk + 1] = w * im;
        }
}

/* ------------------------------------------------------------------------ */
/* Conservation (Sec. 3.3)                                                  */
/* ------------------------------------------------------------------------ */

/* Rows of the integration matrix C at grid point j: dv^3 * (1, v1, v2, v3, |v|^2). */
static void ora_c_column(int N, double L, int j, double *col) {
    double dv = 2.0 * L / N, w = dv * dv * dv;
    int h = N / 2;
    double v1 = dv * (j / (N * N) - h), v2 = dv * ((j / N) % N - h), v3 = dv * (j % N - h);
    col[0] = w;
    col[1] = w * v1;
    col[2] = w * v2;
    col[3] = w * v3;
    col[4] = w * (v1 * v1 + v2 * v2 + v3 * v3);
}

/* mom[5 * c + i] = (C f_c)_i: mass, momentum, energy integrals by the trapezoid rule. */
void ora_moments(int N, double L, int ncells, const double *f, double *mom) {
    int M = N * N * N;
    for (int cidx = 0; cidx < ncells; ++cidx) {
        double s[5] = {0, 0, 0, 0, 0}, col[5];
        for (int j = 0; j < M; ++j) {
            ora_c_column(N, L, j, col);
            for (int i = 0; i < 5; ++i) s[i] += col[i] * f[(size_t)cidx * M + j];
        }
        for (int i = 0; i < 5; ++i) mom[5 * cidx + i] = s[i];
    }
}

/* Solve the SPD n x n system A x = b (n <= 5) by Cholesky (A is overwritten). */
static void ora_chol(int n, double A[5][5], double *b) {
    for (int j = 0; j < n; ++j) {
        double d = A[j][j];
        for (int k = 0; k < j; ++k) d -= A[j][k] * A[j][k];
        A[j][j] = sqrt(d);
        for (int i = j + 1; i < n; ++i) {
            double s = A[i][j];
            for (int k = 0; k < j; ++k) s -= A[i][k] * A[j][k];
            A[i][j] = s / A[j][j];
        }
    }
    for (int i = 0; i < n; ++i) {
        double s = b[i];
        for (int k = 0; k < i; ++k) s -= A[i][k] * b[k];
        b[i] = s / A[i][i];
    }
    for (int i = n - 1; i >= 0; --i) {
        double s = b[i];
        for (int k = i + 1; k < n; ++k) s -= A[k][i] * b[k];
        b[i] = s / A[i][i];
    }
}

/* Q <- Q - C^T (C C^T)^{-1} C Q with the first nrows rows of C, in place,
 * followed by one refinement pass (the same correction applied to the
 * corrected Q). nrows = 5: mass, momentum and energy (elastic collisions);
 * nrows = 4: mass and momentum only (inelastic collisions do not conserve
 * energy, Sec. 3.3). */
void ora_project_rows(int N, double L, int ncells, int nrows, double *Q) {
    int M = N * N * N;
    if (nrows < 1 || nrows > 5) return;
    double A0[5][5] = {{0}};
    double col[5];
    for (int j = 0; j < M; ++j) {
        ora_c_column(N, L, j, col);
        for (int a = 0; a < nrows; ++a)
            for (int b = 0; b < nrows; ++b) A0[a][b] += col[a] * col[b];
    }
#pragma omp parallel for schedule(static)
    for (int cidx = 0; cidx < ncells; ++cidx) {
        double *q = Q + (size_t)cidx * M;
        for (int pass = 0; pass < 2; ++pass) {
            double mu[5] = {0, 0, 0, 0, 0}, c5[5];
            for (int j = 0; j < M; ++j) {
                ora_c_column(N, L, j, c5);
                for (int i = 0; i < nrows; ++i) mu[i] += c5[i] * q[j];
            }
            double A[5][5];
            memcpy(A, A0, sizeof(A));
            ora_chol(nrows, A, mu);
            for (int j = 0; j < M; ++j) {
                ora_c_column(N, L, j, c5);
                double corr = 0.0;
                for (int i = 0; i < nrows; ++i) corr += c5[i] * mu[i];
                q[j] -= corr;
            }
        }
    }
}

/* The elastic projection: all five rows of C. */
void ora_project(int N, double L, int ncells, double *Q) { ora_project_rows(N, L, ncells, 5, Q); }

/* ------------------------------------------------------------------------ */
/* Collision operator                                                       */
/* ------------------------------------------------------------------------ */

/* Q = P_N Qt(f) for ncells cells (f, Q: ncells x M). Optional outputs: the raw
 * (unprojected) Qt and ||Im|| / ||Re|| of the inverse transform. part selects
 * the weight (0 full, 1 loss only, 2 gain only); project = 0 skips P_N. */
void ora_collide(int N, double L, int ncells, const double *Itab, const double *Jtab, int part,
                 int project, const double *f, double *Q, double *Qraw, double *imag_ratio) {
    int M = N * N * N;
    double *fh = (double *)malloc(sizeof(double) * 2 * (size_t)M * ncells);
    double *qh = (double *)malloc(sizeof(double) * 2 * (size_t)M * ncells);
    ora_dft_forward(N, L, ncells, f, fh);
    ora_convolve(N, L, ncells, Itab, Jtab, part, fh, qh);
    ora_dft_inverse(N, L, ncells, qh, Q, imag_ratio);
    if (Qraw) memcpy(Qraw, Q, sizeof(double) * (size_t)M * ncells);
    if (project) ora_project(N, L, ncells, Q);
    free(fh);
    free(qh);
}

/* Space-homogeneous Heun step on df/dt = Q(f,f)/eps with the projection at each
 * stage (Sec. 3.1):  Q1 = P Qt(f); f* = f + dt/eps Q1; Q2 = P Qt(f*);
 * f <- f + dt/(2 eps) (Q1 + Q2). */
void ora_rk2_homogeneous(int N, double L, int ncells, const double *Itab, const double *Jtab,
                         double dt, double eps, double *f) {
    size_t n = (size_t)N * N * N * ncells;
    double *q1 = (double *)malloc(sizeof(double) * n);
    double *q2 = (double *)malloc(sizeof(double) * n);
    double *fs = (double *)malloc(sizeof(double) * n);
    ora_collide(N, L, ncells, Itab, Jtab, 0, 1, f, q1, NULL, NULL);
    for (size_t i = 0; i < n; ++i) fs[i] = f[i] + dt / eps * q1[i];
    ora_collide(N, L, ncells, Itab, Jtab, 0, 1, fs, q2, NULL, NULL);
    for (size_t i = 0; i < n; ++i) f[i] += 0.5 * dt / eps * (q1[i] + q2[i]);
    free(q1);
    free(q2);
    free(fs);
}

/* ------------------------------------------------------------------------ */
/* Inelastic collisions (beta in Eq. G_eqn and Eq. GHat_calc; Sec. 3.3)     */
/* ------------------------------------------------------------------------ */
/* The collision rule with restitution parameter beta is
 * v' = v + (beta/2)(|u| sigma - u) (beta = 1: the elastic rule of
 * Eq. velocity_interact), and Eq. GHat_calc keeps beta in the gain term:
 *   Ghat = 4 pi/(2 pi)^{3/2} int_0^L r^{lam+2} [sinc(beta r |zeta|/2) sinc(r |xi - beta zeta/2|)
 *                                              - sinc(r |xi|)] dr.
 * On the grid the gain arguments are a = beta hz sqrt(p) and
 * b = hz |2 m' - beta k'| = hz sqrt(4 s - 4 beta t + beta^2 p), hz = dz/2, with the
 * integers p = |k'|^2, s = |m'|^2, t = k'.m'; so the gain integrals are
 * tabulated on the triple (p, s, t) (only the triples some zero-extended pair
 * uses are evaluated) and the loss integrals on s, as for beta = 1.
 * I3[(p * np + s) * nt + t + 3h^2], np = 3h^2 + 1, nt = 6h^2 + 1 (N <= 16). */

void ora_weights_sizes_beta(int N, int *np, int *nt) {
    int h = N / 2;
    *np = 3 * h * h + 1;
    *nt = 6 * h * h + 1;
}

int ora_weights_build_beta(int N, double L, double lam, double beta, double *I3, double *Jtab) {
    if (N < 2 || (N % 2) != 0 || N > 16 || L <= 0.0 || !(beta > 0.0 && beta <= 1.0)) return -1;
    int np, nt, h = N / 2, M = N * N * N, T0 = 3 * h * h;
    ora_weights_sizes_beta(N, &np, &nt);
    size_t nI = (size_t)np * np * nt;
    unsigned char *need = (unsigned char *)calloc(nI, 1);
    if (!need) return -2;
    for (int kk = 0; kk < M; ++kk) {
        int k[3] = {kk / (N * N) - h, (kk / N) % N - h, kk % N - h};
        for (int mm = 0; mm < M; ++mm) {
            int m[3] = {mm / (N * N) - h, (mm / N) % N - h, mm % N - h};
            int p = 0, sm = 0, t = 0, valid = 1;
            for (int d = 0; d < 3; ++d) {
                int n = k[d] - m[d] + h; /* grid index of zeta - xi (k, m here are k', m') */
                if (n < 0 || n >= N) valid = 0;
                p += k[d] * k[d];
                sm += m[d] * m[d];
                t += k[d] * m[d];
            }
            if (valid) need[((size_t)p * np + sm) * nt + (t + T0)] = 1;
        }
    }
    double hz = 0.5 * ORA_PI / L;
#pragma omp parallel for schedule(dynamic, 256)
    for (long long idx = 0; idx < (long long)nI; ++idx) {
        if (!need[idx]) {
            I3[idx] = NAN;
            continue;
        }
        int t = (int)(idx % nt) - T0;
        int sm = (int)((idx / nt) % np);
        int p = (int)(idx / ((size_t)nt * np));
        double a = beta * hz * sqrt((double)p);
        double b2 = 4.0 * sm - 4.0 * beta * t + beta * beta * p; /* |2m' - beta k'|^2 >= 0 */
        double b = hz * sqrt(b2 > 0.0 ? b2 : 0.0);
        I3[idx] = ora_radial_I(lam, L, a, b);
    }
    for (int sm = 0; sm < np; ++sm) Jtab[sm] = ora_radial_J(lam, L, hz * sqrt((double)(4 * sm)));
    free(need);
    return 0;
}

static double ora_ghat_lookup_beta(int N, const double *I3, const double *Jtab, int part, const int *k,
                                   const int *m) {
    int np, nt, h = N / 2;
    ora_weights_sizes_beta(N, &np, &nt);
    int p = 0, sm = 0, t = 0;
    for (int d = 0; d < 3; ++d) {
        int kp = k[d] - h, mp = m[d] - h;
        p += kp * kp;
        sm += mp * mp;
        t += kp * mp;
    }
    double pref = 4.0 * ORA_PI / pow(2.0 * ORA_PI, 1.5);
    double gain = I3[((size_t)p * np + sm) * nt + (t + 3 * h * h)], loss = Jtab[sm];
    if (part == 1) return -pref * loss;
    if (part == 2) return pref * gain;
    return pref * (gain - loss);
}

/* The weighted convolution of Sec. 3.2 with the inelastic weights. */
void ora_convolve_beta(int N, double L, int ncells, const double *I3, const double *Jtab, int part,
                       const double *fh, double *qh) {
    int M = N * N * N, h = N / 2;
    double dz = ORA_PI / L;
    double w = dz * dz * dz;
#pragma omp parallel for collapse(2) schedule(dynamic, 16)
    for (int cidx = 0; cidx < ncells; ++cidx)
        for (int kk = 0; kk < M; ++kk) {
            const double *F = fh + (size_t)cidx * 2 * M;
            int k[3] = {kk / (N * N), (kk / N) % N, kk % N};
            double re = 0.0, im = 0.0;
            for (int mm = 0; mm < M; ++mm) {
                int m[3] = {mm / (N * N), (mm / N) % N, mm % N};
                int n[3] = {k[0] - m[0] + h, k[1] - m[1] + h, k[2] - m[2] + h};
                if (n[0] < 0 || n[0] >= N || n[1] < 0 || n[1] >= N || n[2] < 0 || n[2] >= N) continue;
                int nn = (n[0] * N + n[1]) * N + n[2];
                double g = ora_ghat_lookup_beta(N, I3, Jtab, part, k, m);
                double ar = F[2 * mm], ai = F[2 * mm + 1], br = F[2 * nn], bi = F[2 * nn + 1];
                re += g * (ar * br - ai * bi);
                im += g * (ar * bi + ai * br);
            }
            qh[(size_t)cidx * 2 * M + 2 * kk] = w * re;
            qh[(size_t)cidx * 2 * M + 2 * kk + 1] = w * im;
        }
}

/* Q = P Qt(f) with the inelastic weights and the projection on the first
 * nrows rows of C (4: mass and momentum). Arguments as ora_collide. */
void ora_collide_beta(int N, double L, int ncells, const double *I3, const double *Jtab, int part, int nrows,
                      int project, const double *f, double *Q, double *Qraw, double *imag_ratio) {
    int M = N * N * N;
    double *fh = (double *)malloc(sizeof(double) * 2 * (size_t)M * ncells);
    double *qh = (double *)malloc(sizeof(double) * 2 * (size_t)M * ncells);
    ora_dft_forward(N, L, ncells, f, fh);
    ora_convolve_beta(N, L, ncells, I3, Jtab, part, fh, qh);
    ora_dft_inverse(N, L, ncells, qh, Q, imag_ratio);
    if (Qraw) memcpy(Qraw, Q, sizeof(double) * (size_t)M * ncells);
    if (project) ora_project_rows(N, L, ncells, nrows, Q);
    free(fh);
    free(qh);
}

/* Heun step of Sec. 3.1 with the inelastic operator (projection on nrows rows at each stage). */
void ora_rk2_homogeneous_beta(int N, double L, int ncells, const double *I3, const double *Jtab, int nrows,
                              double dt, double eps, double *f) {
    size_t n = (size_t)N * N * N * ncells;
    double *q1 = (double *)malloc(sizeof(double) * n);
    double *q2 = (double *)malloc(sizeof(double) * n);
    double *fs = (double *)malloc(sizeof(double) * n);
    ora_collide_beta(N, L, ncells, I3, Jtab, 0, nrows, 1, f, q1, NULL, NULL);
    for (size_t i = 0; i < n; ++i) fs[i] = f[i] + dt / eps * q1[i];
    ora_collide_beta(N, L, ncells, I3, Jtab, 0, nrows, 1, fs, q2, NULL, NULL);
    for (size_t i = 0; i < n; ++i) f[i] += 0.5 * dt / eps * (q1[i] + q2[i]);
    free(q1);
    free(q2);
    free(fs);
}

/* ------------------------------------------------------------------------ */
/* Transport (Sec. 3.4, Eq. upwind) with wall boundaries (Sec. 2.1, Eq. BC) */
/* ------------------------------------------------------------------------ */

#define ORA_BC_DIFFUSE 0
#define ORA_BC_SPECULAR 1
#define ORA_BC_NOFLUX 2

static double ora_minmod(double a, double b) {
    if (a * b <= 0.0) return 0.0;
    return a > 0.0 ? (a < b ? a : b) : (a > b ? a : b);
}

/* Wall Maxwellian with unit gas constant and zero wall velocity:
 * M_w(v) = (2 pi T_w)^{-3/2} exp(-|v|^2 / (2 T_w)). */
static double ora_wall_maxwellian(double Tw, double v1, double v2, double v3) {
    return pow(2.0 * ORA_PI * Tw, -1.5) * exp(-(v1 * v1 + v2 * v2 + v3 * v3) / (2.0 * Tw));
}

/* Fill the two ghost cells on one side. side = 0: left wall (inward normal +e1,
 * ghosts g[0] = cell -1, g[1] = cell -2; the adjacent interior cells are
 * f0 = cell 0, f1 = cell 1). side = 1: right wall (inward normal -e1, g[0] =
 * cell nx, g[1] = cell nx+1, f0 = cell nx-1, f1 = cell nx-2). */
static void ora_fill_ghosts(int N, double L, int side, int bc, double Tw, const double *f0,
                            const double *f1, double *g0, double *g1) {
    int M = N * N * N, h = N / 2;
    double dv = 2.0 * L / N;
    if (bc == ORA_BC_NOFLUX) {
        /* no flux for the incoming characteristics (Sec. 3.4, for boundaries
         * without wall interaction): incoming components (v.n > 0) are 0 in the
         * ghosts, outgoing ones copy the adjacent cell (they leave freely). */
        for (int j = 0; j < M; ++j) {
            double v1 = dv * (j / (N * N) - h);
            double vn = side == 0 ? v1 : -v1;
            g0[j] = g1[j] = vn > 0.0 ? 0.0 : f0[j];
        }
        return;
    }
    if (bc == ORA_BC_SPECULAR) {
        /* mirror v1 -> -v1: index i -> N - i; i = 0 (v1 = -L) has no partner on the grid. */
        for (int j = 0; j < M; ++j) {
            int i = j / (N * N), rest = j % (N * N);
            if (i == 0) {
                g0[j] = 0.0;
                g1[j] = 0.0;
            } else {
                int jm = (N - i) * N * N + rest;
                g0[j] = f0[jm];
                g1[j] = f1[jm];
            }
        }
        return;
    }
    /* diffuse: incoming components take sigma_w M_w, outgoing ones copy the
     * adjacent interior cell (zero gradient). sigma_w balances the discrete
     * outgoing flux: sigma_w sum_in |v.n| M_w = sum_out |v.n| f0. */
    double out = 0.0, in = 0.0;
    for (int j = 0; j < M; ++j) {
        int i = j / (N * N);
        double v1 = dv * (i - h), v2 = dv * ((j / N) % N - h), v3 = dv * (j % N - h);
        double vn = side == 0 ? v1 : -v1;
        if (vn < 0.0) out += -vn * f0[j];
        else if (vn > 0.0) in += vn * ora_wall_maxwellian(Tw, v1, v2, v3);
    }
    double sigma = in > 0.0 ? out / in : 0.0;
    for (int j = 0; j < M; ++j) {
        int i = j / (N * N);
        double v1 = dv * (i - h), v2 = dv * ((j / N) % N - h), v3 = dv * (j % N - h);
        double vn = side == 0 ? v1 : -v1;
        if (vn > 0.0) {
            g0[j] = g1[j] = sigma * ora_wall_maxwellian(Tw, v1, v2, v3);
        } else {
            g0[j] = g1[j] = f0[j];
        }
    }
}

/* Right-hand side -(F_{j+1/2} - F_{j-1/2}) / dx_j for all interior cells of the
 * extended array e (nx + 4 cells: two ghosts each side, interior at 2..nx+1),
 * on cells of widths w (nx + 4 entries; the ghosts mirror the widths of the
 * adjacent interior cells). Eq. upwind with the cell width of the upwind cell
 * in the reconstruction, F = v1 (f_j + dx_j/2 s_j) for v1 >= 0, and the minmod
 * slope of divided differences over the distances between cell centres,
 * s_j = minmod((f_j - f_{j-1}) / h_{j-1/2}, (f_{j+1} - f_j) / h_{j+1/2}),
 * h_{j+1/2} = (dx_j + dx_{j+1}) / 2 (on a uniform grid: dx). */
static void ora_transport_rhs(int N, double L, int nx, const double *w, const double *e, double *rhs) {
    int M = N * N * N, h = N / 2;
    double dv = 2.0 * L / N;
#pragma omp parallel for schedule(static)
    for (int j = 0; j < M; ++j) {
        double v1 = dv * (j / (N * N) - h);
        for (int c = 0; c < nx; ++c) {
            int x = c + 2;
            double F[2];
            for (int face = 0; face < 2; ++face) {
                int lft = x - 1 + face, rgt = x + face; /* face between lft and rgt */
                double fl = e[(size_t)lft * M + j], fr = e[(size_t)rgt * M + j];
                double hc = 0.5 * (w[lft] + w[rgt]);
                if (v1 >= 0.0) {
                    double fll = e[(size_t)(lft - 1) * M + j];
                    double hl = 0.5 * (w[lft - 1] + w[lft]);
                    double sig = ora_minmod((fl - fll) / hl, (fr - fl) / hc);
                    F[face] = v1 * (fl + 0.5 * w[lft] * sig);
                } else {
                    double frr = e[(size_t)(rgt + 1) * M + j];
                    double hr = 0.5 * (w[rgt] + w[rgt + 1]);
                    double sig = ora_minmod((fr - fl) / hc, (frr - fr) / hr);
                    F[face] = v1 * (fr - 0.5 * w[rgt] * sig);
                }
            }
            rhs[(size_t)c * M + j] = -(F[1] - F[0]) / w[x];
        }
    }
}

static void ora_extend(int N, double L, int nx, const double *f, int bc_l, int bc_r, double Tw_l,
                       double Tw_r, double *e) {
    size_t M = (size_t)N * N * N;
    memcpy(e + 2 * M, f, sizeof(double) * M * nx);
    ora_fill_ghosts(N, L, 0, bc_l, Tw_l, f, f + M, e + 1 * M, e + 0 * M);
    ora_fill_ghosts(N, L, 1, bc_r, Tw_r, f + (nx - 1) * M, f + (nx - 2) * M, e + (nx + 2) * M,
                    e + (nx + 3) * M);
}

/* Transport sub-step of length tau on f (nx cells of M values, widths dx[0..nx),
 * Sec. 3.4: "cells of size dx_j, not necessarily uniform") by Heun's method:
 * f1 = f + tau R(f); f <- (f + f1 + tau R(f1)) / 2. */
void ora_transport_grid(int N, double L, int nx, const double *dx, int bc_l, int bc_r, double Tw_l,
                        double Tw_r, double tau, double *f) {
    size_t M = (size_t)N * N * N, n = M * nx;
    double *w = (double *)malloc(sizeof(double) * (nx + 4));
    for (int c = 0; c < nx; ++c) w[c + 2] = dx[c];
    w[1] = dx[0]; /* ghost widths mirror the adjacent interior cells */
    w[0] = dx[1];
    w[nx + 2] = dx[nx - 1];
    w[nx + 3] = dx[nx - 2];
    double *e = (double *)malloc(sizeof(double) * M * (nx + 4));
    double *r = (double *)malloc(sizeof(double) * n);
    double *f1 = (double *)malloc(sizeof(double) * n);
    ora_extend(N, L, nx, f, bc_l, bc_r, Tw_l, Tw_r, e);
    ora_transport_rhs(N, L, nx, w, e, r);
    for (size_t i = 0; i < n; ++i) f1[i] = f[i] + tau * r[i];
    ora_extend(N, L, nx, f1, bc_l, bc_r, Tw_l, Tw_r, e);
    ora_transport_rhs(N, L, nx, w, e, r);
    for (size_t i = 0; i < n; ++i) f[i] = 0.5 * (f[i] + f1[i] + tau * r[i]);
    free(w);
    free(e);
    free(r);
    free(f1);
}

/* The same on nx uniform cells of [x0, x1]. */
void ora_transport(int N, double L, int nx, double x0, double x1, int bc_l, int bc_r, double Tw_l,
                   double Tw_r, double tau, double *f) {
    double *dx = (double *)malloc(sizeof(double) * nx);
    for (int c = 0; c < nx; ++c) dx[c] = (x1 - x0) / nx;
    ora_transport_grid(N, L, nx, dx, bc_l, bc_r, Tw_l, Tw_r, tau, f);
    free(dx);
}

/* One Strang step T(dt/2) C(dt) T(dt/2) of the space-inhomogeneous problem. */
void ora_strang_step(int N, double L, int nx, double x0, double x1, int bc_l, int bc_r,
                     double Tw_l, double Tw_r, const double *Itab, const double *Jtab, double dt,
                     double eps, double *f) {
    ora_transport(N, L, nx, x0, x1, bc_l, bc_r, Tw_l, Tw_r, 0.5 * dt, f);
    ora_rk2_homogeneous(N, L, nx, Itab, Jtab, dt, eps, f);
    ora_transport(N, L, nx, x0, x1, bc_l, bc_r, Tw_l, Tw_r, 0.5 * dt, f);
}

/* The Strang step on cells of widths dx[0..nx). */
void ora_strang_step_grid(int N, double L, int nx, const double *dx, int bc_l, int bc_r, double Tw_l,
                          double Tw_r, const double *Itab, const double *Jtab, double dt, double eps,
                          double *f) {
    ora_transport_grid(N, L, nx, dx, bc_l, bc_r, Tw_l, Tw_r, 0.5 * dt, f);
    ora_rk2_homogeneous(N, L, nx, Itab, Jtab, dt, eps, f);
    ora_transport_grid(N, L, nx, dx, bc_l, bc_r, Tw_l, Tw_r, 0.5 * dt, f);
}
