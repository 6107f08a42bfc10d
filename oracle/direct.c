/*
 * Brute-force FP64 oracle routes for the SE(2) convolution on Z^2\SE(2).
 *
 * TEST INFRASTRUCTURE ONLY: built by __graft_entry__.build() into oracle/lib/
 * and loaded only by tests/ and bench.py's CPU legs.  Shares no code with the
 * CUDA library.
 *
 * se2_direct_conv: the discrete periodic convolution that the FFT scheme
 *   computes at output grid N = L (closed form below Eq. MatSKfgonG, Section
 *   6.1), written as the rectangle rule of the convolution integral
 *   Eq. f*gRadialMain with the Haar measure Eq. dg:
 *     out[n] = (1/|L|) sum_m F[m] P[(n - m + c) mod (M, N, N)],
 *   c = (0, N/2, N/2).  The half-period shift comes from the grid offset
 *   x_i = -1/2 + i/N of Eq. OmL: x_n - x_m = x_{n-m+N/2}.  Even N only.
 *
 * se2_group_quadrature: the same rectangle rule, but written from the group
 *   convolution Eq. f*g with the full SE(2) law (Eq. SE2law): the kernel is
 *   evaluated at g^{-1} h = (S^{-1}(x - y - l), S^{-1} R) for every lattice
 *   image l (Eq. TH, the coset convolution Eq. oslash), i.e. the translation
 *   argument is rotated by -alpha.  For a kernel radial in translations this
 *   equals se2_direct_conv (Theorem f*gP(1)); for a non-radial kernel it does
 *   not, which the tests use as a negative check.
 *
 * Kernel families for se2_group_quadrature (kind):
 *   0: radial Gaussian (sigma) * 2pi * wrapped normal (sigma_t, centre nu);
 *      params = {sigma, sigma_t, nu}
 *   1: anisotropic Gaussian (s1 along x, s2 along y) * 2pi * wrapped normal;
 *      params = {s1, s2, sigma_t, nu}  -- NOT radial
 *   2: the SE(2) Gaussian via the matrix logarithm (Eq. gbS0), shifted by nu
 *      in the rotations; radial in translations; params = {sigma^2, nu}
 */
#include <math.h>
#include <stddef.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

static inline long idx3(long l, long j, long i, long N) { return (l * N + j) * N + i; }

/* The same sum with the kernel index shifted by c in x and y: c = N/2 on
 * Omega_L (x_i = -1/2 + i/N), c = 0 for grids sampled at x_i = i/N (the plain
 * cyclic convolution). */
void se2_direct_conv_shift(const double* F, const double* P, int N, int M, int c, double* out) {
    const long L = (long)N * N * M;
    for (int ln = 0; ln < M; ++ln)
        for (int jn = 0; jn < N; ++jn)
            for (int in = 0; in < N; ++in) {
                double acc = 0.0;
                for (int lm = 0; lm < M; ++lm) {
                    const int lp = ((ln - lm) % M + M) % M;
                    for (int jm = 0; jm < N; ++jm) {
                        const int jp = ((jn - jm + c) % N + N) % N;
                        const double* Frow = F + idx3(lm, jm, 0, N);
                        const double* Prow = P + idx3(lp, jp, 0, N);
                        for (int im = 0; im < N; ++im) {
                            const int ip = ((in - im + c) % N + N) % N;
                            acc += Frow[im] * Prow[ip];
                        }
                    }
                }
                out[idx3(ln, jn, in, N)] = acc / (double)L;
            }
}

void se2_direct_conv(const double* F, const double* P, int N, int M, double* out) {
    se2_direct_conv_shift(F, P, N, M, N / 2, out);
}

/* Only the listed output points (flat indices into [M][N][N]). */
void se2_direct_conv_points(const double* F, const double* P, int N, int M,
                            const long* pts, long npts, double* out) {
    const long L = (long)N * N * M;
    const int c = N / 2;
    for (long q = 0; q < npts; ++q) {
        const long n = pts[q];
        const int in = (int)(n % N), jn = (int)((n / N) % N), ln = (int)(n / ((long)N * N));
        double acc = 0.0;
        for (int lm = 0; lm < M; ++lm) {
            const int lp = ((ln - lm) % M + M) % M;
            for (int jm = 0; jm < N; ++jm) {
                const int jp = ((jn - jm + c) % N + N) % N;
                const double* Frow = F + idx3(lm, jm, 0, N);
                const double* Prow = P + idx3(lp, jp, 0, N);
                for (int im = 0; im < N; ++im) {
                    const int ip = ((in - im + c) % N + N) % N;
                    acc += Frow[im] * Prow[ip];
                }
            }
        }
        out[q] = acc / (double)L;
    }
}

static double wrapped_normal(double d, double s) {
    /* d reduced to [-pi, pi); images |m| <= 4 */
    d = fmod(d + M_PI, 2.0 * M_PI);
    if (d < 0) d += 2.0 * M_PI;
    d -= M_PI;
    double acc = 0.0;
    for (int m = -4; m <= 4; ++m) {
        const double e = d + 2.0 * M_PI * m;
        acc += exp(-e * e / (2.0 * s * s));
    }
    return acc / (s * sqrt(2.0 * M_PI));
}

/* Kernel value at translation (vx, vy) (one lattice image, no periodisation)
 * and angle t. */
static double kernel_eval(int kind, const double* p, double vx, double vy, double t) {
    if (kind == 0) {
        const double s = p[0];
        const double g = exp(-(vx * vx + vy * vy) / (2.0 * s * s)) / (2.0 * M_PI * s * s);
        return g * 2.0 * M_PI * wrapped_normal(t - p[2], p[1]);
    } else if (kind == 2) {
        /* rho of Eq. gbS0 shifted by p[1] in the rotations, variance p[0]:
         * exp(-(|v|^2 + phi^2) / (2 sigma^2)) with (v, phi) = log(x, R_phi)^v.
         * Half-angle form: V(phi) = (2 sin(phi/2)/phi) R_{phi/2}, so
         * |v| = |x| (phi/2) / sin(phi/2). */
        double phi = fmod(t - p[1] + M_PI, 2.0 * M_PI);
        if (phi < 0) phi += 2.0 * M_PI;
        phi -= M_PI;
        if (phi == -M_PI) phi = M_PI;
        const double h = 0.5 * phi;
        const double a = (h == 0.0) ? 1.0 : h / sin(h);
        const double r2 = a * a * (vx * vx + vy * vy);
        return exp(-(r2 + phi * phi) / (2.0 * p[0]));
    } else {
        const double s1 = p[0], s2 = p[1];
        const double g = exp(-vx * vx / (2.0 * s1 * s1) - vy * vy / (2.0 * s2 * s2)) /
                         (2.0 * M_PI * s1 * s2);
        return g * 2.0 * M_PI * wrapped_normal(t - p[3], p[2]);
    }
}

void se2_group_quadrature(const double* F, int N, int M, int kind, const double* params,
                          int images, double* out) {
    const long L = (long)N * N * M;
    for (int ln = 0; ln < M; ++ln) {
        const double th = 2.0 * M_PI * ln / M;
        for (int jn = 0; jn < N; ++jn) {
            const double xy = -0.5 + (double)jn / N;
            for (int in = 0; in < N; ++in) {
                const double xx = -0.5 + (double)in / N;
                double acc = 0.0;
                for (int lm = 0; lm < M; ++lm) {
                    const double al = 2.0 * M_PI * lm / M;
                    const double ca = cos(al), sa = sin(al);
                    for (int jm = 0; jm < N; ++jm) {
                        const double yy = -0.5 + (double)jm / N;
                        for (int im = 0; im < N; ++im) {
                            const double f = F[idx3(lm, jm, im, N)];
                            if (f == 0.0) continue;
                            const double yx = -0.5 + (double)im / N;
                            double k = 0.0;
                            for (int a = -images; a <= images; ++a)
                                for (int b = -images; b <= images; ++b) {
                                    /* d = x - y - l; kernel at S^{-1} d, S = R_alpha */
                                    const double dx = xx - yx - a, dy = xy - yy - b;
                                    const double rx = ca * dx + sa * dy;
                                    const double ry = -sa * dx + ca * dy;
                                    k += kernel_eval(kind, params, rx, ry, th - al);
                                }
                            acc += f * k;
                        }
                    }
                }
                out[idx3(ln, jn, in, N)] = acc / (double)L;
            }
        }
    }
}
