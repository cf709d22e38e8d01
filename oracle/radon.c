/*
 * oracle/radon.c -- plain FP64 reference for the parallel-beam operators.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing here is part of the product path: only the
 * test suite, the package smoke check and the CPU-baseline leg of the benchmark
 * may load this library.  It shares no code with the CUDA implementation.
 *
 * Geometry (the paper leaves it open; this is the reading used throughout):
 *   - an N x N slice, pixel pitch 1, pixel (row r, col c) sits at
 *     x = c - N/2, y = r - N/2 (integer division);
 *   - n_d detector bins (n_d even), bin m sits at s_m = m - n_d/2;
 *   - angle theta_a has direction e_a = (cos theta_a, sin theta_a);
 *   - radial frequencies k/n_d with k = -(n_d/2-1) .. n_d/2-1: the Nyquist bin is
 *     dropped so that the forward operator is real and A^T A is exactly Toeplitz.
 *
 * The forward operator is Eq. 3 (type-2 non-uniform DFT onto the polar grid, then
 * the 1D inverse DFT along each ray).  Summing the geometric series over k gives
 * the closed form used here:
 *     (A x)(a, m) = (1/n_d) sum_j x_j D(s_m - e_a . x_j),
 *     D(t) = sum_k exp(2 pi i k t / n_d) = sin(pi (n_d-1) t / n_d) / sin(pi t / n_d).
 * The adjoint (Eq. 4) is its transpose.  The point-spread kernel of Sec. 2.1
 * (the adjoint NUFFT applied to the all-ones polar data) is
 *     K(d) = (1/n_d) sum_a D(e_a . d),  d in [-(N-1), N-1]^2,
 * and A^T A x = K (*) x (Eq. 8) is evaluated here by the direct O(N^4) sum.
 */
#include <math.h>
#include <stddef.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* Dirichlet kernel D(t) for even n_d (period n_d). */
double orc_dirichlet(double t, int nd)
{
    double e = t - (double)nd * nearbyint(t / (double)nd);
    double s = sin(M_PI * e / (double)nd);
    if (s == 0.0) return (double)(nd - 1);
    return sin(M_PI * (double)(nd - 1) * e / (double)nd) / s;
}

/* g[a*nd + m] = (A x)(a, m) for one slice x[r*N + c]. */
void orc_forward(const double *x, int N, const double *theta, int na, int nd, double *g)
{
    int h = N / 2;
#pragma omp parallel for schedule(static)
    for (int a = 0; a < na; ++a) {
        double ca = cos(theta[a]), sa = sin(theta[a]);
        double *ga = g + (size_t)a * nd;
        for (int m = 0; m < nd; ++m) ga[m] = 0.0;
        for (int r = 0; r < N; ++r) {
            for (int c = 0; c < N; ++c) {
                double v = x[(size_t)r * N + c];
                if (v == 0.0) continue;
                double u = (double)(c - h) * ca + (double)(r - h) * sa;
                for (int m = 0; m < nd; ++m) {
                    double s = (double)m - 0.5 * nd;
                    ga[m] += v * orc_dirichlet(s - u, nd);
                }
            }
        }
        for (int m = 0; m < nd; ++m) ga[m] /= (double)nd;
    }
}

/* x[r*N + c] = (A^T g)(r, c). */
void orc_adjoint(const double *g, int N, const double *theta, int na, int nd, double *x)
{
    int h = N / 2;
#pragma omp parallel for schedule(static)
    for (int r = 0; r < N; ++r) {
        for (int c = 0; c < N; ++c) {
            double acc = 0.0;
            for (int a = 0; a < na; ++a) {
                double u = (double)(c - h) * cos(theta[a]) + (double)(r - h) * sin(theta[a]);
                const double *ga = g + (size_t)a * nd;
                for (int m = 0; m < nd; ++m) {
                    double s = (double)m - 0.5 * nd;
                    acc += ga[m] * orc_dirichlet(s - u, nd);
                }
            }
            x[(size_t)r * N + c] = acc / (double)nd;
        }
    }
}

/* K[(dy + N-1) * (2N-1) + (dx + N-1)] = K(dx, dy) for |dx|, |dy| <= N-1. */
void orc_kernel(int N, const double *theta, int na, int nd, double *K)
{
    int W = 2 * N - 1;
#pragma omp parallel for schedule(static)
    for (int iy = 0; iy < W; ++iy) {
        for (int ix = 0; ix < W; ++ix) {
            double dx = (double)(ix - (N - 1)), dy = (double)(iy - (N - 1));
            double acc = 0.0;
            for (int a = 0; a < na; ++a)
                acc += orc_dirichlet(dx * cos(theta[a]) + dy * sin(theta[a]), nd);
            K[(size_t)iy * W + ix] = acc / (double)nd;
        }
    }
}

/* z_j = sum_i K(x_j - x_i) x_i : the direct (unfactored) Toeplitz product. */
void orc_normal_direct(const double *x, int N, const double *K, double *z)
{
    int W = 2 * N - 1;
#pragma omp parallel for schedule(static)
    for (int r = 0; r < N; ++r) {
        for (int c = 0; c < N; ++c) {
            double acc = 0.0;
            for (int r2 = 0; r2 < N; ++r2) {
                const double *Krow = K + (size_t)(r - r2 + N - 1) * W + (N - 1) + c;
                const double *xrow = x + (size_t)r2 * N;
                for (int c2 = 0; c2 < N; ++c2) acc += Krow[-c2] * xrow[c2];
            }
            z[(size_t)r * N + c] = acc;
        }
    }
}

/* Single outputs of the same definitions, for sampled checks on large grids. */
double orc_normal_point(const double *x, int N, const double *K, int r, int c)
{
    int W = 2 * N - 1;
    double acc = 0.0;
    for (int r2 = 0; r2 < N; ++r2) {
        const double *Krow = K + (size_t)(r - r2 + N - 1) * W + (N - 1) + c;
        const double *xrow = x + (size_t)r2 * N;
        for (int c2 = 0; c2 < N; ++c2) acc += Krow[-c2] * xrow[c2];
    }
    return acc;
}

double orc_adjoint_point(const double *g, int N, const double *theta, int na, int nd, int r, int c)
{
    int h = N / 2;
    double acc = 0.0;
    for (int a = 0; a < na; ++a) {
        double u = (double)(c - h) * cos(theta[a]) + (double)(r - h) * sin(theta[a]);
        const double *ga = g + (size_t)a * nd;
        for (int m = 0; m < nd; ++m) acc += ga[m] * orc_dirichlet((double)m - 0.5 * nd - u, nd);
    }
    return acc / (double)nd;
}

/* (A x)(a, m) of one slice at one angle theta_a and one bin m, by the direct sum. */
double orc_forward_point(const double *x, int N, double theta_a, int nd, int m)
{
    int h = N / 2;
    double ca = cos(theta_a), sa = sin(theta_a), s = (double)m - 0.5 * nd, acc = 0.0;
    for (int r = 0; r < N; ++r)
        for (int c = 0; c < N; ++c) {
            double v = x[(size_t)r * N + c];
            if (v != 0.0) acc += v * orc_dirichlet(s - ((double)(c - h) * ca + (double)(r - h) * sa), nd);
        }
    return acc / (double)nd;
}
