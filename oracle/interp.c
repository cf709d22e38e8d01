/*
 * oracle/interp.c -- plain FP64 reference for the warm-start and level-transfer
 * steps: the ramp filter of Sec. 2.2 (Eqs. 12-13), the Lanczos-3 level upsampler of
 * Sec. 2.3 (Eqs. 16-17) and the projection subsampling of Sec. 2.3.
 *
 * TEST INFRASTRUCTURE ONLY (see radon.c).
 */
#include <math.h>
#include <stddef.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/*
 * Ramp filter, Eq. 12 with the band-limited spatial kernel whose spectrum is |omega|
 * (Eq. 13) up to the detector Nyquist frequency, sampled at unit pitch:
 *   h[0] = 1/4, h[n] = -1/(pi^2 n^2) for odd n, h[n] = 0 for even n != 0.
 * Each projection row is convolved linearly (no wrap-around).
 */
void orc_ramp_filter(const double *g, int na, int nd, double *gt)
{
#pragma omp parallel for schedule(static)
    for (int a = 0; a < na; ++a) {
        const double *ga = g + (size_t)a * nd;
        double *ta = gt + (size_t)a * nd;
        for (int m = 0; m < nd; ++m) {
            double acc = 0.0;
            for (int m2 = 0; m2 < nd; ++m2) {
                int n = m - m2;
                double h;
                if (n == 0) h = 0.25;
                else if (n % 2 != 0) h = -1.0 / (M_PI * M_PI * (double)n * (double)n);
                else h = 0.0;
                acc += h * ga[m2];
            }
            ta[m] = acc;
        }
    }
}

/*
 * Lanczos kernel with window a.  The printed Eq. 16 is garbled (it is negative at
 * x = 1/2); the standard windowed sinc is used: L(x) = sinc(x) sinc(x/a) for |x| < a.
 */
double orc_lanczos(double x, int a)
{
    if (x == 0.0) return 1.0;
    if (fabs(x) >= (double)a) return 0.0;
    return (double)a * sin(M_PI * x) * sin(M_PI * x / (double)a) / (M_PI * M_PI * x * x);
}

/*
 * One-dimensional x2 Lanczos-3 upsampling (Eq. 17), centre-aligned: coarse sample i
 * lies on fine sample 2i.  Even fine samples copy the coarse sample; odd fine sample
 * 2i+1 sits half-way between coarse i and i+1 and takes the six taps i-2 .. i+3 with
 * weights L(i + 1/2 - i'), normalised to sum 1.  Samples outside the grid are zero.
 */
static void up1d(const double *in, int n, ptrdiff_t istride, double *out, ptrdiff_t ostride)
{
    double w[6], ws = 0.0;
    for (int t = 0; t < 6; ++t) {
        w[t] = orc_lanczos(2.5 - (double)t, 3); /* tap i-2+t at offset (i+0.5) - (i-2+t) */
        ws += w[t];
    }
    for (int t = 0; t < 6; ++t) w[t] /= ws;
    for (int i = 0; i < n; ++i) {
        out[(2 * i) * ostride] = in[i * istride];
        double acc = 0.0;
        for (int t = 0; t < 6; ++t) {
            int i2 = i - 2 + t;
            if (i2 >= 0 && i2 < n) acc += w[t] * in[i2 * istride];
        }
        out[(2 * i + 1) * ostride] = acc;
    }
}

/* Separable x2 upsampling of S slices: in[S][Nc][Nc] -> out[S][2Nc][2Nc]. */
void orc_lanczos_up(const double *in, int S, int Nc, double *out, double *tmp)
{
    int Nf = 2 * Nc;
    for (int z = 0; z < S; ++z) {
        const double *iz = in + (size_t)z * Nc * Nc;
        double *tz = tmp + (size_t)z * Nc * Nf; /* [Nc rows][Nf cols] */
        double *oz = out + (size_t)z * Nf * Nf;
        for (int r = 0; r < Nc; ++r) up1d(iz + (size_t)r * Nc, Nc, 1, tz + (size_t)r * Nf, 1);
        for (int c = 0; c < Nf; ++c) up1d(tz + c, Nc, Nf, oz + c, Nf);
    }
}

/*
 * Coarse projections for a grid of pitch f (Sec. 2.3, "subsampling"): keep every f-th
 * bin, aligned on the centre bin n_d/2, and divide by f because line integrals are
 * measured in coarse-pixel units.  All angles are kept.
 */
void orc_downsample_sino(const double *g, int S, int na, int nd, int f, double *out)
{
    int ndc = nd / f;
    for (int z = 0; z < S; ++z)
        for (int a = 0; a < na; ++a)
            for (int m = 0; m < ndc; ++m)
                out[((size_t)z * na + a) * ndc + m] = g[((size_t)z * na + a) * nd + (size_t)f * m] / (double)f;
}
