/*
 * oracle/prior.c -- plain FP64 reference for the qGGMRF prior of Eq. 5.
 *
 * TEST INFRASTRUCTURE ONLY (see radon.c).
 *
 * The paper defers the prior's form to its references (Sec. 2); the reading used
 * here is the q-generalised Gaussian MRF potential
 *     rho(D) = |D/sigma|^q / (1 + |D/(c sigma)|^(q-p)),
 * with derivative
 *     rho'(D) = (D/sigma^2) |D/sigma|^(q-2) (q + p u) / (1 + u)^2,  u = |D/(c sigma)|^(q-p),
 * and Phi(x) = sum over unordered neighbour pairs {j,k} of b_jk rho(x_j - x_k).
 * Neighbours are the 26 voxels of the 3x3x3 cube around j (Sec. 2.4); the weight of
 * an offset is proportional to 1/|offset| and the 26 weights sum to 1.  Neighbours
 * outside the volume are dropped (free boundary), so a single slice keeps only its
 * 8 in-plane neighbours with the same weights.
 */
#include <math.h>
#include <stddef.h>

static double rho(double d, double p, double q, double c, double sigma)
{
    double a = fabs(d) / sigma;
    double u = pow(fabs(d) / (c * sigma), q - p);
    return pow(a, q) / (1.0 + u);
}

static double drho(double d, double p, double q, double c, double sigma)
{
    if (d == 0.0) return 0.0;
    double a = fabs(d) / sigma;
    double u = pow(fabs(d) / (c * sigma), q - p);
    return (d / (sigma * sigma)) * pow(a, q - 2.0) * (q + p * u) / ((1.0 + u) * (1.0 + u));
}

double orc_rho(double d, double p, double q, double c, double sigma) { return rho(d, p, q, c, sigma); }
double orc_drho(double d, double p, double q, double c, double sigma) { return drho(d, p, q, c, sigma); }

/* Weight of neighbour offset (dz, dy, dx) in {-1,0,1}^3 \ {0}. */
double orc_neighbour_weight(int dz, int dy, int dx)
{
    double total = 6.0 / 1.0 + 12.0 / sqrt(2.0) + 8.0 / sqrt(3.0);
    int n2 = dz * dz + dy * dy + dx * dx;
    if (n2 == 0) return 0.0;
    return (1.0 / sqrt((double)n2)) / total;
}

/*
 * Volume x[(z*N + r)*N + c], S slices.  grad (may be NULL) receives
 * lambda * dPhi/dx_j; *phi (may be NULL) receives lambda * Phi(x).
 */
void orc_prior(const double *x, int S, int N, double p, double q, double c, double sigma,
               double lambda, double *grad, double *phi)
{
    double phisum = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : phisum)
    for (int z = 0; z < S; ++z) {
        for (int r = 0; r < N; ++r) {
            for (int col = 0; col < N; ++col) {
                size_t j = ((size_t)z * N + r) * N + col;
                double g = 0.0;
                for (int dz = -1; dz <= 1; ++dz) {
                    for (int dy = -1; dy <= 1; ++dy) {
                        for (int dx = -1; dx <= 1; ++dx) {
                            if (dz == 0 && dy == 0 && dx == 0) continue;
                            int z2 = z + dz, r2 = r + dy, c2 = col + dx;
                            if (z2 < 0 || z2 >= S || r2 < 0 || r2 >= N || c2 < 0 || c2 >= N) continue;
                            double b = orc_neighbour_weight(dz, dy, dx);
                            double d = x[j] - x[((size_t)z2 * N + r2) * N + c2];
                            g += b * drho(d, p, q, c, sigma);
                            /* count each unordered pair once: the lexicographically larger offset */
                            int fwd = (dz > 0) || (dz == 0 && dy > 0) || (dz == 0 && dy == 0 && dx > 0);
                            if (fwd) phisum += b * rho(d, p, q, c, sigma);
                        }
                    }
                }
                if (grad) grad[j] = lambda * g;
            }
        }
    }
    if (phi) *phi = lambda * phisum;
}
