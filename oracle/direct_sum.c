/*
 * FP64 direct sums for the MFS oracle.  TEST INFRASTRUCTURE ONLY: this file is
 * compiled into the oracle's helper library and is called by the oracle's
 * Python code; the product library never links it and shares no code with it.
 *
 * Both functions evaluate, for every target x_i, the sum over sources y_j of
 * the fundamental solution times the source strength, restricted to pairs in
 * the same group (suspension), and optionally skipping pairs in the same body:
 *
 *   Laplace (Sec. 2.1, Eq. Skk):   u_i = sum_j alpha_j / (4 pi |x_i - y_j|)
 *   Stokes  (Sec. 2.2, Eq. stokeslet, Eq. repS):
 *       u_i = sum_j 1/(8 pi mu r) (I + r r^T / r^2) lambda_j,   r = x_i - y_j
 *
 * Plain double loops, FP64 throughout, one OpenMP thread per block of targets.
 */
#include <math.h>
#include <stddef.h>
#include <stdlib.h>

static const double PI_ORACLE = 3.14159265358979323846;

void oracle_laplace_sum(long nt, const double *x, const int *tgroup, const int *tbody,
                        long ns, const double *y, const int *sgroup, const int *sbody,
                        const double *alpha, int include_self, double *u)
{
    const double c = 1.0 / (4.0 * PI_ORACLE);
#pragma omp parallel for schedule(dynamic, 64)
    for (long i = 0; i < nt; ++i) {
        double acc = 0.0;
        for (long j = 0; j < ns; ++j) {
            if (sgroup[j] != tgroup[i]) continue;
            if (!include_self && sbody[j] == tbody[i]) continue;
            double rx = x[3 * i + 0] - y[3 * j + 0];
            double ry = x[3 * i + 1] - y[3 * j + 1];
            double rz = x[3 * i + 2] - y[3 * j + 2];
            double r = sqrt(rx * rx + ry * ry + rz * rz);
            acc += alpha[j] / r;
        }
        u[i] = c * acc;
    }
}

void oracle_stokeslet_sum(long nt, const double *x, const int *tgroup, const int *tbody,
                          long ns, const double *y, const int *sgroup, const int *sbody,
                          const double *lam, int include_self, double mu, double *u)
{
    const double c = 1.0 / (8.0 * PI_ORACLE * mu);
#pragma omp parallel for schedule(dynamic, 64)
    for (long i = 0; i < nt; ++i) {
        double ax = 0.0, ay = 0.0, az = 0.0;
        for (long j = 0; j < ns; ++j) {
            if (sgroup[j] != tgroup[i]) continue;
            if (!include_self && sbody[j] == tbody[i]) continue;
            double rx = x[3 * i + 0] - y[3 * j + 0];
            double ry = x[3 * i + 1] - y[3 * j + 1];
            double rz = x[3 * i + 2] - y[3 * j + 2];
            double r2 = rx * rx + ry * ry + rz * rz;
            double r = sqrt(r2);
            double lx = lam[3 * j + 0], ly = lam[3 * j + 1], lz = lam[3 * j + 2];
            double rdotl = rx * lx + ry * ly + rz * lz;
            /* (I + r r^T / r^2) lambda / r */
            ax += (lx + rx * rdotl / r2) / r;
            ay += (ly + ry * rdotl / r2) / r;
            az += (lz + rz * rdotl / r2) / r;
        }
        u[3 * i + 0] = c * ax;
        u[3 * i + 1] = c * ay;
        u[3 * i + 2] = c * az;
    }
}

/*
 * Gradient of w^T G(x_i - y_j) mu_j with respect to r = x_i - y_j, summed into
 * per-body gradients of the centres: targets move with their body centre
 * (dr/dc_target = +I), sources with theirs (dr/dc_source = -I).  Only pairs
 * in different bodies of the same group contribute.  Used by the oracle's
 * adjoint.  d/dr_c of [ (w.mu)/r + (w.r)(r.mu)/r^3 ] / (8 pi mu_visc):
 *   -(w.mu) r_c / r^3 + [w_c (r.mu) + mu_c (w.r)] / r^3 - 3 (w.r)(r.mu) r_c / r^5
 */
void oracle_stokeslet_center_grad(long nt, const double *x, const int *tgroup, const int *tbody,
                                  const double *w, long ns, const double *y, const int *sgroup,
                                  const int *sbody, const double *muv, double visc, int nbody,
                                  double *grad /* nbody x 3, accumulated */)
{
    const double c = 1.0 / (8.0 * PI_ORACLE * visc);
#pragma omp parallel
    {
        double *g = (double *)calloc((size_t)3 * nbody, sizeof(double));
#pragma omp for schedule(dynamic, 64)
        for (long i = 0; i < nt; ++i) {
            double gx = 0.0, gy = 0.0, gz = 0.0;
            double wx = w[3 * i + 0], wy = w[3 * i + 1], wz = w[3 * i + 2];
            for (long j = 0; j < ns; ++j) {
                if (sgroup[j] != tgroup[i]) continue;
                if (sbody[j] == tbody[i]) continue;
                double rx = x[3 * i + 0] - y[3 * j + 0];
                double ry = x[3 * i + 1] - y[3 * j + 1];
                double rz = x[3 * i + 2] - y[3 * j + 2];
                double r2 = rx * rx + ry * ry + rz * rz;
                double r = sqrt(r2);
                double r3 = r2 * r, r5 = r3 * r2;
                double mx = muv[3 * j + 0], my = muv[3 * j + 1], mz = muv[3 * j + 2];
                double wm = wx * mx + wy * my + wz * mz;
                double wr = wx * rx + wy * ry + wz * rz;
                double rm = rx * mx + ry * my + rz * mz;
                double dx = -wm * rx / r3 + (wx * rm + mx * wr) / r3 - 3.0 * wr * rm * rx / r5;
                double dy = -wm * ry / r3 + (wy * rm + my * wr) / r3 - 3.0 * wr * rm * ry / r5;
                double dz = -wm * rz / r3 + (wz * rm + mz * wr) / r3 - 3.0 * wr * rm * rz / r5;
                gx += dx; gy += dy; gz += dz;
                /* the source body moves the other way */
                g[3 * sbody[j] + 0] -= c * dx;
                g[3 * sbody[j] + 1] -= c * dy;
                g[3 * sbody[j] + 2] -= c * dz;
            }
            g[3 * tbody[i] + 0] += c * gx;
            g[3 * tbody[i] + 1] += c * gy;
            g[3 * tbody[i] + 2] += c * gz;
        }
#pragma omp critical
        for (long q = 0; q < 3 * (long)nbody; ++q) grad[q] += g[q];
        free(g);
    }
}
