/* Exact nearest-neighbour projection P_D of the DD method, Eq. (7), as the
 * plain linear search the paper's introduction describes: every query is
 * compared with every data point.  FP64 throughout, distances as a plain sum
 * of squared coordinate differences in the Euclidean map of Sec. 3.2.
 *
 * TEST INFRASTRUCTURE ONLY (part of the oracle); never linked into the
 * product library.  Compiled with -ffp-contract=off so that the sums are the
 * same on every host.
 *
 * Ties: the lowest data index wins (strict < while scanning j upwards); the
 * paper does not say.
 */
#include <math.h>
#include <stdint.h>

/* For each query row q of zq [m x dim]: i1/d1 = nearest data row of zd
 * [n x dim] and its squared distance; i2/d2 = second nearest (for the
 * moving-query radius of Eq. 14).  d2 = +inf, i2 = -1 when n < 2. */
void oracle_nn_top2(const double *zd, int64_t n, const double *zq, int64_t m,
                    int dim, int64_t *i1, double *d1, int64_t *i2, double *d2)
{
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t q = 0; q < m; ++q) {
        const double *x = zq + q * dim;
        double b1 = INFINITY, b2 = INFINITY;
        int64_t j1 = -1, j2 = -1;
        for (int64_t j = 0; j < n; ++j) {
            const double *y = zd + j * dim;
            double s = 0.0;
            for (int k = 0; k < dim; ++k) {
                double t = y[k] - x[k];
                s += t * t;
            }
            if (s < b1) {
                b2 = b1; j2 = j1;
                b1 = s; j1 = j;
            } else if (s < b2) {
                b2 = s; j2 = j;
            }
        }
        i1[q] = j1; d1[q] = b1;
        i2[q] = j2; d2[q] = b2;
    }
}

/* Number of OpenMP threads the scan above uses (reported with timings). */
int oracle_nn_threads(void)
{
    int t = 1;
#pragma omp parallel
    {
#pragma omp single
        {
#ifdef _OPENMP
            extern int omp_get_num_threads(void);
            t = omp_get_num_threads();
#endif
        }
    }
    return t;
}
