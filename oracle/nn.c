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
#include <stdlib.h>

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

/* Streaming form of the same scan for data sets too large to hold: the data
 * points are produced chunk by chunk by the C copy of the input generator
 * (dd_inputs/gen.c, linked into this library), mapped with the given
 * C^{1/2} and C^{-1/2} (row-major 6x6) and the 1/sqrt(2) of the map, and
 * compared with every query.  Returns the nearest index and its squared
 * mapped distance per query. */
void ddi_make_dataset(int law, double lo, double hi, double noise_std, double beta, const double *C,
                      uint64_t seed, int64_t start, int64_t n, float *out);

void oracle_nn_stream(int law, double lo, double hi, double noise_std, double beta, const double *C,
                      uint64_t seed, int64_t N, const double *Ch, const double *Cmh, const double *zq, int64_t m,
                      int64_t *i1, double *d1)
{
    const int64_t chunk = 1 << 20;
    float *raw = (float *)malloc((size_t)chunk * 12 * sizeof(float));
    double *z = (double *)malloc((size_t)chunk * 12 * sizeof(double));
    const double r2 = 0.70710678118654752440;
    for (int64_t q = 0; q < m; ++q) {
        i1[q] = -1;
        d1[q] = INFINITY;
    }
    for (int64_t c0 = 0; c0 < N; c0 += chunk) {
        const int64_t n = (N - c0 < chunk) ? N - c0 : chunk;
        ddi_make_dataset(law, lo, hi, noise_std, beta, C, seed, c0, n, raw);
#pragma omp parallel for schedule(static)
        for (int64_t j = 0; j < n; ++j) {
            for (int a = 0; a < 6; ++a) {
                double e = 0.0, g = 0.0;
                for (int b = 0; b < 6; ++b) {
                    e += Ch[6 * a + b] * (double)raw[j * 12 + b];
                    g += Cmh[6 * a + b] * (double)raw[j * 12 + 6 + b];
                }
                z[j * 12 + a] = e * r2;
                z[j * 12 + 6 + a] = g * r2;
            }
        }
#pragma omp parallel for schedule(dynamic, 1)
        for (int64_t q = 0; q < m; ++q) {
            const double *x = zq + q * 12;
            double b1 = d1[q];
            int64_t j1 = i1[q];
            for (int64_t j = 0; j < n; ++j) {
                const double *y = z + j * 12;
                double s = 0.0;
                for (int k = 0; k < 12; ++k) {
                    double t = y[k] - x[k];
                    s += t * t;
                }
                if (s < b1) {
                    b1 = s;
                    j1 = c0 + j;
                }
            }
            d1[q] = b1;
            i1[q] = j1;
        }
    }
    free(raw);
    free(z);
}
