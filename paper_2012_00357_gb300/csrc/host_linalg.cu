// Host-side 6x6 linear algebra for the metric of Eq. (3): symmetric
// eigen-decomposition by cyclic Jacobi rotations (Golub & Van Loan, Matrix
// Computations, Sec. 8.5), from which C^{1/2}, C^{-1/2} and C^{-1} follow.
#include <cmath>

#include "dd_internal.cuh"

namespace {

// Cyclic Jacobi on the n x n symmetric A (row-major, stride n, destroyed):
// V (row-major) holds the eigenvectors as columns, w the eigenvalues.
void jacobi(int n, double *A, double *V, double *w) {
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) V[i * n + j] = (i == j) ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0, diag = 0.0;
        for (int p = 0; p < n; ++p) {
            diag += A[p * n + p] * A[p * n + p];
            for (int q = p + 1; q < n; ++q) off += A[p * n + q] * A[p * n + q];
        }
        if (off <= 1e-34 * diag) break;
        for (int p = 0; p < n; ++p) {
            for (int q = p + 1; q < n; ++q) {
                double apq = A[p * n + q];
                if (apq == 0.0) continue;
                double theta = (A[q * n + q] - A[p * n + p]) / (2.0 * apq);
                double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < n; ++k) {          // A <- A J
                    double akp = A[k * n + p], akq = A[k * n + q];
                    A[k * n + p] = c * akp - s * akq;
                    A[k * n + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {          // A <- J^T A
                    double apk = A[p * n + k], aqk = A[q * n + k];
                    A[p * n + k] = c * apk - s * aqk;
                    A[q * n + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < n; ++k) {          // V <- V J
                    double vkp = V[k * n + p], vkq = V[k * n + q];
                    V[k * n + p] = c * vkp - s * vkq;
                    V[k * n + q] = s * vkp + c * vkq;
                }
            }
        }
    }
    for (int i = 0; i < n; ++i) w[i] = A[i * n + i];
}

void jacobi6(double A[6][6], double V[6][6], double w[6]) { jacobi(6, &A[0][0], &V[0][0], w); }

void spectral(const double V[6][6], const double f[6], double *out) {
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) {
            double s = 0.0;
            for (int k = 0; k < 6; ++k) s += V[i][k] * f[k] * V[j][k];
            out[6 * i + j] = s;
        }
}

}  // namespace

void dd_sym_eig(int n, double *A, double *V, double *w) { jacobi(n, A, V, w); }

bool dd_metric_maps(const double *C, MetricMaps *M) {
    double amax = 0.0;
    for (int i = 0; i < 36; ++i) {
        if (!std::isfinite(C[i])) return false;
        amax = std::fmax(amax, std::fabs(C[i]));
    }
    if (amax == 0.0) return false;
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j)
            if (std::fabs(C[6 * i + j] - C[6 * j + i]) > 1e-12 * amax) return false;
    double A[6][6], V[6][6], w[6];
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) A[i][j] = 0.5 * (C[6 * i + j] + C[6 * j + i]);
    jacobi6(A, V, w);
    double wmax = 0.0, wmin = INFINITY;
    for (int i = 0; i < 6; ++i) {
        wmax = std::fmax(wmax, w[i]);
        wmin = std::fmin(wmin, w[i]);
    }
    if (!(wmin > 1e-13 * wmax)) return false;
    double fh[6], fmh[6], finv[6];
    for (int i = 0; i < 6; ++i) {
        fh[i] = std::sqrt(w[i]);
        fmh[i] = 1.0 / fh[i];
        finv[i] = 1.0 / w[i];
    }
    for (int i = 0; i < 36; ++i) M->C[i] = 0.5 * (C[i] + C[6 * (i % 6) + i / 6]);
    spectral(V, fh, M->Ch);
    spectral(V, fmh, M->Cmh);
    spectral(V, finv, M->Cinv);
    for (int k = 0; k < 12; ++k) M->mu[k] = 0.0;
    return true;
}
