// Data-derived metric of Sec. 3.1: principal component analysis of the
// 12-d data set.  The six principal component vectors (eigenvectors of the
// covariance with the six largest eigenvalues) are the columns of A (12 x 6);
// with A_eps its upper and A_sig its lower 6 x 6 block the metric is
// C = sym(A_sig A_eps^{-1}), which is C itself for data on a linear law
// sig = C eps (the paper writes the product with the components as rows).
//
// Device: column sums, then the 78 distinct centred second moments, in FP64
// with a fixed assignment of points to threads and fixed-order reductions
// (the same result on every run).  Host: the 12 x 12 eigenproblem and the
// 6 x 6 solve.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "dd_internal.cuh"

namespace {

constexpr int64_t kPcaChunk = (int64_t)1 << 24;   // points per pass (host data is copied chunk by chunk)
constexpr int kMomGroups = 3;                      // point groups of the 78 moment threads

// per block: sums of the 12 columns; thread t < 252 takes column t % 12 of
// every 21st point of the block's share
__global__ void __launch_bounds__(256) k_col_sums(const float *__restrict__ x, int64_t n,
                                                  double *__restrict__ part) {
    __shared__ double sh[256];
    const int t = threadIdx.x, col = t % 12, grp = t / 12;
    double acc = 0.0;
    if (t < 252)
        for (int64_t p = (int64_t)blockIdx.x * 21 + grp; p < n; p += (int64_t)gridDim.x * 21) acc += x[p * 12 + col];
    sh[t] = acc;
    __syncthreads();
    if (t < 12) {
        double s = 0.0;
        for (int g = 0; g < 21; ++g) s += sh[g * 12 + t];
        part[blockIdx.x * 12 + t] = s;
    }
}

// per block: the 78 moments sum (x_r - m_r)(x_c - m_c), r <= c; thread
// t < 234 takes entry t % 78 of every 3rd point of the block's share
__global__ void __launch_bounds__(256) k_moments(const float *__restrict__ x, int64_t n, const double *__restrict__ mean,
                                                 double *__restrict__ part) {
    __shared__ double sh[256];
    const int t = threadIdx.x, e = t % 78, grp = t / 78;
    int r = 0, c = e;
    while (c >= 12 - r) {        // entry e -> (r, c), c >= r, row-major upper triangle
        c -= 12 - r;
        ++r;
    }
    c += r;
    double acc = 0.0;
    if (t < 78 * kMomGroups) {
        const double mr = mean[r], mc = mean[c];
        for (int64_t p = (int64_t)blockIdx.x * kMomGroups + grp; p < n; p += (int64_t)gridDim.x * kMomGroups)
            acc = fma((double)x[p * 12 + r] - mr, (double)x[p * 12 + c] - mc, acc);
    }
    sh[t] = acc;
    __syncthreads();
    if (t < 78) {
        double s = 0.0;
        for (int g = 0; g < kMomGroups; ++g) s += sh[g * 78 + t];
        part[blockIdx.x * 78 + t] = s;
    }
}

}  // namespace

extern "C" dd_status dd_pca_metric(dd_ctx *ctx, const float *eps_sig, int64_t N, double *C_out) {
    if (!ctx) return DD_ERR_ARG;
    if (!eps_sig || !C_out || N < 13) return dd_fail(ctx, DD_ERR_ARG, "dd_pca_metric: bad argument (N >= 13)");
    DD_TRY_CUDA(ctx, cudaSetDevice(ctx->device));
    cudaStream_t s = ctx->stream;
    const bool dev = dd_is_device_ptr(eps_sig);
    const int grid = std::max(1, ctx->n_sm * 4);
    const int64_t chunk = std::min(N, kPcaChunk);
    const size_t b_x = dev ? 0 : ((size_t)chunk * 48 + 255) / 256 * 256, b_p = (size_t)grid * 78 * 8;
    void *w = nullptr;
    DD_TRY(dd_workspace(ctx, WS_MISC, b_x + b_p + 256, &w));
    float *xbuf = (float *)w;
    double *part = (double *)((char *)w + b_x);
    double *mean_dev = part + (size_t)grid * 78;       // 12 doubles after the partials (within the 256 spare bytes)
    std::vector<double> hp((size_t)grid * 78);
    auto chunk_ptr = [&](int64_t c0, int64_t n) -> const float * {
        if (dev) return eps_sig + c0 * 12;
        cudaMemcpyAsync(xbuf, eps_sig + c0 * 12, (size_t)n * 48, cudaMemcpyHostToDevice, s);
        return xbuf;
    };
    // column means
    double sum[12] = {0};
    for (int64_t c0 = 0; c0 < N; c0 += chunk) {
        const int64_t n = std::min(chunk, N - c0);
        const float *x = chunk_ptr(c0, n);
        ctx->launches++;
        k_col_sums<<<grid, 256, 0, s>>>(x, n, part);
        DD_TRY_CUDA(ctx, cudaGetLastError());
        DD_TRY_CUDA(ctx, cudaMemcpyAsync(hp.data(), part, (size_t)grid * 12 * 8, cudaMemcpyDeviceToHost, s));
        DD_TRY_CUDA(ctx, cudaStreamSynchronize(s));
        for (int b = 0; b < grid; ++b)
            for (int k = 0; k < 12; ++k) sum[k] += hp[(size_t)b * 12 + k];
    }
    double mean[12];
    for (int k = 0; k < 12; ++k) mean[k] = sum[k] / (double)N;
    DD_TRY_CUDA(ctx, cudaMemcpyAsync(mean_dev, mean, sizeof(mean), cudaMemcpyHostToDevice, s));
    // centred second moments
    double mom[78] = {0};
    for (int64_t c0 = 0; c0 < N; c0 += chunk) {
        const int64_t n = std::min(chunk, N - c0);
        const float *x = chunk_ptr(c0, n);
        ctx->launches++;
        k_moments<<<grid, 256, 0, s>>>(x, n, mean_dev, part);
        DD_TRY_CUDA(ctx, cudaGetLastError());
        DD_TRY_CUDA(ctx, cudaMemcpyAsync(hp.data(), part, (size_t)grid * 78 * 8, cudaMemcpyDeviceToHost, s));
        DD_TRY_CUDA(ctx, cudaStreamSynchronize(s));
        for (int b = 0; b < grid; ++b)
            for (int k = 0; k < 78; ++k) mom[k] += hp[(size_t)b * 78 + k];
    }
    double S[144], V[144], ev[12];
    for (int r = 0, e = 0; r < 12; ++r)
        for (int c = r; c < 12; ++c, ++e) S[r * 12 + c] = S[c * 12 + r] = mom[e] / (double)N;
    for (int k = 0; k < 144; ++k)
        if (!std::isfinite(S[k])) return dd_fail(ctx, DD_ERR_ARG, "dd_pca_metric: non-finite data");
    dd_sym_eig(12, S, V, ev);
    int order[12];
    for (int k = 0; k < 12; ++k) order[k] = k;
    std::sort(order, order + 12, [&](int a, int b) { return ev[a] > ev[b]; });
    // A = the six leading eigenvectors as columns; C = A_sig A_eps^{-1}:
    // solve A_eps^T X = A_sig^T (Gaussian elimination, partial pivoting), C = X^T
    double At[6][12];                       // At[k] = eigenvector k (12 entries)
    for (int k = 0; k < 6; ++k)
        for (int i = 0; i < 12; ++i) At[k][i] = V[i * 12 + order[k]];
    double Mx[6][12];                       // [A_eps^T | A_sig^T], row k = component k
    for (int k = 0; k < 6; ++k)
        for (int i = 0; i < 12; ++i) Mx[k][i] = At[k][i];
    for (int col = 0; col < 6; ++col) {
        int piv = col;
        for (int r = col + 1; r < 6; ++r)
            if (std::fabs(Mx[r][col]) > std::fabs(Mx[piv][col])) piv = r;
        if (!(std::fabs(Mx[piv][col]) > 1e-12))
            return dd_fail(ctx, DD_ERR_NOT_SPD, "dd_pca_metric: principal strains degenerate (A_eps singular)");
        if (piv != col)
            for (int i = 0; i < 12; ++i) std::swap(Mx[piv][i], Mx[col][i]);
        for (int r = 0; r < 6; ++r) {
            if (r == col) continue;
            const double f = Mx[r][col] / Mx[col][col];
            for (int i = col; i < 12; ++i) Mx[r][i] -= f * Mx[col][i];
        }
    }
    double X[6][6];                         // X = A_eps^{-T} A_sig^T
    for (int r = 0; r < 6; ++r)
        for (int c = 0; c < 6; ++c) X[r][c] = Mx[r][6 + c] / Mx[r][r];
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) C_out[6 * i + j] = 0.5 * (X[j][i] + X[i][j]);   // sym(X^T)
    MetricMaps M;
    if (!dd_metric_maps(C_out, &M)) return dd_fail(ctx, DD_ERR_NOT_SPD, "dd_pca_metric: metric not positive definite");
    return DD_OK;
}
