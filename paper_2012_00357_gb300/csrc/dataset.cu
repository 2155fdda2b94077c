// Material data set on the device: load, validate and pre-transform to the
// Euclidean map of Sec. 3.2,
//     z_j = (C^{1/2} eps_j, C^{-1/2} sig_j) / sqrt(2),
// stored centred (minus a fixed sample mean mu) in FP32 with |z_j|^2, so that
// the exact scans can use the expanded distance |z|^2 - 2 z.q with a small
// rounding error.  The (eps, sig) values themselves stay resident for FP64
// rescoring with Eq. (3).
#include <algorithm>
#include <cmath>
#include <cstring>

#include "dd_internal.cuh"

namespace {

__device__ __forceinline__ void map_row(const MetricMaps &M, const float *row, double z[12]) {
    const double r2 = 0.70710678118654752440;
    double s[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) s[k] = (double)row[k];
#pragma unroll
    for (int a = 0; a < 6; ++a) {
        double e = 0.0, g = 0.0;
#pragma unroll
        for (int b = 0; b < 6; ++b) {
            e += M.Ch[6 * a + b] * s[b];
            g += M.Cmh[6 * a + b] * s[6 + b];
        }
        z[a] = e * r2;
        z[6 + a] = g * r2;
    }
}

// Sum of z over the sample points j_i = floor(i N / S), i < S (block partials).
__global__ void k_sample_sum(const float *__restrict__ raw, int64_t N, int64_t S, MetricMaps M,
                             double *__restrict__ part) {
    __shared__ double sh[12][256];
    double acc[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[k] = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < S; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t j = (int64_t)(((__int128)i * N) / S);
        double z[12];
        map_row(M, raw + j * 12, z);
#pragma unroll
        for (int k = 0; k < 12; ++k) acc[k] += z[k];
    }
#pragma unroll
    for (int k = 0; k < 12; ++k) sh[k][threadIdx.x] = acc[k];
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
#pragma unroll
            for (int k = 0; k < 12; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < 12) part[blockIdx.x * 12 + threadIdx.x] = sh[threadIdx.x][0];
}

// z32 = fl32(z - mu), zn = fl32(|z32|^2); padding rows get z = 0, zn = 1e30.
// stats[0] = max |z32_k| bits, stats[1] = max zn bits, stats[2] = non-finite rows.
__global__ void k_transform(const float *__restrict__ raw, int64_t N, int64_t N_pad, MetricMaps M,
                            float *__restrict__ z32, float *__restrict__ zn, unsigned *__restrict__ stats) {
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    unsigned umx = 0, un = 0;     // contributions to the maxima (0 for inactive lanes)
    if (j < N) {
        const float *row = raw + j * 12;
        bool finite = true;
#pragma unroll
        for (int k = 0; k < 12; ++k) finite &= isfinite(row[k]);
        double z[12];
        map_row(M, row, z);
        float mx = 0.f;
        double n2 = 0.0;
        float zr[12];
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            zr[k] = (float)(z[k] - M.mu[k]);
            mx = fmaxf(mx, fabsf(zr[k]));
            n2 += (double)zr[k] * (double)zr[k];
        }
        float4 *dst = reinterpret_cast<float4 *>(z32 + j * 12);
        dst[0] = make_float4(zr[0], zr[1], zr[2], zr[3]);
        dst[1] = make_float4(zr[4], zr[5], zr[6], zr[7]);
        dst[2] = make_float4(zr[8], zr[9], zr[10], zr[11]);
        float n2f = (float)n2;
        zn[j] = n2f;
        if (finite) {
            umx = __float_as_uint(mx);
            un = __float_as_uint(n2f);
        } else {
            atomicAdd(stats + 2, 1u);
        }
    } else if (j < N_pad) {
#pragma unroll
        for (int k = 0; k < 12; ++k) z32[j * 12 + k] = 0.f;
        zn[j] = 1e30f;
    }
    // non-negative floats order like their bit patterns
    for (int o = 16; o > 0; o >>= 1) {
        umx = max(umx, __shfl_xor_sync(0xffffffffu, umx, o));
        un = max(un, __shfl_xor_sync(0xffffffffu, un, o));
    }
    if ((threadIdx.x & 31) == 0 && (umx | un)) {
        atomicMax(stats + 0, umx);
        atomicMax(stats + 1, un);
    }
}

}  // namespace

dd_status dd_transform_dataset(dd_dataset *ds) {
    dd_ctx *ctx = ds->ctx;
    cudaStream_t s = ctx->stream;
    // centre: mean of z over a fixed sample of at most 65536 points
    const int64_t S = std::min<int64_t>(ds->N, 65536);
    const int blocks = (int)std::min<int64_t>(64, (S + 255) / 256);
    void *w = nullptr;
    DD_TRY(dd_workspace(ctx, WS_MISC, (size_t)blocks * 12 * sizeof(double) + 64, &w));
    double *part = reinterpret_cast<double *>(w);
    ctx->launches += 2;
    k_sample_sum<<<blocks, 256, 0, s>>>(ds->raw, ds->N, S, ds->M, part);
    DD_TRY_CUDA(ctx, cudaGetLastError());
    std::vector<double> hp((size_t)blocks * 12);
    DD_TRY_CUDA(ctx, cudaMemcpyAsync(hp.data(), part, hp.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
    DD_TRY_CUDA(ctx, cudaStreamSynchronize(s));
    for (int k = 0; k < 12; ++k) {
        double acc = 0.0;
        for (int b = 0; b < blocks; ++b) acc += hp[(size_t)b * 12 + k];
        ds->M.mu[k] = acc / (double)S;
    }
    unsigned *stats = reinterpret_cast<unsigned *>(part);
    DD_TRY_CUDA(ctx, cudaMemsetAsync(stats, 0, 3 * sizeof(unsigned), s));
    k_transform<<<(unsigned)((ds->N_pad + 255) / 256), 256, 0, s>>>(ds->raw, ds->N, ds->N_pad, ds->M, ds->z32,
                                                                    ds->zn, stats);
    DD_TRY_CUDA(ctx, cudaGetLastError());
    unsigned hs[3];
    DD_TRY_CUDA(ctx, cudaMemcpyAsync(hs, stats, sizeof(hs), cudaMemcpyDeviceToHost, s));
    DD_TRY_CUDA(ctx, cudaStreamSynchronize(s));
    if (hs[2] != 0) return dd_fail(ctx, DD_ERR_ARG, "data set contains non-finite values");
    float mx, n2;
    std::memcpy(&mx, &hs[0], 4);
    std::memcpy(&n2, &hs[1], 4);
    ds->maxabs = mx;
    ds->R = std::sqrt((double)n2) * (1.0 + 1e-6);
    return DD_OK;
}
