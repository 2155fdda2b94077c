// Device helpers of the constraint projection shared by fem.cu and batch.cu.
#pragma once

#include "fem.cuh"

namespace {

__device__ __forceinline__ void node_ijk(const MeshDev &g, int64_t a, int &i, int &j, int &k) {
    const int64_t nx1 = g.nx + 1, ny1 = g.ny + 1;
    i = (int)(a % nx1);
    j = (int)((a / nx1) % ny1);
    k = (int)(a / (nx1 * ny1));
}

__device__ __forceinline__ int64_t node_id(const MeshDev &g, int i, int j, int k) {
    return i + (int64_t)(g.nx + 1) * (j + (int64_t)(g.ny + 1) * k);
}

__device__ __forceinline__ void bt_times(const double *dN, const double *v, double out[3]) {
    // B_a^T v for the Voigt vector v = (xx, yy, zz, yz, xz, xy)
    out[0] = dN[0] * v[0] + dN[2] * v[4] + dN[1] * v[5];
    out[1] = dN[1] * v[1] + dN[2] * v[3] + dN[0] * v[5];
    out[2] = dN[2] * v[2] + dN[1] * v[3] + dN[0] * v[4];
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Bounded grid barrier for a cooperative launch: one monotonic arrival
// counter (zeroed before the launch); barrier number k of the launch completes
// when the counter reaches k * nblocks.  One release-add per block and
// acquire polling, no reset round trip.  Returns false if any block reported
// a timeout.
struct GridBar {
    unsigned *count;
    unsigned nblocks;
    unsigned epoch;
};

__device__ __forceinline__ void red_release_add(unsigned *p, unsigned v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ bool grid_sync(GridBar &gb, unsigned *err) {
    __shared__ int s_ok;
    __syncthreads();
    gb.epoch++;
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned target = gb.epoch * gb.nblocks;
        red_release_add(gb.count, 1u);
        unsigned long long t0 = 0;
        int spin = 0;
        while ((int)(ld_acquire(gb.count) - target) < 0) {
            if ((++spin & 63) == 0) {
                unsigned long long t = dd_globaltimer();
                if (t0 == 0) t0 = t;
                else if (t - t0 > kWaitLimitNs) {
                    atomicOr(err, DEV_ERR_TIMEOUT);
                    ok = 0;
                    break;
                }
            }
        }
        if (ok && (ld_acquire(err) & DEV_ERR_TIMEOUT)) ok = 0;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Sum NV per-thread values over the block; thread 0 gets the totals.
template <int NV>
__device__ void block_sum(double (&v)[NV], double *sh /* [NV * 32] */) {
#pragma unroll
    for (int c = 0; c < NV; ++c)
        for (int o = 16; o > 0; o >>= 1) v[c] += __shfl_down_sync(0xffffffffu, v[c], o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0)
#pragma unroll
        for (int c = 0; c < NV; ++c) sh[c * 32 + wid] = v[c];
    __syncthreads();
    if (wid == 0) {
        const int nw = blockDim.x >> 5;
#pragma unroll
        for (int c = 0; c < NV; ++c) {
            double t = lane < nw ? sh[c * 32 + lane] : 0.0;
            for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
            v[c] = t;
        }
    }
    __syncthreads();
}

// After a barrier: every block sums the grid partials in the same order.
template <int NV>
__device__ void grid_total(const double *part, int nblk, double (&tot)[NV], double *sh) {
    double v[NV];
#pragma unroll
    for (int c = 0; c < NV; ++c) v[c] = 0.0;
    for (int t = threadIdx.x; t < nblk; t += blockDim.x)
#pragma unroll
        for (int c = 0; c < NV; ++c) v[c] += __ldcg(part + (size_t)t * 8 + c);
    block_sum<NV>(v, sh);
    __shared__ double s_tot[8];
    if (threadIdx.x == 0)
#pragma unroll
        for (int c = 0; c < NV; ++c) s_tot[c] = v[c];
    __syncthreads();
#pragma unroll
    for (int c = 0; c < NV; ++c) tot[c] = s_tot[c];
    __syncthreads();
}

}  // namespace
