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

template <typename T>
__device__ __forceinline__ void spmv_node_t(const MeshDev &g, const T *sKe, int64_t a, const T *vz, const T *vp,
                                            const T beta[2], T y[6]) {
    int i, j, k;
    node_ijk(g, a, i, j, k);
#pragma unroll
    for (int c = 0; c < 6; ++c) y[c] = T(0);
    if (k == 0) return;
    for (int oz = -1; oz <= 0; ++oz)
        for (int oy = -1; oy <= 0; ++oy)
            for (int ox = -1; ox <= 0; ++ox) {
                int ei = i + ox, ej = j + oy, ek = k + oz;
                if (ei < 0 || ej < 0 || ek < 0 || ei >= g.nx || ej >= g.ny || ek >= g.nz) continue;
                int la = (-ox) + 2 * (-oy) + 4 * (-oz);
#pragma unroll
                for (int lb = 0; lb < 8; ++lb) {
                    int64_t nb = node_id(g, ei + (lb & 1), ej + ((lb >> 1) & 1), ek + ((lb >> 2) & 1));
                    T xv[6];
#pragma unroll
                    for (int c = 0; c < 6; ++c) {
                        T t = __ldcg(vz + nb * 6 + c);
                        if (vp) t += beta[c / 3] * __ldcg(vp + nb * 6 + c);
                        xv[c] = t;
                    }
                    const T *kb = sKe + (3 * la) * 24 + 3 * lb;
#pragma unroll
                    for (int r = 0; r < 3; ++r) {
                        T k0 = kb[r * 24 + 0], k1 = kb[r * 24 + 1], k2 = kb[r * 24 + 2];
                        y[r] += k0 * xv[0] + k1 * xv[1] + k2 * xv[2];
                        y[3 + r] += k0 * xv[3] + k1 * xv[4] + k2 * xv[5];
                    }
                }
            }
}

__device__ __forceinline__ void apply_minv_f(const double *Mi, const float *r, float *z) {
    float m[9];
#pragma unroll
    for (int c = 0; c < 9; ++c) m[c] = (float)Mi[c];
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int a = 0; a < 3; ++a)
            z[3 * s + a] = m[3 * a] * r[3 * s] + m[3 * a + 1] * r[3 * s + 1] + m[3 * a + 2] * r[3 * s + 2];
}


// Element-parallel product: the 8 threads of a node group (8 consecutive
// lanes) each take one of the (up to) 8 elements around node a (slot e is the
// element in which a has local index e) and gather Ke[e, :] * v over its 8
// nodes; a group-masked butterfly leaves the sum (K v)_a in all 8 lanes.
// v = vz + beta .* vp (vp may be null).  Fixed nodes (k = 0) give 0.
template <typename T>
__device__ __forceinline__ void spmv_group(const MeshDev &g, const T *sKe, int64_t a, int e, unsigned gmask,
                                           const T *vz, const T *vp, const T beta[2], T y[6]) {
    int i, j, k;
    node_ijk(g, a, i, j, k);
#pragma unroll
    for (int c = 0; c < 6; ++c) y[c] = T(0);
    const int ei = i - (e & 1), ej = j - ((e >> 1) & 1), ek = k - ((e >> 2) & 1);
    if (k > 0 && ei >= 0 && ej >= 0 && ek >= 0 && ei < g.nx && ej < g.ny && ek < g.nz) {
#pragma unroll
        for (int lb = 0; lb < 8; ++lb) {
            int64_t nb = node_id(g, ei + (lb & 1), ej + ((lb >> 1) & 1), ek + ((lb >> 2) & 1));
            T xv[6];
#pragma unroll
            for (int c = 0; c < 6; ++c) {
                T t = __ldcg(vz + nb * 6 + c);
                if (vp) t += beta[c / 3] * __ldcg(vp + nb * 6 + c);
                xv[c] = t;
            }
            const T *kb = sKe + (3 * e) * 24 + 3 * lb;
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                T k0 = kb[r * 24 + 0], k1 = kb[r * 24 + 1], k2 = kb[r * 24 + 2];
                y[r] += k0 * xv[0] + k1 * xv[1] + k2 * xv[2];
                y[3 + r] += k0 * xv[3] + k1 * xv[4] + k2 * xv[5];
            }
        }
    }
#pragma unroll
    for (int o = 1; o < 8; o <<= 1)
#pragma unroll
        for (int c = 0; c < 6; ++c) y[c] += __shfl_xor_sync(gmask, y[c], o);
}

// y[c] for a run-time component c without dynamic register indexing.
template <typename T>
__device__ __forceinline__ T pick6(const T (&y)[6], int c) {
    T r = y[0];
#pragma unroll
    for (int k = 1; k < 6; ++k)
        if (c == k) r = y[k];
    return r;
}

}  // namespace
