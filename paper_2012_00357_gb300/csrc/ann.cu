// Approximate data projection (Sec. 4.2-4.5): the k-means search tree of the
// paper restated for the GPU as one wide level of k-means clusters over the
// mapped data, stored cluster-contiguously.
//
// Build (once per data set):
//   Lloyd iterations on a strided sample (k_assign + k_accum + k_update),
//   assignment of every point to its nearest centroid, a counting sort into
//   cluster order (zs, perm), and the radius d_r of every cluster (largest
//   distance from the centroid to a member, Sec. 4.2).
// Query (every DD iteration):
//   1. rank the centroids of every query (FP32 scan in top-k mode, the
//      kCand nearest centroids kept and sorted by exact FP32 distance);
//   2. warm start (Sec. 4.3): the previous nearest point gives the first
//      current-best distance d_c, and its cluster is scanned first;
//   3. the nearest cluster is always scanned (the descent of the tree);
//      every further candidate cluster is scanned when
//          d(x, q) - f_d d_r < d_c                                  (Eq. 13),
//      in order of centroid distance, d_c shrinking as better points appear;
//      f_d = 1 is exact by the triangle inequality, f_d = 0 scans only
//      clusters whose centroid is nearer than the best point so far;
//   4. backtracking is bounded to the kCand nearest centroids; for f_d = 1 a
//      query whose candidate list might miss a cluster allowed by Eq. 13 (the
//      kCand-th centroid still passes the test with the largest radius) is
//      re-searched by the certified exact scan, so f_d = 1 always returns the
//      exact point;
//   5. the answer is rescored with Eq. (3) in FP64.
// Moving-query radius (Eq. 14): with a motion record (previous query, the
// distance d1 of its answer, a lower bound d2 on the distance of every other
// point) a query that moved less than (d2 - d1)/2 keeps its previous
// neighbour without any scan.  The bound is the smaller of the second-best
// point read and, for every cluster, cell or leaf not searched, its centroid
// distance minus f_d times its radius (the cluster model Eq. 13 uses; at
// f_d = 1 a true lower bound, so a kept answer is the exact nearest point).
// A record made at one f_d is used only by searches at the same or a lower
// f_d.
#include <algorithm>
#include <cmath>
#include <vector>

#include "dd_internal.cuh"

namespace {

constexpr int kCand = kAnnCand;   // candidate clusters per query
constexpr int kTileC = 256;       // centroids per shared-memory tile in k_assign

__device__ __forceinline__ float dist2_12(const float *a, const float (&q)[12]) { return dd_dist2_12(a, q); }

// Nearest centroid of every point (expanded FP32 score |c|^2 - 2 c.z, ties to
// the lower centroid index).  Centroids stream through shared memory.  With
// a list, only the rows list[0 .. *n_list - 1] (the rows the tensor-core
// pass left open).
__global__ void __launch_bounds__(256) k_assign(const float *__restrict__ z, int64_t n,
                                                const float *__restrict__ cent, const float *__restrict__ cn,
                                                int L, int32_t *__restrict__ out, const int32_t *__restrict__ list,
                                                const unsigned *__restrict__ n_list) {
    __shared__ __align__(16) float sc[kTileC * 12];
    __shared__ float sn[kTileC];
    const int64_t nq = list ? ((int64_t)*n_list < n ? (int64_t)*n_list : n) : n;
    if (blockIdx.x * (int64_t)blockDim.x >= nq) return;   // the whole block, before any barrier
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t j = t < nq ? (list ? (int64_t)list[t] : t) : n;
    float q[12];
    if (j < n) {
#pragma unroll
        for (int k = 0; k < 12; ++k) q[k] = -2.f * z[j * 12 + k];
    } else {
#pragma unroll
        for (int k = 0; k < 12; ++k) q[k] = 0.f;
    }
    float best = INFINITY;
    int bi = 0;
    for (int c0 = 0; c0 < L; c0 += kTileC) {
        __syncthreads();
        const int nt = min(kTileC, L - c0);
        for (int t = threadIdx.x; t < nt * 12; t += blockDim.x) sc[t] = cent[(int64_t)c0 * 12 + t];
        for (int t = threadIdx.x; t < nt; t += blockDim.x) sn[t] = cn[c0 + t];
        __syncthreads();
        for (int c = 0; c < nt; ++c) {
            const float4 *p = reinterpret_cast<const float4 *>(sc + c * 12);
            float4 a = p[0], b = p[1], d = p[2];
            float v = sn[c];
            v = fmaf(q[0], a.x, v); v = fmaf(q[1], a.y, v); v = fmaf(q[2], a.z, v); v = fmaf(q[3], a.w, v);
            v = fmaf(q[4], b.x, v); v = fmaf(q[5], b.y, v); v = fmaf(q[6], b.z, v); v = fmaf(q[7], b.w, v);
            v = fmaf(q[8], d.x, v); v = fmaf(q[9], d.y, v); v = fmaf(q[10], d.z, v); v = fmaf(q[11], d.w, v);
            if (v < best) {
                best = v;
                bi = c0 + c;
            }
        }
    }
    if (j < n) out[j] = bi;
}

// Cluster sums are accumulated in 64-bit fixed point (coordinates scaled by
// a power of two fs with |z| fs <= 2^30): integer addition does not depend on
// the order of the atomics, so the k-means build is the same on every run.
__device__ __forceinline__ unsigned long long to_fixed(float v, double fs) {
    return (unsigned long long)__double2ll_rn((double)v * fs);
}

__global__ void k_accum(const float *__restrict__ z, int64_t n, const int32_t *__restrict__ asg, double fs,
                        unsigned long long *__restrict__ sums, unsigned *__restrict__ cnt) {
    int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= n) return;
    int c = asg[j];
#pragma unroll
    for (int k = 0; k < 12; ++k) atomicAdd(sums + (size_t)c * 12 + k, to_fixed(z[j * 12 + k], fs));
    atomicAdd(cnt + c, 1u);
}

// centroid = mean of its members (kept when empty); norms; reset accumulators
__global__ void k_update(unsigned long long *__restrict__ sums, unsigned *__restrict__ cnt, double fs,
                         float *__restrict__ cent, float *__restrict__ cn, int L) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= L) return;
    unsigned k = cnt[c];
    double n2 = 0.0;
#pragma unroll
    for (int a = 0; a < 12; ++a) {
        if (k) cent[(size_t)c * 12 + a] = (float)((double)(long long)sums[(size_t)c * 12 + a] / fs / (double)k);
        double v = cent[(size_t)c * 12 + a];
        n2 += v * v;
        sums[(size_t)c * 12 + a] = 0ull;
    }
    cn[c] = (float)n2;
    cnt[c] = 0;
}

__global__ void k_gather_rows(const float *__restrict__ z, int64_t N, int64_t S, float *__restrict__ out) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= S) return;
    int64_t j = (int64_t)(((__int128)i * N) / S);
#pragma unroll
    for (int k = 0; k < 12; ++k) out[i * 12 + k] = z[j * 12 + k];
}

__global__ void k_hist(const int32_t *__restrict__ asg, int64_t n, unsigned *__restrict__ cnt) {
    int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j < n) atomicAdd(cnt + asg[j], 1u);
}

__global__ void k_scatter(const float *__restrict__ z, const int32_t *__restrict__ asg, int64_t n,
                          const int64_t *__restrict__ offs, unsigned *__restrict__ cursor, float *__restrict__ zs,
                          int32_t *__restrict__ perm) {
    int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= n) return;
    int c = asg[j];
    int64_t p = offs[c] + atomicAdd(cursor + c, 1u);
    const float4 *src = reinterpret_cast<const float4 *>(z + j * 12);
    float4 *dst = reinterpret_cast<float4 *>(zs + p * 12);
    dst[0] = src[0];
    dst[1] = src[1];
    dst[2] = src[2];
    perm[p] = (int32_t)j;
}

__global__ void k_radius(const float *__restrict__ zs, const int32_t *__restrict__ perm,
                         const int32_t *__restrict__ asg, int64_t n, const float *__restrict__ cent,
                         unsigned *__restrict__ rbits) {
    int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= n) return;
    int c = asg[perm[p]];
    float q[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) q[k] = cent[(size_t)c * 12 + k];
    float d = sqrtf(dist2_12(zs + p * 12, q));
    // round up by a relative 1e-6 so FP32 rounding never shrinks the bound
    atomicMax(rbits + c, __float_as_uint(d * 1.000001f + 1e-30f));
}

// ---------------------------------------------------------------------------
// Query side
// ---------------------------------------------------------------------------
// Nearest kCand centroids of every listed query when the centroid set is
// small: each thread ranks kRankQ queries, centroids staged in shared memory
// and read as broadcasts (one read serves all of a thread's queries); top
// kCand by the expanded FP32 score |c|^2 - 2 c.q (ties to the lower index),
// then ordered by the FP32 distance as from k_ann_cands.  `list` (may be
// null: queries 0..m-1) holds the *n_list queries to rank, in any order.
constexpr int kRankTile = 896;      // 896 x 52 B of static shared memory (< 48 KB)
constexpr int kRankMax = 4096;    // larger sets go through the tiled FP32 scan
constexpr int kRankQ = 1;         // queries per thread (two measured no faster)

__global__ void __launch_bounds__(256) k_rank_small(const QueryRec *__restrict__ rec, int64_t m,
                                                    const int32_t *__restrict__ list,
                                                    const unsigned *__restrict__ n_list,
                                                    const float *__restrict__ cent, const float *__restrict__ cn,
                                                    int L, int32_t *__restrict__ out_cl, float *__restrict__ out_d) {
    __shared__ __align__(16) float sc[kRankTile * 12];
    __shared__ float sn[kRankTile];
    const int64_t nq = list ? (int64_t)*n_list : m;
    const int64_t base = blockIdx.x * (int64_t)blockDim.x * kRankQ;
    if (base >= nq) return;           // the whole block: before any barrier
    int64_t qi[kRankQ];
    float qm2[kRankQ][12];
    float bs[kRankQ][kCand];
    int bc[kRankQ][kCand];
#pragma unroll
    for (int r = 0; r < kRankQ; ++r) {
        const int64_t t = base + r * blockDim.x + threadIdx.x;
        qi[r] = t < nq ? (list ? (int64_t)list[t] : t) : -1;
#pragma unroll
        for (int k = 0; k < 12; ++k) qm2[r][k] = qi[r] >= 0 ? -2.f * rec[qi[r]].q[k] : 0.f;
#pragma unroll
        for (int k = 0; k < kCand; ++k) {
            bs[r][k] = INFINITY;
            bc[r][k] = -1;
        }
    }
    for (int t0 = 0; t0 < L; t0 += kRankTile) {
        const int nt = min(kRankTile, L - t0);
        __syncthreads();
        for (int k = threadIdx.x; k < nt * 12; k += blockDim.x) sc[k] = cent[(size_t)t0 * 12 + k];
        for (int k = threadIdx.x; k < nt; k += blockDim.x) sn[k] = cn[t0 + k];
        __syncthreads();
        for (int f = 0; f < nt; ++f) {
            const float4 *pc = reinterpret_cast<const float4 *>(sc + f * 12);
            const float4 a = pc[0], b = pc[1], d = pc[2];
            const float n2 = sn[f];
#pragma unroll
            for (int r = 0; r < kRankQ; ++r) {
                const float *w = qm2[r];
                float v = n2;
                v = fmaf(w[0], a.x, v); v = fmaf(w[1], a.y, v); v = fmaf(w[2], a.z, v); v = fmaf(w[3], a.w, v);
                v = fmaf(w[4], b.x, v); v = fmaf(w[5], b.y, v); v = fmaf(w[6], b.z, v); v = fmaf(w[7], b.w, v);
                v = fmaf(w[8], d.x, v); v = fmaf(w[9], d.y, v); v = fmaf(w[10], d.z, v); v = fmaf(w[11], d.w, v);
                if (v < bs[r][kCand - 1]) {
                    bs[r][kCand - 1] = v;
                    bc[r][kCand - 1] = t0 + f;
#pragma unroll
                    for (int k = kCand - 1; k > 0; --k)
                        if (bs[r][k] < bs[r][k - 1]) {
                            const float tv = bs[r][k];
                            bs[r][k] = bs[r][k - 1];
                            bs[r][k - 1] = tv;
                            const int tc = bc[r][k];
                            bc[r][k] = bc[r][k - 1];
                            bc[r][k - 1] = tc;
                        }
                }
            }
        }
    }
#pragma unroll
    for (int r = 0; r < kRankQ; ++r) {
        if (qi[r] < 0) continue;
        const int64_t i = qi[r];
        float q[12];
#pragma unroll
        for (int k = 0; k < 12; ++k) q[k] = rec[i].q[k];
        float bd[kCand];
        int c8[kCand];
#pragma unroll
        for (int k = 0; k < kCand; ++k) {
            c8[k] = bc[r][k];
            bd[k] = c8[k] >= 0 ? dist2_12(cent + (size_t)c8[k] * 12, q) : INFINITY;
        }
#pragma unroll
        for (int a = 1; a < kCand; ++a)       // insertion sort by (distance, index)
#pragma unroll
            for (int k = a; k > 0; --k)
                if (bd[k] < bd[k - 1] || (bd[k] == bd[k - 1] && c8[k] >= 0 && c8[k] < c8[k - 1])) {
                    const float tv = bd[k];
                    bd[k] = bd[k - 1];
                    bd[k - 1] = tv;
                    const int tc = c8[k];
                    c8[k] = c8[k - 1];
                    c8[k - 1] = tc;
                }
#pragma unroll
        for (int k = 0; k < kCand; ++k) {
            out_cl[i * kCand + k] = c8[k];
            out_d[i * kCand + k] = sqrtf(bd[k]);
        }
    }
}

// Merge the top-k lists of the centroid scan; keep the kCand nearest
// centroids by exact FP32 distance (ties to the lower centroid index).
__global__ void k_ann_cands(const CandHeader *__restrict__ hdr, const float2 *__restrict__ cand, int splits, int cap,
                            const QueryRec *__restrict__ rec, int64_t m, const float *__restrict__ cent,
                            int32_t *__restrict__ out_cl, float *__restrict__ out_d) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= m) return;
    float q[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) q[k] = rec[i].q[k];
    float bd[kCand];
    int bc[kCand];
#pragma unroll
    for (int k = 0; k < kCand; ++k) {
        bd[k] = INFINITY;
        bc[k] = -1;
    }
    for (int s = 0; s < splits; ++s) {
        const CandHeader h = hdr[(size_t)i * splits + s];
        const float2 *c = cand + ((size_t)i * splits + s) * cap;
        for (int e = 0; e < h.cnt; ++e) {
            int l = __float_as_int(c[e].y);
            float d = dist2_12(cent + (size_t)l * 12, q);
            // sorted insertion
            if (d < bd[kCand - 1] || (d == bd[kCand - 1] && l < bc[kCand - 1])) {
                int k = kCand - 1;
                while (k > 0 && (d < bd[k - 1] || (d == bd[k - 1] && l < bc[k - 1]))) {
                    bd[k] = bd[k - 1];
                    bc[k] = bc[k - 1];
                    --k;
                }
                bd[k] = d;
                bc[k] = l;
            }
        }
    }
#pragma unroll
    for (int k = 0; k < kCand; ++k) {
        out_cl[i * kCand + k] = bc[k];
        out_d[i * kCand + k] = sqrtf(bd[k]);
    }
}

struct Best {
    float d;      // squared distance
    int j;        // original index
    float s;      // second-best squared distance
};

__device__ __forceinline__ void best_update(Best &b, float d, int j) {
    if (d < b.d || (d == b.d && j < b.j)) {
        b.s = b.d;
        b.d = d;
        b.j = j;
    } else if (d < b.s) {
        b.s = d;
    }
}

// Offer point p (squared distance d) to b; its original index is read only
// when it can become the best, and the point that already is the best (the
// warm start, met again in its own cluster) is not a second candidate.
__device__ __forceinline__ void best_lazy(Best &b, float d, const int32_t *perm, int64_t p) {
    if (d <= b.d) {
        const int j = __ldg(perm + p);
        if (j != b.j) best_update(b, d, j);
    } else if (d < b.s) {
        b.s = d;
    }
}

// One warp scans the points [p0, p1) of the cluster-sorted copy for query q
// (lane-strided, four points of a lane in flight at a time); the original
// index is read only for a point that can become the best.
__device__ __forceinline__ void scan_range(const float *zs, const int32_t *perm, int64_t p0, int64_t p1, int lane,
                                           const float (&q)[12], Best &b) {
    int64_t p = p0 + lane;
    for (; p + 96 < p1; p += 128) {
        float d[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) d[u] = dist2_12(zs + (p + 32 * u) * 12, q);
#pragma unroll
        for (int u = 0; u < 4; ++u) best_lazy(b, d[u], perm, p + 32 * u);
    }
    for (; p < p1; p += 32) best_lazy(b, dist2_12(zs + p * 12, q), perm, p);
}

// warp-wide merge: every lane ends with the same (best, index, second)
__device__ __forceinline__ void best_warp(Best &b) {
    Best g = b;
    for (int o = 16; o > 0; o >>= 1) {
        float d = __shfl_xor_sync(0xffffffffu, g.d, o);
        int j = __shfl_xor_sync(0xffffffffu, g.j, o);
        if (d < g.d || (d == g.d && j < g.j)) {
            g.d = d;
            g.j = j;
        }
    }
    float t = (b.d == g.d && b.j == g.j) ? b.s : b.d;
    t = fminf(t, b.s);
    if (b.d == g.d && b.j == g.j) t = b.s;
    for (int o = 16; o > 0; o >>= 1) t = fminf(t, __shfl_xor_sync(0xffffffffu, t, o));
    b.d = g.d;
    b.j = g.j;
    b.s = t;
}

struct ProbeArgs {
    const float *zs;
    const int32_t *perm;
    const int64_t *offs;
    const float *radius;
    const int32_t *cluster_of;
    const float *z32;           // original order, for the warm start
    const QueryRec *rec;
    const int32_t *cand_cl;
    const float *cand_d;
    int64_t m, N;
    int L;
    float f_d;
    const float *fd_q;          // per-query f_d (may be null: f_d for all)
    float rmax;
    const int32_t *prev;        // may be null
    const float *mot_q;         // motion record (may be null): previous query [m x 12]
    const float *mot_d;         // [m x 2] previous nearest / second distances (plain)
    int32_t *idx;
    float *d1, *d2;             // plain squared distances of the answer / second
    int64_t *fb_list;
    unsigned long long *fb_count;
    unsigned long long *counters;   // [0] point distances evaluated, [1] queries skipped, [2] exact
                                    // re-searches, [3] leaf centroids ranked, [4] distinct points,
                                    // [5] points read
    unsigned *touched;              // [ceil(L / 32)] clusters scanned by any query of this search
    int gated;                      // 1: k_ann_gate ran; cand_cl[i * kCand] == kGated marks a kept query
    int certified;                  // 1: the second distance is the certified bound (Eq. 14); 0: the
                                    // second-best point read below f_d = 1 (the certified bound at 1)
};

constexpr int kGated = -2;

// Eq. (14) before the cell ranking: a query that moved less than half the gap
// between its previous nearest and second distances keeps its warm-start
// point without a search (its answer is written here and its first candidate
// slot marked kGated); every other query is appended to the list the ranking
// and the probes work on.  One thread per query; one list append, and one
// update of each counter, per block.
struct GateArgs {
    const QueryRec *rec;
    int64_t m, N;
    const int32_t *prev;
    const float *z32;
    const float *mot_q, *mot_d;
    float f_d;
    const float *fd_q;          // per-query f_d (may be null: f_d for all)
    int32_t *idx;
    float *d1, *d2;
    int32_t *cand_cl;
    int32_t *list;
    unsigned *n_list;
    unsigned long long *counters;   // [1] queries kept, [3] += Lr per listed query (centroids ranked)
    int Lr;
};

__global__ void __launch_bounds__(256) k_ann_gate(GateArgs G) {
    __shared__ unsigned s_cnt[2][8];
    __shared__ unsigned s_base;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    bool keep = false;
    if (i < G.m) {
        const int j0 = G.prev[i];
        if (j0 >= 0 && j0 < G.N) {
            float q[12];
#pragma unroll
            for (int k = 0; k < 12; ++k) q[k] = G.rec[i].q[k];
            float mv = 0.f;
#pragma unroll
            for (int k = 0; k < 12; ++k) {
                float t = q[k] - G.mot_q[i * 12 + k];
                mv = fmaf(t, t, mv);
            }
            mv = sqrtf(mv);
            const float4 r = *reinterpret_cast<const float4 *>(G.mot_d + i * kMotStride);
            const float f_d = G.fd_q ? G.fd_q[i] : G.f_d;
            if (mv < 0.5f * (r.y - r.x) && f_d <= r.z) {
                const float r2 = r.y;
                keep = true;
                G.idx[i] = j0;
                G.d1[i] = dist2_12(G.z32 + (size_t)j0 * 12, q);
                float lb = fmaxf(r2 - mv, 0.f);
                G.d2[i] = lb * lb;
                G.cand_cl[i * kCand] = kGated;
            }
        }
    }
    const bool listed = i < G.m && !keep;
    const unsigned mk = __ballot_sync(0xffffffffu, keep), ml = __ballot_sync(0xffffffffu, listed);
    if (lane == 0) {
        s_cnt[0][warp] = __popc(mk);
        s_cnt[1][warp] = __popc(ml);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned nk = 0, nl = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            nk += s_cnt[0][w];
            const unsigned c = s_cnt[1][w];
            s_cnt[1][w] = nl;             // exclusive prefix of the warps' list entries
            nl += c;
        }
        s_base = nl ? atomicAdd(G.n_list, nl) : 0u;
        if (nk) atomicAdd(G.counters + 1, (unsigned long long)nk);
        if (nl) atomicAdd(G.counters + 3, (unsigned long long)nl * (unsigned long long)G.Lr);
    }
    __syncthreads();
    if (listed) G.list[s_base + s_cnt[1][warp] + __popc(ml & ((1u << lane) - 1u))] = (int32_t)i;
}

__global__ void __launch_bounds__(256) k_ann_probe(ProbeArgs A) {
    const int lane = threadIdx.x & 31;
    const int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (i >= A.m) return;
    if (A.gated && A.cand_cl[i * kCand] == kGated) return;   // kept by Eq. (14)
    float q[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) q[k] = A.rec[i].q[k];
    Best b{INFINITY, 0x7fffffff, INFINITY};
    int cl0 = -1;
    unsigned long long scanned = 0;
    if (A.prev) {
        const int j0 = A.prev[i];
        if (j0 >= 0 && j0 < A.N) {
            const float d0 = dist2_12(A.z32 + (size_t)j0 * 12, q);
            if (A.mot_q) {
                // Eq. (14): moved less than (d2 - d1)/2 since the last search
                float mv = 0.f;
#pragma unroll
                for (int k = 0; k < 12; ++k) {
                    float t = q[k] - A.mot_q[i * 12 + k];
                    mv = fmaf(t, t, mv);
                }
                mv = sqrtf(mv);
                const float4 r = *reinterpret_cast<const float4 *>(A.mot_d + i * kMotStride);
                const float fdi = A.fd_q ? A.fd_q[i] : A.f_d;
                if (mv < 0.5f * (r.y - r.x) && fdi <= r.z) {
                    if (lane == 0) {
                        A.idx[i] = j0;
                        A.d1[i] = d0;
                        float lb = fmaxf(r.y - mv, 0.f);
                        A.d2[i] = lb * lb;
                        atomicAdd(A.counters + 1, 1ull);
                    }
                    return;
                }
            }
            b.d = d0;
            b.j = j0;
            cl0 = A.cluster_of[j0];
        }
    }
    auto scan = [&](int l) {
        const int64_t p0 = A.offs[l], p1 = A.offs[l + 1];
        scan_range(A.zs, A.perm, p0, p1, lane, q, b);
        scanned += (unsigned long long)(p1 - p0);
        if (lane == 0) atomicOr(A.touched + (l >> 5), 1u << (l & 31));
        best_warp(b);
    };
    if (cl0 >= 0) scan(cl0);
    float dc = sqrtf(b.d);
    const float f_d = A.fd_q ? A.fd_q[i] : A.f_d;
    const bool cert = A.certified || f_d >= 1.0f;
    float lb = INFINITY;    // Eq. (14): plain bound on the points of the clusters not searched
    for (int k = 0; k < kCand; ++k) {
        const int l = A.cand_cl[i * kCand + k];
        if (l < 0) break;
        if (l == cl0) continue;
        const float dl = A.cand_d[i * kCand + k];
        if (k == 0 || dl - f_d * A.radius[l] < dc) {
            scan(l);
            dc = sqrtf(b.d);
        } else if (cert) {
            lb = fminf(lb, dl - f_d * A.radius[l]);
        }
    }
    // clusters beyond the candidate list: no nearer centroid, no wider radius
    if (cert && A.L > kCand) lb = fminf(lb, A.cand_d[i * kCand + kCand - 1] - f_d * A.rmax);
    // completeness of the candidate list under Eq. (13), for exact requests
    // (f_d = 1) only; below that, backtracking is bounded to the kCand
    // nearest centroids
    bool incomplete = false;
    if (A.L > kCand && f_d >= 1.0f) {
        const float dP = A.cand_d[i * kCand + kCand - 1];
        incomplete = (dP - f_d * A.rmax < dc);
    }
    // every candidate cluster was empty (degenerate data, e.g. many copies of
    // a few points leave most clusters without members): the whole data set,
    // so that the answer is always a data point (b is warp-uniform here)
    if (b.j == 0x7fffffff) {
        scan_range(A.zs, A.perm, 0, A.N, lane, q, b);
        scanned += (unsigned long long)A.N;
        best_warp(b);
    }
    if (lane == 0) {
        atomicAdd(A.counters, scanned);
        atomicAdd(A.counters + 5, scanned);
        if (incomplete) {
            unsigned long long t = atomicAdd(A.fb_count, 1ull);
            A.fb_list[t] = i;
        }
        A.idx[i] = b.j;
        A.d1[i] = b.d;
        A.d2[i] = fminf(b.s, lb > 0.f ? lb * lb : 0.f);
    }
}

// FP64 rescoring of the answer (Eq. 3) and the second distance in Eq. 3 units.
// A query whose candidate leaves were all empty and none handed off
// (degenerate data: many copies of a few points leave most leaves without
// members) has no answer yet: this thread scans the whole data set for it
// (the two-level probe leaves that rare case here to keep its registers).
__global__ void k_ann_finish(const float *__restrict__ raw, MetricMaps M, const double *__restrict__ y, int64_t m,
                             int32_t *__restrict__ idx, float *__restrict__ d2f, double *__restrict__ d2,
                             double *__restrict__ d2nd, const float *__restrict__ z32, int64_t N,
                             const QueryRec *__restrict__ rec) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= m) return;
    if (idx[i] < 0 || idx[i] >= N) {
        float q[12];
#pragma unroll
        for (int k = 0; k < 12; ++k) q[k] = rec[i].q[k];
        float b1 = INFINITY;
        int j1 = 0;
        for (int64_t j = 0; j < N; ++j) {
            const float d = dist2_12(z32 + j * 12, q);
            if (d < b1) {
                b1 = d;
                j1 = (int)j;
            }
        }
        idx[i] = j1;
        d2f[i] = 0.f;   // no second-distance bound: the query is searched again next time
    }
    double yy[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) yy[k] = y[i * 12 + k];
    if (d2) d2[i] = dd_eq3(M, yy, raw + (size_t)idx[i] * 12);
    if (d2nd) d2nd[i] = 2.0 * (double)d2f[i];
}

// ---------------------------------------------------------------------------
// Two-level tree: coarse cells of k-means centroids, each split into L2
// k-means leaves (the k-means tree of Sec. 4.2 with wide branching).
// ---------------------------------------------------------------------------
// Stable counting sort of the point indices by cell (members of a cell in
// increasing index order, the same on every run): per-chunk histograms, their
// per-cell prefix over chunks, then one warp per chunk placing its points in
// index order.
constexpr int kStableChunk = 1 << 16;

__global__ void k_chunk_hist(const int32_t *__restrict__ asg, int64_t n, int nb, unsigned *__restrict__ hist) {
    extern __shared__ unsigned sh_hist[];
    for (int b = threadIdx.x; b < nb; b += blockDim.x) sh_hist[b] = 0u;
    __syncthreads();
    const int64_t j0 = (int64_t)blockIdx.x * kStableChunk, j1 = min(n, j0 + kStableChunk);
    for (int64_t j = j0 + threadIdx.x; j < j1; j += blockDim.x) atomicAdd(sh_hist + asg[j], 1u);
    __syncthreads();
    for (int b = threadIdx.x; b < nb; b += blockDim.x) hist[(size_t)blockIdx.x * nb + b] = sh_hist[b];
}

__global__ void k_chunk_offsets(unsigned *__restrict__ hist, int nchunk, int nb, const int64_t *__restrict__ offs) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    unsigned run = (unsigned)offs[b];
    for (int c = 0; c < nchunk; ++c) {
        const unsigned v = hist[(size_t)c * nb + b];
        hist[(size_t)c * nb + b] = run;
        run += v;
    }
}

__global__ void __launch_bounds__(32) k_stable_scatter(const int32_t *__restrict__ asg, int64_t n, int nb,
                                                       const unsigned *__restrict__ off, int32_t *__restrict__ perm1) {
    extern __shared__ unsigned cur[];
    const int lane = threadIdx.x;
    for (int b = lane; b < nb; b += 32) cur[b] = off[(size_t)blockIdx.x * nb + b];
    __syncwarp();
    const int64_t j0 = (int64_t)blockIdx.x * kStableChunk, j1 = min(n, j0 + kStableChunk);
    for (int64_t g = j0; g < j1; g += 32) {
        const int64_t j = g + lane;
        const bool valid = j < j1;
        const int b = valid ? asg[j] : -1;
        const unsigned same = __match_any_sync(0xffffffffu, b);
        const unsigned rank = __popc(same & ((1u << lane) - 1u));
        const unsigned base = valid ? cur[b] : 0u;
        __syncwarp();
        if (valid) {
            perm1[base + rank] = (int32_t)j;
            if (rank == 0) cur[b] = base + __popc(same);
        }
        __syncwarp();
    }
}

__global__ void k_cell_sorted(const int32_t *__restrict__ perm1, const int32_t *__restrict__ asg1, int64_t n,
                              int32_t *__restrict__ c1s) {
    int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p < n) c1s[p] = asg1[perm1[p]];
}

// leaf f of cell C starts at the cell's member of rank floor(f n_C / L2)
__global__ void k_fine_init(const float *__restrict__ z, const int32_t *__restrict__ perm1,
                            const int64_t *__restrict__ offs1, int L1, int L2, const float *__restrict__ cent1,
                            float *__restrict__ centf) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)L1 * L2) return;
    const int C = (int)(t / L2), f = (int)(t % L2);
    const int64_t n_c = offs1[C + 1] - offs1[C];
    const float *src = cent1 + (size_t)C * 12;
    if (n_c > 0) src = z + (size_t)perm1[offs1[C] + (int64_t)f * n_c / L2] * 12;
#pragma unroll
    for (int k = 0; k < 12; ++k) centf[t * 12 + k] = src[k];
}

// Nearest leaf of every point among its own cell's L2 leaves.  Points are
// visited in cell order (p = sorted position), so a block meets few cells;
// each cell's leaf centroids stream through shared memory once per block.
__global__ void __launch_bounds__(256) k_assign_fine(const float *__restrict__ z, const int32_t *__restrict__ perm1,
                                                     const int32_t *__restrict__ c1s, int64_t n,
                                                     const float *__restrict__ centf, const float *__restrict__ cnf,
                                                     int L2, int32_t *__restrict__ fasg) {
    __shared__ __align__(16) float sc[kTileC * 12];
    __shared__ float sn[kTileC];
    __shared__ int s_first, s_last;
    const int64_t p0 = (int64_t)blockIdx.x * blockDim.x;
    const int64_t p = p0 + threadIdx.x;
    const bool act = p < n;
    float q[12];
    int my_c = -1;
    if (act) {
        my_c = c1s[p];
        const float *zp = z + (size_t)perm1[p] * 12;
#pragma unroll
        for (int k = 0; k < 12; ++k) q[k] = -2.f * zp[k];
    } else {
#pragma unroll
        for (int k = 0; k < 12; ++k) q[k] = 0.f;
    }
    if (threadIdx.x == 0) {
        s_first = c1s[p0];
        s_last = c1s[min(n, p0 + (int64_t)blockDim.x) - 1];
    }
    __syncthreads();
    const int cf = s_first, cl = s_last;
    float best = INFINITY;
    int bi = 0;
    for (int c = cf; c <= cl; ++c) {
        for (int t0 = 0; t0 < L2; t0 += kTileC) {
            const int nt = min(kTileC, L2 - t0);
            __syncthreads();
            const float *src = centf + ((size_t)c * L2 + t0) * 12;
            for (int t = threadIdx.x; t < nt * 12; t += blockDim.x) sc[t] = src[t];
            for (int t = threadIdx.x; t < nt; t += blockDim.x) sn[t] = cnf[(size_t)c * L2 + t0 + t];
            __syncthreads();
            if (my_c == c) {
                for (int f = 0; f < nt; ++f) {
                    const float4 *pc = reinterpret_cast<const float4 *>(sc + f * 12);
                    float4 a = pc[0], b = pc[1], d = pc[2];
                    float v = sn[f];
                    v = fmaf(q[0], a.x, v); v = fmaf(q[1], a.y, v); v = fmaf(q[2], a.z, v); v = fmaf(q[3], a.w, v);
                    v = fmaf(q[4], b.x, v); v = fmaf(q[5], b.y, v); v = fmaf(q[6], b.z, v); v = fmaf(q[7], b.w, v);
                    v = fmaf(q[8], d.x, v); v = fmaf(q[9], d.y, v); v = fmaf(q[10], d.z, v); v = fmaf(q[11], d.w, v);
                    if (v < best) {
                        best = v;
                        bi = t0 + f;
                    }
                }
            }
        }
    }
    if (act) fasg[p] = bi;
}

__global__ void k_accum_fine(const float *__restrict__ z, const int32_t *__restrict__ perm1,
                             const int32_t *__restrict__ c1s, const int32_t *__restrict__ fasg, int64_t n, int L2,
                             double fs, unsigned long long *__restrict__ sums, unsigned *__restrict__ cnt) {
    int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int64_t leaf = (int64_t)c1s[p] * L2 + fasg[p];
    const float *zp = z + (size_t)perm1[p] * 12;
#pragma unroll
    for (int k = 0; k < 12; ++k) atomicAdd(sums + leaf * 12 + k, to_fixed(zp[k], fs));
    atomicAdd(cnt + leaf, 1u);
}

// k_accum_fine with the sums of a run of sorted positions gathered in shared
// memory first: a block takes kAccumRun consecutive positions (the members
// of one or two cells), adds every point to its leaf's shared-memory sum,
// then adds the non-empty leaf sums to the global ones, so that the global
// atomics fall from 13 per point to 13 per (block, leaf).  The sums are
// 64-bit fixed point, so the result does not depend on the order.
constexpr int kAccumRun = 8192;
constexpr int kAccumThreads = 512;

__global__ void __launch_bounds__(kAccumThreads) k_accum_fine_run(const float *__restrict__ z,
                                                                  const int32_t *__restrict__ perm1,
                                                                  const int32_t *__restrict__ c1s,
                                                                  const int32_t *__restrict__ fasg, int64_t n, int L2,
                                                                  double fs, unsigned long long *__restrict__ sums,
                                                                  unsigned *__restrict__ cnt) {
    extern __shared__ __align__(16) unsigned long long s_sum[];   // [L2 x 12], then L2 counts
    unsigned *s_cnt = reinterpret_cast<unsigned *>(s_sum + (size_t)L2 * 12);
    const int64_t p0 = (int64_t)blockIdx.x * kAccumRun;
    const int64_t p1 = min(n, p0 + (int64_t)kAccumRun);
    int64_t start = p0;
    while (start < p1) {   // one cell's positions at a time (the cells are contiguous)
        const int c = c1s[start];
        int64_t lo = start, hi = p1;   // first position of [start, p1) outside cell c
        while (lo + 1 < hi) {
            const int64_t mid = (lo + hi) / 2;
            if (c1s[mid] == c) lo = mid;
            else hi = mid;
        }
        const int64_t end = hi;
        for (int t = threadIdx.x; t < L2 * 12; t += blockDim.x) s_sum[t] = 0ull;
        for (int t = threadIdx.x; t < L2; t += blockDim.x) s_cnt[t] = 0u;
        __syncthreads();
        for (int64_t p = start + threadIdx.x; p < end; p += blockDim.x) {
            const int f = fasg[p];
            const float *zp = z + (size_t)perm1[p] * 12;
#pragma unroll
            for (int k = 0; k < 12; ++k) atomicAdd(s_sum + f * 12 + k, to_fixed(zp[k], fs));
            atomicAdd(s_cnt + f, 1u);
        }
        __syncthreads();
        const int64_t leaf0 = (int64_t)c * L2;
        for (int t = threadIdx.x; t < L2; t += blockDim.x) {
            const unsigned k = s_cnt[t];
            if (!k) continue;
            atomicAdd(cnt + leaf0 + t, k);
#pragma unroll
            for (int a = 0; a < 12; ++a) atomicAdd(sums + (leaf0 + t) * 12 + a, s_sum[t * 12 + a]);
        }
        __syncthreads();
        start = end;
    }
}

__global__ void k_leaf_of(const int32_t *__restrict__ perm1, const int32_t *__restrict__ c1s,
                          const int32_t *__restrict__ fasg, int64_t n, int L2, int32_t *__restrict__ leaf_of) {
    int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p < n) leaf_of[perm1[p]] = c1s[p] * L2 + fasg[p];
}

__global__ void k_radius_orig(const float *__restrict__ z, const int32_t *__restrict__ asg, int64_t n,
                              const float *__restrict__ cent, unsigned *__restrict__ rbits) {
    int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= n) return;
    int c = asg[j];
    float q[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) q[k] = cent[(size_t)c * 12 + k];
    float d = sqrtf(dist2_12(z + j * 12, q));
    atomicMax(rbits + c, __float_as_uint(d * 1.000001f + 1e-30f));
}

struct Probe2Args {
    ProbeArgs A;                // leaves in A.radius / A.offs / A.zs / A.perm / A.cluster_of; cand_* are coarse cells
    const float *centf;         // [L x 12] leaf centroids
    const float *rad1;          // [L1] coarse radii
    const float *lrad1;         // [L1] largest leaf radius of every cell
    int L1, L2;
    float r1max;
    // leaf-major hand-off (all null: every leaf is scanned by the query's warp)
    int budget;                 // leaves a warp scans itself beyond the warm-start leaf
    int32_t *pair_leaf;         // [m x kPairMax] leaves left to the leaf-major scan
    int *n_pairs;               // [m]
    unsigned *leaf_cnt;         // [L] queries per leaf
};

constexpr int kFine = 8;        // leaves visited per cell at most
constexpr int kFinePerLane = 16;   // L2 <= 512
constexpr int kPairMax = kCand * kFine + 1;   // leaves a query can hand off (candidates + warm-start leaf)
constexpr int kLeafBudget = 2;                // default leaves a query's warp scans itself

__global__ void __launch_bounds__(256, 4) k_ann_probe2(Probe2Args P) {
    const ProbeArgs &A = P.A;
    const int lane = threadIdx.x & 31;
    const int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (i >= A.m) return;
    if (A.gated && A.cand_cl[i * kCand] == kGated) {   // kept by Eq. (14)
        if (lane == 0 && P.n_pairs) P.n_pairs[i] = 0;
        return;
    }
    float q[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) q[k] = A.rec[i].q[k];
    Best b{INFINITY, 0x7fffffff, INFINITY};
    int l0 = -1;
    unsigned long long scanned = 0;
    if (A.prev) {
        const int j0 = A.prev[i];
        if (j0 >= 0 && j0 < A.N) {
            const float d0 = dist2_12(A.z32 + (size_t)j0 * 12, q);
            if (A.mot_q) {
                float mv = 0.f;
#pragma unroll
                for (int k = 0; k < 12; ++k) {
                    float t = q[k] - A.mot_q[i * 12 + k];
                    mv = fmaf(t, t, mv);
                }
                mv = sqrtf(mv);
                const float4 r = *reinterpret_cast<const float4 *>(A.mot_d + i * kMotStride);
                const float fdi = A.fd_q ? A.fd_q[i] : A.f_d;
                if (mv < 0.5f * (r.y - r.x) && fdi <= r.z) {      // Eq. (14)
                    if (lane == 0) {
                        A.idx[i] = j0;
                        A.d1[i] = d0;
                        float lb = fmaxf(r.y - mv, 0.f);
                        A.d2[i] = lb * lb;
                        atomicAdd(A.counters + 1, 1ull);
                        if (P.n_pairs) P.n_pairs[i] = 0;
                    }
                    return;
                }
            }
            b.d = d0;
            b.j = j0;
            l0 = A.cluster_of[j0];
        }
    }
    auto scan = [&](int l) {
        const int64_t p0 = A.offs[l], p1 = A.offs[l + 1];
        scan_range(A.zs, A.perm, p0, p1, lane, q, b);
        scanned += (unsigned long long)(p1 - p0);
        if (lane == 0) atomicOr(A.touched + (l >> 5), 1u << (l & 31));
        best_warp(b);
    };
    int nscan = 0, npair = 0;
    if (l0 >= 0) {
        if (!P.pair_leaf || P.budget > 0) {
            scan(l0);
            ++nscan;
        } else {
            // no leaf in the warp: the warm-start leaf goes leaf-major too
            if (lane == 0) {
                P.pair_leaf[i * kPairMax + npair] = l0;
                atomicAdd(P.leaf_cnt + l0, 1u);
            }
            ++npair;
        }
    }
    float dc = sqrtf(b.d);
    const float f_d = A.fd_q ? A.fd_q[i] : A.f_d;
    const bool cert = A.certified || f_d >= 1.0f;
    bool incomplete = false;
    // Eq. (14): plain lower bound on the points of the cells and leaves not
    // searched (per lane over its own leaves; warp minimum at the end)
    float lb = INFINITY;
    for (int k1 = 0; k1 < kCand; ++k1) {
        const int C = A.cand_cl[i * kCand + k1];
        if (C < 0) break;
        const float dC = A.cand_d[i * kCand + k1];
        if (!(k1 == 0 || dC - f_d * P.rad1[C] < dc)) {
            // a cell made of the warm-start leaf alone was searched
            if (cert && !(P.L2 == 1 && C == l0)) lb = fminf(lb, dC - f_d * P.rad1[C]);
            continue;
        }
        // rank the cell's leaves: lane holds leaves f = lane + 32 t (squared
        // centroid distances; the plain distance is taken of the chosen ones)
        float fd[kFinePerLane];
        unsigned vis = 0, srch = 0;
        const float cell_lr = P.lrad1[C];
#pragma unroll
        for (int t = 0; t < kFinePerLane; ++t) {
            const int f = lane + 32 * t;
            fd[t] = (f < P.L2) ? dist2_12(P.centf + ((size_t)C * P.L2 + f) * 12, q) : INFINITY;
        }
        if (lane == 0) atomicAdd(A.counters + 3, (unsigned long long)P.L2);
        for (int k2 = 0; k2 < kFine; ++k2) {
            float md = INFINITY;
            int mt = -1;
#pragma unroll
            for (int t = 0; t < kFinePerLane; ++t)
                if (!((vis >> t) & 1u) && fd[t] < md) {
                    md = fd[t];
                    mt = t;
                }
            int ml = mt >= 0 ? lane + 32 * mt : 0x7fffffff;
            for (int o = 16; o > 0; o >>= 1) {
                float od = __shfl_xor_sync(0xffffffffu, md, o);
                int ol = __shfl_xor_sync(0xffffffffu, ml, o);
                if (od < md || (od == md && ol < ml)) {
                    md = od;
                    ml = ol;
                }
            }
            if (!(md < INFINITY)) break;
            md = sqrtf(md);
            // the remaining leaves of the cell are no nearer and no wider than
            // the cell's widest: none can pass Eq. (13) with this d_c or a
            // smaller one (exact requests keep the ordered walk)
            if (f_d < 1.0f && !(k1 == 0 && k2 == 0) && md - f_d * cell_lr >= dc) break;
            if ((ml & 31) == lane) vis |= 1u << (ml >> 5);
            const int l = C * P.L2 + ml;
            if ((k1 == 0 && k2 == 0) || md - f_d * A.radius[l] < dc) {
                if ((ml & 31) == lane) srch |= 1u << (ml >> 5);
                if (l != l0) {
                    if (!P.pair_leaf || nscan < P.budget) {
                        scan(l);
                        dc = sqrtf(b.d);
                        ++nscan;
                    } else if (A.offs[l + 1] > A.offs[l]) {
                        // hand the leaf to the leaf-major scan (Eq. 13 tested with the current d_c)
                        if (lane == 0) {
                            P.pair_leaf[i * kPairMax + npair] = l;
                            atomicAdd(P.leaf_cnt + l, 1u);
                        }
                        ++npair;
                    }
                }
            }
        }
        // Eq. (14) bound of the cell's leaves not searched (each with its own
        // radius).  A leaf can lower X = min(second read, bound so far) only
        // if its centroid is nearer than X + f_d times the cell's widest leaf
        // radius, so the others are passed over without their radius.
        if (cert) {
            const float X = fminf(sqrtf(b.s), lb);
            const float thr = X + f_d * cell_lr;
            const float thr2 = thr > 0.f ? thr * thr : 0.f;
#pragma unroll
            for (int t = 0; t < kFinePerLane; ++t) {
                const int f = lane + 32 * t;
                if (f < P.L2 && !((srch >> t) & 1u) && fd[t] < thr2) {
                    const int l = C * P.L2 + f;
                    if (l != l0) lb = fminf(lb, sqrtf(fd[t]) - f_d * A.radius[l]);
                }
            }
        }
        // leaves of this cell beyond the kFine nearest (exact requests only)
        if (f_d >= 1.0f && P.L2 > kFine) {
            float md = INFINITY;
#pragma unroll
            for (int t = 0; t < kFinePerLane; ++t)
                if (!((vis >> t) & 1u)) md = fminf(md, fd[t]);
            for (int o = 16; o > 0; o >>= 1) md = fminf(md, __shfl_xor_sync(0xffffffffu, md, o));
            if (sqrtf(md) - f_d * A.rmax < dc) incomplete = true;
        }
    }
    if (f_d >= 1.0f && P.L1 > kCand) {
        const float dP = A.cand_d[i * kCand + kCand - 1];
        if (dP - f_d * P.r1max < dc) incomplete = true;
    }
    // cells beyond the candidate list: no nearer centroid, no wider radius
    if (cert && P.L1 > kCand) lb = fminf(lb, A.cand_d[i * kCand + kCand - 1] - f_d * P.r1max);
    for (int o = 16; o > 0; o >>= 1) lb = fminf(lb, __shfl_xor_sync(0xffffffffu, lb, o));
    if (lane == 0) {
        atomicAdd(A.counters, scanned);
        atomicAdd(A.counters + 5, scanned);
        if (incomplete) {
            unsigned long long t = atomicAdd(A.fb_count, 1ull);
            A.fb_list[t] = i;
        }
        A.idx[i] = b.j;
        A.d1[i] = b.d;
        A.d2[i] = fminf(b.s, lb > 0.f ? lb * lb : 0.f);
        if (P.n_pairs) P.n_pairs[i] = npair;
    }
}

// ---------------------------------------------------------------------------
// Leaf-major scan of the handed-off (leaf, query) pairs: the pairs are bucketed
// by leaf (counting sort), and one warp takes up to 32 queries of one leaf, a
// lane per query, reading each point of the leaf once for all of them.
// ---------------------------------------------------------------------------
constexpr int kScanBlock = 1024;   // leaves per block of the count scans
constexpr int kLeafChunk = 64;     // queries of a leaf per warp of the leaf-major scan

// Inclusive block scan of 1024 values (256 threads x 4); returns the
// exclusive prefix of this thread's first value, the block total in *tot.
__device__ __forceinline__ unsigned block_scan4(unsigned (&v)[4], unsigned *sh, unsigned *tot) {
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    unsigned s = v[0] + v[1] + v[2] + v[3];
    unsigned x = s;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[w] = x;
    __syncthreads();
    if (w == 0) {
        unsigned z = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0u;
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, z, o);
            if (lane >= o) z += y;
        }
        if (lane < (int)(blockDim.x >> 5)) sh[lane] = z;
    }
    __syncthreads();
    const unsigned before = (w ? sh[w - 1] : 0u) + x - s;
    *tot = sh[(blockDim.x >> 5) - 1];
    __syncthreads();
    return before;
}

// per block of 1024 leaves: totals of queries and of kLeafChunk-query chunks
__global__ void __launch_bounds__(256) k_leaf_sums(const unsigned *__restrict__ cnt, int L,
                                                    unsigned *__restrict__ bsum, unsigned *__restrict__ bitem) {
    __shared__ unsigned sh[8];
    const int base = blockIdx.x * kScanBlock + threadIdx.x * 4;
    unsigned a[4], c[4], ta, tc;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        a[k] = base + k < L ? cnt[base + k] : 0u;
        c[k] = (a[k] + (unsigned)kLeafChunk - 1u) / (unsigned)kLeafChunk;
    }
    block_scan4(a, sh, &ta);
    block_scan4(c, sh, &tc);
    if (threadIdx.x == 0) {
        bsum[blockIdx.x] = ta;
        bitem[blockIdx.x] = tc;
    }
}

// exclusive scan of the block totals (one block; nb <= 4096)
__global__ void __launch_bounds__(1024) k_leaf_sums_top(unsigned *__restrict__ bsum, unsigned *__restrict__ bitem,
                                                        int nb) {
    __shared__ unsigned sh[32];
    for (int which = 0; which < 2; ++which) {
        unsigned *a = which ? bitem : bsum;
        unsigned v[4], tot;
        const int base = threadIdx.x * 4;
#pragma unroll
        for (int k = 0; k < 4; ++k) v[k] = base + k < nb ? a[base + k] : 0u;
        unsigned run = block_scan4(v, sh, &tot);
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (base + k < nb) {
                const unsigned x = v[k];
                a[base + k] = run;
                run += x;
            }
        __syncthreads();
    }
}

// per-leaf exclusive offsets of pairs and chunks; entry L holds the totals
__global__ void __launch_bounds__(256) k_leaf_offsets(const unsigned *__restrict__ cnt, int L,
                                                       const unsigned *__restrict__ bsum,
                                                       const unsigned *__restrict__ bitem,
                                                       unsigned *__restrict__ pair_off, unsigned *__restrict__ item_off) {
    __shared__ unsigned sh[8];
    const int base = blockIdx.x * kScanBlock + threadIdx.x * 4;
    unsigned a[4], c[4], ta, tc;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        a[k] = base + k < L ? cnt[base + k] : 0u;
        c[k] = (a[k] + (unsigned)kLeafChunk - 1u) / (unsigned)kLeafChunk;
    }
    unsigned ra = block_scan4(a, sh, &ta) + bsum[blockIdx.x];
    unsigned rc = block_scan4(c, sh, &tc) + bitem[blockIdx.x];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (base + k < L) {
            pair_off[base + k] = ra;
            item_off[base + k] = rc;
        }
        if (base + k == L - 1) {
            pair_off[L] = ra + a[k];
            item_off[L] = rc + c[k];
        }
        ra += a[k];
        rc += c[k];
    }
}

// bucket every handed-off pair by its leaf: bucket holds the pair slot
// i * kPairMax + t (query i = slot / kPairMax)
__global__ void k_pair_scatter(const int32_t *__restrict__ pair_leaf, const int *__restrict__ n_pairs, int64_t m,
                               const unsigned *__restrict__ pair_off, unsigned *__restrict__ cursor,
                               unsigned *__restrict__ bucket) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= m) return;
    const int n = n_pairs[i];
    for (int t = 0; t < n; ++t) {
        const int l = pair_leaf[i * kPairMax + t];
        bucket[pair_off[l] + atomicAdd(cursor + l, 1u)] = (unsigned)(i * kPairMax + t);
    }
}

struct PairRes {
    float d1;       // best squared distance in the leaf
    int p1;         // its sorted position
    float d2;       // second best
};

struct LeafScanArgs {
    const float *zs;
    const float *cent;          // [L x 12] leaf centroids
    const int64_t *offs;
    const QueryRec *rec;
    const unsigned *bucket, *pair_off, *item_off;
    int L;
    PairRes *res;               // [m x kPairMax]
    unsigned long long *counters;
    unsigned *touched;
};

// best and second best of the points [p0, p1) for one query
struct LeafBest {
    float b1 = INFINITY, b2 = INFINITY;
    int j1 = 0x7fffffff;
    __device__ __forceinline__ void offer(float d, int p) {
        if (d < b1) {
            b2 = b1;
            b1 = d;
            j1 = p;
        } else {
            b2 = fminf(b2, d);
        }
    }
};

// One warp per chunk of up to 64 queries of a leaf: lane l takes queries l
// and l + 32, so every point read serves two distances.  A chunk of at most
// 16 queries (a leaf few queries reach, typical of the first DD iterations)
// gives each query several lanes, which split the points.
//
// Distances in the leaf's own frame: the warp stages 32 points at a time in
// shared memory as x' = x - c (c the leaf's centroid) with |x'|^2, and a
// query q' = q - c scores |x'|^2 - 2 x'.q' (12 FMA against the direct form's
// 12 differences and 12 FMA); |q'|^2 is added to the best two at the end.
// In the leaf's frame the magnitudes are those of the leaf and of the query's
// distance to it, so the expanded form keeps the direct form's precision.
constexpr int kStagePts = 32;   // points a warp stages at a time

__global__ void __launch_bounds__(256, 3) k_leaf_scan(LeafScanArgs A) {
    __shared__ unsigned long long sc;
    __shared__ __align__(16) float4 sx[8][kStagePts][4];   // per warp: x' (3 float4) and |x'|^2
    __shared__ __align__(16) float4 scen[8][3];            // per warp: the leaf's centroid
    if (threadIdx.x == 0) sc = 0ull;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    float4(*const px)[4] = sx[threadIdx.x >> 5];
    float4 *const pc = scen[threadIdx.x >> 5];
    const unsigned nw = (gridDim.x * blockDim.x) >> 5;
    const unsigned total = A.item_off[A.L];
    for (unsigned it = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; it < total; it += nw) {
        // the leaf of this chunk: item_off[l] <= it < item_off[l + 1]
        int lo = 0, hi = A.L;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (A.item_off[mid] <= it) lo = mid;
            else hi = mid;
        }
        const int l = lo;
        const unsigned q0 = A.pair_off[l] + (unsigned)kLeafChunk * (it - A.item_off[l]);
        const unsigned qn = min((unsigned)kLeafChunk, A.pair_off[l + 1] - q0);
        const bool two = qn > 32u;                      // warp-uniform
        // at most 16 queries: G lanes per query (G a power of two, qn * G <=
        // 32), each taking every G-th point; the partial results are merged
        const int G = qn <= 1u ? 32 : qn <= 2u ? 16 : qn <= 4u ? 8 : qn <= 8u ? 4 : qn <= 16u ? 2 : 1;
        const unsigned slot = (unsigned)(lane / G), sub = (unsigned)(lane & (G - 1));
        const bool act0 = slot < qn, act1 = (unsigned)lane + 32u < qn;
        const unsigned s0 = act0 ? A.bucket[q0 + slot] : 0u, s1 = act1 ? A.bucket[q0 + 32 + lane] : 0u;
        const QueryRec *ra = A.rec + (act0 ? s0 / kPairMax : 0), *rb = A.rec + (act1 ? s1 / kPairMax : 0);
        __syncwarp();   // the previous chunk's reads of the centroid are done
        if (lane < 3) pc[lane] = __ldg(reinterpret_cast<const float4 *>(A.cent + (size_t)l * 12) + lane);
        __syncwarp();
        float ma[12], mb[12];   // -2 q' of the lane's queries
        float qna = 0.f, qnb = 0.f;
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            const float ck = reinterpret_cast<const float *>(pc)[k];
            const float ua = ra->q[k] - ck, ub = rb->q[k] - ck;
            ma[k] = -2.f * ua;
            mb[k] = -2.f * ub;
            qna = fmaf(ua, ua, qna);
            qnb = fmaf(ub, ub, qnb);
        }
        const int64_t p0 = A.offs[l], p1 = A.offs[l + 1];
        const int n = (int)(p1 - p0);
        LeafBest ba, bb;   // scores |x'|^2 - 2 x'.q' until |q'|^2 is added
        for (int t0 = 0; t0 < n; t0 += kStagePts) {
            const int nc = min(kStagePts, n - t0);
            __syncwarp();
            if (lane < nc) {
                const float4 *v = reinterpret_cast<const float4 *>(A.zs + (size_t)(p0 + t0 + lane) * 12);
                const float4 u0 = __ldg(v), u1 = __ldg(v + 1), u2 = __ldg(v + 2);
                const float4 e0 = pc[0], e1 = pc[1], e2 = pc[2];
                const float4 w0 = make_float4(u0.x - e0.x, u0.y - e0.y, u0.z - e0.z, u0.w - e0.w);
                const float4 w1 = make_float4(u1.x - e1.x, u1.y - e1.y, u1.z - e1.z, u1.w - e1.w);
                const float4 w2 = make_float4(u2.x - e2.x, u2.y - e2.y, u2.z - e2.z, u2.w - e2.w);
                float nx = 0.f;
                nx = fmaf(w0.x, w0.x, nx); nx = fmaf(w0.y, w0.y, nx); nx = fmaf(w0.z, w0.z, nx); nx = fmaf(w0.w, w0.w, nx);
                nx = fmaf(w1.x, w1.x, nx); nx = fmaf(w1.y, w1.y, nx); nx = fmaf(w1.z, w1.z, nx); nx = fmaf(w1.w, w1.w, nx);
                nx = fmaf(w2.x, w2.x, nx); nx = fmaf(w2.y, w2.y, nx); nx = fmaf(w2.z, w2.z, nx); nx = fmaf(w2.w, w2.w, nx);
                px[lane][0] = w0;
                px[lane][1] = w1;
                px[lane][2] = w2;
                px[lane][3] = make_float4(nx, 0.f, 0.f, 0.f);
            }
            __syncwarp();
            auto score = [&](const float (&m)[12], const float4 &w0, const float4 &w1, const float4 &w2, float nx) {
                float s = nx;
                s = fmaf(m[0], w0.x, s); s = fmaf(m[1], w0.y, s); s = fmaf(m[2], w0.z, s); s = fmaf(m[3], w0.w, s);
                s = fmaf(m[4], w1.x, s); s = fmaf(m[5], w1.y, s); s = fmaf(m[6], w1.z, s); s = fmaf(m[7], w1.w, s);
                s = fmaf(m[8], w2.x, s); s = fmaf(m[9], w2.y, s); s = fmaf(m[10], w2.z, s); s = fmaf(m[11], w2.w, s);
                return s;
            };
            if (two) {
                for (int t = 0; t < nc; ++t) {
                    const float4 w0 = px[t][0], w1 = px[t][1], w2 = px[t][2];
                    const float nx = px[t][3].x;
                    ba.offer(score(ma, w0, w1, w2, nx), (int)p0 + t0 + t);
                    bb.offer(score(mb, w0, w1, w2, nx), (int)p0 + t0 + t);
                }
            } else {
                for (int t = (int)sub; t < nc; t += G)
                    ba.offer(score(ma, px[t][0], px[t][1], px[t][2], px[t][3].x), (int)p0 + t0 + t);
            }
        }
        // back to squared distances (rounding can take a score below -|q'|^2)
        ba.b1 = fmaxf(ba.b1 + qna, 0.f);
        ba.b2 = fmaxf(ba.b2 + qna, 0.f);
        bb.b1 = fmaxf(bb.b1 + qnb, 0.f);
        bb.b2 = fmaxf(bb.b2 + qnb, 0.f);
        if (!two) {
            // merge the G partial results of a query (ties to the lower point;
            // the second distance is the second smallest of all points read)
            for (int o = 1; o < G; o <<= 1) {
                const float o1 = __shfl_xor_sync(0xffffffffu, ba.b1, o), o2 = __shfl_xor_sync(0xffffffffu, ba.b2, o);
                const int oj = __shfl_xor_sync(0xffffffffu, ba.j1, o);
                if (o1 < ba.b1 || (o1 == ba.b1 && oj < ba.j1)) {
                    ba.b2 = fminf(ba.b1, o2);
                    ba.b1 = o1;
                    ba.j1 = oj;
                } else {
                    ba.b2 = fminf(ba.b2, o1);
                }
            }
        }
        if (act0 && sub == 0u) A.res[s0] = PairRes{ba.b1, ba.j1, ba.b2};
        if (act1) A.res[s1] = PairRes{bb.b1, bb.j1, bb.b2};
        if (lane == 0) {
            atomicOr(A.touched + (l >> 5), 1u << (l & 31));
            atomicAdd(&sc, (unsigned long long)qn * (unsigned long long)n);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0 && sc) {
        atomicAdd(A.counters, sc);
        atomicAdd(A.counters + 5, sc);
    }
}

// fold the leaf-major results into every query's answer (ties to the lower
// data index; the second distance over all points read)
__global__ void k_pair_merge(const int *__restrict__ n_pairs, const PairRes *__restrict__ res,
                             const int32_t *__restrict__ perm, int64_t m, int32_t *__restrict__ idx,
                             float *__restrict__ d1, float *__restrict__ d2) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= m) return;
    const int n = n_pairs[i];
    if (!n) return;
    float bd = d1[i], bs = d2[i];
    int bj = idx[i];
    for (int t = 0; t < n; ++t) {
        const PairRes r = res[i * kPairMax + t];
        if (!(r.d1 < INFINITY)) continue;
        const int j = perm[r.p1];
        if (j == bj) {              // the warm-start point, met again in its handed-off leaf
            bs = fminf(bs, r.d2);
            continue;
        }
        if (r.d1 < bd || (r.d1 == bd && j < bj)) {
            bs = fminf(bs, bd);
            bd = r.d1;
            bj = j;
        } else {
            bs = fminf(bs, r.d1);
        }
        bs = fminf(bs, r.d2);
    }
    idx[i] = bj;
    d1[i] = bd;
    d2[i] = bs;
}

// Points in the clusters marked in the bitmap (the data a search must read
// at least once).
__global__ void k_touched_points(const unsigned *__restrict__ touched, int L, const int64_t *__restrict__ offs,
                                 unsigned long long *__restrict__ out) {
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long n = 0;
    if (w < (L + 31) / 32) {
        unsigned bits = touched[w];
        while (bits) {
            const int b = __ffs(bits) - 1;
            bits &= bits - 1;
            const int l = w * 32 + b;
            if (l < L) n += (unsigned long long)(offs[l + 1] - offs[l]);
        }
    }
    for (int o = 16; o > 0; o >>= 1) n += __shfl_xor_sync(0xffffffffu, n, o);
    if ((threadIdx.x & 31) == 0 && n) atomicAdd(out, n);
}

__global__ void k_motion_update(const QueryRec *__restrict__ rec, int64_t m, const double *__restrict__ d2,
                                const double *__restrict__ d2nd, float f_d, const float *__restrict__ fd_q,
                                int rule, float *__restrict__ mq, float *__restrict__ md) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= m) return;
#pragma unroll
    for (int k = 0; k < 12; ++k) mq[i * 12 + k] = rec[i].q[k];
    // Eq. 3 distances -> plain distances in the mapped coordinates (|dq|^2 = d_e^2 / 2);
    // the nearest one rounded up and the second rounded down (by more than the
    // FP32 rounding of the mapped coordinates and of the bounds) keep the test
    // conservative
    float4 r;
    r.x = (float)(sqrt(0.5 * d2[i]) * (1.0 + 1e-5));
    r.y = (float)(sqrt(0.5 * d2nd[i]) * (1.0 - 1e-5));
    // the f_d the record serves: a certified bound serves its own f_d and any
    // lower one; the second-best point found (rule 1, below f_d = 1) serves
    // every f_d below 1 and never an exact (f_d = 1) search
    const float fd = fd_q ? fd_q[i] : f_d;
    r.z = (rule == 1 && fd < 1.0f) ? 0.99999994f : fd;
    r.w = 0.f;
    *reinterpret_cast<float4 *>(md + i * kMotStride) = r;
}

__global__ void k_export_index(const float *__restrict__ cent, const float *__restrict__ radius, int L, MetricMaps M,
                               double *__restrict__ c_out, double *__restrict__ r_out) {
    int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= L) return;
    for (int k = 0; k < 12; ++k) c_out[(size_t)l * 12 + k] = (double)cent[(size_t)l * 12 + k] + M.mu[k];
    r_out[l] = radius[l];
}

__global__ void k_gather_queries(const double *__restrict__ y, const int64_t *__restrict__ list, int64_t n,
                                 double *__restrict__ ys) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n) return;
    const int64_t i = list[t];
#pragma unroll
    for (int k = 0; k < 12; ++k) ys[t * 12 + k] = y[i * 12 + k];
}

__global__ void k_scatter_results(const int64_t *__restrict__ list, int64_t n, const int32_t *__restrict__ si,
                                  const double *__restrict__ sd, const double *__restrict__ sd2,
                                  int32_t *__restrict__ idx, double *__restrict__ d2, double *__restrict__ d2nd) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n) return;
    const int64_t i = list[t];
    idx[i] = si[t];
    if (d2) d2[i] = sd[t];
    if (d2nd) d2nd[i] = sd2[t];
}

}  // namespace

// Power-of-two scale of the fixed-point cluster sums: |z| fs <= 2^30, so the
// sum of up to 2^31 members stays below 2^61.
static double fixed_scale(double maxabs) {
    const double m = maxabs > 0 ? maxabs : 1.0;
    return std::ldexp(1.0, 30 - (int)std::ceil(std::log2(m)));
}

// Certified exact search (FP32 scan + FP64 rescoring) of the listed queries,
// with the exact second-nearest distance (the two nearest points), so that
// an exhaustively searched query records its true second distance for
// Eq. (14).
static dd_status ann_exact_subset(dd_dataset *ds, const double *y_dev, const int64_t *list, int64_t n, SearchOut out,
                                  cudaStream_t s) {
    dd_ctx *ctx = ds->ctx;
    auto r256 = [](size_t b) { return (b + 255) / 256 * 256; };
    void *w = nullptr;
    DD_TRY(dd_workspace(ctx, WS_ANN_BUILD,
                        r256((size_t)n * 96) + r256((size_t)n * 4) + 2 * r256((size_t)n * 8) + r256((size_t)n * 8) +
                            r256((size_t)n * 16),
                        &w));
    char *c = (char *)w;
    double *ys = (double *)c;
    int32_t *si = (int32_t *)(c + r256((size_t)n * 96));
    double *sd = (double *)(c + r256((size_t)n * 96) + r256((size_t)n * 4));
    double *sd2 = (double *)(c + r256((size_t)n * 96) + r256((size_t)n * 4) + r256((size_t)n * 8));
    int32_t *tk = (int32_t *)(c + r256((size_t)n * 96) + r256((size_t)n * 4) + 2 * r256((size_t)n * 8));
    double *tkd = (double *)(c + r256((size_t)n * 96) + r256((size_t)n * 4) + 2 * r256((size_t)n * 8) +
                             r256((size_t)n * 8));
    ctx->launches += 2;
    k_gather_queries<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(y_dev, list, n, ys);
    DD_TRY_CUDA(ctx, cudaGetLastError());
    SearchOut so{si, sd, sd2};
    so.k = 2;
    so.topk_idx = tk;
    so.topk_d2 = tkd;
    DD_TRY(dd_search_exact_fp32(ds, ys, n, 1, so, nullptr, s));
    k_scatter_results<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(list, n, si, sd, sd2, out.idx, out.d2, out.d2nd);
    DD_TRY_CUDA(ctx, cudaGetLastError());
    return DD_OK;
}

dd_status dd_ann_motion_update(dd_ctx *ctx, const QueryRec *rec, int64_t m, const double *d2, const double *d2nd,
                               double f_d, const float *fd_q, int eq14, AnnMotion *mot, cudaStream_t s) {
    ctx->launches++;
    k_motion_update<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(rec, m, d2, d2nd, (float)f_d, fd_q, eq14,
                                                                 mot->q, mot->d);
    DD_TRY_CUDA(ctx, cudaGetLastError());
    return DD_OK;
}

extern "C" int dd_dataset_ann_nlist(const dd_dataset *ds) { return ds ? ds->ann.nlist : 0; }

extern "C" dd_status dd_dataset_ann_index(dd_dataset *ds, int32_t *cluster_of, double *centroids, double *radii) {
    if (!ds) return DD_ERR_ARG;
    dd_ctx *ctx = ds->ctx;
    AnnIndex &a = ds->ann;
    if (!a.nlist) return dd_fail(ctx, DD_ERR_STATE, "dd_dataset_ann_index: no partition built");
    DD_TRY_CUDA(ctx, cudaSetDevice(ctx->device));
    cudaStream_t s = ctx->stream;
    if (cluster_of)
        DD_TRY_CUDA(ctx, cudaMemcpyAsync(cluster_of, a.cluster_of, (size_t)ds->N * 4, cudaMemcpyDeviceToHost, s));
    if (centroids || radii) {
        void *w = nullptr;
        DD_TRY(dd_workspace(ctx, WS_MISC, (size_t)a.nlist * 13 * 8 + 256, &w));
        double *c = (double *)w, *r = c + (size_t)a.nlist * 12;
        ctx->launches++;
        k_export_index<<<(a.nlist + 255) / 256, 256, 0, s>>>(a.cent, a.radius, a.nlist, ds->M, c, r);
        DD_TRY_CUDA(ctx, cudaGetLastError());
        if (centroids)
            DD_TRY_CUDA(ctx, cudaMemcpyAsync(centroids, c, (size_t)a.nlist * 96, cudaMemcpyDeviceToHost, s));
        if (radii) DD_TRY_CUDA(ctx, cudaMemcpyAsync(radii, r, (size_t)a.nlist * 8, cudaMemcpyDeviceToHost, s));
    }
    DD_TRY_CUDA(ctx, cudaStreamSynchronize(s));
    return DD_OK;
}

extern "C" int64_t dd_dataset_ann_build_fallback(const dd_dataset *ds) { return ds ? ds->ann.build_fallback : 0; }

extern "C" dd_status dd_dataset_ann_cells(dd_dataset *ds, int32_t *L1, int32_t *L2, double *centroids,
                                          double *radii) {
    if (!ds) return DD_ERR_ARG;
    dd_ctx *ctx = ds->ctx;
    AnnIndex &a = ds->ann;
    if (!a.nlist || a.levels != 2) return dd_fail(ctx, DD_ERR_STATE, "dd_dataset_ann_cells: no two-level partition");
    if (L1) *L1 = a.L1;
    if (L2) *L2 = a.L2;
    DD_TRY_CUDA(ctx, cudaSetDevice(ctx->device));
    cudaStream_t s = ctx->stream;
    if (centroids || radii) {
        void *w = nullptr;
        DD_TRY(dd_workspace(ctx, WS_MISC, (size_t)a.L1 * 13 * 8 + 256, &w));
        double *c = (double *)w, *r = c + (size_t)a.L1 * 12;
        ctx->launches++;
        k_export_index<<<(a.L1 + 255) / 256, 256, 0, s>>>(a.cent1, a.rad1, a.L1, ds->M, c, r);
        DD_TRY_CUDA(ctx, cudaGetLastError());
        if (centroids)
            DD_TRY_CUDA(ctx, cudaMemcpyAsync(centroids, c, (size_t)a.L1 * 96, cudaMemcpyDeviceToHost, s));
        if (radii) DD_TRY_CUDA(ctx, cudaMemcpyAsync(radii, r, (size_t)a.L1 * 8, cudaMemcpyDeviceToHost, s));
    }
    DD_TRY_CUDA(ctx, cudaStreamSynchronize(s));
    return DD_OK;
}

void dd_free_ann(dd_dataset *ds) {
    AnnIndex &a = ds->ann;
    if (!a.nlist) return;
    dd_ctx *ctx = ds->ctx;
    size_t Lp = (size_t)(a.nlist + 255) / 256 * 256;
    dd_free(ctx, a.cent, Lp * 48);
    dd_free(ctx, a.cn, Lp * 4);
    dd_free(ctx, a.radius, Lp * 4);
    dd_free(ctx, a.offs, (Lp + 1) * 8);
    dd_free(ctx, a.perm, (size_t)ds->N * 4);
    dd_free(ctx, a.cluster_of, (size_t)ds->N * 4);
    dd_free(ctx, a.zs, (size_t)ds->N * 48);
    if (a.levels == 2) {
        size_t L1p = (size_t)(a.L1 + 255) / 256 * 256;
        dd_free(ctx, a.cent1, L1p * 48);
        dd_free(ctx, a.cn1, L1p * 4);
        dd_free(ctx, a.rad1, L1p * 4);
        if (a.lrad1) dd_free(ctx, a.lrad1, L1p * 4);
    }
    dd_near_tc_free(ctx, &a.rank_tc);
    a = AnnIndex();
}

static dd_status build_tree2(dd_dataset *ds, const dd_dataset_opts &o);

// The nearest-centroid passes of a build.  The assignment to the cells runs
// on the tensor cores (near_tc.cu, the same answers) unless the options ask
// for the ALU or the cells are a handful; the rows that the tensor-core
// scores leave open are finished by the ALU kernel.
struct BuildNear {
    dd_ctx *ctx = nullptr;
    bool tc = false;
    double s = 0.0;
    float R = 0.f;
    NearTcSet C;
    int32_t *fb = nullptr;
    unsigned *fb_n = nullptr;
    int64_t cap = 0;
    int64_t fallback = 0;

    dd_status init(dd_dataset *ds, const dd_dataset_opts &o) {
        ctx = ds->ctx;
        tc = o.ann_alu == 0;
        if (!tc) return DD_OK;
        s = dd_tc_scale(ds->maxabs);
        R = (float)(ds->R * (1.0 + 1e-6));
        cap = std::min<int64_t>(ds->N, (int64_t)1 << 24);
        void *p = nullptr;
        DD_TRY(dd_alloc(ctx, &p, (size_t)cap * 4 + 256, "build fallback list"));
        fb = (int32_t *)p;
        fb_n = (unsigned *)((char *)p + (size_t)cap * 4);
        return DD_OK;
    }
    void release() {
        if (fb) dd_free(ctx, fb, (size_t)cap * 4 + 256);
        fb = nullptr;
        if (ctx) dd_near_tc_free(ctx, &C);
    }
    ~BuildNear() { release(); }
    // rows the tensor-core pass left open (host count; synchronous)
    dd_status open_rows(cudaStream_t st, int64_t *n) {
        unsigned h = 0;
        DD_TRY_CUDA(ctx, cudaMemcpyAsync(&h, fb_n, 4, cudaMemcpyDeviceToHost, st));
        DD_TRY_CUDA(ctx, cudaStreamSynchronize(st));
        *n = h;
        fallback += h;
        return DD_OK;
    }
    // out[j] = nearest of the L centroids to z[j], j < n
    dd_status assign(const float *z, int64_t n, const float *cent, const float *cn, int L, int32_t *out,
                     cudaStream_t st) {
        if (n == 0) return DD_OK;
        const unsigned g = (unsigned)((n + 255) / 256);
        if (!tc || L < 16) {   // a handful of centroids: the ALU kernel
            ctx->launches++;
            k_assign<<<g, 256, 0, st>>>(z, n, cent, cn, L, out, nullptr, nullptr);
            DD_TRY_CUDA(ctx, cudaGetLastError());
            return DD_OK;
        }
        DD_TRY(dd_near_tc_operands(ctx, cent, cn, L, s, R, &C, st));
        DD_TRY_CUDA(ctx, cudaMemsetAsync(fb_n, 0, 4, st));
        DD_TRY(dd_near_tc_assign(ctx, C, z, n, out, fb, fb_n, cap, st));
        int64_t nf = 0;
        DD_TRY(open_rows(st, &nf));
        if (nf == 0) return DD_OK;
        ctx->launches++;
        if (nf > cap) k_assign<<<g, 256, 0, st>>>(z, n, cent, cn, L, out, nullptr, nullptr);
        else k_assign<<<(unsigned)((nf + 255) / 256), 256, 0, st>>>(z, n, cent, cn, L, out, fb, fb_n);
        DD_TRY_CUDA(ctx, cudaGetLastError());
        return DD_OK;
    }
    // fasg[p] = nearest of the L2 leaves of cell c1s[p] to z[perm1[p]] (on
    // the ALU: with four centroid tiles per 128 points the tensor-core
    // kernel was slower, 0.6 s per pass at 10^9 points against 0.38 s)
    dd_status assign_fine(const float *z, const int32_t *perm1, const int32_t *c1s, int64_t n, const float *cent,
                          const float *cn, int L2, int32_t *fasg, cudaStream_t st) {
        ctx->launches++;
        k_assign_fine<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(z, perm1, c1s, n, cent, cn, L2, fasg);
        DD_TRY_CUDA(ctx, cudaGetLastError());
        return DD_OK;
    }
};

// Tensor-core operands of the centroid set the search ranks (kept with the
// index; the ranking falls back to the ALU kernel without them).
static dd_status build_rank_operands(dd_dataset *ds, const dd_dataset_opts &o) {
    AnnIndex &a = ds->ann;
    const bool two = a.levels == 2;
    const int Lr = two ? a.L1 : a.nlist;
    if (o.ann_alu || Lr < 16 || Lr > kRankMax) return DD_OK;
    DD_TRY(dd_near_tc_operands(ds->ctx, two ? a.cent1 : a.cent, two ? a.cn1 : a.cn, Lr, dd_tc_scale(ds->maxabs),
                               (float)(ds->R * (1.0 + 1e-6)), &a.rank_tc, ds->ctx->stream));
    ds->bytes += (size_t)a.rank_tc.rows_pad * 64;
    return DD_OK;
}

dd_status dd_build_ann(dd_dataset *ds, const dd_dataset_opts &o) {
    if (o.ann_levels == 2) return build_tree2(ds, o);
    dd_ctx *ctx = ds->ctx;
    cudaStream_t s = ctx->stream;
    AnnIndex &a = ds->ann;
    const int L = o.ann_nlist;
    const int64_t N = ds->N;
    const int64_t Lp = (L + 255) / 256 * 256;
    int64_t S = o.ann_sample > 0 ? o.ann_sample : (int64_t)64 * L;
    S = std::max<int64_t>(std::min<int64_t>(S, N), L);
    const int iters = o.ann_train_iters > 0 ? o.ann_train_iters : 8;
    void *p = nullptr;
    a.nlist = L;
    DD_TRY(dd_alloc(ctx, &p, Lp * 48, "ANN centroids"));
    a.cent = (float *)p;
    DD_TRY(dd_alloc(ctx, &p, Lp * 4, "ANN centroid norms"));
    a.cn = (float *)p;
    DD_TRY(dd_alloc(ctx, &p, Lp * 4, "ANN radii"));
    a.radius = (float *)p;
    DD_TRY(dd_alloc(ctx, &p, (Lp + 1) * 8, "ANN offsets"));
    a.offs = (int64_t *)p;
    DD_TRY(dd_alloc(ctx, &p, (size_t)N * 4, "ANN permutation"));
    a.perm = (int32_t *)p;
    DD_TRY(dd_alloc(ctx, &p, (size_t)N * 4, "ANN cluster map"));
    a.cluster_of = (int32_t *)p;
    DD_TRY(dd_alloc(ctx, &p, (size_t)N * 48, "ANN sorted data"));
    a.zs = (float *)p;
    ds->bytes += Lp * 60 + (size_t)N * 56;

    // scratch: sample rows, sample assignment, sums, counts
    const size_t b_sample = (size_t)S * 48, b_asg = (size_t)std::max<int64_t>(S, N) * 4, b_sums = (size_t)Lp * 96,
                 b_cnt = (size_t)Lp * 4 + 256;
    void *w = nullptr;
    DD_TRY(dd_workspace(ctx, WS_ANN_BUILD, b_sample + b_asg + b_sums + b_cnt + 1024, &w));
    char *c = (char *)w;
    float *sample = (float *)c;
    int32_t *asg = (int32_t *)(c + (b_sample + 255) / 256 * 256);
    unsigned long long *sums = (unsigned long long *)((char *)asg + (b_asg + 255) / 256 * 256);
    const double fs = fixed_scale(ds->maxabs);
    unsigned *cnt = (unsigned *)((char *)sums + b_sums);

    ctx->launches++;
    k_gather_rows<<<(unsigned)((S + 255) / 256), 256, 0, s>>>(ds->z32, N, S, sample);
    DD_TRY_CUDA(ctx, cudaGetLastError());
    // initial centroids: L rows of the sample, evenly spaced; padding rows never win
    DD_TRY_CUDA(ctx, cudaMemsetAsync(a.cent, 0, Lp * 48, s));
    ctx->launches++;
    k_gather_rows<<<(unsigned)((L + 255) / 256), 256, 0, s>>>(sample, S, L, a.cent);
    DD_TRY_CUDA(ctx, cudaMemsetAsync(sums, 0, b_sums, s));
    DD_TRY_CUDA(ctx, cudaMemsetAsync(cnt, 0, (size_t)Lp * 4, s));
    ctx->launches++;
    k_update<<<(unsigned)((L + 255) / 256), 256, 0, s>>>(sums, cnt, fs, a.cent, a.cn, L);   // norms only
    BuildNear near;
    DD_TRY(near.init(ds, o));
    for (int it = 0; it < iters; ++it) {
        DD_TRY(near.assign(sample, S, a.cent, a.cn, L, asg, s));
        ctx->launches += 2;
        k_accum<<<(unsigned)((S + 255) / 256), 256, 0, s>>>(sample, S, asg, fs, sums, cnt);
        k_update<<<(unsigned)((L + 255) / 256), 256, 0, s>>>(sums, cnt, fs, a.cent, a.cn, L);
    }
    DD_TRY_CUDA(ctx, cudaGetLastError());
    // padding centroids: never selected by the scans
    if (Lp > L) {
        std::vector<float> big((size_t)(Lp - L), 1e30f);
        DD_TRY_CUDA(ctx, cudaMemcpyAsync(a.cn + L, big.data(), (Lp - L) * 4, cudaMemcpyHostToDevice, s));
        DD_TRY_CUDA(ctx, cudaStreamSynchronize(s));
    }
    // assignment of every point, counting sort
    DD_TRY(near.assign(ds->z32, N, a.cent, a.cn, L, asg, s));
    a.build_fallback = near.fallback;
    near.release();
    ctx->launches++;
    DD_TRY_CUDA(ctx, cudaMemsetAsync(cnt, 0, (size_t)Lp * 4, s));
    k_hist<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(asg, N, cnt);
    DD_TRY_CUDA(ctx, cudaGetLastError());
    std::vector<unsigned> hc(L);
    std::vector<int64_t> ho((size_t)Lp + 1, 0);
    DD_TRY_CUDA(ctx, cudaMemcpyAsync(hc.data(), cnt, (size_t)L * 4, cudaMemcpyDeviceToHost, s));
    DD_TRY_CUDA(ctx, cudaStreamSynchronize(s));
    for (int l = 0; l < L; ++l) ho[l + 1] = ho[l] + hc[l];
    for (int64_t l = L; l < Lp; ++l) ho[l + 1] = ho[l];
    DD_TRY_CUDA(ctx, cudaMemcpyAsync(a.offs, ho.data(), (Lp + 1) * 8, cudaMemcpyHostToDevice, s));
    DD_TRY_CUDA(ctx, cudaMemsetAsync(cnt, 0, (size_t)Lp * 4, s));
    DD_TRY_CUDA(ctx, cudaMemcpyAsync(a.cluster_of, asg, (size_t)N * 4, cudaMemcpyDeviceToDevice, s));
    ctx->launches += 2;
    k_scatter<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(ds->z32, asg, N, a.offs, cnt, a.zs, a.perm);
    DD_TRY_CUDA(ctx, cudaMemsetAsync(a.radius, 0, Lp * 4, s));
    k_radius<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(a.zs, a.perm, asg, N, a.cent, (unsigned *)a.radius);
    DD_TRY_CUDA(ctx, cudaGetLastError());
    std::vector<float> hr(L);
    DD_TRY_CUDA(ctx, cudaMemcpyAsync(hr.data(), a.radius, (size_t)L * 4, cudaMemcpyDeviceToHost, s));
    DD_TRY_CUDA(ctx, cudaStreamSynchronize(s));
    a.rmax = 0.f;
    int nonempty = 0;
    for (int l = 0; l < L; ++l) {
        a.rmax = std::max(a.rmax, hr[l]);
        nonempty += hc[l] > 0;
    }
    a.nonempty = nonempty;
    return build_rank_operands(ds, o);
}

// Two-level tree: coarse k-means cells (Lloyd on a sample), every cell split
// into L2 k-means leaves (Lloyd over the cell's members), points stored in
// leaf order.  Leaf C * L2 + f belongs to cell C.
static dd_status build_tree2(dd_dataset *ds, const dd_dataset_opts &o) {
    dd_ctx *ctx = ds->ctx;
    cudaStream_t s = ctx->stream;
    AnnIndex &a = ds->ann;
    const int64_t N = ds->N;
    int L1 = 1 << (int)std::lround(std::log2(std::sqrt((double)std::max(1, o.ann_nlist))));
    L1 = (int)std::max<int64_t>(1, std::min<int64_t>(L1, N));
    const int L2 = (int)std::min<int64_t>(512, std::max<int64_t>(1, (o.ann_nlist + L1 - 1) / L1));
    const int L = L1 * L2;
    const int64_t Lp = (L + 255) / 256 * 256, L1p = (L1 + 255) / 256 * 256;
    const int iters = o.ann_train_iters > 0 ? o.ann_train_iters : 8;
    int64_t S1 = o.ann_sample > 0 ? o.ann_sample : (int64_t)64 * L1;
    S1 = std::max<int64_t>(std::min<int64_t>(S1, N), L1);
    a.levels = 2;
    a.nlist = L;
    a.L1 = L1;
    a.L2 = L2;
    void *p = nullptr;
    DD_TRY(dd_alloc(ctx, &p, Lp * 48, "ANN leaf centroids"));
    a.cent = (float *)p;
    DD_TRY(dd_alloc(ctx, &p, Lp * 4, "ANN leaf norms"));
    a.cn = (float *)p;
    DD_TRY(dd_alloc(ctx, &p, Lp * 4, "ANN leaf radii"));
    a.radius = (float *)p;
    DD_TRY(dd_alloc(ctx, &p, (Lp + 1) * 8, "ANN offsets"));
    a.offs = (int64_t *)p;
    DD_TRY(dd_alloc(ctx, &p, (size_t)N * 4, "ANN permutation"));
    a.perm = (int32_t *)p;
    DD_TRY(dd_alloc(ctx, &p, (size_t)N * 4, "ANN leaf map"));
    a.cluster_of = (int32_t *)p;
    DD_TRY(dd_alloc(ctx, &p, (size_t)N * 48, "ANN sorted data"));
    a.zs = (float *)p;
    DD_TRY(dd_alloc(ctx, &p, L1p * 48, "ANN cell centroids"));
    a.cent1 = (float *)p;
    DD_TRY(dd_alloc(ctx, &p, L1p * 4, "ANN cell norms"));
    a.cn1 = (float *)p;
    DD_TRY(dd_alloc(ctx, &p, L1p * 4, "ANN cell radii"));
    a.rad1 = (float *)p;
    ds->bytes += Lp * 60 + (size_t)N * 56 + L1p * 56;

    auto r256 = [](size_t b) { return (b + 255) / 256 * 256; };
    const size_t b_sample = r256((size_t)S1 * 48), b_n = r256((size_t)N * 4), b_sums = r256((size_t)Lp * 96),
                 b_cnt = r256((size_t)Lp * 4), b_offs1 = r256((size_t)(L1p + 1) * 8);
    void *w = nullptr;
    DD_TRY(dd_workspace(ctx, WS_ANN_BUILD, b_sample + 4 * b_n + b_sums + b_cnt + b_offs1, &w));
    char *c = (char *)w;
    float *sample = (float *)c;
    int32_t *asg1 = (int32_t *)(c + b_sample);
    int32_t *perm1 = (int32_t *)(c + b_sample + b_n);
    int32_t *c1s = (int32_t *)(c + b_sample + 2 * b_n);
    int32_t *fasg = (int32_t *)(c + b_sample + 3 * b_n);
    unsigned long long *sums = (unsigned long long *)(c + b_sample + 4 * b_n);
    const double fs = fixed_scale(ds->maxabs);
    unsigned *cnt = (unsigned *)(c + b_sample + 4 * b_n + b_sums);
    int64_t *offs1 = (int64_t *)(c + b_sample + 4 * b_n + b_sums + b_cnt);
    const unsigned gN = (unsigned)((N + 255) / 256);

    // ---- coarse level ----
    ctx->launches += 2;
    k_gather_rows<<<(unsigned)((S1 + 255) / 256), 256, 0, s>>>(ds->z32, N, S1, sample);
    DD_TRY_CUDA(ctx, cudaMemsetAsync(a.cent1, 0, L1p * 48, s));
    k_gather_rows<<<(unsigned)((L1 + 255) / 256), 256, 0, s>>>(sample, S1, L1, a.cent1);
    DD_TRY_CUDA(ctx, cudaMemsetAsync(sums, 0, b_sums, s));
    DD_TRY_CUDA(ctx, cudaMemsetAsync(cnt, 0, b_cnt, s));
    ctx->launches++;
    k_update<<<(unsigned)((L1 + 255) / 256), 256, 0, s>>>(sums, cnt, fs, a.cent1, a.cn1, L1);
    BuildNear near;
    DD_TRY(near.init(ds, o));
    for (int it = 0; it < iters; ++it) {
        DD_TRY(near.assign(sample, S1, a.cent1, a.cn1, L1, asg1, s));
        ctx->launches += 2;
        k_accum<<<(unsigned)((S1 + 255) / 256), 256, 0, s>>>(sample, S1, asg1, fs, sums, cnt);
        k_update<<<(unsigned)((L1 + 255) / 256), 256, 0, s>>>(sums, cnt, fs, a.cent1, a.cn1, L1);
    }
    if (L1p > L1) {
        std::vector<float> big((size_t)(L1p - L1), 1e30f);
        DD_TRY_CUDA(ctx, cudaMemcpyAsync(a.cn1 + L1, big.data(), (L1p - L1) * 4, cudaMemcpyHostToDevice, s));
    }
    DD_TRY(near.assign(ds->z32, N, a.cent1, a.cn1, L1, asg1, s));
    ctx->launches++;
    DD_TRY_CUDA(ctx, cudaMemsetAsync(cnt, 0, b_cnt, s));
    k_hist<<<gN, 256, 0, s>>>(asg1, N, cnt);
    DD_TRY_CUDA(ctx, cudaGetLastError());
    std::vector<unsigned> hc1(L1);
    std::vector<int64_t> ho1((size_t)L1p + 1, 0);
    DD_TRY_CUDA(ctx, cudaMemcpyAsync(hc1.data(), cnt, (size_t)L1 * 4, cudaMemcpyDeviceToHost, s));
    DD_TRY_CUDA(ctx, cudaStreamSynchronize(s));
    for (int l = 0; l < L1; ++l) ho1[l + 1] = ho1[l] + hc1[l];
    for (int64_t l = L1; l < L1p; ++l) ho1[l + 1] = ho1[l];
    DD_TRY_CUDA(ctx, cudaMemcpyAsync(offs1, ho1.data(), (L1p + 1) * 8, cudaMemcpyHostToDevice, s));
    DD_TRY_CUDA(ctx, cudaMemsetAsync(cnt, 0, b_cnt, s));
    ctx->launches += 3;
    {
        // stable: the members of a cell in index order
        const int nchunk = (int)((N + kStableChunk - 1) / kStableChunk);
        void *wh = nullptr;
        DD_TRY(dd_workspace(ctx, WS_ANN_PAIRS, (size_t)nchunk * L1 * 4, &wh));
        unsigned *hist = (unsigned *)wh;
        ctx->launches += 2;
        k_chunk_hist<<<nchunk, 256, (size_t)L1 * 4, s>>>(asg1, N, L1, hist);
        k_chunk_offsets<<<(L1 + 255) / 256, 256, 0, s>>>(hist, nchunk, L1, offs1);
        k_stable_scatter<<<nchunk, 32, (size_t)L1 * 4, s>>>(asg1, N, L1, hist, perm1);
    }
    k_cell_sorted<<<gN, 256, 0, s>>>(perm1, asg1, N, c1s);
    // ---- leaves: Lloyd inside every cell ----
    k_fine_init<<<(unsigned)((L + 255) / 256), 256, 0, s>>>(ds->z32, perm1, offs1, L1, L2, a.cent1, a.cent);
    DD_TRY_CUDA(ctx, cudaMemsetAsync(sums, 0, b_sums, s));
    DD_TRY_CUDA(ctx, cudaMemsetAsync(cnt, 0, b_cnt, s));
    ctx->launches++;
    k_update<<<(unsigned)((L + 255) / 256), 256, 0, s>>>(sums, cnt, fs, a.cent, a.cn, L);
    const size_t accum_smem = (size_t)L2 * (12 * 8 + 4);
    if (near.tc && accum_smem <= 160 * 1024 && accum_smem > 48 * 1024)
        DD_TRY_CUDA(ctx, cudaFuncSetAttribute(k_accum_fine_run, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)accum_smem));
    for (int it = 0; it < iters; ++it) {
        DD_TRY(near.assign_fine(ds->z32, perm1, c1s, N, a.cent, a.cn, L2, fasg, s));
        ctx->launches += 2;
        if (near.tc && accum_smem <= 160 * 1024)
            k_accum_fine_run<<<(unsigned)((N + kAccumRun - 1) / kAccumRun), kAccumThreads, accum_smem, s>>>(
                ds->z32, perm1, c1s, fasg, N, L2, fs, sums, cnt);
        else
            k_accum_fine<<<gN, 256, 0, s>>>(ds->z32, perm1, c1s, fasg, N, L2, fs, sums, cnt);
        k_update<<<(unsigned)((L + 255) / 256), 256, 0, s>>>(sums, cnt, fs, a.cent, a.cn, L);
    }
    DD_TRY(near.assign_fine(ds->z32, perm1, c1s, N, a.cent, a.cn, L2, fasg, s));
    a.build_fallback = near.fallback;
    near.release();
    ctx->launches++;
    k_leaf_of<<<gN, 256, 0, s>>>(perm1, c1s, fasg, N, L2, a.cluster_of);
    // ---- leaf order, radii ----
    DD_TRY_CUDA(ctx, cudaMemsetAsync(cnt, 0, b_cnt, s));
    ctx->launches++;
    k_hist<<<gN, 256, 0, s>>>(a.cluster_of, N, cnt);
    DD_TRY_CUDA(ctx, cudaGetLastError());
    std::vector<unsigned> hc(L);
    std::vector<int64_t> ho((size_t)Lp + 1, 0);
    DD_TRY_CUDA(ctx, cudaMemcpyAsync(hc.data(), cnt, (size_t)L * 4, cudaMemcpyDeviceToHost, s));
    DD_TRY_CUDA(ctx, cudaStreamSynchronize(s));
    for (int l = 0; l < L; ++l) ho[l + 1] = ho[l] + hc[l];
    for (int64_t l = L; l < Lp; ++l) ho[l + 1] = ho[l];
    DD_TRY_CUDA(ctx, cudaMemcpyAsync(a.offs, ho.data(), (Lp + 1) * 8, cudaMemcpyHostToDevice, s));
    DD_TRY_CUDA(ctx, cudaMemsetAsync(cnt, 0, b_cnt, s));
    DD_TRY_CUDA(ctx, cudaMemsetAsync(a.radius, 0, Lp * 4, s));
    DD_TRY_CUDA(ctx, cudaMemsetAsync(a.rad1, 0, L1p * 4, s));
    ctx->launches += 3;
    k_scatter<<<gN, 256, 0, s>>>(ds->z32, a.cluster_of, N, a.offs, cnt, a.zs, a.perm);
    k_radius<<<gN, 256, 0, s>>>(a.zs, a.perm, a.cluster_of, N, a.cent, (unsigned *)a.radius);
    k_radius_orig<<<gN, 256, 0, s>>>(ds->z32, asg1, N, a.cent1, (unsigned *)a.rad1);
    DD_TRY_CUDA(ctx, cudaGetLastError());
    std::vector<float> hr(L), hr1(L1);
    DD_TRY_CUDA(ctx, cudaMemcpyAsync(hr.data(), a.radius, (size_t)L * 4, cudaMemcpyDeviceToHost, s));
    DD_TRY_CUDA(ctx, cudaMemcpyAsync(hr1.data(), a.rad1, (size_t)L1 * 4, cudaMemcpyDeviceToHost, s));
    DD_TRY_CUDA(ctx, cudaStreamSynchronize(s));
    a.rmax = 0.f;
    a.r1max = 0.f;
    a.nonempty = 0;
    for (int l = 0; l < L; ++l) {
        a.rmax = std::max(a.rmax, hr[l]);
        a.nonempty += hc[l] > 0;
    }
    for (int l = 0; l < L1; ++l) a.r1max = std::max(a.r1max, hr1[l]);
    // largest leaf radius per cell: no leaf of a cell can pass Eq. (13) once
    // its centroid distance minus f_d times this exceeds d_c
    {
        std::vector<float> lr((size_t)L1p, 0.f);
        for (int l = 0; l < L; ++l) lr[l / L2] = std::max(lr[l / L2], hr[l]);
        void *p = nullptr;
        DD_TRY(dd_alloc(ctx, &p, L1p * 4, "ANN cell leaf radii"));
        a.lrad1 = (float *)p;
        DD_TRY_CUDA(ctx, cudaMemcpy(a.lrad1, lr.data(), L1p * 4, cudaMemcpyHostToDevice));
    }
    return build_rank_operands(ds, o);
}

static bool rank_small(const AnnIndex &a) { return (a.levels == 2 ? a.L1 : a.nlist) <= kRankMax; }

// As dd_ann_rank_cells, for the *n_list queries of `list` only (list and
// n_list on the device; both null: every query).  A list needs the small
// centroid set (rank_small).
static dd_status ann_rank_listed(dd_dataset *ds, const QueryRec *rec, int64_t m, const int32_t *list,
                                 const unsigned *n_list, int32_t *cand_cl, float *cand_d, cudaStream_t s) {
    dd_ctx *ctx = ds->ctx;
    const AnnIndex &a = ds->ann;
    const bool two = a.levels == 2;
    const float *rank_cent = two ? a.cent1 : a.cent;
    const float *rank_cn = two ? a.cn1 : a.cn;
    const int Lr = two ? a.L1 : a.nlist;
    if (Lr <= kRankMax && a.rank_tc.hi) {
        // tensor cores; the queries their scores leave open go to the ALU kernel
        const size_t b_fb = ((size_t)m * 4 + 255) / 256 * 256;
        void *w = nullptr;
        DD_TRY(dd_workspace(ctx, WS_NEAR, b_fb + 256, &w));
        int32_t *fb = (int32_t *)w;
        unsigned *fb_n = (unsigned *)((char *)w + b_fb);
        DD_TRY_CUDA(ctx, cudaMemsetAsync(fb_n, 0, 4, s));
        DD_TRY(dd_near_tc_rank(ctx, a.rank_tc, rec, m, list, n_list, cand_cl, cand_d, fb, fb_n, s));
        ctx->launches++;
        k_rank_small<<<(unsigned)((m + 256 * kRankQ - 1) / (256 * kRankQ)), 256, 0, s>>>(
            rec, m, fb, fb_n, rank_cent, rank_cn, Lr, cand_cl, cand_d);
    } else if (Lr <= kRankMax) {
        ctx->launches++;
        k_rank_small<<<(unsigned)((m + 256 * kRankQ - 1) / (256 * kRankQ)), 256, 0, s>>>(
            rec, m, list, n_list, rank_cent, rank_cn, Lr, cand_cl, cand_d);
    } else {
        if (list) return dd_fail(ctx, DD_ERR_STATE, "cell ranking: a query list needs the small centroid set");
        int splits = 0, cap = 0;
        CandHeader *hdr = nullptr;
        float2 *cand = nullptr;
        DD_TRY(dd_scan_fp32_raw(ctx, rank_cent, rank_cn, Lr, rec, m, true, WS_ANN_SCAN, &splits, &cap, &hdr, &cand,
                                s));
        ctx->launches += 2;
        k_ann_cands<<<(unsigned)((m + 127) / 128), 128, 0, s>>>(hdr, cand, splits, cap, rec, m, rank_cent, cand_cl,
                                                                cand_d);
    }
    DD_TRY_CUDA(ctx, cudaGetLastError());
    return DD_OK;
}

dd_status dd_ann_rank_cells(dd_dataset *ds, const QueryRec *rec, int64_t m, int32_t *cand_cl, float *cand_d,
                            cudaStream_t s) {
    return ann_rank_listed(ds, rec, m, nullptr, nullptr, cand_cl, cand_d, s);
}

dd_status dd_ann_finish(dd_dataset *ds, const double *y_dev, int64_t m, const QueryRec *rec, int32_t *idx,
                        float *d2f, double *d2, double *d2nd, cudaStream_t s) {
    dd_ctx *ctx = ds->ctx;
    ctx->launches++;
    k_ann_finish<<<(unsigned)((m + 127) / 128), 128, 0, s>>>(ds->raw, ds->M, y_dev, m, idx, d2f, d2, d2nd, ds->z32,
                                                             ds->N, rec);
    DD_TRY_CUDA(ctx, cudaGetLastError());
    return DD_OK;
}

dd_status dd_search_ann(dd_dataset *ds, const double *y_dev, int64_t m, double f_d, const int32_t *prev_idx_dev,
                        int budget, SearchOut out, dd_search_stats *st, cudaStream_t s) {
    return dd_search_ann_motion(ds, y_dev, m, f_d, nullptr, prev_idx_dev, nullptr, budget, out, st, s);
}

dd_status dd_search_ann_motion(dd_dataset *ds, const double *y_dev, int64_t m, double f_d, const float *fd_q,
                               const int32_t *prev_idx_dev, AnnMotion *mot, int budget, SearchOut out,
                               dd_search_stats *st, cudaStream_t s, int eq14) {
    dd_ctx *ctx = ds->ctx;
    AnnIndex &a = ds->ann;
    if (m == 0) return DD_OK;
    auto r256 = [](size_t b) { return (b + 255) / 256 * 256; };
    const size_t b_rec = r256((size_t)m * sizeof(QueryRec)), b_cl = r256((size_t)m * kCand * 4),
                 b_cd = r256((size_t)m * kCand * 4), b_f = r256((size_t)m * 4), b_list = r256((size_t)m * 8),
                 b_bits = r256((size_t)(a.nlist + 31) / 32 * 4);
    void *w = nullptr;
    DD_TRY(dd_workspace(ctx, WS_ANN, b_rec + b_cl + b_cd + 3 * b_f + b_list + 256 + b_bits, &w));
    char *c = (char *)w;
    QueryRec *rec = (QueryRec *)c;
    int32_t *cand_cl = (int32_t *)(c + b_rec);
    float *cand_d = (float *)(c + b_rec + b_cl);
    float *d1f = (float *)(c + b_rec + b_cl + b_cd);
    float *d2f = (float *)(c + b_rec + b_cl + b_cd + b_f);
    int64_t *fb_list = (int64_t *)(c + b_rec + b_cl + b_cd + 2 * b_f);
    unsigned long long *counters = (unsigned long long *)(c + b_rec + b_cl + b_cd + 2 * b_f + b_list);
    unsigned *touched = (unsigned *)(c + b_rec + b_cl + b_cd + 2 * b_f + b_list + 256);
    int32_t *qlist = (int32_t *)(c + b_rec + b_cl + b_cd + 2 * b_f + b_list + 256 + b_bits);
    unsigned *n_list = (unsigned *)(counters + 8);
    DD_TRY_CUDA(ctx, cudaMemsetAsync(counters, 0, 128, s));
    DD_TRY_CUDA(ctx, cudaMemsetAsync(touched, 0, b_bits, s));

    DD_TRY(dd_map_queries(ds, y_dev, m, nullptr, rec, s));
    if (st) DD_TRY_CUDA(ctx, dd_event_record(ctx, ctx->ev_scan[0], s));
    const bool two = a.levels == 2;
    const int Lr = two ? a.L1 : a.nlist;
    // Eq. (14) ahead of the ranking: kept queries are neither ranked nor probed
    const bool gate = prev_idx_dev && mot && mot->q && rank_small(a);
    if (gate) {
        GateArgs G{rec,     m,        ds->N,    prev_idx_dev, ds->z32, mot->q, mot->d,   (float)f_d,
                   fd_q,    out.idx,  d1f,      d2f,          cand_cl, qlist,  n_list, counters, Lr};
        ctx->launches++;
        k_ann_gate<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(G);
        DD_TRY_CUDA(ctx, cudaGetLastError());
    }
    DD_TRY(ann_rank_listed(ds, rec, m, gate ? qlist : nullptr, gate ? n_list : nullptr, cand_cl, cand_d, s));
    ProbeArgs A;
    A.zs = a.zs;
    A.perm = a.perm;
    A.offs = a.offs;
    A.radius = a.radius;
    A.cluster_of = a.cluster_of;
    A.z32 = ds->z32;
    A.rec = rec;
    A.cand_cl = cand_cl;
    A.cand_d = cand_d;
    A.m = m;
    A.N = ds->N;
    A.L = a.nlist;
    A.f_d = (float)f_d;
    A.fd_q = fd_q;
    A.rmax = a.rmax;
    A.prev = prev_idx_dev;
    A.mot_q = (mot && !gate) ? mot->q : nullptr;
    A.mot_d = (mot && !gate) ? mot->d : nullptr;
    A.gated = gate ? 1 : 0;
    A.certified = eq14 == 1 ? 0 : 1;
    A.idx = out.idx;
    A.d1 = d1f;
    A.d2 = d2f;
    A.fb_list = fb_list;
    A.fb_count = counters + 2;
    A.counters = counters;
    A.touched = touched;
    ctx->launches++;
    if (budget == 0) budget = kLeafBudget;
    if (budget < -1) budget = 0;
    if (two && budget >= 0 && m * kPairMax < ((int64_t)1 << 31)) {
        // the query's warp scans `budget` leaves itself (the warm-start leaf
        // first); the further candidates of Eq. (13) go to the leaf-major scan
        const int L = a.nlist, nb = (L + kScanBlock - 1) / kScanBlock;
        const size_t b_pl = r256((size_t)m * kPairMax * 4), b_np = r256((size_t)m * 4),
                     b_res = r256((size_t)m * kPairMax * sizeof(PairRes)), b_L = r256((size_t)L * 4),
                     b_L1 = r256((size_t)(L + 1) * 4), b_nb = r256((size_t)nb * 4);
        void *wp = nullptr;
        DD_TRY(dd_workspace(ctx, WS_ANN_PAIRS, 2 * b_pl + b_np + b_res + 2 * b_L + 2 * b_L1 + 2 * b_nb, &wp));
        char *cp = (char *)wp;
        int32_t *pair_leaf = (int32_t *)cp;
        cp += b_pl;
        unsigned *bucket = (unsigned *)cp;
        cp += b_pl;
        int *n_pairs = (int *)cp;
        cp += b_np;
        PairRes *res = (PairRes *)cp;
        cp += b_res;
        unsigned *leaf_cnt = (unsigned *)cp;
        cp += b_L;
        unsigned *cursor = (unsigned *)cp;
        cp += b_L;
        unsigned *pair_off = (unsigned *)cp;
        cp += b_L1;
        unsigned *item_off = (unsigned *)cp;
        cp += b_L1;
        unsigned *bsum = (unsigned *)cp;
        cp += b_nb;
        unsigned *bitem = (unsigned *)cp;
        DD_TRY_CUDA(ctx, cudaMemsetAsync(leaf_cnt, 0, 2 * b_L, s));   // counts and cursors
        Probe2Args P2{A, a.cent, a.rad1, a.lrad1, a.L1, a.L2, a.r1max, budget, pair_leaf, n_pairs, leaf_cnt};
        k_ann_probe2<<<(unsigned)((m * 32 + 255) / 256), 256, 0, s>>>(P2);
        DD_TRY_CUDA(ctx, cudaGetLastError());
        ctx->launches += 6;
        k_leaf_sums<<<nb, 256, 0, s>>>(leaf_cnt, L, bsum, bitem);
        k_leaf_sums_top<<<1, 1024, 0, s>>>(bsum, bitem, nb);
        k_leaf_offsets<<<nb, 256, 0, s>>>(leaf_cnt, L, bsum, bitem, pair_off, item_off);
        k_pair_scatter<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(pair_leaf, n_pairs, m, pair_off, cursor, bucket);
        LeafScanArgs LS{a.zs, a.cent, a.offs, rec, bucket, pair_off, item_off, L, res, counters, touched};
        k_leaf_scan<<<(unsigned)(ctx->n_sm * 8), 256, 0, s>>>(LS);
        k_pair_merge<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(n_pairs, res, a.perm, m, out.idx, d1f, d2f);
    } else if (two) {
        Probe2Args P2{A, a.cent, a.rad1, a.lrad1, a.L1, a.L2, a.r1max, 0, nullptr, nullptr, nullptr};
        k_ann_probe2<<<(unsigned)((m * 32 + 255) / 256), 256, 0, s>>>(P2);
    } else {
        k_ann_probe<<<(unsigned)((m * 32 + 255) / 256), 256, 0, s>>>(A);
    }
    DD_TRY_CUDA(ctx, cudaGetLastError());
    if (st) DD_TRY_CUDA(ctx, dd_event_record(ctx, ctx->ev_scan[1], s));
    DD_TRY(dd_ann_finish(ds, y_dev, m, rec, out.idx, d2f, out.d2, out.d2nd, s));
    // exact re-search where the candidate list may be incomplete (f_d = 1)
    unsigned long long n_fb = 0;
    // (a captured step never holds f_d = 1: its caller checks)
    if ((f_d >= 1.0 || fd_q) && !ctx->defer) {
        DD_TRY_CUDA(ctx, cudaMemcpyAsync(&n_fb, counters + 2, sizeof(n_fb), cudaMemcpyDeviceToHost, s));
        DD_TRY_CUDA(ctx, cudaStreamSynchronize(s));
        if (n_fb) DD_TRY(ann_exact_subset(ds, y_dev, fb_list, (int64_t)n_fb, out, s));
    }
    if (mot && out.d2 && out.d2nd)
        DD_TRY(dd_ann_motion_update(ctx, rec, m, out.d2, out.d2nd, f_d, fd_q, eq14, mot, s));
    if (st) {
        const int words = (a.nlist + 31) / 32;
        ctx->launches++;
        k_touched_points<<<(unsigned)((words + 255) / 256), 256, 0, s>>>(touched, a.nlist, a.offs, counters + 4);
        DD_TRY_CUDA(ctx, cudaGetLastError());
    }
    if (st && ctx->defer) {
        DD_TRY_CUDA(ctx, cudaMemcpyAsync(ctx->defer->ann, counters, 8 * sizeof(unsigned long long),
                                         cudaMemcpyDeviceToDevice, s));
        st->distances += gate ? 0 : m * (int64_t)Lr;   // gated: the ranked centroids are in counters[3]
    } else if (st) {
        unsigned long long h[6];
        DD_TRY_CUDA(ctx, cudaMemcpyAsync(h, counters, sizeof(h), cudaMemcpyDeviceToHost, s));
        DD_TRY_CUDA(ctx, cudaStreamSynchronize(s));
        float ms = 0.f;
        DD_TRY_CUDA(ctx, cudaEventElapsedTime(&ms, ctx->ev_scan[0], ctx->ev_scan[1]));
        st->scan_ms += ms;
        st->distances += (int64_t)h[0] + (int64_t)h[3] + (gate ? 0 : m * (int64_t)Lr) + (int64_t)n_fb * ds->N;
        st->points += (int64_t)h[5] + (int64_t)n_fb * ds->N;
        st->unique_points += n_fb ? ds->N : (int64_t)h[4];
        st->skipped += (int64_t)h[1];
        st->uncertified += (int64_t)n_fb;
    }
    return DD_OK;
}
