// Exact data projection P_D (Eq. 7) on CUDA cores.
//
// The linear search of the paper (every query against every data point) is
// restated for the GPU as a certified two-stage scan:
//
//  1. k_scan_fp32 streams the centred mapped coordinates z_j (FP32, 48 B per
//     point) through shared memory with the TMA bulk-copy engine and scores
//     every (query, point) pair with the expanded form
//         s_j = |z_j|^2 - 2 z_j . q   ( = |z_j - q|^2 - |q|^2 ),
//     12 FFMA per pair.  Each query keeps every point whose score lies within
//     a window w of its running minimum; w is twice a bound on the score
//     error (FP32 storage of z and q plus FP32 arithmetic), so the exact
//     nearest point is always inside the final window.
//  2. dd_merge_rescore merges the windows of the data splits, rescores the
//     survivors with Eq. (3) in FP64 from the stored (eps, sig) values and
//     picks the minimum (lowest index on ties).  A query whose window
//     overflowed the candidate buffer is re-searched by an FP64 scan over all
//     points, so the returned neighbour is the exact one.
//
// Candidate layout, per (query q, split s): header hdr[q * S + s] and
// entries cand[(q * S + s) * CAP + c] = (score, index bits).
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <mutex>
#include <string>

#include "dd_internal.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kRQ = 4;                       // queries per thread
constexpr int kCap = 8;                      // candidate buffer per query
constexpr int kT = 128;                      // data points per stage
constexpr int kStages = 4;
constexpr int kQT = kThreads * kRQ;          // queries per CTA

constexpr size_t kScanSmem =
    size_t(kStages) * kT * 12 * 4 + size_t(kStages) * kT * 4 + size_t(kRQ) * kCap * kThreads * 8;

// ---------------------------------------------------------------------------
// Query map: y = (eps, sig) -> centred q = (C^{1/2} eps, C^{-1/2} sig)/sqrt(2) - mu
// ---------------------------------------------------------------------------
__global__ void k_map_queries(const double *__restrict__ y, int64_t m, MetricMaps M, double R,
                              double *__restrict__ zq64, QueryRec *__restrict__ rec) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= m) return;
    double s[12], z[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) s[k] = y[i * 12 + k];
    const double r2 = 0.70710678118654752440;
#pragma unroll
    for (int a = 0; a < 6; ++a) {
        double e = 0.0, g = 0.0;
#pragma unroll
        for (int b = 0; b < 6; ++b) {
            e += M.Ch[6 * a + b] * s[b];
            g += M.Cmh[6 * a + b] * s[6 + b];
        }
        z[a] = e * r2 - M.mu[a];
        z[6 + a] = g * r2 - M.mu[6 + a];
    }
    QueryRec r;
    double qn = 0.0;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        if (zq64) zq64[i * 12 + k] = z[k];
        r.q[k] = (float)z[k];
        qn += (double)r.q[k] * (double)r.q[k];
    }
    // score error bound: storage rounding of z and q (2^-24 relative each),
    // 12-term FFMA chain and the rounded |z|^2, bounded by 2^-18 (R + |q|)^2.
    double b = R + sqrt(qn);
    double E = ldexp(b * b, -18);
    r.w2 = (float)(2.0 * E * 1.0001);
    r.qn = (float)qn;
    r.pad[0] = r.pad[1] = 0.f;
    bool finite = isfinite(qn);
    if (!finite) r.w2 = INFINITY;
    rec[i] = r;
}

// ---------------------------------------------------------------------------
// FP32 streaming scan with candidate windows
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads, 2)
    k_scan_fp32(const float *__restrict__ z32, const float *__restrict__ zn, int64_t N,
                int64_t n_tiles, const QueryRec *__restrict__ rec, int64_t m, int splits,
                int64_t tiles_per_split, CandHeader *__restrict__ hdr, float2 *__restrict__ cand,
                bool topk, unsigned *__restrict__ err) {
    extern __shared__ __align__(128) unsigned char smem[];
    float *sz = reinterpret_cast<float *>(smem);
    float *sn = sz + kStages * kT * 12;
    float2 *buf = reinterpret_cast<float2 *>(sn + kStages * kT);
    __shared__ __align__(8) uint64_t full[kStages];

    const int tid = threadIdx.x;
    const int split = blockIdx.y;
    const int64_t qbase = (int64_t)blockIdx.x * kQT;
    const int64_t t_begin = split * tiles_per_split;
    const int64_t t_end = min(n_tiles, t_begin + tiles_per_split);
    const int64_t ntl = t_end > t_begin ? t_end - t_begin : 0;

    float q[kRQ][12], w2[kRQ];
    CandState cs[kRQ];
#pragma unroll
    for (int r = 0; r < kRQ; ++r) {
        int64_t qi = qbase + r * kThreads + tid;
        cand_init(cs[r], qi < m);
        if (qi < m) {
#pragma unroll
            for (int k = 0; k < 12; ++k) q[r][k] = -2.0f * rec[qi].q[k];
            w2[r] = topk ? INFINITY : rec[qi].w2;   // top-k: keep the best kCap, no window
        } else {
#pragma unroll
            for (int k = 0; k < 12; ++k) q[r][k] = 0.f;
            w2[r] = 0.f;
        }
    }

    const uint32_t zbytes = kT * 12 * 4, nbytes = kT * 4;
    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) dd_mbar_init(dd_smem_addr(&full[s]), 1);
        dd_fence_mbar_init();
        for (int s = 0; s < kStages && s < ntl; ++s) {
            int64_t j0 = (t_begin + s) * kT;
            uint32_t bar = dd_smem_addr(&full[s]);
            dd_mbar_expect_tx(bar, zbytes + nbytes);
            dd_bulk_g2s(dd_smem_addr(sz + s * kT * 12), z32 + j0 * 12, zbytes, bar);
            dd_bulk_g2s(dd_smem_addr(sn + s * kT), zn + j0, nbytes, bar);
        }
    }
    __syncthreads();

    bool ok = true;
    for (int64_t it = 0; it < ntl; ++it) {
        const int s = (int)(it % kStages);
        const uint32_t parity = (uint32_t)((it / kStages) & 1);
        if (ok && !dd_mbar_wait(dd_smem_addr(&full[s]), parity)) {
            ok = false;
            atomicOr(err, DEV_ERR_TIMEOUT);
        }
        const float4 *tz = reinterpret_cast<const float4 *>(sz + s * kT * 12);
        const float *tn = sn + s * kT;
        const int64_t j0 = (t_begin + it) * kT;
#pragma unroll 2
        for (int p = 0; p < kT; ++p) {
            const float4 a = tz[3 * p + 0], b = tz[3 * p + 1], c = tz[3 * p + 2];
            const float n = tn[p];
            float sc[kRQ];
            bool any = false;
#pragma unroll
            for (int r = 0; r < kRQ; ++r) {
                float v = fmaf(q[r][0], a.x, n);
                v = fmaf(q[r][1], a.y, v);
                v = fmaf(q[r][2], a.z, v);
                v = fmaf(q[r][3], a.w, v);
                v = fmaf(q[r][4], b.x, v);
                v = fmaf(q[r][5], b.y, v);
                v = fmaf(q[r][6], b.z, v);
                v = fmaf(q[r][7], b.w, v);
                v = fmaf(q[r][8], c.x, v);
                v = fmaf(q[r][9], c.y, v);
                v = fmaf(q[r][10], c.z, v);
                v = fmaf(q[r][11], c.w, v);
                sc[r] = v;
                any |= (v <= cs[r].lim);
            }
            if (any) {
                const int64_t j = j0 + p;
                if (j < N) {
#pragma unroll
                    for (int r = 0; r < kRQ; ++r)
                        if (sc[r] <= cs[r].lim)
                            cand_insert(cs[r], sc[r], (int)j, w2[r], buf + (size_t)r * kCap * kThreads + tid,
                                        kThreads, kCap, topk);
                }
            }
        }
        __syncthreads();
        if (tid == 0 && it + kStages < ntl) {
            int64_t j0n = (t_begin + it + kStages) * kT;
            uint32_t bar = dd_smem_addr(&full[s]);
            dd_mbar_expect_tx(bar, zbytes + nbytes);
            dd_bulk_g2s(dd_smem_addr(sz + s * kT * 12), z32 + j0n * 12, zbytes, bar);
            dd_bulk_g2s(dd_smem_addr(sn + s * kT), zn + j0n, nbytes, bar);
        }
    }

#pragma unroll
    for (int r = 0; r < kRQ; ++r) {
        int64_t qi = qbase + r * kThreads + tid;
        if (qi >= m) continue;
        cand_store(cs[r], buf + (size_t)r * kCap * kThreads + tid, kThreads, kCap, (size_t)qi * splits + split, hdr,
                   cand);
    }
}

// ---------------------------------------------------------------------------
// Merge + FP64 rescoring (thread per query)
// ---------------------------------------------------------------------------
__global__ void k_merge_rescore(const float *__restrict__ raw, MetricMaps M,
                                const double *__restrict__ y, int64_t m, int splits, int cap,
                                const CandHeader *__restrict__ hdr, const float2 *__restrict__ cand,
                                const QueryRec *__restrict__ rec, int certify, double inv_s2,
                                int32_t *__restrict__ idx, double *__restrict__ d2,
                                double *__restrict__ d2nd, int64_t *__restrict__ fb_list,
                                unsigned long long *__restrict__ fb_count) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= m) return;
    const CandHeader *h = hdr + (size_t)i * splits;
    float gmin = INFINITY;
    for (int s = 0; s < splits; ++s) gmin = fminf(gmin, h[s].mrun);
    const float w2 = rec[i].w2;
    // the window (two-product tensor-core scan: with its q_lo term)
    const float lim = gmin + cand_window(gmin, w2, rec[i].pad[0], rec[i].pad[1]);
    bool uncert = !(w2 < INFINITY);
    for (int s = 0; s < splits; ++s) uncert |= (h[s].dropped <= lim);
    double yy[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) yy[k] = y[i * 12 + k];
    double best = INFINITY, second = INFINITY;
    int32_t bj = -1;
    for (int s = 0; s < splits; ++s) {
        const float2 *c = cand + ((size_t)i * splits + s) * cap;
        for (int e = 0; e < h[s].cnt; ++e) {
            float2 v = c[e];
            if (!(v.x <= lim)) continue;
            int32_t j = __float_as_int(v.y);
            double d = dd_eq3(M, yy, raw + (size_t)j * 12);
            if (d < best || (d == best && j < bj)) {
                second = best;
                best = d;
                bj = j;
            } else if (d < second) {
                second = d;
            }
        }
    }
    if (bj < 0) uncert = true;
    // every point outside the window has |z - q|^2 >= gmin + qn + w2/2 (in
    // score units; inv_s2 converts to the mapped coordinates); with the q_lo
    // term (two-product scan) a score s outside it bounds the distance by
    // s + |q_hi|^2 - (qlo4/2) sqrt(s + |q_hi|^2) - w2/2, increasing in s
    double lb;
    if (rec[i].pad[0] > 0.f) {
        const double a = fmax((double)lim + (double)rec[i].pad[1], 0.0);
        lb = 2.0 * inv_s2 * fmax(a - 0.5 * (double)rec[i].pad[0] * sqrt(a) - 0.5 * (double)w2, 0.0);
    } else {
        lb = 2.0 * inv_s2 * ((double)gmin + (double)rec[i].qn + 0.5 * (double)w2);
    }
    if (uncert && certify) {
        unsigned long long k = atomicAdd(fb_count, 1ull);
        fb_list[k] = i;
        return;
    }
    idx[i] = bj;
    if (d2) d2[i] = best;
    if (d2nd) d2nd[i] = fmin(second, lb);
}

// ---------------------------------------------------------------------------
// FP64 exhaustive re-search of uncertified queries (block per query)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_fallback_fp64(const float *__restrict__ raw, int64_t N,
                                                       MetricMaps M, const double *__restrict__ y,
                                                       const int64_t *__restrict__ list,
                                                       const unsigned long long *__restrict__ count,
                                                       int32_t *__restrict__ idx,
                                                       double *__restrict__ d2,
                                                       double *__restrict__ d2nd) {
    __shared__ double sb[256], ss[256];
    __shared__ int32_t sj[256];
    const unsigned long long n = *count;
    for (unsigned long long t = blockIdx.x; t < n; t += gridDim.x) {
        const int64_t i = list[t];
        double yy[12];
#pragma unroll
        for (int k = 0; k < 12; ++k) yy[k] = y[i * 12 + k];
        double b1 = INFINITY, b2 = INFINITY;
        int32_t j1 = -1;
        for (int64_t j = threadIdx.x; j < N; j += blockDim.x) {
            double d = dd_eq3(M, yy, raw + (size_t)j * 12);
            if (d < b1) {
                b2 = b1;
                b1 = d;
                j1 = (int32_t)j;
            } else if (d < b2) {
                b2 = d;
            }
        }
        sb[threadIdx.x] = b1;
        ss[threadIdx.x] = b2;
        sj[threadIdx.x] = j1;
        __syncthreads();
        for (int w = 128; w > 0; w >>= 1) {
            if (threadIdx.x < w) {
                double a1 = sb[threadIdx.x], a2 = ss[threadIdx.x];
                double c1 = sb[threadIdx.x + w], c2 = ss[threadIdx.x + w];
                int32_t ja = sj[threadIdx.x], jc = sj[threadIdx.x + w];
                bool take_c = (c1 < a1) || (c1 == a1 && jc >= 0 && (ja < 0 || jc < ja));
                double n1 = take_c ? c1 : a1;
                double n2 = take_c ? fmin(a1, c2) : fmin(a2, c1);
                sb[threadIdx.x] = n1;
                ss[threadIdx.x] = n2;
                sj[threadIdx.x] = take_c ? jc : ja;
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            idx[i] = sj[0];
            if (d2) d2[i] = sb[0];
            if (d2nd) d2nd[i] = ss[0];
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// The k nearest points (k = 2 .. kTopMax) from scans run in top-k mode
// ---------------------------------------------------------------------------
constexpr int kTopMax = DD_TOPK_MAX;

// Keep (d, j) among the k smallest of a list sorted by (d, j) ascending.
template <typename T>
__device__ __forceinline__ void topk_insert(T (&bd)[kTopMax], int (&bj)[kTopMax], int k, T d, int j) {
    if (!(d < bd[k - 1] || (d == bd[k - 1] && j < bj[k - 1]))) return;
    int p = k - 1;
    while (p > 0 && (d < bd[p - 1] || (d == bd[p - 1] && j < bj[p - 1]))) {
        bd[p] = bd[p - 1];
        bj[p] = bj[p - 1];
        --p;
    }
    bd[p] = d;
    bj[p] = j;
}

// Thread per query.  Every split kept its best `cap` scores (score s =
// |z|^2 - 2 z.q, error at most E = w2/2 against the exact score), so a point
// left out of a full split scores at least that split's worst kept score.
// The true k nearest points all score at most S_k + w2 (S_k the k-th smallest
// kept score): if every full split's worst kept score exceeds S_k + w2, the
// kept entries up to S_k + w2 hold them, and FP64 rescoring of those entries
// gives the exact k nearest.  Otherwise (certify) the query is listed for the
// FP64 re-search.
__global__ void k_merge_topk(const float *__restrict__ raw, MetricMaps M, const double *__restrict__ y, int64_t m,
                             int splits, int cap, const CandHeader *__restrict__ hdr, const float2 *__restrict__ cand,
                             const QueryRec *__restrict__ rec, int k, int certify, double inv_s2,
                             int32_t *__restrict__ idx, double *__restrict__ d2, double *__restrict__ d2nd,
                             int32_t *__restrict__ tk_idx, double *__restrict__ tk_d2, int64_t *__restrict__ fb_list,
                             unsigned long long *__restrict__ fb_count) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= m) return;
    const CandHeader *h = hdr + (size_t)i * splits;
    // pass 1: the k smallest kept scores, and the least worst-kept score of the full splits
    float sk[kTopMax];
    int sj[kTopMax];
#pragma unroll
    for (int e = 0; e < kTopMax; ++e) {
        sk[e] = INFINITY;
        sj[e] = 0x7fffffff;
    }
    float full_min = INFINITY;
    for (int s = 0; s < splits; ++s) {
        const float2 *c = cand + ((size_t)i * splits + s) * cap;
        float mx = -INFINITY;
        for (int e = 0; e < h[s].cnt; ++e) {
            const float2 v = c[e];
            mx = fmaxf(mx, v.x);
            topk_insert(sk, sj, k, v.x, __float_as_int(v.y));
        }
        if (h[s].cnt >= cap) full_min = fminf(full_min, fminf(mx, h[s].dropped));
    }
    const float w2 = rec[i].w2;
    const float lim = certify ? sk[k - 1] + w2 : INFINITY;
    const bool uncert = certify && (!(w2 < INFINITY) || (full_min < INFINITY && !(full_min > lim)));
    if (uncert) {
        const unsigned long long t = atomicAdd(fb_count, 1ull);
        fb_list[t] = i;
        return;
    }
    // pass 2: FP64 rescoring (Eq. 3) of the kept entries up to lim
    double yy[12];
#pragma unroll
    for (int q = 0; q < 12; ++q) yy[q] = y[i * 12 + q];
    double bd[kTopMax];
    int bj[kTopMax];
#pragma unroll
    for (int e = 0; e < kTopMax; ++e) {
        bd[e] = INFINITY;
        bj[e] = 0x7fffffff;
    }
    for (int s = 0; s < splits; ++s) {
        const float2 *c = cand + ((size_t)i * splits + s) * cap;
        for (int e = 0; e < h[s].cnt; ++e) {
            const float2 v = c[e];
            if (!(v.x <= lim)) continue;
            const int j = __float_as_int(v.y);
            topk_insert(bd, bj, k, dd_eq3(M, yy, raw + (size_t)j * 12), j);
        }
    }
    for (int e = 0; e < k; ++e) {
        const bool ok = bd[e] < INFINITY;
        tk_idx[i * k + e] = ok ? bj[e] : -1;
        if (tk_d2) tk_d2[i * k + e] = bd[e];
    }
    idx[i] = bd[0] < INFINITY ? bj[0] : -1;
    if (d2) d2[i] = bd[0];
    if (d2nd) {
        // points outside the kept entries score at least full_min, at least
        // full_min - E exactly (plus |q|^2 for the squared distance)
        const double out = full_min < INFINITY
                               ? 2.0 * inv_s2 * ((double)full_min + (double)rec[i].qn - 0.5 * (double)w2)
                               : INFINITY;
        d2nd[i] = certify ? bd[1] : fmin(bd[1], out);
    }
}

// FP64 exhaustive k-nearest search of the listed queries (block per query):
// every thread keeps the k best of its points, then the block merges the
// sorted lists pairwise.
__global__ void __launch_bounds__(256) k_fallback_topk_fp64(const float *__restrict__ raw, int64_t N, MetricMaps M,
                                                            const double *__restrict__ y,
                                                            const int64_t *__restrict__ list,
                                                            const unsigned long long *__restrict__ count, int k,
                                                            int32_t *__restrict__ idx, double *__restrict__ d2,
                                                            double *__restrict__ d2nd, int32_t *__restrict__ tk_idx,
                                                            double *__restrict__ tk_d2) {
    __shared__ double sd[256 * kTopMax];
    __shared__ int sjx[256 * kTopMax];
    const unsigned long long n = *count;
    const int tid = threadIdx.x;
    for (unsigned long long t = blockIdx.x; t < n; t += gridDim.x) {
        const int64_t i = list[t];
        double yy[12];
#pragma unroll
        for (int q = 0; q < 12; ++q) yy[q] = y[i * 12 + q];
        double bd[kTopMax];
        int bj[kTopMax];
#pragma unroll
        for (int e = 0; e < kTopMax; ++e) {
            bd[e] = INFINITY;
            bj[e] = 0x7fffffff;
        }
        for (int64_t j = tid; j < N; j += blockDim.x) topk_insert(bd, bj, k, dd_eq3(M, yy, raw + (size_t)j * 12), (int)j);
        for (int e = 0; e < k; ++e) {
            sd[tid * k + e] = bd[e];
            sjx[tid * k + e] = bj[e];
        }
        __syncthreads();
        for (int w = blockDim.x / 2; w > 0; w >>= 1) {
            if (tid < w) {
                // merge the sorted lists of threads tid and tid + w into bd/bj
                int a = 0, b = 0;
                const double *da = sd + tid * k, *db = sd + (tid + w) * k;
                const int *ja = sjx + tid * k, *jb = sjx + (tid + w) * k;
                for (int e = 0; e < k; ++e) {
                    const bool take_a = (da[a] < db[b]) || (da[a] == db[b] && ja[a] <= jb[b]);
                    bd[e] = take_a ? da[a] : db[b];
                    bj[e] = take_a ? ja[a] : jb[b];
                    if (take_a) ++a;
                    else ++b;
                }
            }
            __syncthreads();
            if (tid < w)
                for (int e = 0; e < k; ++e) {
                    sd[tid * k + e] = bd[e];
                    sjx[tid * k + e] = bj[e];
                }
            __syncthreads();
        }
        if (tid < k) {
            const bool ok = sd[tid] < INFINITY;
            tk_idx[i * k + tid] = ok ? sjx[tid] : -1;
            if (tk_d2) tk_d2[i * k + tid] = sd[tid];
        }
        if (tid == 0) {
            idx[i] = sd[0] < INFINITY ? sjx[0] : -1;
            if (d2) d2[i] = sd[0];
            if (d2nd) d2nd[i] = sd[1];
        }
        __syncthreads();
    }
}

int pick_splits(int64_t qtiles, int64_t n_tiles, int n_sm, int per_sm) {
    const int64_t slots = (int64_t)n_sm * per_sm;
    if (qtiles >= slots) return 1;
    int64_t best_s = 1;
    double best_eff = 0.0;
    for (int64_t s = 1; s <= slots && s <= n_tiles; ++s) {
        int64_t ctas = qtiles * s;
        int64_t waves = (ctas + slots - 1) / slots;
        double eff = (double)ctas / (double)(waves * slots);
        // prefer full waves, then fewer splits
        if (eff > best_eff + 1e-9) {
            best_eff = eff;
            best_s = s;
        }
        if (ctas >= slots && eff > 0.94) break;
    }
    return (int)best_s;
}

}  // namespace

dd_status dd_map_queries(dd_dataset *ds, const double *y_dev, int64_t m, double *zq64,
                         QueryRec *rec, cudaStream_t s) {
    if (m == 0) return DD_OK;
    ds->ctx->launches++;
    k_map_queries<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(y_dev, m, ds->M, ds->R, zq64, rec);
    DD_TRY_CUDA(ds->ctx, cudaGetLastError());
    return DD_OK;
}

dd_status dd_fallback_exact(dd_dataset *ds, const double *y_dev, const int64_t *fb_list,
                            const unsigned long long *fb_count, int64_t m, SearchOut out, cudaStream_t s) {
    dd_ctx *ctx = ds->ctx;
    int grid = (int)std::min<int64_t>(m, (int64_t)ctx->n_sm * 4);
    ctx->launches++;
    k_fallback_fp64<<<grid, 256, 0, s>>>(ds->raw, ds->N, ds->M, y_dev, fb_list, fb_count, out.idx, out.d2, out.d2nd);
    DD_TRY_CUDA(ctx, cudaGetLastError());
    return DD_OK;
}

namespace {
__global__ void k_gather_listed(const double *__restrict__ y, const int64_t *__restrict__ list, int64_t n,
                                double *__restrict__ ys, int64_t *__restrict__ list_copy) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n) return;
    const int64_t i = list[t];
    list_copy[t] = i;
#pragma unroll
    for (int k = 0; k < 12; ++k) ys[t * 12 + k] = y[i * 12 + k];
}

__global__ void k_scatter_listed(const int64_t *__restrict__ list, int64_t n, const int32_t *__restrict__ si,
                                 const double *__restrict__ sd, const double *__restrict__ sd2,
                                 int32_t *__restrict__ idx, double *__restrict__ d2, double *__restrict__ d2nd) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n) return;
    const int64_t i = list[t];
    idx[i] = si[t];
    if (d2) d2[i] = sd[t];
    if (d2nd) d2nd[i] = sd2[t];
}
}  // namespace

// The listed queries searched again by the certified FP32 scan (which
// re-searches its own uncertified ones in FP64), results written back.
static dd_status exact_fp32_subset(dd_dataset *ds, const double *y_dev, const int64_t *list, int64_t n,
                                   SearchOut out, cudaStream_t s) {
    dd_ctx *ctx = ds->ctx;
    auto r256 = [](size_t b) { return (b + 255) / 256 * 256; };
    void *w = nullptr;
    DD_TRY(dd_workspace(ctx, WS_SUBSET,
                        r256((size_t)n * 96) + r256((size_t)n * 8) + r256((size_t)n * 4) + 2 * r256((size_t)n * 8),
                        &w));
    char *c = (char *)w;
    double *ys = (double *)c;
    c += r256((size_t)n * 96);
    int64_t *lc = (int64_t *)c;
    c += r256((size_t)n * 8);
    int32_t *si = (int32_t *)c;
    c += r256((size_t)n * 4);
    double *sd = (double *)c;
    c += r256((size_t)n * 8);
    double *sd2 = (double *)c;
    ctx->launches++;
    k_gather_listed<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(y_dev, list, n, ys, lc);
    DD_TRY_CUDA(ctx, cudaGetLastError());
    DD_TRY(dd_search_exact_fp32(ds, ys, n, 1, SearchOut{si, sd, sd2}, nullptr, s));
    ctx->launches++;
    k_scatter_listed<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(lc, n, si, sd, sd2, out.idx, out.d2, out.d2nd);
    DD_TRY_CUDA(ctx, cudaGetLastError());
    return DD_OK;
}

dd_status dd_merge_rescore(dd_dataset *ds, const double *y_dev, int64_t m, int splits, int cap,
                           const CandHeader *hdr, const float2 *cand, const QueryRec *rec,
                           int certify, double inv_s2, SearchOut out, dd_search_stats *st, cudaStream_t s,
                           bool fp32_first) {
    dd_ctx *ctx = ds->ctx;
    void *w = nullptr;
    size_t need = (size_t)m * sizeof(int64_t) + 256;
    DD_TRY(dd_workspace(ctx, WS_MISC, need, &w));
    unsigned long long *fb_count = reinterpret_cast<unsigned long long *>(w);
    int64_t *fb_list = reinterpret_cast<int64_t *>(reinterpret_cast<char *>(w) + 256);
    DD_TRY_CUDA(ctx, cudaMemsetAsync(fb_count, 0, sizeof(unsigned long long), s));
    ctx->launches++;
    k_merge_rescore<<<(unsigned)((m + 127) / 128), 128, 0, s>>>(
        ds->raw, ds->M, y_dev, m, splits, cap, hdr, cand, rec, certify, inv_s2, out.idx, out.d2, out.d2nd,
        fb_list, fb_count);
    DD_TRY_CUDA(ctx, cudaGetLastError());
    if (certify && fp32_first && !ctx->capturing && !ctx->defer) {
        unsigned long long n = 0;
        DD_TRY_CUDA(ctx, cudaMemcpyAsync(&n, fb_count, sizeof(n), cudaMemcpyDeviceToHost, s));
        DD_TRY_CUDA(ctx, cudaStreamSynchronize(s));
        if (n) DD_TRY(exact_fp32_subset(ds, y_dev, fb_list, (int64_t)n, out, s));
        if (st) {
            st->uncertified += (int64_t)n;
            st->distances += (int64_t)n * ds->N;
        }
        return DD_OK;
    }
    if (certify) {
        int grid = (int)std::min<int64_t>(m, (int64_t)ctx->n_sm * 4);
        ctx->launches++;
        k_fallback_fp64<<<grid, 256, 0, s>>>(ds->raw, ds->N, ds->M, y_dev, fb_list, fb_count,
                                             out.idx, out.d2, out.d2nd);
        DD_TRY_CUDA(ctx, cudaGetLastError());
    }
    if (st && ctx->defer) {
        DD_TRY_CUDA(ctx, cudaMemcpyAsync(&ctx->defer->fb, fb_count, sizeof(*fb_count), cudaMemcpyDeviceToDevice, s));
    } else if (st) {
        unsigned long long n = 0;
        DD_TRY_CUDA(ctx, cudaMemcpyAsync(&n, fb_count, sizeof(n), cudaMemcpyDeviceToHost, s));
        DD_TRY_CUDA(ctx, cudaStreamSynchronize(s));
        st->uncertified += (int64_t)n;
        st->distances += (int64_t)n * ds->N;
    }
    return DD_OK;
}

dd_status dd_merge_topk(dd_dataset *ds, const double *y_dev, int64_t m, int splits, int cap, const CandHeader *hdr,
                        const float2 *cand, const QueryRec *rec, int certify, double inv_s2, SearchOut out,
                        dd_search_stats *st, cudaStream_t s) {
    dd_ctx *ctx = ds->ctx;
    if (out.k < 2 || out.k > kTopMax || !out.topk_idx) return dd_fail(ctx, DD_ERR_ARG, "top-k merge: k out of range");
    void *w = nullptr;
    DD_TRY(dd_workspace(ctx, WS_MISC, (size_t)m * sizeof(int64_t) + 256, &w));
    unsigned long long *fb_count = reinterpret_cast<unsigned long long *>(w);
    int64_t *fb_list = reinterpret_cast<int64_t *>(reinterpret_cast<char *>(w) + 256);
    DD_TRY_CUDA(ctx, cudaMemsetAsync(fb_count, 0, sizeof(unsigned long long), s));
    ctx->launches++;
    k_merge_topk<<<(unsigned)((m + 127) / 128), 128, 0, s>>>(ds->raw, ds->M, y_dev, m, splits, cap, hdr, cand, rec,
                                                             out.k, certify, inv_s2, out.idx, out.d2, out.d2nd,
                                                             out.topk_idx, out.topk_d2, fb_list, fb_count);
    DD_TRY_CUDA(ctx, cudaGetLastError());
    if (certify) {
        const int grid = (int)std::min<int64_t>(m, (int64_t)ctx->n_sm * 4);
        ctx->launches++;
        k_fallback_topk_fp64<<<grid, 256, 0, s>>>(ds->raw, ds->N, ds->M, y_dev, fb_list, fb_count, out.k, out.idx,
                                                  out.d2, out.d2nd, out.topk_idx, out.topk_d2);
        DD_TRY_CUDA(ctx, cudaGetLastError());
    }
    if (st && ctx->defer) {
        DD_TRY_CUDA(ctx, cudaMemcpyAsync(&ctx->defer->fb, fb_count, sizeof(*fb_count), cudaMemcpyDeviceToDevice, s));
    } else if (st) {
        unsigned long long n = 0;
        DD_TRY_CUDA(ctx, cudaMemcpyAsync(&n, fb_count, sizeof(n), cudaMemcpyDeviceToHost, s));
        DD_TRY_CUDA(ctx, cudaStreamSynchronize(s));
        st->uncertified += (int64_t)n;
        st->distances += (int64_t)n * ds->N;
    }
    return DD_OK;
}

dd_status dd_scan_fp32_raw(dd_ctx *ctx, const float *z32, const float *zn, int64_t N, const QueryRec *rec, int64_t m,
                           bool topk, int slot, int *splits_out, int *cap_out, CandHeader **hdr_out, float2 **cand_out,
                           cudaStream_t s) {
    const int64_t n_tiles = (N + kT - 1) / kT;
    const int64_t qtiles = (m + kQT - 1) / kQT;
    const int splits = pick_splits(qtiles, n_tiles, ctx->n_sm, 2);
    const int64_t tps = (n_tiles + splits - 1) / splits;
    size_t hdr_bytes = ((size_t)m * splits * sizeof(CandHeader) + 255) / 256 * 256;
    size_t cand_bytes = (size_t)m * splits * kCap * sizeof(float2);
    void *w = nullptr;
    DD_TRY(dd_workspace(ctx, slot, hdr_bytes + cand_bytes, &w));
    CandHeader *hdr = reinterpret_cast<CandHeader *>(w);
    float2 *cand = reinterpret_cast<float2 *>(reinterpret_cast<char *>(w) + hdr_bytes);
    DD_TRY_CUDA(ctx, cudaFuncSetAttribute(k_scan_fp32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kScanSmem));
    ctx->launches++;
    k_scan_fp32<<<dim3((unsigned)qtiles, (unsigned)splits), kThreads, kScanSmem, s>>>(
        z32, zn, N, n_tiles, rec, m, splits, tps, hdr, cand, topk, ctx->dev_err);
    DD_TRY_CUDA(ctx, cudaGetLastError());
    *splits_out = splits;
    *cap_out = kCap;
    *hdr_out = hdr;
    *cand_out = cand;
    return DD_OK;
}

dd_status dd_search_exact_fp32(dd_dataset *ds, const double *y_dev, int64_t m, int certify,
                               SearchOut out, dd_search_stats *st, cudaStream_t s) {
    dd_ctx *ctx = ds->ctx;
    if (m == 0) return DD_OK;
    const int64_t n_tiles = (ds->N + kT - 1) / kT;
    const int64_t qtiles = (m + kQT - 1) / kQT;
    // Split count (data ranges per query tile, merged afterwards): the
    // heuristic fills whole waves of CTAs; the autotuner times it, half and
    // twice it on the first call of every query-tile count with 10^9 to
    // 5 x 10^12 pairs and keeps the fastest for this context (all give the
    // same answers); larger problems take the heuristic.
    const int s0 = pick_splits(qtiles, n_tiles, ctx->n_sm, 2);
    int cands[3] = {s0, (int)std::max<int64_t>(1, s0 / 2), (int)std::min<int64_t>(n_tiles, (int64_t)s0 * 2)};
    int splits = s0;
    bool tune = false;
    {
        auto it = ctx->fp32_splits.find(qtiles);
        if (it != ctx->fp32_splits.end()) splits = it->second;
        // the trials run the whole problem (the split count decides the grid
        // shape), so only where one trial costs tens of milliseconds
        else tune = !ctx->capturing && (double)m * (double)ds->N >= 1e9 && (double)m * (double)ds->N <= 5e12;
    }
    const int s_max = tune ? std::max(cands[0], std::max(cands[1], cands[2])) : splits;

    size_t rec_bytes = ((size_t)m * sizeof(QueryRec) + 255) / 256 * 256;
    size_t hdr_bytes = ((size_t)m * s_max * sizeof(CandHeader) + 255) / 256 * 256;
    size_t cand_bytes = (size_t)m * s_max * kCap * sizeof(float2);
    void *w = nullptr;
    DD_TRY(dd_workspace(ctx, WS_SEARCH, rec_bytes + hdr_bytes + cand_bytes, &w));
    QueryRec *rec = reinterpret_cast<QueryRec *>(w);
    CandHeader *hdr = reinterpret_cast<CandHeader *>(reinterpret_cast<char *>(w) + rec_bytes);
    float2 *cand = reinterpret_cast<float2 *>(reinterpret_cast<char *>(w) + rec_bytes + hdr_bytes);

    DD_TRY(dd_map_queries(ds, y_dev, m, nullptr, rec, s));
    DD_TRY_CUDA(ctx, cudaFuncSetAttribute(k_scan_fp32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kScanSmem));
    // top-k mode (the best kCap scores of every split, no window) for the k
    // nearest points or an uncertified search; else the certified window
    const bool topk = certify == 0 || out.k >= 2;
    if (tune) {
        float best = 1e30f;
        for (int c = 0; c < 3; ++c) {
            if (c > 0 && (cands[c] == cands[0] || (c == 2 && cands[2] == cands[1]))) continue;
            const int sp = cands[c];
            const int64_t tp = (n_tiles + sp - 1) / sp;
            DD_TRY_CUDA(ctx, dd_event_record(ctx, ctx->ev_scan[0], s));
            ctx->launches++;
            k_scan_fp32<<<dim3((unsigned)qtiles, (unsigned)sp), kThreads, kScanSmem, s>>>(
                ds->z32, ds->zn, ds->N, n_tiles, rec, m, sp, tp, hdr, cand, topk, ctx->dev_err);
            DD_TRY_CUDA(ctx, cudaGetLastError());
            DD_TRY_CUDA(ctx, dd_event_record(ctx, ctx->ev_scan[1], s));
            DD_TRY_CUDA(ctx, cudaEventSynchronize(ctx->ev_scan[1]));
            float ms = 0.f;
            DD_TRY_CUDA(ctx, cudaEventElapsedTime(&ms, ctx->ev_scan[0], ctx->ev_scan[1]));
            if (ms < best) {
                best = ms;
                splits = sp;
            }
        }
        ctx->fp32_splits[qtiles] = splits;
    }
    const int64_t tps = (n_tiles + splits - 1) / splits;
    dim3 grid((unsigned)qtiles, (unsigned)splits);
    ctx->launches++;
    if (st) DD_TRY_CUDA(ctx, dd_event_record(ctx, ctx->ev_scan[0], s));
    k_scan_fp32<<<grid, kThreads, kScanSmem, s>>>(ds->z32, ds->zn, ds->N, n_tiles, rec, m, splits, tps,
                                                  hdr, cand, topk, ctx->dev_err);
    DD_TRY_CUDA(ctx, cudaGetLastError());
    if (st) DD_TRY_CUDA(ctx, dd_event_record(ctx, ctx->ev_scan[1], s));
    if (st) st->distances += m * ds->N;
    if (out.k >= 2) DD_TRY(dd_merge_topk(ds, y_dev, m, splits, kCap, hdr, cand, rec, certify, 1.0, out, st, s));
    else DD_TRY(dd_merge_rescore(ds, y_dev, m, splits, kCap, hdr, cand, rec, certify, 1.0, out, st, s));
    if (st && !ctx->defer) {
        float ms = 0.f;
        DD_TRY_CUDA(ctx, cudaEventElapsedTime(&ms, ctx->ev_scan[0], ctx->ev_scan[1]));
        st->scan_ms += ms;
    }
    return DD_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free variant of the exact FP32 projection.
//
// For callers that cannot allocate device memory during a call: for example a
// serving loop whose device memory is fully reserved up front by another
// allocator (a framework's caching allocator owning the HBM), or a real-time
// caller that cannot accept cudaMalloc/cudaFree, which may fail under memory
// pressure and (cudaFree) synchronise the whole device.  The scratch of the
// FP32 scan (query records, candidate windows, the re-search list) lives in
// the file-scope array below instead of the context's workspaces.  Every GPU
// that loads the library holds this array (32 MiB) until the process exits.
// ---------------------------------------------------------------------------
static constexpr size_t kNoAllocScratchBytes = 32ull << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

namespace {
constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mu;
void *g_noalloc_ptr[kNoAllocMaxDevices] = {};
}  // namespace

namespace {
// Makes ctx's device current for the lifetime of the guard and restores the
// caller's current device afterwards.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) {
            cudaGetLastError();
            prev = -1;
        }
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};
}  // namespace

extern "C" dd_status dd_project_nearest_noalloc(dd_dataset *ds, const double *y_dev, int64_t m, int32_t *idx_dev,
                                               double *d2_dev, void *stream, int wait) {
    if (!ds) return DD_ERR_ARG;
    dd_ctx *ctx = ds->ctx;
    if (m < 0 || m > DD_NOALLOC_MAX_QUERIES)
        return dd_fail(ctx, DD_ERR_ARG,
                       "dd_project_nearest_noalloc: m must be in [0, " + std::to_string(DD_NOALLOC_MAX_QUERIES) + "]");
    if (m == 0) return DD_OK;
    if (!y_dev || !idx_dev || !d2_dev) return dd_fail(ctx, DD_ERR_ARG, "dd_project_nearest_noalloc: NULL argument");
    if (ctx->device < 0 || ctx->device >= kNoAllocMaxDevices)
        return dd_fail(ctx, DD_ERR_ARG, "dd_project_nearest_noalloc: device index too large");
    DeviceGuard guard(ctx->device);
    {
        int cur = -1;
        DD_TRY_CUDA(ctx, cudaGetDevice(&cur));
        if (cur != ctx->device) return dd_fail(ctx, DD_ERR_CUDA, "dd_project_nearest_noalloc: cannot select the device");
    }
    // Set-up, once per device, with that device current: the device address
    // of the scratch array (host code only sees a host-side stand-in).
    void *base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        if (!g_noalloc_ptr[ctx->device]) {
            void *p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess)
                return dd_fail(ctx, DD_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            g_noalloc_ptr[ctx->device] = p;
        }
        base = g_noalloc_ptr[ctx->device];
    }
    cudaStream_t s = stream ? (cudaStream_t)stream : ctx->stream;
    const int64_t n_tiles = (ds->N + kT - 1) / kT;
    const int64_t qtiles = (m + kQT - 1) / kQT;
    auto r256 = [](size_t b) { return (b + 255) / 256 * 256; };
    const size_t fixed = r256((size_t)m * sizeof(QueryRec)) + r256((size_t)m * sizeof(int64_t)) + 256;
    const size_t per_split = (size_t)m * (sizeof(CandHeader) + kCap * sizeof(float2));
    const int64_t s_fit = (int64_t)((kNoAllocScratchBytes - fixed - 512) / per_split);
    const int splits = (int)std::max<int64_t>(1, std::min<int64_t>(pick_splits(qtiles, n_tiles, ctx->n_sm, 2), s_fit));
    const int64_t tps = (n_tiles + splits - 1) / splits;
    char *c = (char *)base;
    // head of the array: the re-search counter (8 bytes) and this call's
    // device status word (4 bytes), both cleared below
    unsigned long long *fb_count = (unsigned long long *)c;
    unsigned *err = (unsigned *)(c + 8);
    QueryRec *rec = (QueryRec *)(c + 256);
    int64_t *fb_list = (int64_t *)(c + 256 + r256((size_t)m * sizeof(QueryRec)));
    CandHeader *hdr = (CandHeader *)(c + fixed);
    float2 *cand = (float2 *)(c + fixed + r256((size_t)m * splits * sizeof(CandHeader)));
    // the re-search counter and the status word must start at zero; every
    // other region is fully written before it is read
    DD_TRY_CUDA(ctx, cudaMemsetAsync(c, 0, 16, s));
    ctx->launches += 4;
    k_map_queries<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(y_dev, m, ds->M, ds->R, nullptr, rec);
    DD_TRY_CUDA(ctx, cudaFuncSetAttribute(k_scan_fp32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kScanSmem));
    k_scan_fp32<<<dim3((unsigned)qtiles, (unsigned)splits), kThreads, kScanSmem, s>>>(
        ds->z32, ds->zn, ds->N, n_tiles, rec, m, splits, tps, hdr, cand, false, err);
    k_merge_rescore<<<(unsigned)((m + 127) / 128), 128, 0, s>>>(ds->raw, ds->M, y_dev, m, splits, kCap, hdr, cand,
                                                                rec, 1, 1.0, idx_dev, d2_dev, nullptr, fb_list,
                                                                fb_count);
    const int grid = (int)std::min<int64_t>(m, (int64_t)ctx->n_sm * 4);
    k_fallback_fp64<<<grid, 256, 0, s>>>(ds->raw, ds->N, ds->M, y_dev, fb_list, fb_count, idx_dev, d2_dev, nullptr);
    DD_TRY_CUDA(ctx, cudaGetLastError());
    if (wait) {
        unsigned h = 0;
        DD_TRY_CUDA(ctx, cudaMemcpyAsync(&h, err, sizeof(h), cudaMemcpyDeviceToHost, s));
        DD_TRY_CUDA(ctx, cudaStreamSynchronize(s));
        if (h & DEV_ERR_TIMEOUT)
            return dd_fail(ctx, DD_ERR_TIMEOUT, "dd_project_nearest_noalloc: a device wait timed out");
    }
    return DD_OK;
}
