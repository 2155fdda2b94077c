// Nearest centroids on the tensor cores, with exactly the answers of the ALU
// kernels they replace.
//
// Two places of the approximate search rank centroids by the expanded FP32
// score v(c) = |c|^2 - 2 c.q (the nearest centroid is the one of least v):
//  * the cell ranking of every listed query (Sec. 4.2: the kCand = 8 nearest
//    cells, then ordered by distance; ann.cu k_rank_small), and
//  * the k-means assignment of the tree build to the nearest cell
//    (ann.cu k_assign).
// Each is a (rows x centroids) contraction of width 12.  Here it runs as split
// FP16 MMAs (tcgen05, FP32 accumulators in TMEM; three products per score as
// in the certified exact scan of search_tc.cu), an epilogue keeps, per row,
// the best tensor-core scores within a window above its K-th best (at most
// CAP), and the row is finished in FP32 with the ALU kernels' own arithmetic
// on those candidates only:
//
//   Let Delta bound |S_t(c) / s^2 - v(c)| for every centroid (S_t the
//   tensor-core score with operands scaled by s, v the FP32 score).  If c is
//   among the K best by v, then S_t(c) <= T_K + 2 Delta s^2, T_K the K-th
//   best tensor-core score (the K best by S_t all have v <= T_K / s^2 +
//   Delta, so the K-th best v is at most that, and S_t(c) / s^2 <= v(c) +
//   Delta).  A score is offered to the list only while it is within
//   2 Delta s^2 of the K-th best so far (which only falls), and the least
//   offered score that did not fit is remembered: when that exceeds
//   T_K + 2 Delta s^2 the list holds every centroid that can be among the K
//   best in FP32; they are rescored with
//   the ALU formula (same operands, same fused multiply-adds in the same
//   order) and the K best by (v, index) are exactly the ALU kernel's.
//   Otherwise the row goes on a list that the ALU kernel finishes.
//
// Delta: the tensor-core error of the split-FP16 product (as for the exact
// scan: 2^-15 B^2 + 2^-18 with B = s (R + |q|), R bounding |c|) plus the FP32
// score's own rounding, at most 2^-19 (R^2 + 2 R |q|) s^2.
//
// The assignment of points to the leaves of their own cell (ann.cu
// k_assign_fine: 512 leaves per cell) stays on the ALU: with its four
// centroid tiles per 128 points this kernel measured 0.6 s per pass at 10^9
// points against 0.38 s for the ALU kernel (tensor pipe 3 % busy; the time
// goes to the per-tile hand-offs).
//
// Persistent CTAs (two per SM), each taking every grid-th tile of 128 rows.
// Warp 0 streams the centroid operand tiles (hi and lo, 4 KB each) into a
// ring of stages with 1-D bulk copies; warp 1 allocates TMEM and issues the
// three MMAs of every 128-centroid tile into one of two accumulators; warps
// 2..5 take one row each per thread: they write the rows' operands into one
// of two A buffers (A0 = (q_hi, 1, 1), A1 = (q_lo), A2 = A0; the next row
// tile's while the current one runs), and per accumulator a min-reducing
// 32-column TMEM load per chunk, walking only chunks whose minimum is within
// the window.  Every mbarrier wait is bounded; on a timeout the kernel flags
// the error, stops issuing work, drains what is in flight and frees TMEM.
#include <algorithm>
#include <cmath>

#include "dd_internal.cuh"
#include "tc_ptx.cuh"

namespace {

using namespace dd_tc;

constexpr int kRows = 128;          // rows per CTA (MMA M)
constexpr int kCols = 128;          // centroids per tile (MMA N)
constexpr int kStages = 4;
constexpr int kThreads = 192;       // producer warp, MMA warp, 4 epilogue warps
constexpr uint32_t kStageBytes = 2 * kTileBytes;
constexpr uint32_t kTmemCols = 256;

// MODE 0: cell ranking of listed queries (K = kAnnCand nearest by v, then
// ordered by distance); MODE 1: nearest centroid of every row.
template <int MODE>
struct NearCfg {
    static constexpr int K = MODE == 0 ? kAnnCand : 1;
    static constexpr int CAP = MODE == 0 ? 12 : 8;
};

struct NearArgs {
    const float *z;            // MODE 1: point coordinates [.. x 12]
    const QueryRec *rec;       // MODE 0: query records
    const int32_t *list;       // MODE 0: listed queries (null: 0..n-1)
    const unsigned *n_list;    // MODE 0: device count of `list` (null: n)
    int64_t n;                 // rows (MODE 0: the capacity of the list)
    const __half *chi, *clo;   // split FP16 centroid operand tiles
    const float *cent, *cn;    // FP32 centroids [.. x 12] and |c|^2: the ALU kernels' operands
    int Lc;                    // centroids
    int tpg;                   // their operand tiles
    float s;                   // operand scale (a power of two)
    float R;                   // bound on |c|
    int32_t *out;              // MODE 1: nearest centroid
    int32_t *out_cl;           // MODE 0: [m x K] cells, nearest first
    float *out_d;              // MODE 0: [m x K] their FP32 distances
    int32_t *fb;               // rows (MODE 0: queries) left to the ALU kernel
    unsigned *fb_n;            // their count (may exceed fb_cap: then only fb_cap are listed)
    int64_t fb_cap;
    unsigned *err;
};

__device__ __forceinline__ bool better(float v1, int c1, float v2, int c2) {
    return v1 < v2 || (v1 == v2 && c1 < c2);
}

// The ALU kernels' score of centroid c: |c|^2 stored, then the 12 fused
// multiply-adds of -2 q against c in coordinate order.
__device__ __forceinline__ float alu_score(const float *__restrict__ cent, const float *__restrict__ cn, int64_t c,
                                           const float (&qm2)[12]) {
    const float4 *p = reinterpret_cast<const float4 *>(cent + c * 12);
    const float4 a = __ldg(p), b = __ldg(p + 1), d = __ldg(p + 2);
    float v = __ldg(cn + c);
    v = fmaf(qm2[0], a.x, v); v = fmaf(qm2[1], a.y, v); v = fmaf(qm2[2], a.z, v); v = fmaf(qm2[3], a.w, v);
    v = fmaf(qm2[4], b.x, v); v = fmaf(qm2[5], b.y, v); v = fmaf(qm2[6], b.z, v); v = fmaf(qm2[7], b.w, v);
    v = fmaf(qm2[8], d.x, v); v = fmaf(qm2[9], d.y, v); v = fmaf(qm2[10], d.z, v); v = fmaf(qm2[11], d.w, v);
    return v;
}

// Operands of one row (this thread's row of a row tile), fetched in two
// steps so that the loads of the next row tile overlap the current one's
// epilogue: the row's index, then its coordinates.
struct RowSrc {
    int64_t idx;     // MODE 0: query; MODE 1: row (-1: no row)
    float q[12];
};

template <int MODE>
__device__ __forceinline__ void fetch_index(const NearArgs &P, int64_t nrows, int64_t r, RowSrc &S) {
    S.idx = r < nrows ? (MODE == 0 && P.list ? (int64_t)P.list[r] : r) : -1;
}

template <int MODE>
__device__ __forceinline__ void fetch_coords(const NearArgs &P, RowSrc &S) {
    if (S.idx < 0) {
#pragma unroll
        for (int k = 0; k < 12; ++k) S.q[k] = 0.f;
        return;
    }
    const float *src = MODE == 0 ? P.rec[S.idx].q : P.z + S.idx * 12;
#pragma unroll
    for (int k = 0; k < 12; ++k) S.q[k] = src[k];
}

// The row's operands into A buffer sA (A0 = (q_hi, 1, 1), A1 = (q_lo),
// A2 = A0 at `row`), its FP32 coordinates into sQ and its window into sW.
__device__ __forceinline__ void build_row(const RowSrc &S, float sc, float R, int row, unsigned char *sA, float *sQ,
                                          float *sW) {
    __half h[16], l[16];
    float qn = 0.f;      // |q|^2
    bool in_range = true;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        const float x = S.q[k] * sc;   // exact: the scale is a power of two
        in_range &= fabsf(x) < 30000.f;
        qn = fmaf(S.q[k], S.q[k], qn);
        h[k] = __float2half_rn(x);
        l[k] = __float2half_rn(x - __half2float(h[k]));   // the difference is exact in FP32
        sQ[row * 12 + k] = S.q[k];
    }
    h[12] = h[13] = __float2half_rn(in_range ? 1.f : 0.f);
    h[14] = h[15] = l[12] = l[13] = l[14] = l[15] = __float2half_rn(0.f);
    if (!in_range)
#pragma unroll
        for (int k = 0; k < 12; ++k) h[k] = l[k] = __float2half_rn(0.f);
    // the norm is rounded up by a relative 1e-5 for its FP32 evaluation
    const float qa = sqrtf(qn) * 1.00001f;
    const float B = sc * (R + qa);
    const float Et = ldexpf(B * B, -15) + ldexpf(1.f, -18);
    const float Ef = ldexpf(R * R + 2.f * R * qa, -19) * sc * sc;
    sW[row] = in_range ? 2.f * (Et + Ef) * 1.0001f : INFINITY;
#pragma unroll
    for (int half8 = 0; half8 < 2; ++half8) {
        uint4 vh, vl;
        __half *th = reinterpret_cast<__half *>(&vh), *tl = reinterpret_cast<__half *>(&vl);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            th[k] = h[8 * half8 + k];
            tl[k] = l[8 * half8 + k];
        }
        const uint32_t off = canon_off(row, 8 * half8);
        *reinterpret_cast<uint4 *>(sA + off) = vh;
        *reinterpret_cast<uint4 *>(sA + kTileBytes + off) = vl;
        *reinterpret_cast<uint4 *>(sA + 2 * kTileBytes + off) = vh;
    }
    // generic-proxy writes that the tensor cores (async proxy) will read
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Persistent: CTA b takes row tiles b, b + gridDim.x, ...  The epilogue warps
// build the next row tile's operands into the other A buffer while the MMAs
// of the current one run; stage, accumulator and A-buffer phases run on
// across row tiles.
template <int MODE>
__global__ void __launch_bounds__(kThreads, 2) k_near_tc(NearArgs P) {
    constexpr int K = NearCfg<MODE>::K, CAP = NearCfg<MODE>::CAP;
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char *sA = smem;                          // 2 buffers x 3 x 4 KB
    unsigned char *sB = smem + 6 * kTileBytes;         // kStages x 8 KB
    float *sQ = reinterpret_cast<float *>(sB + kStages * kStageBytes);   // 2 x kRows x 12
    float *sW = sQ + 2 * kRows * 12;                                     // 2 x kRows
    __shared__ __align__(8) uint64_t bar_full[kStages], bar_empty[kStages], bar_tfull[2], bar_tempty[2],
        bar_afull[2], bar_adone[2], bar_done;
    __shared__ uint32_t tmem_slot;

    const int64_t nrows = (MODE == 0 && P.n_list) ? (int64_t)*P.n_list : P.n;
    const int64_t n_rt = (nrows + kRows - 1) / kRows;
    if ((int64_t)blockIdx.x >= n_rt) return;   // the whole CTA, before any barrier
    const int64_t stride = gridDim.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            dd_mbar_init(dd_smem_addr(&bar_full[s]), 1);
            dd_mbar_init(dd_smem_addr(&bar_empty[s]), 1);
        }
        for (int a = 0; a < 2; ++a) {
            dd_mbar_init(dd_smem_addr(&bar_tfull[a]), 1);
            dd_mbar_init(dd_smem_addr(&bar_tempty[a]), 4);
            dd_mbar_init(dd_smem_addr(&bar_afull[a]), 4);
            dd_mbar_init(dd_smem_addr(&bar_adone[a]), 1);
        }
        dd_mbar_init(dd_smem_addr(&bar_done), 1);
        dd_fence_mbar_init();
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         dd_smem_addr(&tmem_slot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- producer ----------------
            bool ok = true;
            int64_t gt = 0;   // operand tiles issued over all row tiles
            for (int64_t rt = blockIdx.x; ok && rt < n_rt; rt += stride) {
                for (int t = 0; t < P.tpg; ++t, ++gt) {
                    const int s = (int)(gt % kStages);
                    if (gt >= kStages &&
                        !dd_mbar_wait(dd_smem_addr(&bar_empty[s]), (uint32_t)(((gt / kStages) - 1) & 1))) {
                        ok = false;
                        break;
                    }
                    const uint32_t bf = dd_smem_addr(&bar_full[s]);
                    const int64_t tile = t;
                    dd_mbar_expect_tx(bf, kStageBytes);
                    dd_bulk_g2s(dd_smem_addr(sB + s * kStageBytes),
                                reinterpret_cast<const char *>(P.chi) + tile * kTileBytes, kTileBytes, bf);
                    dd_bulk_g2s(dd_smem_addr(sB + s * kStageBytes + kTileBytes),
                                reinterpret_cast<const char *>(P.clo) + tile * kTileBytes, kTileBytes, bf);
                }
            }
            if (!ok) {
                atomicOr(P.err, DEV_ERR_TIMEOUT);
                // drain: wait (bounded) for every issued copy that nobody consumed
                for (int64_t t = (gt > kStages ? gt - kStages : 0); t < gt; ++t)
                    dd_mbar_wait(dd_smem_addr(&bar_full[t % kStages]), (uint32_t)((t / kStages) & 1));
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------- MMA issuer ----------------
            bool ok = true;
            constexpr uint32_t idesc = idesc_f16(kRows, kCols);
            int64_t gt = 0;
            int64_t i = 0;   // row tiles of this CTA
            for (int64_t rt = blockIdx.x; ok && rt < n_rt; rt += stride, ++i) {
                const int b = (int)(i & 1);
                if (!dd_mbar_wait(dd_smem_addr(&bar_afull[b]), (uint32_t)((i >> 1) & 1))) {
                    ok = false;
                    break;
                }
                const uint32_t a0 = dd_smem_addr(sA + b * 3 * kTileBytes);
                for (int t = 0; t < P.tpg; ++t, ++gt) {
                    const int s = (int)(gt % kStages);
                    const int ab = (int)(gt & 1);
                    if (!dd_mbar_wait(dd_smem_addr(&bar_full[s]), (uint32_t)((gt / kStages) & 1))) {
                        ok = false;
                        break;
                    }
                    if (gt >= 2 && !dd_mbar_wait(dd_smem_addr(&bar_tempty[ab]), (uint32_t)(((gt >> 1) - 1) & 1))) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t d = tmem + (uint32_t)ab * kCols;
                    const uint32_t bh = dd_smem_addr(sB + s * kStageBytes);
                    umma_f16(d, umma_desc(a0), umma_desc(bh), idesc, 0u);
                    umma_f16(d, umma_desc(a0 + kTileBytes), umma_desc(bh), idesc, 1u);
                    umma_f16(d, umma_desc(a0 + 2 * kTileBytes), umma_desc(bh + kTileBytes), idesc, 1u);
                    umma_commit(dd_smem_addr(&bar_empty[s]));
                    umma_commit(dd_smem_addr(&bar_tfull[ab]));
                }
                umma_commit(dd_smem_addr(&bar_adone[b]));   // A buffer b is free once these MMAs complete
            }
            if (!ok) atomicOr(P.err, DEV_ERR_TIMEOUT);
            // all issued MMAs complete before TMEM is released
            umma_commit(dd_smem_addr(&bar_done));
            if (!dd_mbar_wait(dd_smem_addr(&bar_done), 0)) atomicOr(P.err, DEV_ERR_TIMEOUT);
        }
    } else {
        // ---------------- epilogue: one row per thread ----------------
        const int quarter = warp & 3;          // the TMEM lane quarter this warp may read
        const int row = quarter * 32 + lane;
        auto publish = [&](int b) {            // this warp's rows of A buffer b are written
            __syncwarp();
            if (lane == 0) dd_mbar_arrive(dd_smem_addr(&bar_afull[b]));
        };
        RowSrc src;
        fetch_index<MODE>(P, nrows, (int64_t)blockIdx.x * kRows + row, src);
        fetch_coords<MODE>(P, src);
        build_row(src, P.s, P.R, row, sA, sQ, sW);
        publish(0);
        bool ok = true;
        int64_t gt = 0;
        int64_t i = 0;
        for (int64_t rt = blockIdx.x; ok && rt < n_rt; rt += stride, ++i) {
            const int b = (int)(i & 1);
            // the next row tile's operands go into the other buffer (free once
            // the MMAs of the row tile before this one are complete): its
            // index now, its coordinates after the first tile, the operands
            // after the second (or the last) one, so that the loads overlap
            // this row tile's epilogue
            const bool next = rt + stride < n_rt;
            if (next) fetch_index<MODE>(P, nrows, (rt + stride) * kRows + row, src);
            auto stage_next = [&](int t, int ntl) {
                if (!next) return true;
                if (t == 0) fetch_coords<MODE>(P, src);
                if (t != (ntl > 1 ? 1 : 0)) return true;
                const int nb = b ^ 1;
                if (i >= 1 &&
                    !__all_sync(0xffffffffu, dd_mbar_wait(dd_smem_addr(&bar_adone[nb]), (uint32_t)(((i - 1) >> 1) & 1)))) {
                    if (lane == 0) atomicOr(P.err, DEV_ERR_TIMEOUT);
                    return false;
                }
                build_row(src, P.s, P.R, row, sA + nb * 3 * kTileBytes, sQ + nb * kRows * 12, sW + nb * kRows);
                publish(nb);
                return true;
            };
            const int64_t r = rt * kRows + row;
            const bool active = r < nrows;
            // the row's kept list: the best tensor-core scores within the
            // window W of its K-th best so far (sorted; +inf: empty);
            // `dropped` is the least score that was within that window when
            // offered but did not fit
            const float W = active ? sW[b * kRows + row] : INFINITY;
            const bool rowok = active && W < INFINITY;
            float sv[CAP];
            int sc[CAP];
            float dropped = INFINITY;
#pragma unroll
            for (int e = 0; e < CAP; ++e) {
                sv[e] = INFINITY;
                sc[e] = -1;
            }
            auto insert = [&](float v, int col) {
                sv[CAP - 1] = v;
                sc[CAP - 1] = col;
#pragma unroll
                for (int e = CAP - 1; e > 0; --e)
                    if (sv[e] < sv[e - 1]) {
                        const float tv = sv[e];
                        sv[e] = sv[e - 1];
                        sv[e - 1] = tv;
                        const int tc = sc[e];
                        sc[e] = sc[e - 1];
                        sc[e - 1] = tc;
                    }
            };
            // scores above the gate can never be needed: the K-th best only falls
            auto gate = [&]() { return sv[K - 1] + W; };
            auto offer = [&](float v, int col) {
                if (v < sv[CAP - 1]) {
                    dropped = fminf(dropped, sv[CAP - 1]);   // the entry pushed out (+inf: none)
                    insert(v, col);
                } else {
                    dropped = fminf(dropped, v);
                }
            };
            for (int t = 0; t < P.tpg; ++t, ++gt) {
                const int ab = (int)(gt & 1);
                // warp-uniform outcome: tcgen05.ld below is .sync.aligned
                if (!__all_sync(0xffffffffu, dd_mbar_wait(dd_smem_addr(&bar_tfull[ab]), (uint32_t)((gt >> 1) & 1)))) {
                    if (lane == 0) atomicOr(P.err, DEV_ERR_TIMEOUT);
                    ok = false;
                    break;
                }
                tc_fence_after();
                const bool use = rowok;
                const int colbase = t * kCols;
                const uint32_t base = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)ab * kCols;
                uint32_t ra[32], rb[32];
                float mina = 0.f, minb = 0.f;
                auto filter = [&](const uint32_t(&rr)[32], float mred, int c) {
                    if (!use || !(mred <= gate())) return;   // most chunks: nothing within the gate
                    const float g = gate();
                    unsigned msk = 0;
#pragma unroll
                    for (int k = 0; k < 32; ++k) msk |= (__uint_as_float(rr[k]) <= g ? 1u : 0u) << k;
                    while (msk) {
                        const int k = __ffs(msk) - 1;
                        msk &= msk - 1;
                        float vk = __uint_as_float(rr[0]);
#pragma unroll
                        for (int kk = 1; kk < 32; ++kk) vk = (k == kk) ? __uint_as_float(rr[kk]) : vk;
                        const int col = colbase + c * 32 + k;
                        if (col < P.Lc && vk <= gate()) offer(vk, col);
                    }
                };
                auto release = [&]() {   // every column of this accumulator is in registers
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) dd_mbar_arrive(dd_smem_addr(&bar_tempty[ab]));
                };
                tmem_ld32_red_async(base, ra, mina);
                tmem_wait_red(ra, mina);
#pragma unroll 1
                for (int c = 0; c < 4; c += 2) {   // ra holds chunk c
                    tmem_ld32_red_async(base + (uint32_t)((c + 1) * 32), rb, minb);
                    filter(ra, mina, c);
                    tmem_wait_red(rb, minb);       // rb holds chunk c + 1
                    if (c + 2 < 4) tmem_ld32_red_async(base + (uint32_t)((c + 2) * 32), ra, mina);
                    else release();
                    filter(rb, minb, c + 1);
                    if (c + 2 < 4) tmem_wait_red(ra, mina);
                }
                if (!stage_next(t, P.tpg)) {
                    ok = false;
                    break;
                }
            }
            if (!ok || !active) continue;
            // every score not kept exceeds thr, unless `dropped` says otherwise
            const float thr = sv[K - 1] + W;
            const bool cert = rowok && sv[K - 1] < INFINITY && dropped > thr;
            if (!cert) {
                const unsigned slot = atomicAdd(P.fb_n, 1u);
                if (slot < P.fb_cap) P.fb[slot] = (MODE == 0) ? (P.list ? P.list[r] : (int32_t)r) : (int32_t)r;
                continue;
            }
            float q[12], qm2[12];
#pragma unroll
            for (int k = 0; k < 12; ++k) {
                q[k] = sQ[(b * kRows + row) * 12 + k];
                qm2[k] = -2.f * q[k];
            }
            float bv[K];
            int bc[K];
#pragma unroll
            for (int k = 0; k < K; ++k) {
                bv[k] = INFINITY;
                bc[k] = -1;
            }
#pragma unroll
            for (int e = 0; e < CAP; ++e) {
                if (!(sv[e] <= thr)) continue;
                const int col = sc[e];
                const float v = alu_score(P.cent, P.cn, col, qm2);
                if (!better(v, col, bv[K - 1], bc[K - 1] < 0 ? 0x7fffffff : bc[K - 1])) continue;
                bv[K - 1] = v;
                bc[K - 1] = col;
#pragma unroll
                for (int k = K - 1; k > 0; --k)
                    if (better(bv[k], bc[k], bv[k - 1], bc[k - 1] < 0 ? 0x7fffffff : bc[k - 1])) {
                        const float tv = bv[k];
                        bv[k] = bv[k - 1];
                        bv[k - 1] = tv;
                        const int tc = bc[k];
                        bc[k] = bc[k - 1];
                        bc[k - 1] = tc;
                    }
            }
            if (MODE == 0) {
                // as the ALU ranking: the K cells ordered by (FP32 distance, index)
                const int64_t qi = P.list ? (int64_t)P.list[r] : r;
                float bd[K];
#pragma unroll
                for (int k = 0; k < K; ++k) bd[k] = bc[k] >= 0 ? dd_dist2_12(P.cent + (size_t)bc[k] * 12, q) : INFINITY;
#pragma unroll
                for (int a = 1; a < K; ++a)
#pragma unroll
                    for (int k = a; k > 0; --k)
                        if (bd[k] < bd[k - 1] || (bd[k] == bd[k - 1] && bc[k] >= 0 && bc[k] < bc[k - 1])) {
                            const float tv = bd[k];
                            bd[k] = bd[k - 1];
                            bd[k - 1] = tv;
                            const int tc = bc[k];
                            bc[k] = bc[k - 1];
                            bc[k - 1] = tc;
                        }
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    P.out_cl[qi * K + k] = bc[k];
                    P.out_d[qi * K + k] = sqrtf(bd[k]);
                }
            } else {
                P.out[r] = bc[0];
            }
        }
    }
    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
    }
}

constexpr size_t kNearSmem = 100 * 1024;   // at most two CTAs (2 x 256 TMEM columns) per SM

template <int MODE>
dd_status launch_near(dd_ctx *ctx, const NearArgs &P, int64_t rows, cudaStream_t s) {
    if (rows <= 0) return DD_OK;
    static_assert(6 * kTileBytes + kStages * kStageBytes + 2 * kRows * 13 * 4 + 1024 <= kNearSmem, "shared memory");
    DD_TRY_CUDA(ctx, cudaFuncSetAttribute(k_near_tc<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)kNearSmem));
    ctx->launches++;
    // persistent: two CTAs per SM at most, each taking every grid-th row tile
    const int64_t tiles = (rows + kRows - 1) / kRows;
    const int64_t grid = std::min<int64_t>(tiles, 2 * (int64_t)ctx->n_sm);
    k_near_tc<MODE><<<(unsigned)grid, kThreads, kNearSmem, s>>>(P);
    DD_TRY_CUDA(ctx, cudaGetLastError());
    return DD_OK;
}

NearArgs base_args(dd_ctx *ctx, const NearTcSet &C, int32_t *fb, unsigned *fb_n, int64_t fb_cap) {
    NearArgs P{};
    P.chi = C.hi;
    P.clo = C.lo;
    P.cent = C.cent;
    P.cn = C.cn;
    P.Lc = (int)C.L;
    P.tpg = (int)((C.L + kCols - 1) / kCols);
    P.s = (float)C.s;
    P.R = C.R;
    P.fb = fb;
    P.fb_n = fb_n;
    P.fb_cap = fb_cap;
    P.err = ctx->dev_err;
    return P;
}

}  // namespace

dd_status dd_near_tc_operands(dd_ctx *ctx, const float *cent, const float *cn, int64_t L, double s,
                              float R, NearTcSet *C, cudaStream_t st) {
    const int64_t L_pad = (L + kCols - 1) / kCols * kCols;
    if (!C->hi || C->rows_pad < L_pad) {
        if (C->hi) dd_free(ctx, C->hi, (size_t)C->rows_pad * 64);
        C->hi = C->lo = nullptr;
        void *p = nullptr;
        DD_TRY(dd_alloc(ctx, &p, (size_t)L_pad * 64, "tensor-core centroid operands"));
        C->hi = (__half *)p;
        C->lo = C->hi + (size_t)L_pad * 16;
        C->rows_pad = L_pad;
    }
    C->cent = cent;
    C->cn = cn;
    C->L = L;
    C->s = s;
    C->R = R;
    return dd_tc_split_rows(ctx, cent, L, L_pad, s, C->hi, C->lo, st);
}

void dd_near_tc_free(dd_ctx *ctx, NearTcSet *C) {
    if (C->hi) dd_free(ctx, C->hi, (size_t)C->rows_pad * 64);
    *C = NearTcSet{};
}

dd_status dd_near_tc_rank(dd_ctx *ctx, const NearTcSet &C, const QueryRec *rec, int64_t m, const int32_t *list,
                          const unsigned *n_list, int32_t *out_cl, float *out_d, int32_t *fb, unsigned *fb_n,
                          cudaStream_t s) {
    if (C.L < NearCfg<0>::CAP) return dd_fail(ctx, DD_ERR_STATE, "tensor-core ranking needs 16 centroids or more");
    NearArgs P = base_args(ctx, C, fb, fb_n, m);
    P.rec = rec;
    P.list = list;
    P.n_list = n_list;
    P.n = m;
    P.out_cl = out_cl;
    P.out_d = out_d;
    return launch_near<0>(ctx, P, m, s);
}

dd_status dd_near_tc_assign(dd_ctx *ctx, const NearTcSet &C, const float *z, int64_t n, int32_t *out, int32_t *fb,
                            unsigned *fb_n, int64_t fb_cap, cudaStream_t s) {
    if (C.L < NearCfg<1>::CAP) return dd_fail(ctx, DD_ERR_STATE, "tensor-core assignment needs 4 centroids or more");
    NearArgs P = base_args(ctx, C, fb, fb_n, fb_cap);
    P.z = z;
    P.n = n;
    P.out = out;
    return launch_near<1>(ctx, P, n, s);
}
