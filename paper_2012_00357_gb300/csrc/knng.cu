// Approximate data projection by a greedy walk in the k-nearest-neighbour
// graph of the data set (Sec. 4.4).
//
// Graph (built once per data set, after the two-level k-means tree, as the
// paper builds it with its k-means tree): every point is linked to the k
// nearest other points that a search of the tree at accuracy f_d (Eq. 13)
// finds for it, nearest first.  One warp per point keeps the k best in a
// lane-distributed sorted list (bitonic sort and merge of 32 candidates at a
// time, candidates that cannot enter the list are dropped by one compare).
// Nodes are positions in the cluster-sorted copy zs, so that neighbours lie
// mostly in the point's own leaf and a walk reads nearby rows.
//
// Walk (every DD iteration): one warp per query, one lane per neighbour.  The
// walk starts at the previous nearest point (warm start, Sec. 4.4), or without
// one at data point SplitMix64(i) mod N for query i (the first output of a
// SplitMix64 generator seeded with i); it evaluates all neighbours of the
// current point and moves to the nearest of them while that one is strictly
// nearer to the query, ending at a local minimum of the graph or after f_s node
// changes.  The moving-query radius of Eq. (14) keeps queries that moved less
// than (d2 - d1)/2 without a walk.  The answer is rescored with Eq. (3) in FP64.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <vector>

#include "dd_internal.cuh"

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kBuildChunk = 1 << 20;     // points searched per build launch
constexpr int kFineB = 8;                // leaves visited per cell at most
constexpr int kFinePerLaneB = 16;        // leaves per cell <= 512

__device__ __forceinline__ float dist2_12(const float *a, const float (&q)[12]) {
    const float4 *p = reinterpret_cast<const float4 *>(a);
    const float4 u = __ldg(p), v = __ldg(p + 1), w = __ldg(p + 2);
    float d, s = 0.f;
    d = u.x - q[0]; s = fmaf(d, d, s);
    d = u.y - q[1]; s = fmaf(d, d, s);
    d = u.z - q[2]; s = fmaf(d, d, s);
    d = u.w - q[3]; s = fmaf(d, d, s);
    d = v.x - q[4]; s = fmaf(d, d, s);
    d = v.y - q[5]; s = fmaf(d, d, s);
    d = v.z - q[6]; s = fmaf(d, d, s);
    d = v.w - q[7]; s = fmaf(d, d, s);
    d = w.x - q[8]; s = fmaf(d, d, s);
    d = w.y - q[9]; s = fmaf(d, d, s);
    d = w.z - q[10]; s = fmaf(d, d, s);
    d = w.w - q[11]; s = fmaf(d, d, s);
    return s;
}

__device__ __forceinline__ bool pair_less(float a, int pa, float b, int pb) { return a < b || (a == b && pa < pb); }

// Lane-distributed list of R x 32 (squared distance, position) entries in
// ascending order: entry 32 r + lane is (d[r], p[r]) of that lane; entries
// with d = +inf are empty.
template <int R>
struct TopK {
    float d[R];
    int p[R];
};

__device__ __forceinline__ void cas(float &d, int &p, int st, bool keep_min, int lane) {
    const float od = __shfl_xor_sync(kFull, d, st);
    const int op = __shfl_xor_sync(kFull, p, st);
    const bool olt = pair_less(od, op, d, p);
    if (keep_min == ((lane & st) == 0) ? olt : !olt) {
        d = od;
        p = op;
    }
}

// ascending sort of a bitonic sequence held one entry per lane
__device__ __forceinline__ void bitonic_clean(float &d, int &p, int lane) {
#pragma unroll
    for (int st = 16; st > 0; st >>= 1) cas(d, p, st, true, lane);
}

// Offer one candidate per lane (d = +inf: none).  Keeps the R x 32 smallest
// of list and candidates in order; candidates not below entry k-1 are
// dropped.  The sorted candidates cascade through the list: at level r the
// 32 smallest of (level r, carry) stay and the 32 largest are carried on,
// so every level stays sorted and not below the one before it.
template <int R>
__device__ __forceinline__ void topk_offer(TopK<R> &L, float d, int p, int k, int lane) {
    const int rk = (k - 1) >> 5, lk = (k - 1) & 31;
    float td = L.d[0];
    int tp = L.p[0];
#pragma unroll
    for (int r = 1; r < R; ++r)
        if (r == rk) {
            td = L.d[r];
            tp = L.p[r];
        }
    td = __shfl_sync(kFull, td, lk);
    tp = __shfl_sync(kFull, tp, lk);
    const bool pass = pair_less(d, p, td, tp);
    if (!__any_sync(kFull, pass)) return;
    if (!pass) {
        d = INFINITY;
        p = INT_MAX;
    }
    // bitonic sort of the candidates, ascending over the lanes
#pragma unroll
    for (int size = 2; size <= 32; size <<= 1) {
#pragma unroll
        for (int st = size >> 1; st > 0; st >>= 1) cas(d, p, st, (lane & size) == 0, lane);
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        // the i-th entry of the level against the (31-i)-th carried one:
        // elementwise min and max are bitonic halves of the 64
        const float rd = __shfl_sync(kFull, d, 31 - lane);
        const int rp = __shfl_sync(kFull, p, 31 - lane);
        const bool rl = pair_less(rd, rp, L.d[r], L.p[r]);
        const float hd = rl ? L.d[r] : rd;
        const int hp = rl ? L.p[r] : rp;
        if (rl) {
            L.d[r] = rd;
            L.p[r] = rp;
        }
        bitonic_clean(L.d[r], L.p[r], lane);
        if (r + 1 == R || !__any_sync(kFull, hd < INFINITY)) break;
        d = hd;
        p = hp;
        bitonic_clean(d, p, lane);
    }
}

// Query records of the build: the rows p0 .. p0+n-1 of zs.
__global__ void k_rec_rows(const float *__restrict__ zs, int64_t p0, int64_t n, QueryRec *__restrict__ rec) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n) return;
    QueryRec r;
    float qn = 0.f;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        r.q[k] = zs[(p0 + t) * 12 + k];
        qn = fmaf(r.q[k], r.q[k], qn);
    }
    r.w2 = 0.f;
    r.qn = qn;
    r.pad[0] = r.pad[1] = 0.f;
    rec[t] = r;
}

struct BuildArgs {
    const float *zs;            // [N x 12] cluster-sorted mapped coordinates
    const int64_t *offs;        // [L + 1] leaf ranges of zs
    const float *radius;        // [L] leaf radii
    const float *centf;         // [L x 12] leaf centroids
    const float *rad1;          // [L1] cell radii
    int L2;                     // leaves per cell
    const QueryRec *rec;        // [n] rows p0 .. p0+n-1
    const int32_t *cand_cl;     // [n x kAnnCand] nearest cells
    const float *cand_d;
    int64_t p0, n;
    int k;
    float f_d;
    int32_t *nbr;               // [N x k] neighbour positions (output)
    unsigned long long *evals;  // point distances evaluated
};

// k nearest other points of every row by the tree search of Eq. (13) with d_c
// the current k-th distance: the nearest cell and its nearest leaf always, a
// further cell or leaf (in order of centroid distance, at most kFineB leaves
// per cell) when d(x, c) - f_d r < d_c.
template <int R>
__global__ void __launch_bounds__(256) k_knn_build(BuildArgs A) {
    const int lane = threadIdx.x & 31;
    const int64_t t = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (t >= A.n) return;
    const int64_t self = A.p0 + t;
    float q[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) q[k] = A.rec[t].q[k];
    TopK<R> L;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        L.d[r] = INFINITY;
        L.p[r] = INT_MAX;
    }
    unsigned long long ev = 0;
    const int rk = (A.k - 1) >> 5, lk = (A.k - 1) & 31;
    auto dc = [&]() {
        float v = L.d[0];
#pragma unroll
        for (int r = 1; r < R; ++r)
            if (r == rk) v = L.d[r];
        return sqrtf(__shfl_sync(kFull, v, lk));
    };
    auto scan = [&](int l) {
        const int64_t a = A.offs[l], b = A.offs[l + 1];
        for (int64_t base = a; base < b; base += 32) {
            const int64_t p = base + lane;
            float d = INFINITY;
            int pp = INT_MAX;
            if (p < b && p != self) {
                d = dist2_12(A.zs + p * 12, q);
                pp = (int)p;
            }
            topk_offer<R>(L, d, pp, A.k, lane);
        }
        ev += (unsigned long long)(b - a);
    };
    for (int k1 = 0; k1 < kAnnCand; ++k1) {
        const int C = A.cand_cl[t * kAnnCand + k1];
        if (C < 0) break;
        const float dC = A.cand_d[t * kAnnCand + k1];
        if (!(k1 == 0 || dC - A.f_d * A.rad1[C] < dc())) continue;
        float fd[kFinePerLaneB];
        unsigned vis = 0;
#pragma unroll
        for (int u = 0; u < kFinePerLaneB; ++u) {
            const int f = lane + 32 * u;
            fd[u] = (f < A.L2) ? sqrtf(dist2_12(A.centf + ((size_t)C * A.L2 + f) * 12, q)) : INFINITY;
        }
        for (int k2 = 0; k2 < kFineB; ++k2) {
            float md = INFINITY;
            int mu = -1;
#pragma unroll
            for (int u = 0; u < kFinePerLaneB; ++u)
                if (!((vis >> u) & 1u) && fd[u] < md) {
                    md = fd[u];
                    mu = u;
                }
            int ml = mu >= 0 ? lane + 32 * mu : INT_MAX;
            for (int o = 16; o > 0; o >>= 1) {
                const float od = __shfl_xor_sync(kFull, md, o);
                const int ol = __shfl_xor_sync(kFull, ml, o);
                if (od < md || (od == md && ol < ml)) {
                    md = od;
                    ml = ol;
                }
            }
            if (!(md < INFINITY)) break;
            if ((ml & 31) == lane) vis |= 1u << (ml >> 5);
            const int l = C * A.L2 + ml;
            if ((k1 == 0 && k2 == 0) || md - A.f_d * A.radius[l] < dc()) scan(l);
        }
    }
#pragma unroll
    for (int r = 0; r < R; ++r)
        if (32 * r + lane < A.k) A.nbr[self * A.k + 32 * r + lane] = L.d[r] < INFINITY ? L.p[r] : -1;
    if (lane == 0) atomicAdd(A.evals, ev);
}

__global__ void k_pos_of(const int32_t *__restrict__ perm, int64_t N, int32_t *__restrict__ pos_of) {
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p < N) pos_of[perm[p]] = (int32_t)p;
}

// Export: neighbour positions -> data indices.
__global__ void k_graph_export(const int32_t *__restrict__ nbr, const int32_t *__restrict__ perm, int64_t n,
                               int32_t *__restrict__ out) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n) return;
    const int32_t p = nbr[t];
    out[t] = p >= 0 ? perm[p] : -1;
}

__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

struct WalkArgs {
    const float *zs;
    const int32_t *perm;        // sorted position -> data index
    const int32_t *pos_of;      // data index -> sorted position
    const int32_t *nbr;         // [N x k]
    int k;
    const float *z32;           // original order, for the warm start
    const QueryRec *rec;
    int64_t m, N;
    int f_s;
    const int32_t *prev;        // may be null
    const float *mot_q;         // motion record (may be null)
    const float *mot_d;
    int32_t *idx;
    float *d1, *d2;             // plain squared distances of the answer / second
    unsigned long long *counters;   // [0] distances, [1] skipped, [5] points read, [6] node changes,
                                    // [7] walks stopped by f_s
};

template <int NC>
__device__ __forceinline__ void walk_one(const WalkArgs &A, int64_t i, int lane, unsigned long long *sc) {
    float q[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) q[k] = A.rec[i].q[k];
    int p;
    float dcur;
    const int j0 = A.prev ? A.prev[i] : -1;
    if (j0 >= 0 && j0 < A.N) {
        dcur = dist2_12(A.z32 + (size_t)j0 * 12, q);
        if (A.mot_q) {
            float mv = 0.f;
#pragma unroll
            for (int k = 0; k < 12; ++k) {
                const float t = q[k] - A.mot_q[i * 12 + k];
                mv = fmaf(t, t, mv);
            }
            mv = sqrtf(mv);
            const float r1 = A.mot_d[i * kMotStride], r2 = A.mot_d[i * kMotStride + 1];
            if (mv < 0.5f * (r2 - r1)) {          // Eq. (14)
                if (lane == 0) {
                    A.idx[i] = j0;
                    A.d1[i] = dcur;
                    const float lb = fmaxf(r2 - mv, 0.f);
                    A.d2[i] = lb * lb;
                    atomicAdd(sc + 1, 1ull);
                }
                return;
            }
        }
        p = A.pos_of[j0];
    } else {
        // no previous neighbour: data point SplitMix64(i) mod N
        const int64_t j = (int64_t)(splitmix64((uint64_t)i) % (uint64_t)A.N);
        p = A.pos_of[j];
        dcur = dist2_12(A.z32 + (size_t)j * 12, q);
    }
    float second = INFINITY;
    int moves = 0;
    bool bounded = false;
    unsigned long long ev = 1;
    for (;;) {
        if (A.f_s > 0 && moves >= A.f_s) {
            bounded = true;
            break;
        }
        // every lane takes up to NC neighbours (all loads issued before any
        // reduction); nearest one (ties to the lower data index) and the
        // smallest distance among the others
        int t[NC];
        float d[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) t[c] = 32 * c + lane < A.k ? A.nbr[(size_t)p * A.k + 32 * c + lane] : -1;
#pragma unroll
        for (int c = 0; c < NC; ++c) d[c] = t[c] >= 0 ? dist2_12(A.zs + (size_t)t[c] * 12, q) : INFINITY;
        float ld = INFINITY, ls = INFINITY;      // lane's nearest and the lane's other minimum
        int lt = -1, nv = 0;
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            if (t[c] < 0) continue;
            ++nv;
            bool better = d[c] < ld;
            if (d[c] == ld && lt >= 0) better = A.perm[t[c]] < A.perm[lt];
            if (better) {
                ls = fminf(ls, ld);
                ld = d[c];
                lt = t[c];
            } else {
                ls = fminf(ls, d[c]);
            }
        }
        for (int o = 16; o > 0; o >>= 1) nv += __shfl_xor_sync(kFull, nv, o);
        ev += (unsigned long long)nv;
        float bd = ld;
        for (int o = 16; o > 0; o >>= 1) bd = fminf(bd, __shfl_xor_sync(kFull, bd, o));
        const bool at_min = lt >= 0 && ld == bd;
        const unsigned tie = __ballot_sync(kFull, at_min);
        int bt = -1, wl = -1;
        if (__popc(tie) == 1) {
            wl = __ffs(tie) - 1;
        } else if (tie) {
            const int j = at_min ? A.perm[lt] : INT_MAX;
            int jb = j;
            for (int o = 16; o > 0; o >>= 1) jb = min(jb, __shfl_xor_sync(kFull, jb, o));
            wl = __ffs(__ballot_sync(kFull, at_min && j == jb)) - 1;
        }
        if (wl >= 0) bt = __shfl_sync(kFull, lt, wl);
        float od = lane == wl ? ls : fminf(ld, ls);
        for (int o = 16; o > 0; o >>= 1) od = fminf(od, __shfl_xor_sync(kFull, od, o));
        if (bt >= 0 && bd < dcur) {
            second = fminf(second, fminf(dcur, od));
            dcur = bd;
            p = bt;
            ++moves;
        } else {
            second = fminf(second, bd);
            break;
        }
    }
    // a walk stopped by f_s is not at a local minimum: radius 0 for Eq. (14)
    if (bounded) second = dcur;
    if (lane == 0) {
        A.idx[i] = A.perm[p];
        A.d1[i] = dcur;
        A.d2[i] = second;
        atomicAdd(sc + 0, ev);
        atomicAdd(sc + 2, (unsigned long long)moves);
        if (bounded) atomicAdd(sc + 3, 1ull);
    }
}

template <int NC>
__global__ void __launch_bounds__(256) k_knng_walk(WalkArgs A) {
    __shared__ unsigned long long sc[4];
    if (threadIdx.x < 4) sc[threadIdx.x] = 0ull;
    __syncthreads();
    const int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (i < A.m) walk_one<NC>(A, i, threadIdx.x & 31, sc);
    __syncthreads();
    if (threadIdx.x == 0) {
        if (sc[0]) {
            atomicAdd(A.counters + 0, sc[0]);
            atomicAdd(A.counters + 5, sc[0]);
        }
        if (sc[1]) atomicAdd(A.counters + 1, sc[1]);
        if (sc[2]) atomicAdd(A.counters + 6, sc[2]);
        if (sc[3]) atomicAdd(A.counters + 7, sc[3]);
    }
}

}  // namespace

dd_status dd_build_knng(dd_dataset *ds, const dd_dataset_opts &o) {
    dd_ctx *ctx = ds->ctx;
    const AnnIndex &a = ds->ann;
    KnnGraph &g = ds->knn;
    if (o.knn_k < 1 || o.knn_k > 128) return dd_fail(ctx, DD_ERR_ARG, "knn_k must be 1 .. 128");
    if (!(o.knn_fd >= 0.0 && o.knn_fd <= 1.0)) return dd_fail(ctx, DD_ERR_ARG, "knn_fd outside [0, 1]");
    if (a.levels != 2 || !a.nlist)
        return dd_fail(ctx, DD_ERR_ARG, "the k-NN graph is built with the two-level tree (ann_levels = 2)");
    cudaStream_t s = ctx->stream;
    const int64_t N = ds->N;
    void *p = nullptr, *p2 = nullptr;
    DD_TRY(dd_alloc(ctx, &p, (size_t)N * o.knn_k * 4, "k-NN graph"));
    if (dd_status st = dd_alloc(ctx, &p2, (size_t)N * 4, "k-NN graph positions"); st != DD_OK) {
        dd_free(ctx, p, (size_t)N * o.knn_k * 4);
        return st;
    }
    g.k = o.knn_k;
    g.fd = (float)o.knn_fd;
    g.nbr = (int32_t *)p;
    g.pos_of = (int32_t *)p2;
    ctx->launches++;
    k_pos_of<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(a.perm, N, g.pos_of);
    DD_TRY_CUDA(ctx, cudaGetLastError());

    auto r256 = [](size_t b) { return (b + 255) / 256 * 256; };
    const int64_t B = std::min<int64_t>(N, kBuildChunk);
    const size_t b_rec = r256((size_t)B * sizeof(QueryRec)), b_c = r256((size_t)B * kAnnCand * 4);
    void *w = nullptr;
    DD_TRY(dd_workspace(ctx, WS_ANN_BUILD, b_rec + 2 * b_c + 256, &w));
    char *c = (char *)w;
    QueryRec *rec = (QueryRec *)c;
    int32_t *cand_cl = (int32_t *)(c + b_rec);
    float *cand_d = (float *)(c + b_rec + b_c);
    unsigned long long *evals = (unsigned long long *)(c + b_rec + 2 * b_c);
    DD_TRY_CUDA(ctx, cudaMemsetAsync(evals, 0, 8, s));
    for (int64_t p0 = 0; p0 < N; p0 += B) {
        const int64_t n = std::min<int64_t>(B, N - p0);
        ctx->launches += 2;
        k_rec_rows<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(a.zs, p0, n, rec);
        DD_TRY_CUDA(ctx, cudaGetLastError());
        DD_TRY(dd_ann_rank_cells(ds, rec, n, cand_cl, cand_d, s));
        BuildArgs A{a.zs, a.offs, a.radius, a.cent, a.rad1, a.L2, rec, cand_cl, cand_d, p0, n, g.k, g.fd, g.nbr,
                    evals};
        const unsigned grid = (unsigned)((n * 32 + 255) / 256);
        if (g.k <= 32) k_knn_build<1><<<grid, 256, 0, s>>>(A);
        else if (g.k <= 64) k_knn_build<2><<<grid, 256, 0, s>>>(A);
        else if (g.k <= 96) k_knn_build<3><<<grid, 256, 0, s>>>(A);
        else k_knn_build<4><<<grid, 256, 0, s>>>(A);
        DD_TRY_CUDA(ctx, cudaGetLastError());
    }
    ds->bytes += (size_t)N * (g.k + 1) * 4;
    return DD_OK;
}

void dd_free_knng(dd_dataset *ds) {
    KnnGraph &g = ds->knn;
    if (!g.k) return;
    dd_free(ds->ctx, g.nbr, (size_t)ds->N * g.k * 4);
    dd_free(ds->ctx, g.pos_of, (size_t)ds->N * 4);
    g = KnnGraph();
}

dd_status dd_search_knng(dd_dataset *ds, const double *y_dev, int64_t m, int f_s, const int32_t *prev_idx_dev,
                         AnnMotion *mot, SearchOut out, dd_search_stats *st, cudaStream_t s) {
    dd_ctx *ctx = ds->ctx;
    const KnnGraph &g = ds->knn;
    if (!g.k) return dd_fail(ctx, DD_ERR_STATE, "graph search needs the k-NN graph (knn_k)");
    if (f_s < 0) return dd_fail(ctx, DD_ERR_ARG, "f_s < 0");
    if (m == 0) return DD_OK;
    auto r256 = [](size_t b) { return (b + 255) / 256 * 256; };
    const size_t b_rec = r256((size_t)m * sizeof(QueryRec)), b_f = r256((size_t)m * 4);
    void *w = nullptr;
    DD_TRY(dd_workspace(ctx, WS_ANN, b_rec + 2 * b_f + 256, &w));
    char *c = (char *)w;
    QueryRec *rec = (QueryRec *)c;
    float *d1f = (float *)(c + b_rec);
    float *d2f = (float *)(c + b_rec + b_f);
    unsigned long long *counters = (unsigned long long *)(c + b_rec + 2 * b_f);
    DD_TRY_CUDA(ctx, cudaMemsetAsync(counters, 0, 64, s));
    DD_TRY(dd_map_queries(ds, y_dev, m, nullptr, rec, s));
    if (st) DD_TRY_CUDA(ctx, dd_event_record(ctx, ctx->ev_scan[0], s));
    WalkArgs A{ds->ann.zs, ds->ann.perm, g.pos_of, g.nbr, g.k, ds->z32, rec, m, ds->N, f_s, prev_idx_dev,
               mot ? mot->q : nullptr, mot ? mot->d : nullptr, out.idx, d1f, d2f, counters};
    ctx->launches++;
    const unsigned grid = (unsigned)((m * 32 + 255) / 256);
    if (g.k <= 32) k_knng_walk<1><<<grid, 256, 0, s>>>(A);
    else if (g.k <= 64) k_knng_walk<2><<<grid, 256, 0, s>>>(A);
    else if (g.k <= 96) k_knng_walk<3><<<grid, 256, 0, s>>>(A);
    else k_knng_walk<4><<<grid, 256, 0, s>>>(A);
    DD_TRY_CUDA(ctx, cudaGetLastError());
    if (st) DD_TRY_CUDA(ctx, dd_event_record(ctx, ctx->ev_scan[1], s));
    DD_TRY(dd_ann_finish(ds, y_dev, m, rec, out.idx, d2f, out.d2, out.d2nd, s));
    // the walk's skip does not depend on f_d (its record is stored as made at f_d = 1)
    if (mot && out.d2 && out.d2nd) DD_TRY(dd_ann_motion_update(ctx, rec, m, out.d2, out.d2nd, 1.0, nullptr, 0, mot, s));
    if (st && ctx->defer) {
        DD_TRY_CUDA(ctx, cudaMemcpyAsync(ctx->defer->ann, counters, 8 * sizeof(unsigned long long),
                                         cudaMemcpyDeviceToDevice, s));
    } else if (st) {
        unsigned long long h[8];
        DD_TRY_CUDA(ctx, cudaMemcpyAsync(h, counters, sizeof(h), cudaMemcpyDeviceToHost, s));
        DD_TRY_CUDA(ctx, cudaStreamSynchronize(s));
        float ms = 0.f;
        DD_TRY_CUDA(ctx, cudaEventElapsedTime(&ms, ctx->ev_scan[0], ctx->ev_scan[1]));
        st->scan_ms += ms;
        st->distances += (int64_t)h[0];
        st->points += (int64_t)h[5];
        st->skipped += (int64_t)h[1];
        st->moves += (int64_t)h[6];
    }
    return DD_OK;
}

extern "C" int dd_dataset_knn_k(const dd_dataset *ds) { return ds ? ds->knn.k : 0; }

extern "C" dd_status dd_dataset_knn_graph(dd_dataset *ds, int32_t *nbr) {
    if (!ds) return DD_ERR_ARG;
    dd_ctx *ctx = ds->ctx;
    const KnnGraph &g = ds->knn;
    if (!g.k) return dd_fail(ctx, DD_ERR_STATE, "dd_dataset_knn_graph: no graph built");
    if (!nbr) return dd_fail(ctx, DD_ERR_ARG, "dd_dataset_knn_graph: NULL argument");
    DD_TRY_CUDA(ctx, cudaSetDevice(ctx->device));
    cudaStream_t s = ctx->stream;
    const int64_t n = ds->N * g.k;
    void *w = nullptr;
    DD_TRY(dd_workspace(ctx, WS_MISC, (size_t)n * 4, &w));
    int32_t *tmp = (int32_t *)w;
    // rows in sorted order -> rows in data order: row of point j is row pos_of[j]
    ctx->launches++;
    k_graph_export<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(g.nbr, ds->ann.perm, n, tmp);
    DD_TRY_CUDA(ctx, cudaGetLastError());
    std::vector<int32_t> h((size_t)n), pos((size_t)ds->N);
    DD_TRY_CUDA(ctx, cudaMemcpyAsync(h.data(), tmp, (size_t)n * 4, cudaMemcpyDeviceToHost, s));
    DD_TRY_CUDA(ctx, cudaMemcpyAsync(pos.data(), g.pos_of, (size_t)ds->N * 4, cudaMemcpyDeviceToHost, s));
    DD_TRY_CUDA(ctx, cudaStreamSynchronize(s));
    for (int64_t j = 0; j < ds->N; ++j)
        std::memcpy(nbr + j * g.k, h.data() + (size_t)pos[j] * g.k, (size_t)g.k * 4);
    return DD_OK;
}
