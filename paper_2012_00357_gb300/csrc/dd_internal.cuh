// Internal declarations shared by the translation units of libdd.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/dd.h"

// ---------------------------------------------------------------------------
// Error plumbing
// ---------------------------------------------------------------------------
struct DDError {
    dd_status st;
    std::string msg;
};

#define DD_TRY_CUDA(ctx, call)                                                      \
    do {                                                                            \
        cudaError_t e_ = (call);                                                    \
        if (e_ != cudaSuccess) {                                                    \
            return dd_fail((ctx), DD_ERR_CUDA, std::string(#call) + ": " +          \
                                                   cudaGetErrorString(e_));         \
        }                                                                           \
    } while (0)

#define DD_TRY(x)                                                                   \
    do {                                                                            \
        dd_status s_ = (x);                                                         \
        if (s_ != DD_OK) return s_;                                                 \
    } while (0)

// Device error word bits (written by kernels, read by the host after a call).
enum : unsigned {
    DEV_ERR_TIMEOUT = 1u,      // a bounded wait expired
    DEV_ERR_BOUNDS = 2u,       // an index failed its bounds check
};

// Wall-clock limit of every device-side spin wait.
constexpr unsigned long long kWaitLimitNs = 2000000000ull;   // 2 s

__device__ __forceinline__ unsigned long long dd_globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// ---------------------------------------------------------------------------
// Metric maps of a data set: C, C^{-1}, C^{1/2}, C^{-1/2}, the centre of the
// stored coordinates.  Passed to kernels by value.
// ---------------------------------------------------------------------------
struct MetricMaps {
    double C[36];
    double Cinv[36];
    double Ch[36];
    double Cmh[36];
    double mu[12];
};

// ---------------------------------------------------------------------------
// Context and data set
// ---------------------------------------------------------------------------
struct Workspace {
    void *ptr = nullptr;
    size_t bytes = 0;
};

// Search counters that a step captured into a CUDA graph copies to device
// memory instead of reading them back in the middle of the step; the host
// reads them after the step.
struct DeferredStats {
    unsigned long long fb;       // exact search: queries re-searched in FP64
    unsigned long long ann[8];   // approximate search: point distances, skipped, exact re-search, fine
                                 // centroids, distinct points, points read, graph node changes,
                                 // walks stopped by f_s
};

struct StepPlan;

struct dd_ctx {
    int device = 0;
    int n_sm = 0;
    size_t budget = 0;
    size_t in_use = 0;
    cudaStream_t stream = nullptr;
    std::string err;
    unsigned *dev_err = nullptr;        // device error word
    // grow-only scratch buffers keyed by purpose
    Workspace ws[13];
    int64_t launches = 0;               // kernels launched (instrumentation)
    int tc_epi[3] = {0, 0, 0};          // tuned tensor-core scan variants (uncertified, certified nearest, certified k nearest)
    std::map<int64_t, int> fp32_splits; // tuned data splits of the FP32 scan, per query-tile count
    cudaEvent_t ev_scan[2] = {nullptr, nullptr};   // brackets the dominant scan kernel
    uint64_t ws_gen = 0;                // bumped whenever a workspace is reallocated
    bool capturing = false;             // a step is being captured: no host syncs, no allocation
    DeferredStats *defer = nullptr;     // set while enqueuing a captured step (device counters)
    std::vector<StepPlan *> plans;      // cached batched-step plans (batch.cu)
    std::vector<uint64_t> last_batch;   // solver ids of the previous batched step
};

// Record a timing event on s; while a step is being captured the record
// becomes a node of the graph, so that every replay records it again.
inline cudaError_t dd_event_record(const dd_ctx *ctx, cudaEvent_t e, cudaStream_t s) {
    return ctx->capturing ? cudaEventRecordWithFlags(e, s, cudaEventRecordExternal) : cudaEventRecord(e, s);
}

// Free the cached batched-step plans that hold solver `id` (all plans if id
// is 0); they keep device pointers into the solvers' state.
void dd_plans_drop(dd_ctx *ctx, uint64_t id);

enum WsSlot {
    WS_SEARCH = 0, WS_QUERY = 1, WS_MISC = 2, WS_SOLVE = 3, WS_TC = 4, WS_ANN = 5, WS_ANN_SCAN = 6, WS_ANN_BUILD = 7,
    WS_BATCH = 8, WS_BATCH_CG = 9, WS_ANN_PAIRS = 10, WS_SUBSET = 11, WS_NEAR = 12
};

// Coarse cells a tree search ranks per query (ann.cu).
constexpr int kAnnCand = 8;

// k-nearest-neighbour graph of DD_SEARCH_KNNG (knng.cu).  Nodes are positions
// of the cluster-sorted copy AnnIndex::zs.
struct KnnGraph {
    int k = 0;
    float fd = 0.f;
    int32_t *nbr = nullptr;     // [N x k] neighbour positions, nearest first (-1: none)
    int32_t *pos_of = nullptr;  // [N] sorted position of every original point
};

// Tensor-core operands of a centroid set (near_tc.cu).
struct NearTcSet {
    __half *hi = nullptr, *lo = nullptr;   // split FP16 operand tiles [rows_pad x 16] each
    int64_t rows_pad = 0;
    const float *cent = nullptr;           // FP32 centroids [L x 12] and |c|^2 [L]
    const float *cn = nullptr;
    int64_t L = 0;
    double s = 0.0;                        // operand scale
    float R = 0.f;                         // bound on |c|
};

struct AnnIndex {
    int nlist = 0;
    float *cent = nullptr;      // [Lp x 12] centroids (centred mapped coordinates)
    float *cn = nullptr;        // [Lp] |centroid|^2 (padding rows: huge)
    float *radius = nullptr;    // [Lp] max distance centroid -> member
    int64_t *offs = nullptr;    // [Lp + 1] cluster ranges in the sorted order
    int32_t *perm = nullptr;    // [N] original index of sorted position
    int32_t *cluster_of = nullptr; // [N] cluster of each original point
    float *zs = nullptr;        // [N x 12] mapped coordinates in sorted order
    float rmax = 0.f;           // largest radius
    int nonempty = 0;
    // two-level tree (levels == 2): L1 coarse cells, each with L2 leaves
    // (leaf C * L2 + f belongs to cell C); the leaves above are the fine level
    int levels = 1;
    int L1 = 0, L2 = 0;
    float *cent1 = nullptr;     // [L1p x 12]
    float *cn1 = nullptr;       // [L1p]
    float *rad1 = nullptr;      // [L1p]
    float r1max = 0.f;
    float *lrad1 = nullptr;     // [L1p] largest leaf radius of every cell
    // tensor-core operands of the ranked centroid set (cells, or the clusters
    // of one level); hi null: the ranking runs on the ALU only
    NearTcSet rank_tc;
    int64_t build_fallback = 0; // build rows the tensor-core passes left to the ALU
};

// Moving-query record of the approximate search (Eq. 14), per query:
// previous mapped query (centred FP32), the plain distance of its answer
// (rounded up), a plain lower bound on the distance of every other data
// point (rounded down; the bound of the search's cluster model at its f_d)
// and the f_d the record was made at.  A record is used only by a search at
// the same or a lower f_d; d = 0 disables the skip.
constexpr int kMotStride = 4;   // floats per query in AnnMotion::d: (d1, d2 bound, f_d, unused)
struct AnnMotion {
    float *q;      // [m x 12]
    float *d;      // [m x kMotStride]
};

// Host-side setup of the constraint projection for one mesh: element
// stiffness, stencil tables, smoother weight and coarse-level inverse.  A
// function of the mesh and the metric only, so the solves of a data set on
// the same mesh share one copy.
struct SolverSetup {
    int nx = 0, ny = 0, nz = 0, top = 0;
    double lx = 0, ly = 0, lz = 0;
    std::vector<double> Ke, St64;
    std::vector<float> St32, Kinv;
    double omega = 0;
};

struct dd_dataset {
    dd_ctx *ctx = nullptr;
    int64_t N = 0, N_pad = 0;
    const float *raw = nullptr;  // [N x 12] (eps, sig) as loaded
    bool owns_raw = true;
    float *z32 = nullptr;        // [N_pad x 12] centred mapped coordinates, FP32
    float *zn = nullptr;         // [N_pad] |z32|^2 (padding: huge)
    double R = 0.0;              // max_j |z32_j|
    double maxabs = 0.0;         // max_j,k |z32_jk|
    MetricMaps M;
    // tensor-core operands (search_tc.cu): split FP16 copies of s*z32 in the
    // UMMA canonical K-major layout, hi = fp16(s z), lo = fp16(s z - hi)
    __half *z16hi = nullptr;     // [N_pad x 16]
    __half *z16lo = nullptr;     // [N_pad x 16]
    double scale16 = 0.0;        // power-of-two scale s
    AnnIndex ann;
    KnnGraph knn;
    size_t bytes = 0;
    std::vector<std::shared_ptr<const SolverSetup>> setups;   // most recent last
    std::mutex setup_mu;
};

dd_status dd_fail(dd_ctx *ctx, dd_status st, const std::string &msg);
dd_status dd_alloc(dd_ctx *ctx, void **p, size_t bytes, const char *what);
void dd_free(dd_ctx *ctx, void *p, size_t bytes);
dd_status dd_workspace(dd_ctx *ctx, int slot, size_t bytes, void **out);
dd_status dd_check_device_error(dd_ctx *ctx, cudaStream_t s, const char *where);
bool dd_is_device_ptr(const void *p);

// Host linear algebra (host_linalg.cu)
bool dd_metric_maps(const double *C, MetricMaps *M);   // false: not SPD
// Eigen-decomposition of the symmetric n x n A (n <= 12, row-major,
// destroyed) by cyclic Jacobi rotations: eigenvectors as the columns of V.
void dd_sym_eig(int n, double *A, double *V, double *w);

// Padding granule of the data arrays (points).
constexpr int64_t kDataTile = 256;

// ---------------------------------------------------------------------------
// Search (search_fp32.cu / search_tc.cu / ann.cu)
// ---------------------------------------------------------------------------
// Per-query record consumed by the low-precision scans.
struct QueryRec {
    float q[12];      // centred mapped coordinates, FP32
    float w2;         // candidate window (twice the score error bound)
    float qn;         // |q|^2
    float pad[2];
};

struct SearchOut {
    int32_t *idx;     // [m]
    double *d2;       // [m] Eq. (3) distance, may be null
    double *d2nd;     // [m] second-best distance lower bound, may be null
    int k = 0;                   // exact modes: >= 2 also fills the k nearest points
    int32_t *topk_idx = nullptr; // [m x k] (k >= 2)
    double *topk_d2 = nullptr;   // [m x k], may be null
};

dd_status dd_map_queries(dd_dataset *ds, const double *y_dev, int64_t m, double *zq64,
                         QueryRec *rec, cudaStream_t s);
dd_status dd_search_exact_fp32(dd_dataset *ds, const double *y_dev, int64_t m, int certify,
                               SearchOut out, dd_search_stats *st, cudaStream_t s);
// terms: FP16 products per distance of the certified nearest-point scan (2 or
// 3; 0 = the autotuner's choice)
dd_status dd_search_exact_tc(dd_dataset *ds, const double *y_dev, int64_t m, int certify,
                             SearchOut out, dd_search_stats *st, cudaStream_t s, int terms = 0);
dd_status dd_build_fp16(dd_dataset *ds);
// Power-of-two operand scale of the tensor-core kernels (max |s z| <= 32 for
// coordinates bounded by maxabs).
double dd_tc_scale(double maxabs);
// Split FP16 operand tiles (UMMA canonical layout, 128 rows per 4 KB tile) of
// the n rows z [n x 12]: hi row (-2 x_hi, |x_hi|^2 in two terms, 0, 0), lo row
// (-2 x_lo, |x_hi + x_lo|^2 - |x_hi|^2 in two terms, 0, 0), x = s z; rows n ..
// n_pad - 1 are padding.  hi and lo hold n_pad x 16 halves each.
dd_status dd_tc_split_rows(dd_ctx *ctx, const float *z, int64_t n, int64_t n_pad, double s, __half *hi, __half *lo,
                           cudaStream_t st);

// Nearest centroids on the tensor cores (near_tc.cu), answers equal to the ALU
// kernels of ann.cu; rows that the tensor-core scores cannot settle are
// appended to fb (count fb_n, zeroed by the caller; at most fb_cap entries
// are written, the count keeps counting) for the ALU kernel.
dd_status dd_near_tc_operands(dd_ctx *ctx, const float *cent, const float *cn, int64_t L, double s, float R,
                              NearTcSet *C, cudaStream_t st);
void dd_near_tc_free(dd_ctx *ctx, NearTcSet *C);
// kAnnCand nearest cells of the listed queries (list/n_list on the device;
// both null: queries 0..m-1), as k_rank_small writes them; fb holds m entries.
dd_status dd_near_tc_rank(dd_ctx *ctx, const NearTcSet &C, const QueryRec *rec, int64_t m, const int32_t *list,
                          const unsigned *n_list, int32_t *out_cl, float *out_d, int32_t *fb, unsigned *fb_n,
                          cudaStream_t s);
// Nearest centroid of every row of z [n x 12] (ties to the lower index).
dd_status dd_near_tc_assign(dd_ctx *ctx, const NearTcSet &C, const float *z, int64_t n, int32_t *out, int32_t *fb,
                            unsigned *fb_n, int64_t fb_cap, cudaStream_t s);
dd_status dd_search_ann(dd_dataset *ds, const double *y_dev, int64_t m, double f_d,
                        const int32_t *prev_idx_dev, int budget, SearchOut out, dd_search_stats *st,
                        cudaStream_t s);
dd_status dd_build_ann(dd_dataset *ds, const dd_dataset_opts &o);
// budget (two-level tree): leaves a query's warp scans itself (the
// warm-start leaf first) before the further Eq. (13) candidates go to the
// leaf-major scan; 0 = the default, -1 = all leaves in the query's warp,
// < -1 = none.
dd_status dd_search_ann_motion(dd_dataset *ds, const double *y_dev, int64_t m, double f_d, const float *fd_q,
                               const int32_t *prev_idx_dev, AnnMotion *mot, int budget, SearchOut out,
                               dd_search_stats *st, cudaStream_t s, int eq14 = 0);
// FP64 exhaustive re-search of the queries listed in fb_list (count on device).
dd_status dd_fallback_exact(dd_dataset *ds, const double *y_dev, const int64_t *fb_list,
                            const unsigned long long *fb_count, int64_t m, SearchOut out, cudaStream_t s);
// Record (q, d1, d2 bound, f_d) of the last search for the moving-query test
// (f_d per query from fd_q when given, else f_d).
// eq14: the rule that made d2nd (0 the certified bound, 1 the second-closest
// point found; a rule-1 record below f_d = 1 serves every f_d below 1).
dd_status dd_ann_motion_update(dd_ctx *ctx, const QueryRec *rec, int64_t m, const double *d2, const double *d2nd,
                               double f_d, const float *fd_q, int eq14, AnnMotion *mot, cudaStream_t s);
dd_status dd_run_search(dd_dataset *ds, int mode, int certify, double f_d, int f_s, int budget,
                        const int32_t *prev_dev,
                        const double *y_dev, int64_t m, SearchOut out, dd_search_stats *st, cudaStream_t s);
void dd_free_ann(dd_dataset *ds);
// The kAnnCand nearest coarse cells of every query (two-level tree), sorted by
// FP32 distance (plain, not squared); -1 pads.
dd_status dd_ann_rank_cells(dd_dataset *ds, const QueryRec *rec, int64_t m, int32_t *cand_cl, float *cand_d,
                            cudaStream_t s);
// FP64 Eq. (3) distance of every answer, and the second distance (FP32 plain
// squared, mapped coordinates) in Eq. (3) units; a query left without an
// answer (every candidate leaf empty) is searched over the whole data set
// here.
dd_status dd_ann_finish(dd_dataset *ds, const double *y_dev, int64_t m, const QueryRec *rec, int32_t *idx,
                        float *d2f, double *d2, double *d2nd, cudaStream_t s);

// k-nearest-neighbour graph (knng.cu)
dd_status dd_build_knng(dd_dataset *ds, const dd_dataset_opts &o);
dd_status dd_search_knng(dd_dataset *ds, const double *y_dev, int64_t m, int f_s, const int32_t *prev_idx_dev,
                         AnnMotion *mot, SearchOut out, dd_search_stats *st, cudaStream_t s);
void dd_free_knng(dd_dataset *ds);

// FP32 scan of mapped queries against any point set (z32 [N_pad x 12], zn
// [N_pad], rows padded to 128): per (query, split) candidate windows, or the
// best kCap scores in top-k mode.  Buffers live in workspace `slot`.
struct CandHeader;
dd_status dd_scan_fp32_raw(dd_ctx *ctx, const float *z32, const float *zn, int64_t N, const QueryRec *rec, int64_t m,
                           bool topk, int slot, int *splits_out, int *cap_out, CandHeader **hdr_out, float2 **cand_out,
                           cudaStream_t s);

// Shared by the exact scans: merge split candidates, rescore in FP64 and
// re-search uncertified queries.  Candidate layout described in search_fp32.cu.
struct CandHeader {
    float mrun;       // smallest score seen in the split
    float dropped;    // smallest score that did not fit in the buffer (+inf: none)
    int cnt;          // valid entries
    int pad;
};
// fp32_first: uncertified queries are re-searched by the certified FP32 scan
// (a window 8x narrower than the tensor-core scan's) before any FP64 scan,
// when the call may synchronise (not while a step is captured).
dd_status dd_merge_rescore(dd_dataset *ds, const double *y_dev, int64_t m, int splits, int cap,
                           const CandHeader *hdr, const float2 *cand, const QueryRec *rec,
                           int certify, double inv_s2, SearchOut out, dd_search_stats *st, cudaStream_t s,
                           bool fp32_first = false);
// As dd_merge_rescore for the k >= 2 nearest points (out.k), from scans run
// in top-k mode (the best `cap` scores of every split, no window): the k
// nearest candidates by FP64 Eq. (3); with certify, a query whose k-th
// score is not separated by the score window from every full split's worst
// kept score is re-searched in FP64.
dd_status dd_merge_topk(dd_dataset *ds, const double *y_dev, int64_t m, int splits, int cap, const CandHeader *hdr,
                        const float2 *cand, const QueryRec *rec, int certify, double inv_s2, SearchOut out,
                        dd_search_stats *st, cudaStream_t s);

// Eq. (3) in FP64 between a state y (eps, sig) and data point j (raw FP32).
__device__ __forceinline__ double dd_eq3(const MetricMaps &M, const double *y, const float *row) {
    double de[6], ds[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        de[k] = y[k] - (double)row[k];
        ds[k] = y[6 + k] - (double)row[6 + k];
    }
    double a = 0.0, b = 0.0;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        double ce = 0.0, cs = 0.0;
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            ce += M.C[6 * i + k] * de[k];
            cs += M.Cinv[6 * i + k] * ds[k];
        }
        a += ce * de[i];
        b += cs * ds[i];
    }
    return a + b;
}

// Bounded mbarrier wait.  Returns false on timeout.
__device__ __forceinline__ bool dd_mbar_wait(uint32_t bar, uint32_t parity) {
    uint32_t done = 0;
    unsigned long long t0 = 0;
    for (int spin = 0;; ++spin) {
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
        // the clock is read only once a wait has lasted (the fast path of a
        // pipeline wait does not pay for it), then every 64 tries
        if (spin >= 256 && (spin & 63) == 0) {
            unsigned long long t = dd_globaltimer();
            if (t0 == 0) t0 = t;
            else if (t - t0 > kWaitLimitNs) return false;
        }
    }
}

// Plain FP32 squared distance of a 12-float row (16-byte aligned) to q, in
// coordinate order: the arithmetic every FP32 distance of the tree search
// uses, so that kernels sharing it agree bit for bit.
__device__ __forceinline__ float dd_dist2_12(const float *a, const float (&q)[12]) {
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

__device__ __forceinline__ uint32_t dd_smem_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void dd_mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void dd_fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void dd_mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void dd_mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// 1-D bulk copy global -> shared (TMA engine), completion on an mbarrier.
// dst, src 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void dd_bulk_g2s(uint32_t dst, const void *src, uint32_t bytes,
                                            uint32_t bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
        "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}

// ---------------------------------------------------------------------------
// Candidate window of one query inside a low-precision scan.
//
// Every point whose score s lies within w2 of the running minimum mrun is
// kept (w2 = twice the score error bound, so the exact nearest point is
// always inside the final window).  The buffer holds `cap` entries; when it
// is full of in-window entries the worst one is evicted and the smallest
// evicted score is remembered in `dropped`: the result is certified exact
// iff dropped > final mrun + w2.  In top-k mode (no certification wanted)
// the entry threshold `lim` also falls to the buffer's worst score once it
// is full, so the buffer ends as the best `cap` scores.
// ---------------------------------------------------------------------------
struct CandState {
    float mrun, wl, lim, dropped;
    int cnt;
};

__device__ __forceinline__ void cand_init(CandState &c, bool active) {
    c.mrun = INFINITY;
    c.wl = INFINITY;
    c.lim = active ? INFINITY : -INFINITY;
    c.dropped = INFINITY;
    c.cnt = 0;
}

// Window above the running minimum m: w2, plus, for a score taken against
// a query rounded to q_hi (the two-product tensor-core scan), the q_lo term
// qlo4 * D with qlo4 = 4 |q_lo| and D = sqrt(m + |q_hi|^2) + qlo4 / 2 bounding
// the distance to q_hi of every point that can lie in the window.
__device__ __forceinline__ float cand_window(float m, float w2, float qlo4, float qhn) {
    if (!(qlo4 > 0.f)) return w2;
    const float D = sqrtf(fmaxf(m + qhn + w2, 0.f)) + 0.5f * qlo4;
    return w2 + qlo4 * D * 1.001f;
}

// buf: this query's entry 0; consecutive entries are `st` float2 apart.
__device__ __forceinline__ void cand_insert(CandState &c, float s, int j, float w2, float2 *buf, int st, int cap,
                                            bool topk, float qlo4 = 0.f, float qhn = 0.f) {
    if (s < c.mrun) {
        c.mrun = s;
        c.wl = s + cand_window(s, w2, qlo4, qhn);
    }
    if (!(s <= c.wl)) return;
    if (c.cnt == cap) {
        int c2 = 0;
        for (int e = 0; e < cap; ++e) {
            float2 v = buf[e * st];
            if (v.x <= c.wl) buf[(c2++) * st] = v;
        }
        c.cnt = c2;
    }
    if (c.cnt < cap) {
        buf[c.cnt * st] = make_float2(s, __int_as_float(j));
        c.cnt++;
    } else {
        int pm = 0;
        float mx = buf[0].x;
        for (int e = 1; e < cap; ++e) {
            float v = buf[e * st].x;
            if (v > mx) {
                mx = v;
                pm = e;
            }
        }
        if (s < mx) {
            c.dropped = fminf(c.dropped, mx);
            buf[pm * st] = make_float2(s, __int_as_float(j));
        } else {
            c.dropped = fminf(c.dropped, s);
        }
    }
    c.lim = c.wl;
    if (topk && c.cnt == cap) {
        float mx = buf[0].x;
        for (int e = 1; e < cap; ++e) mx = fmaxf(mx, buf[e * st].x);
        c.lim = fminf(c.wl, mx);
    }
}

// Write the window's surviving entries and header for (query slot).
__device__ __forceinline__ void cand_store(const CandState &c, const float2 *buf, int st, int cap, size_t slot,
                                           CandHeader *hdr, float2 *cand) {
    int c2 = 0;
    for (int e = 0; e < c.cnt; ++e) {
        float2 v = buf[e * st];
        if (v.x <= c.wl) cand[slot * cap + (c2++)] = v;
    }
    CandHeader h;
    h.mrun = c.mrun;
    h.dropped = c.dropped;
    h.cnt = c2;
    h.pad = 0;
    hdr[slot] = h;
}
