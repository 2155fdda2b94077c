/*
 * dd.h - C ABI of a GB300 (sm_103a) library for the hot path of model-free
 * data-driven (DD) computational mechanics: per-iteration projection of every
 * material point's (strain, stress) state onto its nearest point of a material
 * data set, alternating with the projection onto the constraint set.
 *
 * Method: Eggersmann, Stainier, Ortiz & Reese, "Efficient Data Structures for
 * Model-free Data-Driven Computational Mechanics" (arXiv:2012.00357).
 *   Sec. 2, Eq. (1)-(3): DD problem, global distance, C-weighted local metric.
 *   Sec. 2, Eq. (4)-(6): constraint projection P_C (two solves with K).
 *   Sec. 2, Eq. (7)-(8): data projection P_D and the fixed-point iteration.
 *   Sec. 3.2:            Euclidean map q = (C^{1/2} eps, C^{-1/2} sig).
 *   Sec. 4.2-4.5, Eq. (11), (13), (14): approximate k-means search, accuracy
 *                        ramp of f_d, warm start and moving-query radius.
 *
 * Conventions shared by every call
 *   - States are rows of 12 values (eps[6], sig[6]) in Voigt order
 *     (xx, yy, zz, yz, xz, xy), engineering shear strains, row-major.
 *   - The metric C is a symmetric positive definite 6x6 Voigt matrix, given
 *     as 36 row-major doubles in host memory.
 *   - Pointers documented "host or device" may point to either; the library
 *     detects the kind with cudaPointerGetAttributes.  Device pointers must
 *     belong to the context's device.  Host-pointer calls are synchronous;
 *     device-pointer calls are ordered on the given stream and the caller
 *     synchronises before reading the results.
 *   - Every call returns a dd_status; no call aborts or throws.  After an
 *     error dd_last_error(ctx) returns a message.  A DD_ERR_CUDA or
 *     DD_ERR_TIMEOUT status leaves the context usable unless the CUDA
 *     context itself was lost (then every later call returns DD_ERR_CUDA).
 *   - Objects are owned by the caller once returned and are released with
 *     the matching *_free / dd_destroy call.  Calls on one context are not
 *     thread-safe; use one context per host thread.
 */
#ifndef DD_H
#define DD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#pragma GCC visibility push(default)
#endif

typedef enum dd_status {
    DD_OK = 0,
    DD_ERR_ARG = 1,            /* invalid argument: null, size, range, NaN */
    DD_ERR_NOT_SPD = 2,        /* metric not symmetric positive definite */
    DD_ERR_OOM = 3,            /* device allocation failed or HBM budget exceeded */
    DD_ERR_CUDA = 4,           /* CUDA runtime error */
    DD_ERR_TIMEOUT = 5,        /* a bounded device-side wait expired */
    DD_ERR_NOT_CONVERGED = 6,  /* iteration limit reached; outputs are filled */
    DD_ERR_STATE = 7           /* call not valid for this object */
} dd_status;

typedef struct dd_ctx dd_ctx;
typedef struct dd_dataset dd_dataset;

/* Search modes of the data projection P_D (Eq. 7). */
enum {
    DD_SEARCH_EXACT_FP32 = 0,  /* exact: FP32 streaming scan + FP64 rescoring */
    DD_SEARCH_EXACT_TC = 1,    /* exact: FP16 tensor-core contraction, FP32
                                  accumulation, candidates rescored in FP64 */
    DD_SEARCH_ANN = 2,         /* approximate k-means partition search (Eq. 13),
                                  warm-started from the previous neighbour */
    DD_SEARCH_KNNG = 3         /* approximate greedy walk in the k-nearest-
                                  neighbour graph (Sec. 4.4), warm-started from
                                  the previous neighbour; needs a data set
                                  loaded with knn_k > 0 */
};

/* ------------------------------------------------------------------------ */
/* Context                                                                   */
/* ------------------------------------------------------------------------ */

/* Create a context on CUDA device `device`.  `hbm_budget` caps the device
 * bytes the context may hold (0 = no cap beyond the device's free memory).
 * Allocates a stream and small bookkeeping buffers.  *out is set on DD_OK. */
dd_status dd_create(int device, size_t hbm_budget, dd_ctx **out);

/* Release the context.  Every dataset created from it must be freed first. */
void dd_destroy(dd_ctx *ctx);

/* Message of the last failed call on ctx ("" if none).  Valid until the next
 * call on ctx.  ctx may be NULL (then: the last dd_create failure). */
const char *dd_last_error(const dd_ctx *ctx);

/* Device bytes currently held by the context (datasets, workspaces). */
size_t dd_bytes_in_use(const dd_ctx *ctx);

/* ------------------------------------------------------------------------ */
/* Material data set                                                         */
/* ------------------------------------------------------------------------ */

typedef struct dd_dataset_opts {
    int build_fp16;     /* 1: also build the FP16 operand copy used by
                           DD_SEARCH_EXACT_TC (32 bytes per point) */
    int ann_nlist;      /* >0: build the k-means partition used by DD_SEARCH_ANN
                           with this many clusters; 0: none */
    int ann_train_iters;/* Lloyd iterations of the partition build (default 8) */
    int64_t ann_sample; /* training sample size (0: min(N, 64 * ann_nlist)) */
    uint64_t seed;      /* seed of the partition build's initial centroids */
    int borrow;         /* 1 and eps_sig is a device pointer: keep using the
                           caller's buffer instead of copying it; it must stay
                           valid and unchanged until dd_free_dataset */
    int ann_levels;     /* 1 (default): ann_nlist k-means clusters in one level;
                           2: a two-level k-means tree, about sqrt(ann_nlist)
                           coarse cells each split into leaves, ann_nlist
                           leaves in total (for 10^8 - 10^9 points) */
    int knn_k;          /* 1..128: also build the k-nearest-neighbour graph
                           of DD_SEARCH_KNNG (Sec. 4.4): every point linked to
                           the knn_k nearest other points that a search of
                           the two-level tree (ann_levels = 2, required)
                           finds for it at accuracy knn_fd (Eq. 13);
                           4 * knn_k + 4 bytes per point.  0: no graph */
    double knn_fd;      /* f_d of the graph build (0 .. 1; 1 with at most 8
                           coarse cells of at most 8 leaves gives the exact
                           graph) */
    int ann_alu;        /* 0 (default): the nearest-centroid passes of the
                           partition build and the search's cell ranking run
                           on the tensor cores, with answers equal to the ALU
                           kernels' (rows the low-precision scores cannot
                           settle are finished on the ALU), and the leaf sums
                           of the build are gathered per run of points in
                           shared memory first; 1: the plain ALU kernels
                           throughout (same partition, same answers) */
} dd_dataset_opts;

/* Load a material data set D = {(eps_j, sig_j)}, j = 0..N-1 (Sec. 2) and
 * pre-transform it to the Euclidean map of Sec. 3.2,
 *     z_j = (C^{1/2} eps_j, C^{-1/2} sig_j) / sqrt(2),
 * so that |z_j - z(y)|^2 = d_e^2(y, (eps_j, sig_j)) / 2 with d_e of Eq. (3).
 *   eps_sig  host or device, float32 [N x 12] row-major (eps[6], sig[6]).
 *            These values are the data set; FP64 rescoring reads them.
 *   N        1 .. 2^31 - 1.
 *   C        host, 36 doubles, the SPD metric of Eq. (3).
 *   opts     may be NULL (all zero).
 * Errors: DD_ERR_ARG (N out of range, null pointers, non-finite data),
 * DD_ERR_NOT_SPD, DD_ERR_OOM, DD_ERR_CUDA.  Synchronous. */
dd_status dd_load_dataset(dd_ctx *ctx, const float *eps_sig, int64_t N,
                          const double *C, const dd_dataset_opts *opts,
                          dd_dataset **out);

void dd_free_dataset(dd_dataset *ds);

/* Number of points and the byte size of the device-resident copies. */
int64_t dd_dataset_size(const dd_dataset *ds);
size_t dd_dataset_bytes(const dd_dataset *ds);

/* The k-means partition of DD_SEARCH_ANN (built when ann_nlist > 0):
 * number of clusters L (0 if none), and a host copy of the index.
 *   cluster_of  host int32 [N]: cluster of every data point, or NULL
 *   centroids   host float64 [L x 12]: centroids in the mapped coordinates
 *               z = (C^{1/2} eps, C^{-1/2} sig)/sqrt(2), or NULL
 *   radii       host float64 [L]: radius d_r of every cluster (largest
 *               centroid-member distance, rounded up), or NULL
 * Errors: DD_ERR_STATE if no partition was built.  Synchronous. */
int dd_dataset_ann_nlist(const dd_dataset *ds);
dd_status dd_dataset_ann_index(dd_dataset *ds, int32_t *cluster_of, double *centroids, double *radii);

/* The cell level of a two-level partition (ann_levels = 2; the leaves are
 * the clusters of dd_dataset_ann_index, leaf l lying in cell l / L2).
 *   L1, L2      host int32: number of cells, leaves per cell (may be NULL)
 *   centroids   host float64 [L1 x 12]: cell centroids in the mapped
 *               coordinates, or NULL
 *   radii       host float64 [L1]: radius of every cell (largest
 *               centroid-member distance over its points, rounded up), or NULL
 * The cells order the descent and pass Eq. (13) with these radii (Sec. 4.2).
 * Errors: DD_ERR_STATE if no two-level partition was built.  Synchronous. */
dd_status dd_dataset_ann_cells(dd_dataset *ds, int32_t *L1, int32_t *L2, double *centroids, double *radii);

/* Rows of the partition build's nearest-centroid passes that the tensor-core
 * scores could not settle and the ALU kernel finished (0 with ann_alu = 1 or
 * no partition).  Not an error: the build's answers are the same either way. */
int64_t dd_dataset_ann_build_fallback(const dd_dataset *ds);

/* The k-nearest-neighbour graph of DD_SEARCH_KNNG (Sec. 4.4, built when
 * knn_k > 0): its k (0 if none), and a host copy.
 *   nbr  host int32 [N x k]: row j holds the data indices of the neighbours
 *        of point j, nearest first (FP32 distances in the mapped coordinates,
 *        ties to the lower sorted position); -1 where fewer than k were found
 * Errors: DD_ERR_STATE if no graph was built.  Synchronous. */
int dd_dataset_knn_k(const dd_dataset *ds);
dd_status dd_dataset_knn_graph(dd_dataset *ds, int32_t *nbr);

/* The data-derived metric of Sec. 3.1 (principal component analysis):
 * the six principal component vectors of the data (eigenvectors of the
 * covariance about the mean with the six largest eigenvalues) are the columns
 * of A (12 x 6), A_eps its upper and A_sig its lower 6 x 6 block, and
 *     C = sym(A_sig A_eps^{-1}),
 * the paper's sym(A_eps^{-1} A_sig) with the components as rows of A; for
 * data on a linear law sig = C0 eps it returns C0.  The moments are summed in
 * FP64 on the device in a fixed order (the same result on every run).
 *   eps_sig  host or device, float32 [N x 12] (eps[6], sig[6]), N >= 13.
 *   C_out    host, 36 doubles (row-major), written on DD_OK.
 * Errors: DD_ERR_ARG (null, N < 13, non-finite data), DD_ERR_NOT_SPD (the
 * principal strain block is singular or the metric is not positive
 * definite), DD_ERR_CUDA.  Synchronous. */
dd_status dd_pca_metric(dd_ctx *ctx, const float *eps_sig, int64_t N, double *C_out);

/* Write points start .. start+N-1 of the seeded synthetic data set into the
 * device buffer out_dev (float32 [N x 12]).  This is the device copy of the
 * input generator of the Python module dd_inputs (SplitMix64 counter stream,
 * uniform strains in [eps_lo, eps_hi], stress from the law `law` = 0:
 * sig = C eps, 1: sig = C eps (1 + beta |eps|), 2: the cubic isotropic law
 * of Eq. (9), sig = 2 mu (eps + beta eps^3) + lam (tr eps + beta (tr eps)^3) I
 * with lam = C[0][1], mu = C[3][3] and eps^3 the tensor power, plus
 * Irwin-Hall noise of std
 * noise_std), bit-identical to it.  It is not part of the DD method; it
 * exists so that data sets of 10^8-10^9 points can be made in place.
 * Asynchronous on `stream` (a cudaStream_t, NULL = the context's stream). */
dd_status dd_synth_dataset(dd_ctx *ctx, int law, double eps_lo, double eps_hi,
                           double noise_std, double beta, const double *C,
                           uint64_t seed, int64_t start, int64_t N,
                           float *out_dev, void *stream);

/* ------------------------------------------------------------------------ */
/* Data projection P_D                                                       */
/* ------------------------------------------------------------------------ */

typedef struct dd_search_opts {
    int mode;                 /* DD_SEARCH_* */
    int certify;              /* exact modes: 1 (default when opts is NULL)
                                 = queries whose low-precision candidate window
                                 overflowed are re-searched exactly in FP64,
                                 so the result is the exact argmin; 0 = keep
                                 the best rescored candidate (reported) */
    double f_d;               /* DD_SEARCH_ANN: accuracy parameter of Eq. (13),
                                 0 = no backtracking .. 1 = exact */
    const int32_t *prev_idx;  /* DD_SEARCH_ANN: previous neighbour of each
                                 query (warm start), host or device, or NULL */
    void *stream;             /* cudaStream_t for device pointers, NULL = ctx */
    int f_s;                  /* DD_SEARCH_KNNG: at most f_s node changes per
                                 walk (the bound of Sec. 4.4); 0 = walk to a
                                 local minimum of the graph.  Without
                                 prev_idx the walk of query i starts at data
                                 point SplitMix64(i) mod N (the first output
                                 of SplitMix64 seeded with i) */
    int ann_budget;           /* DD_SEARCH_ANN with the two-level tree: leaves
                                 a query's warp scans itself, the warm-start
                                 leaf first (d_c shrinking after each, as in
                                 Sec. 4.3); its further Eq. (13) candidates,
                                 tested with the d_c reached then, are scanned
                                 leaf-major, up to 32 queries per read of a
                                 leaf.  0 = default (2), -1 = every leaf in
                                 the query's warp, < -1 = none (all leaves,
                                 the warm-start one included, leaf-major) */
    int topk;                 /* exact modes: number k (1 .. DD_TOPK_MAX) of
                                 nearest data points written to topk_out;
                                 0 = none (topk_out must then be NULL) */
    double *topk_d2;          /* [m x topk] FP64 d_e^2 (Eq. 3) of topk_out,
                                 or NULL */
    double *d2nd;             /* [m] output, or NULL: a lower bound on d_e^2
                                 of every data point other than idx[i] - the
                                 second-nearest distance of Eq. (14).  Exact
                                 modes: certified (the exact second-nearest
                                 distance when topk >= 2).  DD_SEARCH_ANN: the
                                 smaller of the second-best point read and,
                                 for every cluster, cell or leaf not
                                 searched, (centroid distance - f_d radius)^2
                                 in the mapped coordinates, times 2: a true
                                 lower bound at f_d = 1, the bound of Eq.
                                 (13)'s cluster model below.  DD_SEARCH_KNNG:
                                 the nearest other point the walk evaluated
                                 (0 when f_s stopped it), which keeps a query
                                 exactly where the walk from its warm start
                                 would stay */
    const double *prev_y;     /* DD_SEARCH_ANN / DD_SEARCH_KNNG: moving-query
                                 record of Eq. (14), or NULL.  The states
                                 [m x 12] of the previous call, with prev_d2
                                 and prev_d2nd [m] the d2 and d2nd it returned
                                 and prev_idx its idx: a query whose mapped
                                 state moved by less than
                                 (sqrt(prev_d2nd / 2) - sqrt(prev_d2 / 2)) / 2
                                 keeps prev_idx without a search.  For
                                 DD_SEARCH_ANN the previous call must have
                                 used an f_d no smaller than this call's (the
                                 bound is that f_d's).  Same memory kind as y;
                                 requires prev_idx, prev_d2 and prev_d2nd */
    const double *prev_d2;
    const double *prev_d2nd;
    int eq14;                 /* DD_SEARCH_ANN: d2nd (and so the record a
                                 later call makes of it) is 0 (default) the
                                 certified bound above, 1 the second-closest
                                 point found below f_d = 1 (the paper's
                                 estimate; see dd_solve_opts.eq14) */
    int tc_terms;             /* DD_SEARCH_EXACT_TC, certify = 1, topk < 2:
                                 FP16 products per distance, 3 (split query
                                 and data) or 2 (split data, single FP16
                                 query, wider window); both certified exact.
                                 0 = the autotuner's choice */
} dd_search_opts;

/* Largest k of dd_search_opts.topk.  k < DD_TOPK_MAX is certified from the
 * low-precision candidates for almost every query; k = DD_TOPK_MAX re-searches
 * most queries in FP64. */
#define DD_TOPK_MAX 8

typedef struct dd_search_stats {
    int64_t uncertified;      /* queries re-searched in FP64 (exact modes) */
    int64_t distances;        /* point distances evaluated (the paper's
                                 "comparisons", Sec. 3.1) */
    int64_t skipped;          /* queries answered by the moving-query radius */
    double ms;                /* device time of the call (CUDA events) */
    double scan_ms;           /* device time of the dominant scan kernel alone
                                 (CUDA events on the launching stream) */
    int64_t points;           /* data points read by the approximate search
                                 (the rest of `distances` are centroids) */
    int64_t unique_points;    /* approximate search: points of the distinct
                                 clusters it read (what it must fetch from
                                 memory at least once) */
    int64_t moves;            /* DD_SEARCH_KNNG: node changes of all walks */
} dd_search_stats;

/* Nearest data point of each state y_i (Eq. 7):
 *     idx[i] = argmin_j d_e^2(y_i, (eps_j, sig_j)),  d2[i] = that d_e^2 (Eq. 3,
 *     without the 1/2 of Eq. 2), evaluated in FP64 from the stored data.
 * Ties between data points with equal FP64 distance go to the lowest index.
 *   y         host or device, float64 [m x 12] states (eps, sig).
 *   m         >= 0 (0 is a no-op).
 *   idx       host or device, int32 [m] (output).
 *   d2        host or device, float64 [m] (output), may be NULL.
 *   topk_out  host or device, int32 [m x opts->topk] (output), or NULL:
 *             exact modes only.  Row i lists the topk nearest data points of
 *             y_i, nearest first by FP64 Eq. (3) distance (ties to the lower
 *             index), -1 past the N-th.  With certify = 1 they are the exact
 *             k nearest points (the low-precision scan keeps the best 8
 *             scores per data range; a query whose k-th candidate is not
 *             separated from the scores left out by the scan's error bound
 *             is re-searched in FP64).  With certify = 0 they are the best of
 *             those candidates after FP64 rescoring (the tensor-core top-k
 *             form; the caller can measure their error against an exact
 *             search).
 *   stats     host, may be NULL.
 * All of y, idx, d2, topk_out and the opts arrays must be of the same kind
 * (all host or all device).  Errors: DD_ERR_ARG (bad sizes, f_d outside
 * [0, 1], topk outside 0 .. DD_TOPK_MAX or with an approximate mode, a
 * motion record without prev_idx, mixed memory kinds), DD_ERR_STATE (the
 * mode's index or operand copy was not built), DD_ERR_OOM, DD_ERR_CUDA,
 * DD_ERR_TIMEOUT. */
dd_status dd_project_nearest(dd_dataset *ds, const double *y, int64_t m,
                             const dd_search_opts *opts, int32_t *idx,
                             double *d2, int32_t *topk_out,
                             dd_search_stats *stats);

/* Largest query count accepted by dd_project_nearest_noalloc. */
#define DD_NOALLOC_MAX_QUERIES 65536

/* Exact nearest-data projection that allocates no device memory.  The paper
 * has no counterpart: this exists for callers that cannot allocate during a
 * call, for example a serving loop whose device memory is fully reserved by
 * another allocator, or a latency-bound caller that cannot accept cudaMalloc /
 * cudaFree (which can fail under memory pressure, and cudaFree synchronises
 * the device).  Same result as dd_project_nearest with DD_SEARCH_EXACT_FP32
 * and certify = 1: idx[i], and d2[i] the FP64 squared energy-norm distance
 * of that point, as dd_project_nearest returns it.
 *   y_dev    device, float64 [m x 12] states (eps, sig)
 *   m        0 .. DD_NOALLOC_MAX_QUERIES; larger m returns DD_ERR_ARG
 *   idx_dev  device, int32 [m] (output); d2_dev device, float64 [m] (output)
 *   stream   cudaStream_t, NULL = the context's stream
 *   wait     0: asynchronous on stream; a device-side wait that gave up
 *            leaves the outputs unspecified and is not reported.  1: the call
 *            synchronises the stream and returns DD_ERR_TIMEOUT if a bounded
 *            device wait of this call gave up (the status word lives in the
 *            scratch array and is cleared at the start of every call, so it
 *            never reports another call's failure).
 * The calling thread's current device is the same on return as on entry.
 * Scratch is one file-scope device array of 32 MiB that every GPU loading the
 * library holds until exit.  The first call on a device looks up the array's
 * device address (cudaGetSymbolAddress) with that device current; make that
 * first call before any stream capture.  All calls share the array: calls
 * whose work overlaps on the GPU (different streams, or several host threads)
 * race on it and must be serialised by the caller. */
dd_status dd_project_nearest_noalloc(dd_dataset *ds, const double *y_dev, int64_t m,
                                     int32_t *idx_dev, double *d2_dev, void *stream, int wait);

/* ------------------------------------------------------------------------ */
/* DD solve: z_{i+1} = P_D(P_C(z_i)), Eq. (8)                               */
/* ------------------------------------------------------------------------ */

/* Box [0,lx]x[0,ly]x[0,lz] of nx*ny*nz trilinear hexahedra, 2x2x2 Gauss
 * points.  Node (i,j,k) = i + (nx+1)(j + (ny+1)k), dof = 3 node + component;
 * element (i,j,k) = i + nx(j + ny k); Gauss point g = gx + 2gy + 4gz at
 * (2g* - 1)/sqrt(3); material point = 8 element + g. */
typedef struct dd_mesh {
    int nx, ny, nz;
    double lx, ly, lz;
} dd_mesh;

/* Boundary conditions: every dof on z = 0 is clamped.  With rot_z == 0 the
 * face z = lz carries the traction t(x,y) = t0 + tx (x - lx/2) + ty (y - ly/2),
 * integrated into consistent nodal forces f (2x2 Gauss per face).  With
 * rot_z != 0 the face z = lz is turned rigidly by rot_z radians about the
 * vertical axis through its centre instead: u = (R(rot_z) - I)(x - lx/2,
 * y - ly/2, 0) there, eta = 0 there, no traction (the paper's torsion
 * problem); t0, tx, ty must then be zero (DD_ERR_ARG otherwise) and nz >= 2. */
typedef struct dd_load {
    double t0[3], tx[3], ty[3];
    double rot_z;             /* prescribed rotation of the top face (radians), 0: traction */
} dd_load;

typedef struct dd_solve_opts {
    int mode;                 /* DD_SEARCH_* used for P_D */
    int certify;              /* as in dd_search_opts (exact modes) */
    double f_d0, f_d_final;   /* DD_SEARCH_ANN: f_d ramps linearly from f_d0
                                 to f_d_final over ramp_iters iterations
                                 (Sec. 4.5), then stays at f_d_final */
    int ramp_iters;
    int max_iter;             /* DD iterations (default 100) */
    double cg_rtol;           /* CG relative residual (default 1e-12) */
    int cg_max_iter;          /* CG iterations per solve (default 20000) */
    uint64_t seed;            /* initial association when init_idx is NULL:
                                 idx_e = SplitMix64(key(seed, 3), e) mod N */
    const int32_t *init_idx;  /* host, int32 [n_gp], or NULL */
    int stall_iters;          /* DD_SEARCH_ANN: stop when the global distance
                                 has not decreased by more than 1e-12 relative
                                 for this many iterations (default 3) */
    int cg_mode;              /* P_C solves: 0 (default) = FP32 Krylov
                                 iterations inside FP64 iterative refinement
                                 (residual b - K x and x in FP64, stop test
                                 |b - K x| <= cg_rtol |b| in FP64); 1 = FP64
                                 preconditioned CG throughout */
    int f_s;                  /* DD_SEARCH_KNNG: node-change bound of every
                                 walk, as in dd_search_opts (0 = none) */
    int ann_budget;           /* DD_SEARCH_ANN: as in dd_search_opts */
    int fd_rule;              /* DD_SEARCH_ANN: the accuracy schedule
                                 f = f(d, d_e, i) of Eq. (11):
                                 0 (default) the linear ramp above;
                                 1 global: f starts at f_d0 and rises by
                                 (f_d_final - f_d0) / ramp_iters after every
                                 iteration in which P_D reduced the global
                                 distance by less than the fraction fd_tau
                                 (1 - d_after_PD / d_after_PC < fd_tau), up to
                                 f_d_final; fd_tau = 1 gives the ramp;
                                 2 local: a material point whose distance
                                 after P_C is at most fd_tau times the mean of
                                 the previous iteration is searched with
                                 f_d_final, the others with the ramp value.
                                 The stop tests apply once f has reached
                                 f_d_final (rule 1) or the ramp has ended. */
    double fd_tau;            /* parameter of fd_rule 1 and 2 (>= 0) */
    int eq14;                 /* DD_SEARCH_ANN: second distance of the
                                 moving-query radius of Eq. (14).  0 (default)
                                 = the certified bound of dd_search_opts.d2nd:
                                 a kept query gets the answer a search would
                                 certify at that f_d (the exact nearest point
                                 at f_d = 1).  1 = the second-closest point the
                                 search found, the paper's estimate: faster
                                 (more queries kept) but a kept answer can be
                                 stale where a pruned cluster holds a nearer
                                 point; used only below f_d = 1 (an exact search
                                 always takes the certified bound) */
} dd_solve_opts;

/* Result of a solve: the constraint-set state y = (u, eps, sig) of the last
 * P_C and the data association idx it was computed from (Sec. 2).  All
 * arrays are host memory allocated by the library; release with
 * dd_result_free. */
typedef struct dd_result {
    int64_t n_nodes, n_gp;
    int iters;                /* P_C solves performed */
    int converged;            /* association unchanged in the last P_D */
    double *u;                /* [n_nodes x 3] displacement */
    double *eta;              /* [n_nodes x 3] Lagrange multiplier of Eq. 5b */
    double *eps;              /* [n_gp x 6] */
    double *sig;              /* [n_gp x 6] */
    int32_t *idx;             /* [n_gp] association of the last P_C */
    double *d2_pc;            /* [iters] global distance Eq. 2 after P_C */
    double *d2_pd;            /* [iters] global distance Eq. 2 after P_D */
    int64_t *changed;         /* [iters] associations changed by P_D */
    int *cg_iters;            /* [iters] CG iterations (max of the two solves) */
    double search_ms, cg_ms, other_ms;  /* device time per phase, summed */
    int64_t uncertified;      /* exact modes: FP64 re-searches, summed */
    int64_t distances;        /* point distances evaluated, summed */
} dd_result;

/* Solve one DD problem on the data set.  Returns DD_OK when the association
 * stopped changing (exact modes) or the distance stalled (ANN),
 * DD_ERR_NOT_CONVERGED when max_iter was reached (result filled), or an
 * error.  Synchronous. */
dd_status dd_solve(dd_dataset *ds, const dd_mesh *mesh, const dd_load *load,
                   const dd_solve_opts *opts, dd_result *out);

void dd_result_free(dd_result *r);

/* ------------------------------------------------------------------------ */
/* Stepwise solve: the state of one DD problem kept on the device            */
/* ------------------------------------------------------------------------ */

typedef struct dd_solver dd_solver;

/* Statistics of one iteration z_{i+1} = P_D(P_C(z_i)). */
typedef struct dd_iter_info {
    int iter;                 /* 1-based iteration number */
    int64_t changed;          /* associations changed by P_D */
    double d2_pc, d2_pd;      /* global distance Eq. 2 after P_C, after P_D */
    int cg_iters;             /* CG iterations (max of the two systems) */
    double cg_ms, search_ms, other_ms, scan_ms;   /* device times */
    int64_t uncertified, distances;
    double f_d;               /* accuracy parameter used (ANN) */
    int done;                 /* 1: the stop rule fired or max_iter reached */
    int64_t skipped;          /* ANN: queries kept by the moving-query radius
                                 (Eq. 14) without a search */
    int64_t points;           /* ANN: data points read by the search */
    int64_t unique_points;    /* ANN: points of the distinct clusters read */
    int graph;                /* 1: dd_solvers_step replayed (or captured) the
                                 step as a CUDA graph; 0: launched eagerly */
    int64_t moves;            /* DD_SEARCH_KNNG: node changes of the walks */
} dd_iter_info;

/* Set up a DD problem (mesh, load, options as for dd_solve) on the data set:
 * builds the element operators and the preconditioner, draws or copies the
 * initial association and allocates the per-problem device state (about
 * 700 bytes per node + 600 bytes per material point).  The data set must
 * outlive the solver. */
dd_status dd_solver_create(dd_dataset *ds, const dd_mesh *mesh, const dd_load *load,
                           const dd_solve_opts *opts, dd_solver **out);

/* One DD iteration (P_C, then P_D, then the stop test of Sec. 2).
 * Synchronous; info may be NULL.  Returns DD_ERR_STATE once done. */
dd_status dd_solver_step(dd_solver *sv, dd_iter_info *info);

/* 1 once the stop rule fired or max_iter iterations ran. */
int dd_solver_done(const dd_solver *sv);

/* Copy the current state to a host result (as dd_solve returns it). */
dd_status dd_solver_result(dd_solver *sv, dd_result *out);

void dd_solver_free(dd_solver *sv);

/* One DD iteration of n solves on the same data set at once: the P_C solves
 * of all of them run in ONE cooperative CG launch (each solve on its own range
 * of thread blocks, meshes of any size) and the P_D searches of all material
 * points in ONE search over the concatenated states.  Every solver must be
 * unfinished, appear once, and share the search mode, certify and cg_mode;
 * the approximate search uses each solve's own f_d ramp position.  infos
 * (host, n entries) may be NULL.  Synchronous.  Results are those of stepping
 * each solver alone. */
dd_status dd_solvers_step(dd_solver **svs, int n, dd_iter_info *infos);

/* Solve nsolves problems (meshes[i], loads[i], the same options) on one data
 * set together, stepping all unfinished solves with dd_solvers_step until
 * every one has stopped.  outs: host array of nsolves results (free each
 * with dd_result_free).  Returns DD_ERR_NOT_CONVERGED if any solve reached
 * max_iter.  init_idx in opts, if given, is used for every solve. */
dd_status dd_solve_batch(dd_dataset *ds, int nsolves, const dd_mesh *meshes, const dd_load *loads,
                         const dd_solve_opts *opts, dd_result *outs);

/* ------------------------------------------------------------------------ */
/* Serving: one resident data set, requests admitted by memory and batched   */
/* ------------------------------------------------------------------------ */

typedef struct dd_server dd_server;

typedef struct dd_server_opts {
    dd_solve_opts solve;      /* options of every solve; init_idx is ignored and
                                 each request's seed draws its association */
    size_t state_budget;      /* device bytes the active solves' states may
                                 hold; a request waits while it does not fit
                                 (0 = no cap).  Search workspaces are extra. */
    int max_batch;            /* most solves stepped together (0 = 64) */
} dd_server_opts;

typedef struct dd_server_stats {
    int64_t submitted, completed, active, pending, steps, max_active;
    double busy_ms;           /* host time spent in batched steps */
    double cg_ms, search_ms, other_ms;   /* device time of those steps by phase:
                                            P_C solves, P_D search, the rest */
    int64_t graph_steps;      /* steps replayed as a CUDA graph */
} dd_server_stats;

/* Start a worker thread that serves DD solves on ds.  From then on the worker
 * owns the context: other calls on it (and on ds) must wait until
 * dd_server_stop.  Each tick the worker admits pending requests in arrival
 * order while their states fit in state_budget, runs one iteration of every
 * active solve with dd_solvers_step (requests that arrived meanwhile join
 * the next tick) and retires finished solves. */
dd_status dd_server_start(dd_dataset *ds, const dd_server_opts *opts, dd_server **out);

/* Queue a solve (mesh, load, seed of its initial association).  Thread-safe.
 * *ticket identifies the request. */
dd_status dd_server_submit(dd_server *sv, const dd_mesh *mesh, const dd_load *load, uint64_t seed,
                           int64_t *ticket);

/* Wait up to timeout_s seconds (0 = do not wait) for a request.  On
 * completion returns the solve's status (DD_OK or DD_ERR_NOT_CONVERGED with
 * *out filled; free with dd_result_free) and *latency_ms = time from submit
 * to result; DD_ERR_TIMEOUT if not finished yet.  A ticket can be collected
 * once.  Thread-safe. */
dd_status dd_server_poll(dd_server *sv, int64_t ticket, double timeout_s, dd_result *out, double *latency_ms);

dd_status dd_server_get_stats(dd_server *sv, dd_server_stats *out);

/* Finish every queued and active request, stop the worker and release the
 * server (results not collected are freed). */
dd_status dd_server_stop(dd_server *sv);

/* Number of kernels the context has launched so far (instrumentation). */
int64_t dd_launch_count(const dd_ctx *ctx);

#if defined(__GNUC__)
#pragma GCC visibility pop
#endif

#ifdef __cplusplus
}
#endif

#endif /* DD_H */
