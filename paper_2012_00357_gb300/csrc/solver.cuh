// State of one DD problem on the device (solver.cu, batch.cu).
#pragma once

#include <vector>

#include "dd_internal.cuh"
#include "fem.cuh"

struct dd_solver {
    dd_dataset *ds = nullptr;
    dd_ctx *ctx = nullptr;
    dd_mesh mesh;
    dd_solve_opts o;
    MeshDev g;
    ElemOps ops;
    void *block = nullptr;
    size_t block_bytes = 0;
    double *Ke = nullptr, *f = nullptr, *Minv = nullptr, *star = nullptr, *ce = nullptr, *y = nullptr;
    double *St64 = nullptr;
    float *St32 = nullptr;
    double *dpc = nullptr, *d2 = nullptr, *d2nd = nullptr, *stats = nullptr;
    int32_t *cur = nullptr, *nxt = nullptr;
    int32_t *idx_a = nullptr;           // the first of the two association buffers (cur or nxt)
    uint64_t id = 0;                    // unique per process (keys the cached step plans)
    AnnMotion mot{nullptr, nullptr};    // Eq. 14 record of the approximate search
    CGBuffers cb;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    int it = 0;
    bool converged = false, done = false;
    int stall = 0;
    double best_pd = INFINITY;
    int fd_steps = 0;                   // ramp steps taken by the global-distance rule (fd_rule 1)
    float *fdq = nullptr;               // [n_gp] per-point f_d (fd_rule 2)
    std::vector<double> h_pc, h_pd;
    std::vector<int64_t> h_ch;
    std::vector<int> h_cg;
    double cg_ms = 0, search_ms = 0, other_ms = 0;
    int64_t uncertified = 0, distances = 0;
};

// Host-side bookkeeping after one iteration's statistics are on the host:
// history, stop rule, association swap.  Returns true when the solve stops.
bool dd_solver_account(dd_solver *sv, const double hs[3], int cg_it, float cg_ms, float other_ms, float search_ms,
                       const dd_search_stats &sst, double f_d, dd_iter_info *info);
double dd_solver_fd(const dd_solver *sv, int it);

// f_d of the queries of one solve in one iteration: f_near for a point whose
// distance after P_C (dpc) is at most thr, f_far for the others (thr < 0:
// f_far for all).
struct FdParam {
    float f_far, f_near, thr, pad;
};
FdParam dd_solver_fd_param(const dd_solver *sv, int it);
// p[e] = f_d of point e from the parameter in device memory (pd) or, when pd
// is null, from hp.
dd_status dd_fill_fd(dd_ctx *ctx, float *p, int64_t n, const FdParam *pd, FdParam hp, const double *dpc,
                     cudaStream_t s);
