// Several DD problems stepped together.
//
// One batched iteration of solves s = 1..S on one data set:
//   * P_C: gather, right-hand sides and recovery per solve, and ONE
//     cooperative launch that runs the mixed-precision CG of every solve:
//     each solve owns a contiguous range of thread blocks, reduces its dot
//     products over that range only (fixed order), and all solves share the
//     grid barriers; a solve that has converged idles until the others have;
//   * P_D: ONE search over the concatenated states of all solves (the
//     per-material-point search is independent of the solve it belongs to),
//     with per-query f_d for the approximate search, whose ramp depends on
//     each solve's own iteration count;
//   * statistics and the stop rule per solve.
// Solves can have meshes of different sizes; they share the search mode and
// the CG mode.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "dd_internal.cuh"
#include "fem.cuh"
#include "fem_dev.cuh"
#include "solver.cuh"

namespace {

constexpr int kBThreads = 256;
constexpr int kGroups = kBThreads / 8;     // nodes per block and pass

struct SegCG {
    MeshDev g;
    const double *Ke, *Minv, *b;
    double *x;
    float *r, *z, *p0, *p1, *q, *d;
    int blk0, nblk;
};

struct BCGArgs {
    const SegCG *seg;
    const int *blk_seg;        // [grid] solve of every block
    int S;
    double *part;              // [2 x grid x 8]
    int *flags;                // [2 x S]: outer activity, inner activity (written by segment leaders)
    unsigned *bar, *err;
    double rtol2, in_rtol2;
    int max_outer, max_inner;
    int *it_out;               // [S] inner iterations of every solve
};

// Sum over the partials of blocks [b0, b0 + nb) in a fixed order.
template <int NV>
__device__ void range_total(const double *part, int b0, int nb, double (&tot)[NV], double *sh) {
    double v[NV];
#pragma unroll
    for (int c = 0; c < NV; ++c) v[c] = 0.0;
    for (int t = threadIdx.x; t < nb; t += blockDim.x)
#pragma unroll
        for (int c = 0; c < NV; ++c) v[c] += __ldcg(part + (size_t)(b0 + t) * 8 + c);
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

__device__ int count_flags(const int *flags, int S, double *sh) {
    double v[1] = {0.0};
    for (int t = threadIdx.x; t < S; t += blockDim.x) v[0] += (double)__ldcg(flags + t);
    block_sum<1>(v, sh);
    __shared__ int s_cnt;
    if (threadIdx.x == 0) s_cnt = (int)v[0];
    __syncthreads();
    int r = s_cnt;
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kBThreads) k_cg_batch(BCGArgs A) {
    __shared__ double sKe[576];
    __shared__ float sKf[576];
    __shared__ double sh[8 * 32];
    const int sidx = A.blk_seg[blockIdx.x];
    const SegCG S = A.seg[sidx];
    const MeshDev &g = S.g;
    for (int t = threadIdx.x; t < 576; t += blockDim.x) {
        sKe[t] = S.Ke[t];
        sKf[t] = (float)S.Ke[t];
    }
    __syncthreads();
    // node groups: 8 consecutive lanes per node, lane slot e = element slot
    // for the product and component c = e (< 6) for the per-node updates
    const int e = threadIdx.x & 7;
    const int lane = threadIdx.x & 31;
    const unsigned gmask = 0xffu << (lane & 24);
    const int gbase = lane & 24;
    const bool comp = e < 6;
    const int c = comp ? e : 0, sy = c / 3;
    const unsigned G = gridDim.x;
    GridBar gbar{A.bar, G, 0u};
    const int lb = blockIdx.x - S.blk0;
    const bool leader = (lb == 0 && threadIdx.x == 0);
    const int64_t gstride = (int64_t)S.nblk * kGroups;
    const int64_t a0 = (int64_t)lb * kGroups + (threadIdx.x >> 3);
    double *partA = A.part, *partB = A.part + (size_t)G * 8;
    int *outer_flag = A.flags, *inner_flag = A.flags + A.S;
    const double zb64[2] = {0.0, 0.0};
    double rr_true[2] = {0.0, 0.0}, bb[2] = {0.0, 0.0};
    int inner_count = 0;
    // z_c = M^-1 r for component c of the node: the system's 3 residuals come
    // from the group's lanes 3 sy .. 3 sy + 2
    auto precond = [&](int64_t a, float rc) -> float {
        float r0 = __shfl_sync(gmask, rc, gbase + 3 * sy + 0);
        float r1 = __shfl_sync(gmask, rc, gbase + 3 * sy + 1);
        float r2 = __shfl_sync(gmask, rc, gbase + 3 * sy + 2);
        const double *Mi = S.Minv + a * 9 + 3 * (c % 3);
        return (float)Mi[0] * r0 + (float)Mi[1] * r1 + (float)Mi[2] * r2;
    };
    for (int outer = 0;; ++outer) {
        double v[6] = {0, 0, 0, 0, 0, 0};
        for (int64_t a = a0; a < g.n_nodes; a += gstride) {
            double kx[6];
            spmv_group<double>(g, sKe, a, e, gmask, S.x, nullptr, zb64, kx);
            const double bc = comp ? S.b[a * 6 + c] : 0.0;
            const double r64 = comp ? bc - pick6(kx, c) : 0.0;
            const float rf = (float)r64;
            const float zf = precond(a, rf);
            if (comp) {
                S.r[a * 6 + c] = rf;
                S.z[a * 6 + c] = zf;
                S.p0[a * 6 + c] = zf;
                S.d[a * 6 + c] = 0.f;
                (sy ? v[1] : v[0]) += (double)rf * (double)zf;
                (sy ? v[3] : v[2]) += r64 * r64;
                (sy ? v[5] : v[4]) += bc * bc;
            }
        }
        block_sum<6>(v, sh);
        if (threadIdx.x == 0)
            for (int k = 0; k < 6; ++k) partB[blockIdx.x * 8 + k] = v[k];
        if (!grid_sync(gbar, A.err)) return;
        double tot[6];
        range_total<6>(partB, S.blk0, S.nblk, tot, sh);
        double rz[2] = {tot[0], tot[1]};
        bool conv[2];
        for (int s2 = 0; s2 < 2; ++s2) {
            rr_true[s2] = tot[2 + s2];
            bb[s2] = tot[4 + s2];
            conv[s2] = !(rr_true[s2] > A.rtol2 * bb[s2]) || bb[s2] == 0.0;
        }
        const bool more = !(conv[0] && conv[1]) && outer < A.max_outer;
        if (leader) {
            outer_flag[sidx] = more ? 1 : 0;
            inner_flag[sidx] = more ? 1 : 0;
        }
        if (!grid_sync(gbar, A.err)) return;
        if (count_flags(outer_flag, A.S, sh) == 0) {
            for (int s2 = 0; s2 < 2; ++s2)
                if (bb[s2] == 0.0 && comp && sy == s2)
                    for (int64_t a = a0; a < g.n_nodes; a += gstride) S.x[a * 6 + c] = 0.0;
            break;
        }
        // gain four digits per refinement step, but never solve below a tenth
        // of the final tolerance
        const double target[2] = {fmax(A.in_rtol2 * rr_true[0], 0.01 * A.rtol2 * bb[0]),
                                  fmax(A.in_rtol2 * rr_true[1], 0.01 * A.rtol2 * bb[1])};
        bool ic[2] = {conv[0] || !more, conv[1] || !more};
        float beta[2] = {0.f, 0.f};
        float *pold = S.p0, *pnew = S.p1;
        for (int it = 0; it < A.max_inner; ++it) {
            const bool act = !(ic[0] && ic[1]);
            double w[2] = {0, 0};
            if (act) {
                for (int64_t a = a0; a < g.n_nodes; a += gstride) {
                    float kq[6];
                    spmv_group<float>(g, sKf, a, e, gmask, S.z, pold, beta, kq);
                    if (comp) {
                        const float pn = S.z[a * 6 + c] + (sy ? beta[1] : beta[0]) * pold[a * 6 + c];
                        const float qc = pick6(kq, c);
                        pnew[a * 6 + c] = pn;
                        S.q[a * 6 + c] = qc;
                        (sy ? w[1] : w[0]) += (double)pn * (double)qc;
                    }
                }
            }
            block_sum<2>(w, sh);
            if (threadIdx.x == 0) {
                partA[blockIdx.x * 8 + 0] = w[0];
                partA[blockIdx.x * 8 + 1] = w[1];
            }
            if (!grid_sync(gbar, A.err)) return;
            // lagged stop: the leaders published their activity before this barrier
            if (count_flags(inner_flag, A.S, sh) == 0) break;
            double pq[2];
            range_total<2>(partA, S.blk0, S.nblk, pq, sh);
            float alpha[2];
            for (int s2 = 0; s2 < 2; ++s2) alpha[s2] = (ic[s2] || !(pq[s2] > 0.0)) ? 0.f : (float)(rz[s2] / pq[s2]);
            double u[4] = {0, 0, 0, 0};
            if (act) {
                for (int64_t a = a0; a < g.n_nodes; a += gstride) {
                    float rv = 0.f;
                    if (comp) {
                        S.d[a * 6 + c] += (sy ? alpha[1] : alpha[0]) * pnew[a * 6 + c];
                        rv = S.r[a * 6 + c] - (sy ? alpha[1] : alpha[0]) * S.q[a * 6 + c];
                        S.r[a * 6 + c] = rv;
                    }
                    const float zv = precond(a, rv);
                    if (comp) {
                        S.z[a * 6 + c] = zv;
                        (sy ? u[1] : u[0]) += (double)rv * (double)zv;
                        (sy ? u[3] : u[2]) += (double)rv * (double)rv;
                    }
                }
            }
            block_sum<4>(u, sh);
            if (threadIdx.x == 0)
                for (int k = 0; k < 4; ++k) partB[blockIdx.x * 8 + k] = u[k];
            if (!grid_sync(gbar, A.err)) return;
            double t4[4];
            range_total<4>(partB, S.blk0, S.nblk, t4, sh);
            for (int s2 = 0; s2 < 2; ++s2) {
                if (!ic[s2]) {
                    beta[s2] = (rz[s2] != 0.0) ? (float)(t4[s2] / rz[s2]) : 0.f;
                    rz[s2] = t4[s2];
                    ic[s2] = !(t4[2 + s2] > target[s2]) || !(pq[s2] > 0.0);
                } else {
                    beta[s2] = 0.f;
                }
            }
            if (act) ++inner_count;
            if (leader) inner_flag[sidx] = (ic[0] && ic[1]) ? 0 : 1;
            float *t = pold;
            pold = pnew;
            pnew = t;
        }
        if (comp)
            for (int64_t a = a0; a < g.n_nodes; a += gstride) S.x[a * 6 + c] += (double)S.d[a * 6 + c];
        if (!grid_sync(gbar, A.err)) return;
    }
    if (leader) A.it_out[sidx] = inner_count;
}

__global__ void k_fill_f(float *p, int64_t n, float v) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}

}  // namespace

// Mixed-precision CG of n systems in one cooperative launch.  *it_dev points
// at the per-system inner iteration counts (device) after the launch.
dd_status dd_cg_segments(dd_ctx *ctx, const MeshDev *const *gs, const CGBuffers *const *cbs, int n, double rtol,
                         int max_it, cudaStream_t s, int **it_dev) {
    int64_t nodes = 0;
    for (int i = 0; i < n; ++i) nodes += gs[i]->n_nodes;
    int occ = 0;
    DD_TRY_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_cg_batch, kBThreads, 0));
    const int cap = std::max(1, std::min(occ, 1)) * ctx->n_sm;   // one block per SM: fewer barrier arrivals
    if (n > cap) return dd_fail(ctx, DD_ERR_ARG, "more solves than resident CG blocks");
    std::vector<int> nblk(n);
    int total = 0;
    for (int i = 0; i < n; ++i) {
        const int64_t nn = gs[i]->n_nodes;
        int64_t want = (nn + kGroups - 1) / kGroups;
        int64_t share = (int64_t)((double)cap * (double)nn / (double)nodes);
        nblk[i] = (int)std::max<int64_t>(1, std::min(want, share));
        total += nblk[i];
    }
    while (total > cap) {   // trim the largest shares until the grid is co-resident
        int k = (int)(std::max_element(nblk.begin(), nblk.end()) - nblk.begin());
        if (nblk[k] <= 1) return dd_fail(ctx, DD_ERR_ARG, "cannot fit the CG grid");
        --nblk[k];
        --total;
    }
    std::vector<SegCG> seg(n);
    std::vector<int> blk_seg(total);
    int b0 = 0;
    for (int i = 0; i < n; ++i) {
        const CGBuffers &cb = *cbs[i];
        const size_t n6 = (size_t)gs[i]->n_nodes * 6;
        SegCG &S = seg[i];
        S.g = *gs[i];
        S.Ke = cb.Ke;
        S.Minv = cb.Minv;
        S.b = cb.b;
        S.x = cb.x;
        S.r = reinterpret_cast<float *>(cb.r);
        S.d = S.r + n6;                 // the FP64 work arrays hold two FP32 vectors each
        S.z = reinterpret_cast<float *>(cb.z);
        S.p0 = reinterpret_cast<float *>(cb.p0);
        S.p1 = reinterpret_cast<float *>(cb.p1);
        S.q = reinterpret_cast<float *>(cb.q);
        S.blk0 = b0;
        S.nblk = nblk[i];
        for (int k = 0; k < nblk[i]; ++k) blk_seg[b0 + k] = i;
        b0 += nblk[i];
    }
    auto r256 = [](size_t b) { return (b + 255) / 256 * 256; };
    const size_t b_seg = r256(n * sizeof(SegCG)), b_bs = r256(total * sizeof(int)),
                 b_part = r256((size_t)2 * total * 8 * 8), b_flags = r256((size_t)2 * n * sizeof(int)),
                 b_it = r256(n * sizeof(int));
    void *w = nullptr;
    DD_TRY(dd_workspace(ctx, WS_BATCH_CG, b_seg + b_bs + b_part + b_flags + b_it + 256, &w));
    char *c = (char *)w;
    SegCG *d_seg = (SegCG *)c;
    int *d_bs = (int *)(c + b_seg);
    double *d_part = (double *)(c + b_seg + b_bs);
    int *d_flags = (int *)(c + b_seg + b_bs + b_part);
    *it_dev = (int *)(c + b_seg + b_bs + b_part + b_flags);
    unsigned *d_bar = (unsigned *)(c + b_seg + b_bs + b_part + b_flags + b_it);
    DD_TRY_CUDA(ctx, cudaMemcpyAsync(d_seg, seg.data(), n * sizeof(SegCG), cudaMemcpyHostToDevice, s));
    DD_TRY_CUDA(ctx, cudaMemcpyAsync(d_bs, blk_seg.data(), total * sizeof(int), cudaMemcpyHostToDevice, s));
    DD_TRY_CUDA(ctx, cudaMemsetAsync(d_bar, 0, 2 * sizeof(unsigned), s));
    BCGArgs A;
    A.seg = d_seg;
    A.blk_seg = d_bs;
    A.S = n;
    A.part = d_part;
    A.flags = d_flags;
    A.bar = d_bar;
    A.err = ctx->dev_err;
    A.rtol2 = rtol * rtol;
    A.in_rtol2 = 1e-8;                  // each refinement step gains four digits
    A.max_outer = 30;
    A.max_inner = max_it;
    A.it_out = *it_dev;
    void *args[] = {&A};
    ctx->launches++;
    DD_TRY_CUDA(ctx, cudaLaunchCooperativeKernel((const void *)k_cg_batch, dim3(total), dim3(kBThreads), args, 0, s));
    return DD_OK;
}


extern "C" dd_status dd_solvers_step(dd_solver **svs, int n, dd_iter_info *infos) {
    if (!svs || n < 1 || !svs[0]) return DD_ERR_ARG;
    dd_ctx *ctx = svs[0]->ctx;
    dd_dataset *ds = svs[0]->ds;
    const dd_solve_opts &o0 = svs[0]->o;
    int64_t M = 0, nodes = 0;
    for (int i = 0; i < n; ++i) {
        dd_solver *sv = svs[i];
        if (!sv || sv->ds != ds) return dd_fail(ctx, DD_ERR_ARG, "dd_solvers_step: solvers must share one data set");
        if (sv->done) return dd_fail(ctx, DD_ERR_STATE, "dd_solvers_step: a solve has already finished");
        if (sv->o.mode != o0.mode || sv->o.certify != o0.certify || sv->o.cg_mode != o0.cg_mode)
            return dd_fail(ctx, DD_ERR_ARG, "dd_solvers_step: solvers must share search mode, certify and cg_mode");
        for (int j = 0; j < i; ++j)
            if (svs[j] == sv) return dd_fail(ctx, DD_ERR_ARG, "dd_solvers_step: a solver appears twice");
        M += sv->g.n_gp;
        nodes += sv->g.n_nodes;
    }
    DD_TRY_CUDA(ctx, cudaSetDevice(ctx->device));
    cudaStream_t s = ctx->stream;
    cudaEvent_t *ev = svs[0]->ev;   // batch-level phase events
    DD_TRY_CUDA(ctx, cudaEventRecord(ev[0], s));
    for (int i = 0; i < n; ++i) {
        dd_solver *sv = svs[i];
        ++sv->it;
        DD_TRY(fem_gather_star(ds, sv->cur, sv->g.n_gp, sv->star, sv->ce, s));
        DD_TRY(fem_assemble_rhs(ctx, sv->g, sv->ops, sv->star, sv->ce, sv->f, const_cast<double *>(sv->cb.b), s));
    }
    // ---- one cooperative CG launch for every solve ----
    std::vector<int> it_host(n, 0);
    int *it_dev = nullptr;
    if (o0.cg_mode == 1) {
        for (int i = 0; i < n; ++i) DD_TRY(fem_cg(ctx, svs[i]->g, svs[i]->cb, o0.cg_rtol, o0.cg_max_iter, s));
    } else {
        std::vector<const MeshDev *> gs(n);
        std::vector<const CGBuffers *> cbs(n);
        for (int i = 0; i < n; ++i) {
            gs[i] = &svs[i]->g;
            cbs[i] = &svs[i]->cb;
        }
        DD_TRY(dd_cg_segments(ctx, gs.data(), cbs.data(), n, o0.cg_rtol, o0.cg_max_iter, s, &it_dev));
    }
    DD_TRY_CUDA(ctx, cudaEventRecord(ev[1], s));
    for (int i = 0; i < n; ++i) DD_TRY(fem_recover(ds, svs[i]->g, svs[i]->ops, svs[i]->cb.x, svs[i]->star, svs[i]->y,
                                                   svs[i]->dpc, s));
    DD_TRY_CUDA(ctx, cudaEventRecord(ev[2], s));

    // ---- one search over the concatenated states ----
    auto r256 = [](size_t b) { return (b + 255) / 256 * 256; };
    const size_t b_y = r256((size_t)M * 96), b_i = r256((size_t)M * 4), b_d = r256((size_t)M * 8),
                 b_fd = r256((size_t)M * 4), b_mq = r256((size_t)M * 48), b_md = r256((size_t)M * 8);
    void *w = nullptr;
    DD_TRY(dd_workspace(ctx, WS_BATCH, b_y + 2 * b_i + 2 * b_d + b_fd + b_mq + b_md, &w));
    char *c = (char *)w;
    double *y_cat = (double *)c;
    int32_t *prev_cat = (int32_t *)(c + b_y);
    int32_t *idx_cat = (int32_t *)(c + b_y + b_i);
    double *d2_cat = (double *)(c + b_y + 2 * b_i);
    double *d2nd_cat = (double *)(c + b_y + 2 * b_i + b_d);
    float *fd_cat = (float *)(c + b_y + 2 * b_i + 2 * b_d);
    AnnMotion mot_cat{(float *)(c + b_y + 2 * b_i + 2 * b_d + b_fd), (float *)(c + b_y + 2 * b_i + 2 * b_d + b_fd + b_mq)};
    const bool ann = o0.mode == DD_SEARCH_ANN;
    std::vector<double> fds(n);
    int64_t off = 0;
    for (int i = 0; i < n; ++i) {
        dd_solver *sv = svs[i];
        const int64_t ng = sv->g.n_gp;
        fds[i] = dd_solver_fd(sv, sv->it);
        DD_TRY_CUDA(ctx, cudaMemcpyAsync(y_cat + off * 12, sv->y, ng * 96, cudaMemcpyDeviceToDevice, s));
        if (ann) {
            DD_TRY_CUDA(ctx, cudaMemcpyAsync(prev_cat + off, sv->cur, ng * 4, cudaMemcpyDeviceToDevice, s));
            DD_TRY_CUDA(ctx, cudaMemcpyAsync(mot_cat.q + off * 12, sv->mot.q, ng * 48, cudaMemcpyDeviceToDevice, s));
            DD_TRY_CUDA(ctx, cudaMemcpyAsync(mot_cat.d + off * 2, sv->mot.d, ng * 8, cudaMemcpyDeviceToDevice, s));
            ctx->launches++;
            k_fill_f<<<(unsigned)((ng + 255) / 256), 256, 0, s>>>(fd_cat + off, ng, (float)fds[i]);
        }
        off += ng;
    }
    dd_search_stats sst;
    std::memset(&sst, 0, sizeof(sst));
    SearchOut so{idx_cat, d2_cat, d2nd_cat};
    if (ann) {
        if (!ds->ann.nlist) return dd_fail(ctx, DD_ERR_STATE, "ANN search needs the partition (ann_nlist)");
        DD_TRY(dd_search_ann_motion(ds, y_cat, M, fds[0], fd_cat, prev_cat, &mot_cat, so, &sst, s));
    } else {
        DD_TRY(dd_run_search(ds, o0.mode, o0.certify, o0.f_d_final, nullptr, y_cat, M, so, &sst, s));
    }
    off = 0;
    for (int i = 0; i < n; ++i) {
        dd_solver *sv = svs[i];
        const int64_t ng = sv->g.n_gp;
        DD_TRY_CUDA(ctx, cudaMemcpyAsync(sv->nxt, idx_cat + off, ng * 4, cudaMemcpyDeviceToDevice, s));
        DD_TRY_CUDA(ctx, cudaMemcpyAsync(sv->d2, d2_cat + off, ng * 8, cudaMemcpyDeviceToDevice, s));
        DD_TRY_CUDA(ctx, cudaMemcpyAsync(sv->d2nd, d2nd_cat + off, ng * 8, cudaMemcpyDeviceToDevice, s));
        if (ann) {
            DD_TRY_CUDA(ctx, cudaMemcpyAsync(sv->mot.q, mot_cat.q + off * 12, ng * 48, cudaMemcpyDeviceToDevice, s));
            DD_TRY_CUDA(ctx, cudaMemcpyAsync(sv->mot.d, mot_cat.d + off * 2, ng * 8, cudaMemcpyDeviceToDevice, s));
        }
        off += ng;
    }
    DD_TRY_CUDA(ctx, cudaEventRecord(ev[3], s));
    for (int i = 0; i < n; ++i)
        DD_TRY(fem_iter_stats(ctx, svs[i]->nxt, svs[i]->cur, svs[i]->d2, svs[i]->dpc, svs[i]->g.n_gp, svs[i]->g.w,
                              svs[i]->stats, s));
    std::vector<double> hs((size_t)n * 3);
    for (int i = 0; i < n; ++i)
        DD_TRY_CUDA(ctx, cudaMemcpyAsync(&hs[(size_t)i * 3], svs[i]->stats, 3 * sizeof(double), cudaMemcpyDeviceToHost, s));
    if (it_dev) {
        DD_TRY_CUDA(ctx, cudaMemcpyAsync(it_host.data(), it_dev, n * sizeof(int), cudaMemcpyDeviceToHost, s));
    } else {
        for (int i = 0; i < n; ++i)
            DD_TRY_CUDA(ctx, cudaMemcpyAsync(&it_host[i], svs[i]->cb.it_out, sizeof(int), cudaMemcpyDeviceToHost, s));
    }
    DD_TRY_CUDA(ctx, cudaStreamSynchronize(s));
    DD_TRY(dd_check_device_error(ctx, s, "dd_solvers_step"));
    float t01 = 0, t12 = 0, t23 = 0;
    cudaEventElapsedTime(&t01, ev[0], ev[1]);
    cudaEventElapsedTime(&t12, ev[1], ev[2]);
    cudaEventElapsedTime(&t23, ev[2], ev[3]);
    for (int i = 0; i < n; ++i) {
        dd_search_stats si = sst;   // the shared search is reported to every solve
        dd_solver_account(svs[i], &hs[(size_t)i * 3], it_host[i], t01, t12, t23, si, fds[i], infos ? &infos[i] : nullptr);
    }
    return DD_OK;
}

extern "C" dd_status dd_solve_batch(dd_dataset *ds, int nsolves, const dd_mesh *meshes, const dd_load *loads,
                                    const dd_solve_opts *opts, dd_result *outs) {
    if (!ds) return DD_ERR_ARG;
    dd_ctx *ctx = ds->ctx;
    if (nsolves < 1 || !meshes || !loads || !outs) return dd_fail(ctx, DD_ERR_ARG, "dd_solve_batch: bad argument");
    std::vector<dd_solver *> svs(nsolves, nullptr);
    dd_status st = DD_OK;
    for (int i = 0; i < nsolves && st == DD_OK; ++i) {
        std::memset(&outs[i], 0, sizeof(dd_result));
        st = dd_solver_create(ds, &meshes[i], &loads[i], opts, &svs[i]);
    }
    while (st == DD_OK) {
        std::vector<dd_solver *> act;
        for (auto *sv : svs)
            if (!sv->done) act.push_back(sv);
        if (act.empty()) break;
        st = dd_solvers_step(act.data(), (int)act.size(), nullptr);
    }
    bool all_conv = true;
    for (int i = 0; i < nsolves && st == DD_OK; ++i) {
        st = dd_solver_result(svs[i], &outs[i]);
        all_conv &= svs[i]->converged;
    }
    for (auto *sv : svs) dd_solver_free(sv);
    if (st == DD_OK && !all_conv) st = DD_ERR_NOT_CONVERGED;
    return st;
}
