// The DD fixed-point iteration z_{i+1} = P_D(P_C(z_i)) (Sec. 2, Eq. 8) as a
// device-resident solver object.
//
// A dd_solver owns the state of one problem on the device: the element
// operators, the two CG solution vectors (warm start of the next P_C), the
// recovered states y and the association.  One step issues, on one stream:
//   gather (eps*, sig*) of the association, assemble E and S (Eq. 5),
//   cooperative CG for K u = E and K eta = S, recovery of eps and sig
//   (Eq. 6), the nearest-data projection (Eq. 7) and a fixed-order reduction
//   of the iteration statistics;
// then reads back three scalars for the stop rule: the association did not
// change (exact search, Sec. 2), or for the approximate search the global
// distance Eq. (2) stopped decreasing.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "dd_internal.cuh"
#include "fem.cuh"
#include "solver.cuh"

dd_status dd_init_association(dd_ctx *ctx, uint64_t seed, int64_t n, int64_t N, int32_t *idx, cudaStream_t s);


namespace {

void solve_defaults(dd_solve_opts *o) {
    std::memset(o, 0, sizeof(*o));
    o->mode = DD_SEARCH_EXACT_FP32;
    o->certify = 1;
    o->ramp_iters = 20;
    o->max_iter = 100;
    o->cg_rtol = 1e-12;
    o->cg_max_iter = 20000;
    o->stall_iters = 3;
}

struct Bump {
    char *base;
    size_t off = 0;
    template <class T>
    T *take(size_t n) {
        T *p = base ? (T *)(base + off) : nullptr;
        off += (n * sizeof(T) + 255) / 256 * 256;
        return p;
    }
};

// Lay out (or, with base == nullptr, size) the solver's device block.
size_t carve(dd_solver *sv, char *base) {
    Bump bp{base};
    const size_t nn = sv->g.n_nodes, ng = sv->g.n_gp;
    sv->Ke = bp.take<double>(576);
    sv->f = bp.take<double>(nn * 3);
    CGBuffers &cb = sv->cb;
    double *b = bp.take<double>(nn * 6), *x = bp.take<double>(nn * 6);
    cb.b = b;
    cb.x = x;
    cb.r = bp.take<double>(nn * 6);
    cb.z = bp.take<double>(nn * 6);
    cb.p0 = bp.take<double>(nn * 6);
    cb.p1 = bp.take<double>(nn * 6);
    cb.q = bp.take<double>(nn * 6);
    sv->Minv = bp.take<double>(nn * 9);
    cb.Minv = sv->Minv;
    cb.Ke = sv->Ke;
    cb.St64 = sv->St64 = bp.take<double>(27 * 27 * 9);
    cb.St32 = sv->St32 = bp.take<float>(27 * 27 * 12);
    fem_mg_plan(sv->g, cb);
    cb.mg_t0 = bp.take<float>(nn * 6);
    for (int l = 1; l < cb.glev; ++l) {
        const size_t n6 = (size_t)(cb.lnx[l] + 1) * (cb.lny[l] + 1) * (cb.lnz[l] + 1) * 6;
        cb.mg_r[l] = bp.take<float>(n6);
        cb.mg_z[l] = bp.take<float>(n6);
        cb.mg_t[l] = bp.take<float>(n6);
    }
    if (cb.glev < cb.nlev) {
        const int l = cb.glev;
        cb.mg_zg = bp.take<float>((size_t)(cb.lnx[l] + 1) * (cb.lny[l] + 1) * (cb.lnz[l] + 1) * 6);
        cb.mg_inv = bp.take<float>((size_t)cb.mg_ndof * cb.mg_ndof);
    }
    cb.part = bp.take<double>((size_t)2 * sv->ctx->n_sm * 32 * 8);
    cb.bar = bp.take<unsigned>(16);
    cb.it_out = bp.take<int>(16);
    cb.res_out = bp.take<double>(8);
    sv->star = bp.take<double>(ng * 12);
    sv->ce = bp.take<double>(ng * 6);
    sv->y = bp.take<double>(ng * 12);
    sv->dpc = bp.take<double>(ng);
    sv->d2 = bp.take<double>(ng);
    sv->d2nd = bp.take<double>(ng);
    sv->cur = bp.take<int32_t>(ng);
    sv->nxt = bp.take<int32_t>(ng);
    sv->idx_a = sv->cur;
    sv->stats = bp.take<double>(kIterStatsDoubles);
    sv->mot.q = bp.take<float>(ng * 12);
    sv->mot.d = bp.take<float>(ng * kMotStride);
    sv->fdq = bp.take<float>(ng);
    return bp.off;
}

}  // namespace

// f_d after k steps of the ramp from f_d0 to f_d_final in ramp_iters steps
static double ramp_fd(const dd_solve_opts &o, int k) {
    if (o.ramp_iters <= 0) return o.f_d_final;
    return o.f_d0 + (o.f_d_final - o.f_d0) * std::min(1.0, (double)k / (double)o.ramp_iters);
}

double dd_solver_fd(const dd_solver *sv, int it) {
    const dd_solve_opts &o = sv->o;
    if (o.mode != DD_SEARCH_ANN) return o.f_d_final;
    // the ramp takes one step per iteration; the global rule one per stalled iteration
    return ramp_fd(o, o.fd_rule == 1 ? sv->fd_steps : it - 1);
}

FdParam dd_solver_fd_param(const dd_solver *sv, int it) {
    const dd_solve_opts &o = sv->o;
    const float f = (float)dd_solver_fd(sv, it);
    FdParam p{f, f, -1.f, 0.f};
    if (o.mode == DD_SEARCH_ANN && o.fd_rule == 2 && !sv->h_pc.empty()) {
        // Eq. (11) with the local distance: near points at full accuracy
        p.f_near = (float)o.f_d_final;
        p.thr = (float)(o.fd_tau * sv->h_pc.back() / (double)sv->g.n_gp);
    }
    return p;
}

bool dd_solver_account(dd_solver *sv, const double hs[3], int cg_it, float cg_ms, float other_ms, float search_ms,
                       const dd_search_stats &sst, double f_d, dd_iter_info *info) {
    const dd_solve_opts &o = sv->o;
    const int it = sv->it;
    sv->cg_ms += cg_ms;
    sv->other_ms += other_ms;
    sv->search_ms += search_ms;
    sv->uncertified += sst.uncertified;
    sv->distances += sst.distances;
    sv->h_pc.push_back(hs[2]);
    sv->h_pd.push_back(hs[1]);
    sv->h_ch.push_back((int64_t)hs[0]);
    sv->h_cg.push_back(cg_it);
    bool stop = false;
    // an approximate search is still tightening while f_d ramps up: its stop
    // tests apply once f_d has reached its final value
    const int steps = o.fd_rule == 1 ? sv->fd_steps : it - 1;   // ramp steps behind this iteration's f_d
    const bool settled = o.mode != DD_SEARCH_ANN || o.ramp_iters <= 0 || steps >= o.ramp_iters;
    if (o.mode == DD_SEARCH_ANN && o.fd_rule == 1) {
        // Eq. (11) with the global distance: one more ramp step after an
        // iteration in which P_D gained less than the fraction fd_tau
        const double gain = hs[2] > 0.0 ? 1.0 - hs[1] / hs[2] : 0.0;
        if (gain < o.fd_tau && sv->fd_steps < o.ramp_iters) ++sv->fd_steps;
    }
    if (hs[0] == 0.0 && settled) {
        sv->converged = true;
        stop = true;   // nxt == cur: the state was computed from the final association
    } else if (o.mode == DD_SEARCH_ANN || o.mode == DD_SEARCH_KNNG) {
        if (hs[1] < sv->best_pd * (1.0 - 1e-12)) {
            sv->best_pd = hs[1];
            sv->stall = 0;
        } else if (settled && ++sv->stall >= o.stall_iters) {
            sv->converged = true;
            stop = true;   // keep the association the constraint state was computed from
        }
    }
    if (!stop) std::swap(sv->cur, sv->nxt);
    if (stop || it >= o.max_iter) sv->done = true;
    if (info) {
        info->iter = it;
        info->changed = (int64_t)hs[0];
        info->d2_pc = hs[2];
        info->d2_pd = hs[1];
        info->cg_iters = cg_it;
        info->cg_ms = cg_ms;
        info->other_ms = other_ms;
        info->search_ms = search_ms;
        info->scan_ms = sst.scan_ms;
        info->uncertified = sst.uncertified;
        info->distances = sst.distances;
        info->f_d = f_d;
        info->done = sv->done ? 1 : 0;
        info->skipped = sst.skipped;
        info->points = sst.points;
        info->unique_points = sst.unique_points;
        info->graph = 0;
        info->moves = sst.moves;
    }
    return sv->done;
}

// Device bytes of one solve's state (what dd_solver_create allocates).
size_t dd_solver_state_bytes(dd_ctx *ctx, const dd_mesh &mesh) {
    dd_solver tmp;
    tmp.ctx = ctx;
    tmp.g = fem_mesh(mesh);
    return carve(&tmp, nullptr);
}

// The host-side setup of sv's mesh (sv->g and sv->cb planned): computed on
// the first solve of a data set on that mesh, then shared; a data set keeps
// the kSetupCache meshes used last (at most ~0.7 MB each).
constexpr size_t kSetupCache = 64;
static std::shared_ptr<const SolverSetup> solver_setup(dd_dataset *ds, const dd_solver *sv) {
    const MeshDev &g = sv->g;
    const dd_mesh &m = sv->mesh;
    std::lock_guard<std::mutex> lock(ds->setup_mu);
    for (size_t k = 0; k < ds->setups.size(); ++k) {
        const auto p = ds->setups[k];
        if (p->nx == m.nx && p->ny == m.ny && p->nz == m.nz && p->top == g.top_fixed && p->lx == m.lx &&
            p->ly == m.ly && p->lz == m.lz) {
            ds->setups.erase(ds->setups.begin() + (std::ptrdiff_t)k);   // most recently used last
            ds->setups.push_back(p);
            return p;
        }
    }
    auto su = std::make_shared<SolverSetup>();
    su->nx = m.nx;
    su->ny = m.ny;
    su->nz = m.nz;
    su->top = g.top_fixed;
    su->lx = m.lx;
    su->ly = m.ly;
    su->lz = m.lz;
    su->Ke.assign(576, 0.0);
    fem_element_stiffness(g, sv->ops, ds->M.C, su->Ke.data());
    su->St64.assign(27 * 27 * 9, 0.0);
    su->St32.assign(27 * 27 * 12, 0.f);
    fem_stencil_table(su->Ke.data(), su->St64.data());
    su->omega = 4.0 / (3.0 * fem_jacobi_lambda_max(su->St64.data()));
    if (sv->cb.glev < sv->cb.nlev) fem_mg_coarse_inverse(sv->cb, su->St64.data(), su->Kinv);
    for (int cd = 0; cd < 27 * 27; ++cd)
        for (int k = 0; k < 9; ++k) su->St32[cd * 12 + k] = (float)su->St64[cd * 9 + k];
    if (ds->setups.size() >= kSetupCache) ds->setups.erase(ds->setups.begin());   // least recently used
    ds->setups.push_back(su);
    return su;
}

extern "C" dd_status dd_solver_create(dd_dataset *ds, const dd_mesh *mesh, const dd_load *load,
                                      const dd_solve_opts *opts, dd_solver **out) {
    if (!ds) return DD_ERR_ARG;
    dd_ctx *ctx = ds->ctx;
    if (!mesh || !load || !out) return dd_fail(ctx, DD_ERR_ARG, "dd_solver_create: NULL argument");
    *out = nullptr;
    if (mesh->nx < 1 || mesh->ny < 1 || mesh->nz < 1 || !(mesh->lx > 0) || !(mesh->ly > 0) || !(mesh->lz > 0))
        return dd_fail(ctx, DD_ERR_ARG, "dd_solver_create: bad mesh");
    if ((int64_t)mesh->nx * mesh->ny * mesh->nz * 8 > INT32_MAX)
        return dd_fail(ctx, DD_ERR_ARG, "dd_solver_create: mesh too large");
    dd_solve_opts o;
    solve_defaults(&o);
    if (opts) {
        o = *opts;
        if (o.max_iter <= 0) o.max_iter = 100;
        if (!(o.cg_rtol > 0)) o.cg_rtol = 1e-12;
        if (o.cg_max_iter <= 0) o.cg_max_iter = 20000;
        if (o.ramp_iters < 0) o.ramp_iters = 0;
        if (o.stall_iters <= 0) o.stall_iters = 3;
    }
    if (o.mode < 0 || o.mode > 3) return dd_fail(ctx, DD_ERR_ARG, "dd_solver_create: unknown mode");
    if (o.mode == DD_SEARCH_KNNG && o.f_s < 0) return dd_fail(ctx, DD_ERR_ARG, "dd_solver_create: f_s < 0");
    if (o.mode == DD_SEARCH_KNNG && !ds->knn.k)
        return dd_fail(ctx, DD_ERR_STATE, "dd_solver_create: graph search needs the k-NN graph (knn_k)");
    if (o.cg_mode < 0 || o.cg_mode > 1) return dd_fail(ctx, DD_ERR_ARG, "dd_solver_create: unknown cg_mode");
    if (o.mode == DD_SEARCH_ANN && !(o.f_d0 >= 0 && o.f_d0 <= 1 && o.f_d_final >= 0 && o.f_d_final <= 1))
        return dd_fail(ctx, DD_ERR_ARG, "dd_solver_create: f_d outside [0, 1]");
    if (o.fd_rule < 0 || o.fd_rule > 2 || !(o.fd_tau >= 0.0))
        return dd_fail(ctx, DD_ERR_ARG, "dd_solver_create: unknown fd_rule or fd_tau < 0");
    if (o.eq14 < 0 || o.eq14 > 1) return dd_fail(ctx, DD_ERR_ARG, "dd_solver_create: unknown eq14 rule");
    for (int c = 0; c < 3; ++c)
        if (!std::isfinite(load->t0[c]) || !std::isfinite(load->tx[c]) || !std::isfinite(load->ty[c]))
            return dd_fail(ctx, DD_ERR_ARG, "dd_solver_create: non-finite load");
    const bool rotate = load->rot_z != 0.0;
    if (rotate) {
        if (!std::isfinite(load->rot_z)) return dd_fail(ctx, DD_ERR_ARG, "dd_solver_create: non-finite rotation");
        for (int c = 0; c < 3; ++c)
            if (load->t0[c] != 0.0 || load->tx[c] != 0.0 || load->ty[c] != 0.0)
                return dd_fail(ctx, DD_ERR_ARG, "dd_solver_create: traction and prescribed rotation on the same face");
        if (mesh->nz < 2) return dd_fail(ctx, DD_ERR_ARG, "dd_solver_create: a prescribed rotation needs nz >= 2");
    }
    DD_TRY_CUDA(ctx, cudaSetDevice(ctx->device));
    static std::atomic<uint64_t> next_id{1};
    dd_solver *sv = new dd_solver();
    sv->id = next_id++;
    sv->ds = ds;
    sv->ctx = ctx;
    sv->mesh = *mesh;
    sv->o = o;
    sv->o.init_idx = nullptr;
    sv->g = fem_mesh(*mesh);
    sv->g.top_fixed = rotate ? 1 : 0;
    fem_elem_ops(sv->g, &sv->ops);
    auto fail = [&](dd_status st) {
        dd_solver_free(sv);
        return st;
    };
    sv->block_bytes = carve(sv, nullptr);
    dd_status st = dd_alloc(ctx, &sv->block, sv->block_bytes, "solver state");
    if (st != DD_OK) return fail(st);
    carve(sv, (char *)sv->block);
    for (auto &e : sv->ev)
        if (cudaEventCreate(&e) != cudaSuccess) return fail(dd_fail(ctx, DD_ERR_CUDA, "cudaEventCreate"));
    const size_t nn = sv->g.n_nodes, ng = sv->g.n_gp;
    const std::shared_ptr<const SolverSetup> su = solver_setup(ds, sv);
    const std::vector<double> &Ke = su->Ke, &St64 = su->St64;
    const std::vector<float> &St32 = su->St32, &Kinv = su->Kinv;
    sv->cb.omega = su->omega;
    std::vector<double> f(nn * 3);
    fem_traction_force(sv->g, *load, mesh->lx, mesh->ly, f.data());
    // x starts at zero, with the prescribed top displacement in its u part;
    // the solves keep those entries (fixed dofs) and the residual b - K x
    // carries their coupling to the free dofs
    std::vector<double> x0(nn * 6, 0.0);
    if (rotate) fem_top_rotation(sv->g, load->rot_z, mesh->lx, mesh->ly, x0.data());
    cudaStream_t s = ctx->stream;
    if (cudaMemcpyAsync(sv->Ke, Ke.data(), 576 * 8, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(sv->St64, St64.data(), St64.size() * 8, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(sv->St32, St32.data(), St32.size() * 4, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        (!Kinv.empty() &&
         cudaMemcpyAsync(sv->cb.mg_inv, Kinv.data(), Kinv.size() * 4, cudaMemcpyHostToDevice, s) != cudaSuccess) ||
        cudaMemcpyAsync(sv->f, f.data(), nn * 3 * 8, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(sv->cb.x, x0.data(), nn * 6 * 8, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemsetAsync(sv->mot.d, 0, ng * kMotStride * sizeof(float), s) != cudaSuccess ||
        cudaMemsetAsync(sv->stats, 0, kIterStatsDoubles * sizeof(double), s) != cudaSuccess)
        return fail(dd_fail(ctx, DD_ERR_CUDA, "dd_solver_create: upload"));
    if ((st = fem_block_jacobi(ctx, sv->g, sv->Ke, sv->Minv, s)) != DD_OK) return fail(st);
    if (opts && opts->init_idx) {
        cudaMemcpyKind k = dd_is_device_ptr(opts->init_idx) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        if (cudaMemcpyAsync(sv->cur, opts->init_idx, ng * 4, k, s) != cudaSuccess)
            return fail(dd_fail(ctx, DD_ERR_CUDA, "dd_solver_create: copy init_idx"));
    } else if ((st = dd_init_association(ctx, o.seed, ng, ds->N, sv->cur, s)) != DD_OK) {
        return fail(st);
    }
    if (cudaStreamSynchronize(s) != cudaSuccess) return fail(dd_fail(ctx, DD_ERR_CUDA, "dd_solver_create: sync"));
    *out = sv;
    return DD_OK;
}

extern "C" void dd_solver_free(dd_solver *sv) {
    if (!sv) return;
    cudaSetDevice(sv->ctx->device);
    cudaStreamSynchronize(sv->ctx->stream);
    dd_plans_drop(sv->ctx, sv->id);
    for (auto &e : sv->ev)
        if (e) cudaEventDestroy(e);
    dd_free(sv->ctx, sv->block, sv->block_bytes);
    delete sv;
}

extern "C" int dd_solver_done(const dd_solver *sv) { return sv ? (sv->done ? 1 : 0) : 1; }

extern "C" dd_status dd_solver_step(dd_solver *sv, dd_iter_info *info) {
    if (!sv) return DD_ERR_ARG;
    dd_ctx *ctx = sv->ctx;
    if (sv->done) return dd_fail(ctx, DD_ERR_STATE, "dd_solver_step: solve already finished");
    DD_TRY_CUDA(ctx, cudaSetDevice(ctx->device));
    dd_dataset *ds = sv->ds;
    const dd_solve_opts &o = sv->o;
    const MeshDev &g = sv->g;
    const int64_t ng = g.n_gp;
    cudaStream_t s = ctx->stream;
    const int it = ++sv->it;
    DD_TRY_CUDA(ctx, cudaEventRecord(sv->ev[0], s));
    DD_TRY(fem_gather_star(ds, sv->cur, ng, sv->star, sv->ce, s));
    DD_TRY(fem_assemble_rhs(ctx, g, sv->ops, sv->star, sv->ce, sv->f, const_cast<double *>(sv->cb.b), s));
    if (o.cg_mode == 1) DD_TRY(fem_cg(ctx, g, sv->cb, o.cg_rtol, o.cg_max_iter, s));
    else DD_TRY(fem_cg_mixed(ctx, g, sv->cb, o.cg_rtol, o.cg_max_iter, s));
    DD_TRY_CUDA(ctx, cudaEventRecord(sv->ev[1], s));
    DD_TRY(fem_recover(ds, g, sv->ops, sv->cb.x, sv->star, sv->y, sv->dpc, s));
    DD_TRY_CUDA(ctx, cudaEventRecord(sv->ev[2], s));
    const FdParam fp = dd_solver_fd_param(sv, it);
    const double f_d = fp.f_far;
    SearchOut so{sv->nxt, sv->d2, sv->d2nd};
    dd_search_stats sst;
    std::memset(&sst, 0, sizeof(sst));
    if (o.mode == DD_SEARCH_ANN) {
        if (!ds->ann.nlist) return dd_fail(ctx, DD_ERR_STATE, "ANN search needs the partition (ann_nlist)");
        const float *fdq = nullptr;
        if (fp.thr >= 0.f) {
            DD_TRY(dd_fill_fd(ctx, sv->fdq, ng, nullptr, fp, sv->dpc, s));
            fdq = sv->fdq;
        }
        DD_TRY(dd_search_ann_motion(ds, sv->y, ng, f_d, fdq, sv->cur, &sv->mot, o.ann_budget, so, &sst, s, o.eq14));
    } else if (o.mode == DD_SEARCH_KNNG) {
        DD_TRY(dd_search_knng(ds, sv->y, ng, o.f_s, sv->cur, &sv->mot, so, &sst, s));
    } else {
        DD_TRY(dd_run_search(ds, o.mode, o.certify, f_d, o.f_s, o.ann_budget, sv->cur, sv->y, ng, so, &sst, s));
    }
    DD_TRY_CUDA(ctx, cudaEventRecord(sv->ev[3], s));
    DD_TRY(fem_iter_stats(ctx, sv->nxt, sv->cur, sv->d2, sv->dpc, ng, g.w, sv->stats, s));
    double hs[3];
    int cg_it = 0;
    DD_TRY_CUDA(ctx, cudaMemcpyAsync(hs, sv->stats, sizeof(hs), cudaMemcpyDeviceToHost, s));
    DD_TRY_CUDA(ctx, cudaMemcpyAsync(&cg_it, sv->cb.it_out, sizeof(int), cudaMemcpyDeviceToHost, s));
    DD_TRY_CUDA(ctx, cudaStreamSynchronize(s));
    DD_TRY(dd_check_device_error(ctx, s, "dd_solver_step"));
    float t01 = 0, t12 = 0, t23 = 0;
    cudaEventElapsedTime(&t01, sv->ev[0], sv->ev[1]);
    cudaEventElapsedTime(&t12, sv->ev[1], sv->ev[2]);
    cudaEventElapsedTime(&t23, sv->ev[2], sv->ev[3]);
    dd_solver_account(sv, hs, cg_it, t01, t12, t23, sst, f_d, info);
    return DD_OK;
}

extern "C" dd_status dd_solver_result(dd_solver *sv, dd_result *out) {
    if (!sv || !out) return DD_ERR_ARG;
    dd_ctx *ctx = sv->ctx;
    std::memset(out, 0, sizeof(*out));
    const size_t nn = sv->g.n_nodes, ng = sv->g.n_gp;
    out->n_nodes = sv->g.n_nodes;
    out->n_gp = sv->g.n_gp;
    out->iters = (int)sv->h_pc.size();
    out->converged = sv->converged ? 1 : 0;
    size_t ni = sv->h_pc.size() ? sv->h_pc.size() : 1;
    out->u = (double *)std::malloc(nn * 3 * 8);
    out->eta = (double *)std::malloc(nn * 3 * 8);
    out->eps = (double *)std::malloc(ng * 6 * 8);
    out->sig = (double *)std::malloc(ng * 6 * 8);
    out->idx = (int32_t *)std::malloc(ng * 4);
    out->d2_pc = (double *)std::malloc(ni * 8);
    out->d2_pd = (double *)std::malloc(ni * 8);
    out->changed = (int64_t *)std::malloc(ni * 8);
    out->cg_iters = (int *)std::malloc(ni * sizeof(int));
    if (!out->u || !out->eta || !out->eps || !out->sig || !out->idx || !out->d2_pc || !out->d2_pd || !out->changed ||
        !out->cg_iters) {
        dd_result_free(out);
        return dd_fail(ctx, DD_ERR_OOM, "dd_solver_result: host allocation failed");
    }
    // the state of the last P_C and the association it was computed from
    const int32_t *assoc = sv->converged ? sv->cur : sv->nxt;
    if (sv->it == 0) assoc = sv->cur;
    std::vector<double> hx(nn * 6), hy(ng * 12);
    cudaStream_t s = ctx->stream;
    DD_TRY_CUDA(ctx, cudaMemcpyAsync(hx.data(), sv->cb.x, nn * 6 * 8, cudaMemcpyDeviceToHost, s));
    DD_TRY_CUDA(ctx, cudaMemcpyAsync(hy.data(), sv->y, ng * 12 * 8, cudaMemcpyDeviceToHost, s));
    DD_TRY_CUDA(ctx, cudaMemcpyAsync(out->idx, assoc, ng * 4, cudaMemcpyDeviceToHost, s));
    DD_TRY_CUDA(ctx, cudaStreamSynchronize(s));
    for (size_t a = 0; a < nn; ++a)
        for (int c = 0; c < 3; ++c) {
            out->u[a * 3 + c] = hx[a * 6 + c];
            out->eta[a * 3 + c] = hx[a * 6 + 3 + c];
        }
    for (size_t e = 0; e < ng; ++e)
        for (int c = 0; c < 6; ++c) {
            out->eps[e * 6 + c] = hy[e * 12 + c];
            out->sig[e * 6 + c] = hy[e * 12 + 6 + c];
        }
    for (size_t i = 0; i < sv->h_pc.size(); ++i) {
        out->d2_pc[i] = sv->h_pc[i];
        out->d2_pd[i] = sv->h_pd[i];
        out->changed[i] = sv->h_ch[i];
        out->cg_iters[i] = sv->h_cg[i];
    }
    out->search_ms = sv->search_ms;
    out->cg_ms = sv->cg_ms;
    out->other_ms = sv->other_ms;
    out->uncertified = sv->uncertified;
    out->distances = sv->distances;
    return DD_OK;
}

extern "C" dd_status dd_solve(dd_dataset *ds, const dd_mesh *mesh, const dd_load *load, const dd_solve_opts *opts,
                              dd_result *out) {
    if (!ds) return DD_ERR_ARG;
    if (!out) return dd_fail(ds->ctx, DD_ERR_ARG, "dd_solve: NULL argument");
    std::memset(out, 0, sizeof(*out));
    dd_solver *sv = nullptr;
    DD_TRY(dd_solver_create(ds, mesh, load, opts, &sv));
    dd_status st = DD_OK;
    while (!sv->done && (st = dd_solver_step(sv, nullptr)) == DD_OK) {
    }
    if (st == DD_OK) st = dd_solver_result(sv, out);
    if (st == DD_OK && !sv->converged) st = DD_ERR_NOT_CONVERGED;
    dd_solver_free(sv);
    return st;
}

extern "C" void dd_result_free(dd_result *r) {
    if (!r) return;
    std::free(r->u);
    std::free(r->eta);
    std::free(r->eps);
    std::free(r->sig);
    std::free(r->idx);
    std::free(r->d2_pc);
    std::free(r->d2_pd);
    std::free(r->changed);
    std::free(r->cg_iters);
    std::memset(r, 0, sizeof(*r));
}
