// Serving loop: one resident material data set, DD solve requests admitted
// as device memory frees up and stepped together.
//
// A worker thread owns the context.  Every tick it
//   1. admits pending requests in arrival order while their solve states fit
//      in the state budget (and fewer than max_batch solves are active),
//   2. runs one iteration of every active solve with dd_solvers_step: their
//      P_C solves share one cooperative CG launch and all their material
//      points one search, so requests that arrive while others are on the GPU
//      join the next tick (continuous batching),
//   3. retires finished solves: copies the result to the host, frees the
//      state, records the latency (submit -> result ready).
// dd_server_submit / dd_server_poll / dd_server_get_stats may be called from
// any host thread.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "dd_internal.cuh"
#include "solver.cuh"

size_t dd_solver_state_bytes(dd_ctx *ctx, const dd_mesh &mesh);

namespace {

double now_ms() {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

struct Request {
    int64_t ticket;
    dd_mesh mesh;
    dd_load load;
    uint64_t seed;
    double t_submit;
};

struct Finished {
    dd_status st;
    std::string err;
    dd_result res;
    double t_submit, t_admit, t_done;
};

struct Active {
    Request req;
    dd_solver *sv;
    size_t bytes;
    double t_admit;
};

}  // namespace

struct dd_server {
    dd_dataset *ds = nullptr;
    dd_ctx *ctx = nullptr;
    dd_server_opts o;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request> pending;
    std::map<int64_t, Finished> finished;
    std::vector<Active> active;       // worker thread only
    size_t active_bytes = 0;
    bool stopping = false;
    std::thread worker;
    int64_t next_ticket = 1;
    dd_server_stats stats{};
};

static void finish(dd_server *S, const Active &a, dd_status st, const std::string &err) {
    Finished f;
    std::memset(&f.res, 0, sizeof(f.res));
    f.st = st;
    f.err = err;
    f.t_submit = a.req.t_submit;
    f.t_admit = a.t_admit;
    if (st == DD_OK && a.sv) {
        f.st = dd_solver_result(a.sv, &f.res);
        if (f.st == DD_OK && !a.sv->converged) f.st = DD_ERR_NOT_CONVERGED;
        if (f.st != DD_OK && f.st != DD_ERR_NOT_CONVERGED) f.err = S->ctx->err;
    }
    f.t_done = now_ms();
    if (a.sv) dd_solver_free(a.sv);
    std::lock_guard<std::mutex> lk(S->mu);
    S->active_bytes -= std::min(S->active_bytes, a.bytes);
    S->stats.completed++;
    S->stats.active = (int64_t)S->active.size();
    S->finished.emplace(a.req.ticket, std::move(f));
    S->cv_done.notify_all();
}

static void worker_loop(dd_server *S) {
    cudaSetDevice(S->ctx->device);
    const int max_batch = S->o.max_batch > 0 ? S->o.max_batch : 64;
    for (;;) {
        std::vector<Request> admit;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            if (S->active.empty())
                S->cv_work.wait_for(lk, std::chrono::milliseconds(20),
                                    [&] { return S->stopping || !S->pending.empty(); });
            if (S->stopping && S->pending.empty() && S->active.empty()) return;
            size_t bytes = S->active_bytes;
            size_t n_act = S->active.size();
            while (!S->pending.empty() && n_act < (size_t)max_batch) {
                size_t b = dd_solver_state_bytes(S->ctx, S->pending.front().mesh);
                if (S->o.state_budget && n_act > 0 && bytes + b > S->o.state_budget) break;   // wait for room
                admit.push_back(S->pending.front());
                S->pending.pop_front();
                bytes += b;
                ++n_act;
            }
            S->active_bytes = bytes;
            S->stats.pending = (int64_t)S->pending.size();
        }
        for (const Request &r : admit) {
            dd_solve_opts so = S->o.solve;
            so.init_idx = nullptr;
            so.seed = r.seed;
            Active a{r, nullptr, dd_solver_state_bytes(S->ctx, r.mesh), now_ms()};
            dd_status st = dd_solver_create(S->ds, &r.mesh, &r.load, &so, &a.sv);
            if (st != DD_OK) {
                a.sv = nullptr;
                finish(S, a, st, S->ctx->err);
                continue;
            }
            S->active.push_back(a);
        }
        if (S->active.empty()) continue;
        std::vector<dd_solver *> svs;
        for (auto &a : S->active) svs.push_back(a.sv);
        std::vector<dd_iter_info> infos(svs.size());
        const double t0 = now_ms();
        dd_status st = dd_solvers_step(svs.data(), (int)svs.size(), infos.data());
        {
            std::lock_guard<std::mutex> lk(S->mu);
            S->stats.steps++;
            S->stats.busy_ms += now_ms() - t0;
            if (st == DD_OK) {   // the batch's phases are shared by all its solves
                S->stats.cg_ms += infos[0].cg_ms;
                S->stats.search_ms += infos[0].search_ms;
                S->stats.other_ms += infos[0].other_ms;
                S->stats.graph_steps += infos[0].graph;
            }
            S->stats.max_active = std::max<int64_t>(S->stats.max_active, (int64_t)svs.size());
        }
        std::vector<Active> keep;
        for (auto &a : S->active) {
            if (st != DD_OK) finish(S, a, st, S->ctx->err);
            else if (a.sv->done) finish(S, a, DD_OK, "");
            else keep.push_back(a);
        }
        S->active.swap(keep);
        std::lock_guard<std::mutex> lk(S->mu);
        S->stats.active = (int64_t)S->active.size();
    }
}

extern "C" dd_status dd_server_start(dd_dataset *ds, const dd_server_opts *opts, dd_server **out) {
    if (!ds || !out) return DD_ERR_ARG;
    dd_ctx *ctx = ds->ctx;
    *out = nullptr;
    dd_server *S = new dd_server();
    S->ds = ds;
    S->ctx = ctx;
    std::memset(&S->o, 0, sizeof(S->o));
    if (opts) S->o = *opts;
    if (S->o.solve.mode < 0 || S->o.solve.mode > 3) {
        delete S;
        return dd_fail(ctx, DD_ERR_ARG, "dd_server_start: unknown search mode");
    }
    if (S->o.solve.max_iter <= 0) S->o.solve.max_iter = 100;
    if (!(S->o.solve.cg_rtol > 0)) S->o.solve.cg_rtol = 1e-12;
    if (S->o.solve.cg_max_iter <= 0) S->o.solve.cg_max_iter = 20000;
    if (S->o.solve.stall_iters <= 0) S->o.solve.stall_iters = 3;
    if (S->o.solve.mode != DD_SEARCH_ANN && !opts) S->o.solve.certify = 1;
    S->worker = std::thread(worker_loop, S);
    *out = S;
    return DD_OK;
}

extern "C" dd_status dd_server_submit(dd_server *S, const dd_mesh *mesh, const dd_load *load, uint64_t seed,
                                      int64_t *ticket) {
    if (!S || !mesh || !load || !ticket) return DD_ERR_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stopping) return DD_ERR_STATE;
    Request r{S->next_ticket++, *mesh, *load, seed, now_ms()};
    S->pending.push_back(r);
    S->stats.submitted++;
    S->stats.pending = (int64_t)S->pending.size();
    *ticket = r.ticket;
    S->cv_work.notify_one();
    return DD_OK;
}

extern "C" dd_status dd_server_poll(dd_server *S, int64_t ticket, double timeout_s, dd_result *out,
                                    double *latency_ms) {
    if (!S || !out) return DD_ERR_ARG;
    std::memset(out, 0, sizeof(*out));
    std::unique_lock<std::mutex> lk(S->mu);
    auto ready = [&] { return S->finished.count(ticket) != 0; };
    if (!ready()) {
        if (timeout_s <= 0) return DD_ERR_TIMEOUT;
        if (!S->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), ready)) return DD_ERR_TIMEOUT;
    }
    auto it = S->finished.find(ticket);
    Finished f = std::move(it->second);
    S->finished.erase(it);
    *out = f.res;
    if (latency_ms) *latency_ms = f.t_done - f.t_submit;
    // the worker owns the context (and its error string): report the status only
    return f.st;
}

extern "C" dd_status dd_server_get_stats(dd_server *S, dd_server_stats *out) {
    if (!S || !out) return DD_ERR_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    *out = S->stats;
    return DD_OK;
}

extern "C" dd_status dd_server_stop(dd_server *S) {
    if (!S) return DD_ERR_ARG;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stopping = true;
        S->cv_work.notify_all();
    }
    if (S->worker.joinable()) S->worker.join();
    for (auto &kv : S->finished) dd_result_free(&kv.second.res);
    delete S;
    return DD_OK;
}
