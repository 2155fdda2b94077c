// C ABI of libdd: context, data set, data projection P_D and the DD solve.
//
// The DD iteration z_{i+1} = P_D(P_C(z_i)) (Sec. 2, Eq. 8) runs device
// resident: per iteration the host issues the kernels of P_C (fem.cu) and
// P_D (search_*.cu, ann.cu) on one stream and reads back three scalars (the
// number of changed associations and the global distance Eq. 2 after P_C and
// after P_D) for the stop test of Sec. 2.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "dd_internal.cuh"
#include "fem.cuh"

static thread_local std::string g_create_err;

dd_status dd_fail(dd_ctx *ctx, dd_status st, const std::string &msg) {
    if (ctx) ctx->err = msg;
    else g_create_err = msg;
    return st;
}

dd_status dd_alloc(dd_ctx *ctx, void **p, size_t bytes, const char *what) {
    *p = nullptr;
    if (bytes == 0) bytes = 256;
    if (ctx->budget && ctx->in_use + bytes > ctx->budget)
        return dd_fail(ctx, DD_ERR_OOM, std::string("HBM budget exceeded allocating ") + what);
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return dd_fail(ctx, DD_ERR_OOM, std::string("cudaMalloc failed for ") + what + ": " + cudaGetErrorString(e));
    }
    ctx->in_use += bytes;
    return DD_OK;
}

void dd_free(dd_ctx *ctx, void *p, size_t bytes) {
    if (!p) return;
    cudaFree(p);
    if (bytes == 0) bytes = 256;
    ctx->in_use -= std::min(ctx->in_use, bytes);
}

dd_status dd_workspace(dd_ctx *ctx, int slot, size_t bytes, void **out) {
    Workspace &w = ctx->ws[slot];
    if (w.bytes >= bytes && w.ptr) {
        *out = w.ptr;
        return DD_OK;
    }
    if (ctx->capturing) return dd_fail(ctx, DD_ERR_STATE, "workspace would grow while a step is captured");
    if (w.ptr) {
        DD_TRY_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        DD_TRY_CUDA(ctx, cudaDeviceSynchronize());
        dd_free(ctx, w.ptr, w.bytes);
        w.ptr = nullptr;
        w.bytes = 0;
    }
    size_t nb = std::max<size_t>(bytes + bytes / 4, 4096);
    DD_TRY(dd_alloc(ctx, &w.ptr, nb, "workspace"));
    w.bytes = nb;
    ctx->ws_gen++;
    *out = w.ptr;
    return DD_OK;
}

dd_status dd_check_device_error(dd_ctx *ctx, cudaStream_t s, const char *where) {
    unsigned h = 0;
    DD_TRY_CUDA(ctx, cudaMemcpyAsync(&h, ctx->dev_err, sizeof(h), cudaMemcpyDeviceToHost, s));
    DD_TRY_CUDA(ctx, cudaStreamSynchronize(s));
    if (h == 0) return DD_OK;
    DD_TRY_CUDA(ctx, cudaMemsetAsync(ctx->dev_err, 0, sizeof(unsigned), s));
    DD_TRY_CUDA(ctx, cudaStreamSynchronize(s));
    if (h & DEV_ERR_TIMEOUT) return dd_fail(ctx, DD_ERR_TIMEOUT, std::string(where) + ": device wait timed out");
    return dd_fail(ctx, DD_ERR_ARG, std::string(where) + ": index out of range");
}

bool dd_is_device_ptr(const void *p) {
    if (!p) return false;
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

dd_status dd_transform_dataset(dd_dataset *ds);
dd_status dd_init_association(dd_ctx *ctx, uint64_t seed, int64_t n, int64_t N, int32_t *idx, cudaStream_t s);

// ---------------------------------------------------------------------------
// Context
// ---------------------------------------------------------------------------
extern "C" dd_status dd_create(int device, size_t hbm_budget, dd_ctx **out) {
    if (!out) return dd_fail(nullptr, DD_ERR_ARG, "dd_create: out is NULL");
    *out = nullptr;
    int n = 0;
    cudaError_t e = cudaGetDeviceCount(&n);
    if (e != cudaSuccess || n == 0) {
        cudaGetLastError();
        return dd_fail(nullptr, DD_ERR_CUDA, "no CUDA device available");
    }
    if (device < 0 || device >= n) return dd_fail(nullptr, DD_ERR_ARG, "dd_create: device out of range");
    dd_ctx *ctx = new dd_ctx();
    ctx->device = device;
    ctx->budget = hbm_budget;
    auto bail = [&](const char *what, cudaError_t err) {
        g_create_err = std::string(what) + ": " + cudaGetErrorString(err);
        cudaGetLastError();
        if (ctx->dev_err) cudaFree(ctx->dev_err);
        if (ctx->stream) cudaStreamDestroy(ctx->stream);
        delete ctx;
        return DD_ERR_CUDA;
    };
    if ((e = cudaSetDevice(device)) != cudaSuccess) return bail("cudaSetDevice", e);
    if ((e = cudaDeviceGetAttribute(&ctx->n_sm, cudaDevAttrMultiProcessorCount, device)) != cudaSuccess)
        return bail("cudaDeviceGetAttribute", e);
    if ((e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking)) != cudaSuccess)
        return bail("cudaStreamCreate", e);
    if ((e = cudaMalloc((void **)&ctx->dev_err, 256)) != cudaSuccess) return bail("cudaMalloc", e);
    if ((e = cudaMemset(ctx->dev_err, 0, 256)) != cudaSuccess) return bail("cudaMemset", e);
    if ((e = cudaEventCreate(&ctx->ev_scan[0])) != cudaSuccess) return bail("cudaEventCreate", e);
    if ((e = cudaEventCreate(&ctx->ev_scan[1])) != cudaSuccess) return bail("cudaEventCreate", e);
    ctx->in_use = 256;
    *out = ctx;
    return DD_OK;
}

extern "C" void dd_destroy(dd_ctx *ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    dd_plans_drop(ctx, 0);
    for (auto &w : ctx->ws)
        if (w.ptr) cudaFree(w.ptr);
    cudaFree(ctx->dev_err);
    cudaEventDestroy(ctx->ev_scan[0]);
    cudaEventDestroy(ctx->ev_scan[1]);
    cudaStreamDestroy(ctx->stream);
    delete ctx;
}

extern "C" const char *dd_last_error(const dd_ctx *ctx) { return ctx ? ctx->err.c_str() : g_create_err.c_str(); }

extern "C" size_t dd_bytes_in_use(const dd_ctx *ctx) { return ctx ? ctx->in_use : 0; }

extern "C" int64_t dd_launch_count(const dd_ctx *ctx) { return ctx ? ctx->launches : 0; }

// ---------------------------------------------------------------------------
// Data set
// ---------------------------------------------------------------------------
extern "C" dd_status dd_load_dataset(dd_ctx *ctx, const float *eps_sig, int64_t N, const double *C,
                                     const dd_dataset_opts *opts, dd_dataset **out) {
    if (!ctx) return DD_ERR_ARG;
    if (!out || !eps_sig || !C) return dd_fail(ctx, DD_ERR_ARG, "dd_load_dataset: NULL argument");
    *out = nullptr;
    if (N < 1 || N > INT32_MAX) return dd_fail(ctx, DD_ERR_ARG, "dd_load_dataset: N out of range");
    dd_dataset_opts o;
    std::memset(&o, 0, sizeof(o));
    if (opts) o = *opts;
    if (o.ann_nlist < 0 || o.ann_nlist > N) return dd_fail(ctx, DD_ERR_ARG, "dd_load_dataset: ann_nlist out of range");
    DD_TRY_CUDA(ctx, cudaSetDevice(ctx->device));
    dd_dataset *ds = new dd_dataset();
    ds->ctx = ctx;
    if (!dd_metric_maps(C, &ds->M)) {
        delete ds;
        return dd_fail(ctx, DD_ERR_NOT_SPD, "metric C is not symmetric positive definite");
    }
    ds->N = N;
    ds->N_pad = (N + kDataTile - 1) / kDataTile * kDataTile;
    const bool dev = dd_is_device_ptr(eps_sig);
    dd_status st = DD_OK;
    auto fail = [&](dd_status s2) {
        dd_free_dataset(ds);
        return s2;
    };
    if (dev && o.borrow) {
        ds->raw = eps_sig;
        ds->owns_raw = false;
    } else {
        void *p = nullptr;
        if ((st = dd_alloc(ctx, &p, (size_t)N * 48, "data set")) != DD_OK) return fail(st);
        ds->raw = (const float *)p;
        ds->bytes += (size_t)N * 48;
        cudaError_t e = cudaMemcpyAsync(p, eps_sig, (size_t)N * 48, dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                        ctx->stream);
        if (e != cudaSuccess) return fail(dd_fail(ctx, DD_ERR_CUDA, std::string("copy data set: ") + cudaGetErrorString(e)));
    }
    void *p = nullptr;
    if ((st = dd_alloc(ctx, &p, (size_t)ds->N_pad * 48, "mapped data")) != DD_OK) return fail(st);
    ds->z32 = (float *)p;
    if ((st = dd_alloc(ctx, &p, (size_t)ds->N_pad * 4, "norms")) != DD_OK) return fail(st);
    ds->zn = (float *)p;
    ds->bytes += (size_t)ds->N_pad * 52;
    if ((st = dd_transform_dataset(ds)) != DD_OK) return fail(st);
    if (o.build_fp16 && (st = dd_build_fp16(ds)) != DD_OK) return fail(st);
    if (o.ann_nlist > 0 && (st = dd_build_ann(ds, o)) != DD_OK) return fail(st);
    if (o.knn_k != 0 && (st = dd_build_knng(ds, o)) != DD_OK) return fail(st);
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return fail(dd_fail(ctx, DD_ERR_CUDA, cudaGetErrorString(e)));
    *out = ds;
    return DD_OK;
}

extern "C" void dd_free_dataset(dd_dataset *ds) {
    if (!ds) return;
    dd_ctx *ctx = ds->ctx;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    dd_plans_drop(ctx, 0);
    if (ds->owns_raw) dd_free(ctx, (void *)ds->raw, (size_t)ds->N * 48);
    dd_free(ctx, ds->z32, (size_t)ds->N_pad * 48);
    dd_free(ctx, ds->zn, (size_t)ds->N_pad * 4);
    if (ds->z16hi) dd_free(ctx, ds->z16hi, (size_t)ds->N_pad * 32);
    if (ds->z16lo) dd_free(ctx, ds->z16lo, (size_t)ds->N_pad * 32);
    dd_free_knng(ds);
    dd_free_ann(ds);
    delete ds;
}

extern "C" int64_t dd_dataset_size(const dd_dataset *ds) { return ds ? ds->N : 0; }

extern "C" size_t dd_dataset_bytes(const dd_dataset *ds) { return ds ? ds->bytes : 0; }

// ---------------------------------------------------------------------------
// P_D
// ---------------------------------------------------------------------------
dd_status dd_run_search(dd_dataset *ds, int mode, int certify, double f_d, int f_s, int budget,
                        const int32_t *prev_dev,
                            const double *y_dev, int64_t m, SearchOut out, dd_search_stats *st, cudaStream_t s) {
    switch (mode) {
    case DD_SEARCH_EXACT_FP32:
        return dd_search_exact_fp32(ds, y_dev, m, certify, out, st, s);
    case DD_SEARCH_EXACT_TC:
        if (!ds->z16hi) return dd_fail(ds->ctx, DD_ERR_STATE, "tensor-core search needs the FP16 copy (build_fp16)");
        return dd_search_exact_tc(ds, y_dev, m, certify, out, st, s);
    case DD_SEARCH_ANN:
        if (!ds->ann.nlist) return dd_fail(ds->ctx, DD_ERR_STATE, "ANN search needs the partition (ann_nlist)");
        return dd_search_ann(ds, y_dev, m, f_d, prev_dev, budget, out, st, s);
    case DD_SEARCH_KNNG:
        return dd_search_knng(ds, y_dev, m, f_s, prev_dev, nullptr, out, st, s);
    default:
        return dd_fail(ds->ctx, DD_ERR_ARG, "unknown search mode");
    }
}

extern "C" dd_status dd_project_nearest(dd_dataset *ds, const double *y, int64_t m, const dd_search_opts *opts,
                                        int32_t *idx, double *d2, int32_t *topk_out, dd_search_stats *stats) {
    if (!ds) return DD_ERR_ARG;
    dd_ctx *ctx = ds->ctx;
    if (m < 0) return dd_fail(ctx, DD_ERR_ARG, "dd_project_nearest: m < 0");
    if (m == 0) return DD_OK;
    if (!y || !idx) return dd_fail(ctx, DD_ERR_ARG, "dd_project_nearest: NULL argument");
    dd_search_opts o;
    std::memset(&o, 0, sizeof(o));
    o.certify = 1;
    if (opts) o = *opts;
    const bool approx = o.mode == DD_SEARCH_ANN || o.mode == DD_SEARCH_KNNG;
    if (o.mode == DD_SEARCH_ANN && !(o.f_d >= 0.0 && o.f_d <= 1.0))
        return dd_fail(ctx, DD_ERR_ARG, "dd_project_nearest: f_d outside [0, 1]");
    if (o.mode == DD_SEARCH_KNNG && o.f_s < 0) return dd_fail(ctx, DD_ERR_ARG, "dd_project_nearest: f_s < 0");
    const int k = o.topk;
    if (k < 0 || k > DD_TOPK_MAX) return dd_fail(ctx, DD_ERR_ARG, "dd_project_nearest: topk outside 0 .. DD_TOPK_MAX");
    if ((k > 0) != (topk_out != nullptr))
        return dd_fail(ctx, DD_ERR_ARG, "dd_project_nearest: topk_out and opts->topk must be given together");
    if (o.topk_d2 && !topk_out) return dd_fail(ctx, DD_ERR_ARG, "dd_project_nearest: topk_d2 without topk_out");
    if (k > 0 && approx) return dd_fail(ctx, DD_ERR_ARG, "dd_project_nearest: topk needs an exact search mode");
    if (o.eq14 < 0 || o.eq14 > 1) return dd_fail(ctx, DD_ERR_ARG, "dd_project_nearest: unknown eq14 rule");
    if (o.tc_terms != 0 && o.tc_terms != 2 && o.tc_terms != 3)
        return dd_fail(ctx, DD_ERR_ARG, "dd_project_nearest: tc_terms must be 0, 2 or 3");
    const bool motion = o.prev_y != nullptr;
    if (motion && !approx)
        return dd_fail(ctx, DD_ERR_ARG, "dd_project_nearest: the motion record (prev_y) needs an approximate mode");
    if (motion && (!o.prev_idx || !o.prev_d2 || !o.prev_d2nd))
        return dd_fail(ctx, DD_ERR_ARG, "dd_project_nearest: prev_y needs prev_idx, prev_d2 and prev_d2nd");
    DD_TRY_CUDA(ctx, cudaSetDevice(ctx->device));
    const bool dev = dd_is_device_ptr(y);
    for (const void *p : {(const void *)idx, (const void *)d2, (const void *)topk_out, (const void *)o.topk_d2,
                          (const void *)o.d2nd, (const void *)o.prev_y, (const void *)o.prev_d2,
                          (const void *)o.prev_d2nd})
        if (p && dd_is_device_ptr(p) != dev)
            return dd_fail(ctx, DD_ERR_ARG, "dd_project_nearest: all arrays must be host or all device memory");
    if (o.prev_idx && dev && !dd_is_device_ptr(o.prev_idx))
        return dd_fail(ctx, DD_ERR_ARG, "dd_project_nearest: prev_idx must be device memory with device y");
    cudaStream_t s = o.stream ? (cudaStream_t)o.stream : ctx->stream;
    auto r256 = [](size_t b) { return (b + 255) / 256 * 256; };
    // device copies of host arrays, and the buffers the search needs besides
    // the caller's: d2 and d2nd when not asked for (the motion record and the
    // top-k distances read them), the motion record
    const size_t by = r256((size_t)m * 96), bi = r256((size_t)m * 4), bd = r256((size_t)m * 8),
                 bk = r256((size_t)m * (k > 0 ? k : 1) * 4), bkd = r256((size_t)m * (k > 0 ? k : 1) * 8),
                 brec = r256((size_t)m * sizeof(QueryRec)), bmq = r256((size_t)m * 48),
                 bmd = r256((size_t)m * 4 * kMotStride);
    const size_t need = 2 * by + 2 * bi + 4 * bd + bk + bkd + brec + bmq + bmd;
    void *w = nullptr;
    DD_TRY(dd_workspace(ctx, WS_QUERY, need, &w));
    char *c = (char *)w;
    auto take = [&](size_t b) {
        char *p = c;
        c += b;
        return p;
    };
    const double *y_dev = dev ? y : (const double *)take(by);
    const double *py_dev = (dev || !motion) ? o.prev_y : (const double *)take(by);
    int32_t *idx_dev = dev ? idx : (int32_t *)take(bi);
    const int32_t *prev_dev = (dev || !o.prev_idx) ? o.prev_idx : (const int32_t *)take(bi);
    double *d2_dev = (dev && d2) ? d2 : (double *)take(bd);
    double *d2nd_dev = (dev && o.d2nd) ? o.d2nd : (double *)take(bd);
    const double *pd2_dev = (dev || !motion) ? o.prev_d2 : (const double *)take(bd);
    const double *pd2nd_dev = (dev || !motion) ? o.prev_d2nd : (const double *)take(bd);
    int32_t *tk_dev = (dev || !topk_out) ? topk_out : (int32_t *)take(bk);
    double *tkd_dev = (dev && o.topk_d2) ? o.topk_d2 : (k > 0 ? (double *)take(bkd) : nullptr);
    QueryRec *prec = motion ? (QueryRec *)take(brec) : nullptr;
    AnnMotion mot{motion ? (float *)take(bmq) : nullptr, motion ? (float *)take(bmd) : nullptr};
    if (!dev) {
        DD_TRY_CUDA(ctx, cudaMemcpyAsync((void *)y_dev, y, (size_t)m * 96, cudaMemcpyHostToDevice, s));
        if (o.prev_idx)
            DD_TRY_CUDA(ctx, cudaMemcpyAsync((void *)prev_dev, o.prev_idx, (size_t)m * 4, cudaMemcpyHostToDevice, s));
        if (motion) {
            DD_TRY_CUDA(ctx, cudaMemcpyAsync((void *)py_dev, o.prev_y, (size_t)m * 96, cudaMemcpyHostToDevice, s));
            DD_TRY_CUDA(ctx, cudaMemcpyAsync((void *)pd2_dev, o.prev_d2, (size_t)m * 8, cudaMemcpyHostToDevice, s));
            DD_TRY_CUDA(ctx, cudaMemcpyAsync((void *)pd2nd_dev, o.prev_d2nd, (size_t)m * 8, cudaMemcpyHostToDevice, s));
        }
    }
    dd_search_stats local;
    std::memset(&local, 0, sizeof(local));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (stats) {
        DD_TRY_CUDA(ctx, cudaEventCreate(&e0));
        DD_TRY_CUDA(ctx, cudaEventCreate(&e1));
        DD_TRY_CUDA(ctx, cudaEventRecord(e0, s));
    }
    SearchOut out{idx_dev, d2_dev, d2nd_dev};
    if (k >= 2) {
        out.k = k;
        out.topk_idx = tk_dev;
        out.topk_d2 = tkd_dev;
    }
    dd_search_stats *pst = stats ? &local : nullptr;
    dd_status st = DD_OK;
    if (motion) {
        // the record of the previous call: its mapped states and the plain
        // distances of Eq. (14), made at this call's f_d
        DD_TRY(dd_map_queries(ds, py_dev, m, nullptr, prec, s));
        DD_TRY(dd_ann_motion_update(ctx, prec, m, pd2_dev, pd2nd_dev, o.mode == DD_SEARCH_ANN ? o.f_d : 1.0, nullptr,
                                    o.mode == DD_SEARCH_ANN ? o.eq14 : 0, &mot, s));
        if (o.mode == DD_SEARCH_ANN) {
            if (!ds->ann.nlist) return dd_fail(ctx, DD_ERR_STATE, "ANN search needs the partition (ann_nlist)");
            st = dd_search_ann_motion(ds, y_dev, m, o.f_d, nullptr, prev_dev, &mot, o.ann_budget, out, pst, s, o.eq14);
        } else {
            st = dd_search_knng(ds, y_dev, m, o.f_s, prev_dev, &mot, out, pst, s);
        }
    } else if (o.mode == DD_SEARCH_ANN) {
        if (!ds->ann.nlist) return dd_fail(ctx, DD_ERR_STATE, "ANN search needs the partition (ann_nlist)");
        st = dd_search_ann_motion(ds, y_dev, m, o.f_d, nullptr, prev_dev, nullptr, o.ann_budget, out, pst, s, o.eq14);
    } else if (o.mode == DD_SEARCH_EXACT_TC) {
        if (!ds->z16hi) return dd_fail(ctx, DD_ERR_STATE, "tensor-core search needs the FP16 copy (build_fp16)");
        st = dd_search_exact_tc(ds, y_dev, m, o.certify, out, pst, s, o.tc_terms);
    } else {
        st = dd_run_search(ds, o.mode, o.certify, o.f_d, o.f_s, o.ann_budget, prev_dev, y_dev, m, out, pst, s);
    }
    if (st != DD_OK) return st;
    if (k == 1) {
        DD_TRY_CUDA(ctx, cudaMemcpyAsync(tk_dev, idx_dev, (size_t)m * 4, cudaMemcpyDeviceToDevice, s));
        DD_TRY_CUDA(ctx, cudaMemcpyAsync(tkd_dev, d2_dev, (size_t)m * 8, cudaMemcpyDeviceToDevice, s));
    }
    if (stats) {
        DD_TRY_CUDA(ctx, cudaEventRecord(e1, s));
        DD_TRY_CUDA(ctx, cudaEventSynchronize(e1));
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        local.ms = ms;
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        *stats = local;
    }
    if (!dev) {
        DD_TRY_CUDA(ctx, cudaMemcpyAsync(idx, idx_dev, (size_t)m * 4, cudaMemcpyDeviceToHost, s));
        if (d2) DD_TRY_CUDA(ctx, cudaMemcpyAsync(d2, d2_dev, (size_t)m * 8, cudaMemcpyDeviceToHost, s));
        if (o.d2nd) DD_TRY_CUDA(ctx, cudaMemcpyAsync(o.d2nd, d2nd_dev, (size_t)m * 8, cudaMemcpyDeviceToHost, s));
        if (topk_out)
            DD_TRY_CUDA(ctx, cudaMemcpyAsync(topk_out, tk_dev, (size_t)m * k * 4, cudaMemcpyDeviceToHost, s));
        if (o.topk_d2)
            DD_TRY_CUDA(ctx, cudaMemcpyAsync(o.topk_d2, tkd_dev, (size_t)m * k * 8, cudaMemcpyDeviceToHost, s));
        DD_TRY_CUDA(ctx, cudaStreamSynchronize(s));
    }
    if (!dev || stats) DD_TRY(dd_check_device_error(ctx, s, "dd_project_nearest"));
    return DD_OK;
}

