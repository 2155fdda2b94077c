"""Thin ctypes binding of libdd (include/dd.h).

Argument marshalling only: every step of the DD path runs in the CUDA
library.  Functions keep the C names; arrays may be numpy arrays (host memory)
or torch CUDA tensors (device memory), passed as raw pointers.  There is no
fallback: if libdd.so is missing or a call fails, an exception is raised.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_char_p, c_double, c_int, c_int32, c_int64, c_size_t, c_uint64, c_void_p

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdd.so")

DD_OK, DD_ERR_ARG, DD_ERR_NOT_SPD, DD_ERR_OOM, DD_ERR_CUDA, DD_ERR_TIMEOUT, DD_ERR_NOT_CONVERGED, DD_ERR_STATE = range(8)
STATUS_NAMES = ["DD_OK", "DD_ERR_ARG", "DD_ERR_NOT_SPD", "DD_ERR_OOM", "DD_ERR_CUDA", "DD_ERR_TIMEOUT",
                "DD_ERR_NOT_CONVERGED", "DD_ERR_STATE"]
DD_SEARCH_EXACT_FP32, DD_SEARCH_EXACT_TC, DD_SEARCH_ANN, DD_SEARCH_KNNG = 0, 1, 2, 3

# Entry points declared in include/dd.h (checked by the tests).
EXPORTS = [
    "dd_create", "dd_destroy", "dd_last_error", "dd_bytes_in_use", "dd_load_dataset", "dd_free_dataset",
    "dd_dataset_size", "dd_dataset_bytes", "dd_synth_dataset", "dd_project_nearest", "dd_solve",
    "dd_result_free", "dd_solver_create", "dd_solver_step", "dd_solver_done", "dd_solver_result",
    "dd_solver_free", "dd_launch_count", "dd_dataset_ann_nlist", "dd_dataset_ann_index",
    "dd_dataset_ann_cells", "dd_dataset_ann_build_fallback", "dd_dataset_knn_k", "dd_dataset_knn_graph", "dd_pca_metric",
    "dd_project_nearest_noalloc", "dd_solvers_step", "dd_solve_batch", "dd_server_start", "dd_server_submit",
    "dd_server_poll", "dd_server_get_stats", "dd_server_stop",
]
DD_NOALLOC_MAX_QUERIES = 65536
DD_TOPK_MAX = 8


class DDError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 8 else status}: {msg}")
        self.status = status


class dd_dataset_opts(ctypes.Structure):
    _fields_ = [("build_fp16", c_int), ("ann_nlist", c_int), ("ann_train_iters", c_int),
                ("ann_sample", c_int64), ("seed", c_uint64), ("borrow", c_int), ("ann_levels", c_int),
                ("knn_k", c_int), ("knn_fd", c_double), ("ann_alu", c_int)]


class dd_search_opts(ctypes.Structure):
    _fields_ = [("mode", c_int), ("certify", c_int), ("f_d", c_double), ("prev_idx", c_void_p),
                ("stream", c_void_p), ("f_s", c_int), ("ann_budget", c_int), ("topk", c_int),
                ("topk_d2", c_void_p), ("d2nd", c_void_p), ("prev_y", c_void_p), ("prev_d2", c_void_p),
                ("prev_d2nd", c_void_p), ("eq14", c_int), ("tc_terms", c_int)]


class dd_search_stats(ctypes.Structure):
    _fields_ = [("uncertified", c_int64), ("distances", c_int64), ("skipped", c_int64), ("ms", c_double),
                ("scan_ms", c_double), ("points", c_int64), ("unique_points", c_int64),
                ("moves", c_int64)]


class dd_iter_info(ctypes.Structure):
    _fields_ = [("iter", c_int), ("changed", c_int64), ("d2_pc", c_double), ("d2_pd", c_double),
                ("cg_iters", c_int), ("cg_ms", c_double), ("search_ms", c_double), ("other_ms", c_double),
                ("scan_ms", c_double), ("uncertified", c_int64), ("distances", c_int64), ("f_d", c_double),
                ("done", c_int), ("skipped", c_int64), ("points", c_int64), ("unique_points", c_int64),
                ("graph", c_int), ("moves", c_int64)]


class dd_mesh(ctypes.Structure):
    _fields_ = [("nx", c_int), ("ny", c_int), ("nz", c_int), ("lx", c_double), ("ly", c_double),
                ("lz", c_double)]


class dd_load(ctypes.Structure):
    _fields_ = [("t0", c_double * 3), ("tx", c_double * 3), ("ty", c_double * 3), ("rot_z", c_double)]


def _load(L) -> dd_load:
    """dd_load of a dd_inputs.Load (traction field or prescribed top rotation)."""
    return dd_load((c_double * 3)(*L.t0), (c_double * 3)(*L.tx), (c_double * 3)(*L.ty),
                   float(getattr(L, "rot_z", 0.0)))


class dd_solve_opts(ctypes.Structure):
    _fields_ = [("mode", c_int), ("certify", c_int), ("f_d0", c_double), ("f_d_final", c_double),
                ("ramp_iters", c_int), ("max_iter", c_int), ("cg_rtol", c_double), ("cg_max_iter", c_int),
                ("seed", c_uint64), ("init_idx", c_void_p), ("stall_iters", c_int), ("cg_mode", c_int),
                ("f_s", c_int), ("ann_budget", c_int), ("fd_rule", c_int), ("fd_tau", c_double),
                ("eq14", c_int)]


class dd_server_opts(ctypes.Structure):
    _fields_ = [("solve", dd_solve_opts), ("state_budget", c_size_t), ("max_batch", c_int)]


class dd_server_stats(ctypes.Structure):
    _fields_ = [("submitted", c_int64), ("completed", c_int64), ("active", c_int64), ("pending", c_int64),
                ("steps", c_int64), ("max_active", c_int64), ("busy_ms", c_double), ("cg_ms", c_double),
                ("search_ms", c_double), ("other_ms", c_double), ("graph_steps", c_int64)]


class dd_result(ctypes.Structure):
    _fields_ = [("n_nodes", c_int64), ("n_gp", c_int64), ("iters", c_int), ("converged", c_int),
                ("u", POINTER(c_double)), ("eta", POINTER(c_double)), ("eps", POINTER(c_double)),
                ("sig", POINTER(c_double)), ("idx", POINTER(c_int32)), ("d2_pc", POINTER(c_double)),
                ("d2_pd", POINTER(c_double)), ("changed", POINTER(c_int64)), ("cg_iters", POINTER(c_int)),
                ("search_ms", c_double), ("cg_ms", c_double), ("other_ms", c_double),
                ("uncertified", c_int64), ("distances", c_int64)]


_lib = None


def lib():
    """The loaded libdd (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libdd.so not built ({LIB_PATH}); run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        vp = c_void_p
        L.dd_create.argtypes = [c_int, c_size_t, POINTER(vp)]
        L.dd_destroy.argtypes = [vp]
        L.dd_destroy.restype = None
        L.dd_last_error.argtypes = [vp]
        L.dd_last_error.restype = c_char_p
        L.dd_bytes_in_use.argtypes = [vp]
        L.dd_bytes_in_use.restype = c_size_t
        L.dd_load_dataset.argtypes = [vp, vp, c_int64, POINTER(c_double), POINTER(dd_dataset_opts), POINTER(vp)]
        L.dd_free_dataset.argtypes = [vp]
        L.dd_free_dataset.restype = None
        L.dd_dataset_size.argtypes = [vp]
        L.dd_dataset_size.restype = c_int64
        L.dd_dataset_bytes.argtypes = [vp]
        L.dd_dataset_bytes.restype = c_size_t
        L.dd_synth_dataset.argtypes = [vp, c_int, c_double, c_double, c_double, c_double, POINTER(c_double),
                                       c_uint64, c_int64, c_int64, vp, vp]
        L.dd_project_nearest.argtypes = [vp, vp, c_int64, POINTER(dd_search_opts), vp, vp, vp,
                                         POINTER(dd_search_stats)]
        L.dd_solve.argtypes = [vp, POINTER(dd_mesh), POINTER(dd_load), POINTER(dd_solve_opts), POINTER(dd_result)]
        L.dd_result_free.argtypes = [POINTER(dd_result)]
        L.dd_result_free.restype = None
        L.dd_solver_create.argtypes = [vp, POINTER(dd_mesh), POINTER(dd_load), POINTER(dd_solve_opts), POINTER(vp)]
        L.dd_solver_step.argtypes = [vp, POINTER(dd_iter_info)]
        L.dd_solver_done.argtypes = [vp]
        L.dd_solver_done.restype = c_int
        L.dd_solver_result.argtypes = [vp, POINTER(dd_result)]
        L.dd_solver_free.argtypes = [vp]
        L.dd_solver_free.restype = None
        L.dd_launch_count.argtypes = [vp]
        L.dd_launch_count.restype = c_int64
        L.dd_dataset_ann_nlist.argtypes = [vp]
        L.dd_dataset_ann_nlist.restype = c_int
        L.dd_dataset_ann_index.argtypes = [vp, vp, vp, vp]
        L.dd_dataset_ann_cells.argtypes = [vp, POINTER(c_int32), POINTER(c_int32), vp, vp]
        L.dd_dataset_ann_build_fallback.argtypes = [vp]
        L.dd_dataset_ann_build_fallback.restype = c_int64
        L.dd_dataset_knn_k.argtypes = [vp]
        L.dd_dataset_knn_k.restype = c_int
        L.dd_dataset_knn_graph.argtypes = [vp, vp]
        L.dd_pca_metric.argtypes = [vp, vp, c_int64, POINTER(c_double)]
        L.dd_project_nearest_noalloc.argtypes = [vp, vp, c_int64, vp, vp, vp, c_int]
        L.dd_solvers_step.argtypes = [POINTER(vp), c_int, POINTER(dd_iter_info)]
        L.dd_server_start.argtypes = [vp, POINTER(dd_server_opts), POINTER(vp)]
        L.dd_server_submit.argtypes = [vp, POINTER(dd_mesh), POINTER(dd_load), c_uint64, POINTER(c_int64)]
        L.dd_server_poll.argtypes = [vp, c_int64, c_double, POINTER(dd_result), POINTER(c_double)]
        L.dd_server_get_stats.argtypes = [vp, POINTER(dd_server_stats)]
        L.dd_server_stop.argtypes = [vp]
        L.dd_solve_batch.argtypes = [vp, c_int, POINTER(dd_mesh), POINTER(dd_load), POINTER(dd_solve_opts),
                                     POINTER(dd_result)]
        for name in EXPORTS:
            getattr(L, name)
        _lib = L
    return _lib


def _ptr(a) -> int | None:
    """Raw pointer of a numpy array or torch tensor (None passes NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"], "array must be C-contiguous"
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        assert a.is_contiguous(), "tensor must be contiguous"
        return a.data_ptr()
    raise TypeError(type(a))


def _check(ctx, st: int):
    if st != DD_OK:
        msg = lib().dd_last_error(ctx)
        raise DDError(st, msg.decode() if msg else "")


def _Cmat(C) -> ctypes.Array:
    C = np.ascontiguousarray(C, dtype=np.float64).reshape(36)
    return (c_double * 36)(*C.tolist())


# ---------------------------------------------------------------------------
# Same names as the C ABI
# ---------------------------------------------------------------------------
def dd_create(device: int = 0, hbm_budget: int = 0):
    ctx = c_void_p()
    _check(None, lib().dd_create(device, hbm_budget, ctypes.byref(ctx)))
    return ctx


def dd_destroy(ctx) -> None:
    lib().dd_destroy(ctx)


def dd_last_error(ctx) -> str:
    m = lib().dd_last_error(ctx)
    return m.decode() if m else ""


def dd_bytes_in_use(ctx) -> int:
    return int(lib().dd_bytes_in_use(ctx))


def dd_load_dataset(ctx, eps_sig, C, build_fp16: bool = False, ann_nlist: int = 0, ann_train_iters: int = 0,
                    ann_sample: int = 0, seed: int = 0, borrow: bool = False, ann_levels: int = 1,
                    knn_k: int = 0, knn_fd: float = 0.6, ann_alu: bool = False):
    N = int(eps_sig.shape[0])
    assert tuple(eps_sig.shape[1:]) == (12,)
    opts = dd_dataset_opts(int(build_fp16), int(ann_nlist), int(ann_train_iters), int(ann_sample), int(seed),
                           int(borrow), int(ann_levels), int(knn_k), float(knn_fd), int(ann_alu))
    ds = c_void_p()
    _check(ctx, lib().dd_load_dataset(ctx, _ptr(eps_sig), N, _Cmat(C), ctypes.byref(opts), ctypes.byref(ds)))
    return ds


def dd_free_dataset(ds) -> None:
    lib().dd_free_dataset(ds)


def dd_dataset_size(ds) -> int:
    return int(lib().dd_dataset_size(ds))


def dd_dataset_bytes(ds) -> int:
    return int(lib().dd_dataset_bytes(ds))


def dd_synth_dataset(ctx, out_dev, law, C, seed: int = 0, start: int = 0, stream=None) -> None:
    """law: a dd_inputs.DataLaw; out_dev: torch float32 CUDA tensor [N, 12]."""
    N = int(out_dev.shape[0])
    _check(ctx, lib().dd_synth_dataset(ctx, law.code, law.eps_lo, law.eps_hi, law.noise_std, law.beta, _Cmat(C),
                                       int(seed), int(start), N, _ptr(out_dev), stream))


def dd_project_nearest(ds, ctx, y, idx, d2=None, mode: int = DD_SEARCH_EXACT_FP32, certify: bool = True,
                       f_d: float = 0.0, prev_idx=None, stream=None, want_stats: bool = True, f_s: int = 0,
                       ann_budget: int = 0, topk_out=None, topk_d2=None, d2nd=None, prev_y=None, prev_d2=None,
                       prev_d2nd=None, eq14: int = 0, tc_terms: int = 0):
    """topk_out: [m x k] int32 array (its second dimension gives k); the
    other optional arrays as in dd_search_opts."""
    m = int(y.shape[0])
    k = int(topk_out.shape[1]) if topk_out is not None else 0
    opts = dd_search_opts(int(mode), int(certify), float(f_d), _ptr(prev_idx), stream, int(f_s), int(ann_budget),
                          k, _ptr(topk_d2), _ptr(d2nd), _ptr(prev_y), _ptr(prev_d2), _ptr(prev_d2nd), int(eq14), int(tc_terms))
    st = dd_search_stats()
    _check(ctx, lib().dd_project_nearest(ds, _ptr(y), m, ctypes.byref(opts), _ptr(idx), _ptr(d2), _ptr(topk_out),
                                         ctypes.byref(st) if want_stats else None))
    return st


class Result:
    """Host copy of a dd_result."""

    def __init__(self, r: dd_result):
        nn, ng, it = r.n_nodes, r.n_gp, r.iters
        arr = np.ctypeslib.as_array
        self.n_nodes, self.n_gp, self.iters, self.converged = nn, ng, it, bool(r.converged)
        self.u = arr(r.u, shape=(nn * 3,)).copy()
        self.eta = arr(r.eta, shape=(nn * 3,)).copy()
        self.eps = arr(r.eps, shape=(ng, 6)).copy()
        self.sig = arr(r.sig, shape=(ng, 6)).copy()
        self.idx = arr(r.idx, shape=(ng,)).copy()
        self.d2_pc = arr(r.d2_pc, shape=(max(it, 1),))[:it].copy()
        self.d2_pd = arr(r.d2_pd, shape=(max(it, 1),))[:it].copy()
        self.changed = arr(r.changed, shape=(max(it, 1),))[:it].copy()
        self.cg_iters = arr(r.cg_iters, shape=(max(it, 1),))[:it].copy()
        self.search_ms, self.cg_ms, self.other_ms = r.search_ms, r.cg_ms, r.other_ms
        self.uncertified, self.distances = r.uncertified, r.distances


def dd_solve(ds, ctx, n_el, load, mode: int = DD_SEARCH_EXACT_FP32, init_idx=None, max_iter: int = 100,
             cg_rtol: float = 1e-12, cg_max_iter: int = 20000, certify: bool = True, f_d0: float = 0.0,
             f_d_final: float = 0.0, ramp_iters: int = 20, seed: int = 0, stall_iters: int = 3,
             lengths=(1.0, 1.0, 1.0), allow_not_converged: bool = True, cg_mode: int = 0, f_s: int = 0,
             ann_budget: int = 0, fd_rule: int = 0, fd_tau: float = 0.0, eq14: int = 0):
    """Solve one cube problem; `load` is a dd_inputs.Load.  Returns a Result."""
    nx, ny, nz = (n_el, n_el, n_el) if np.isscalar(n_el) else n_el
    mesh = dd_mesh(nx, ny, nz, *lengths)
    L = _load(load)
    ii = None if init_idx is None else np.ascontiguousarray(init_idx, dtype=np.int32)
    opts = dd_solve_opts(int(mode), int(certify), float(f_d0), float(f_d_final), int(ramp_iters), int(max_iter),
                         float(cg_rtol), int(cg_max_iter), int(seed), _ptr(ii), int(stall_iters), int(cg_mode),
                         int(f_s), int(ann_budget), int(fd_rule), float(fd_tau), int(eq14))
    r = dd_result()
    st = lib().dd_solve(ds, ctypes.byref(mesh), ctypes.byref(L), ctypes.byref(opts), ctypes.byref(r))
    try:
        if st != DD_OK and not (allow_not_converged and st == DD_ERR_NOT_CONVERGED):
            _check(ctx, st)
        return Result(r)
    finally:
        lib().dd_result_free(ctypes.byref(r))


def dd_result_free(r: dd_result) -> None:
    """Release the library-allocated arrays of a raw dd_result (dd_solve's
    wrapper above already copies and frees them)."""
    lib().dd_result_free(ctypes.byref(r))


def _solve_args(n_el, load, mode, init_idx, max_iter, cg_rtol, cg_max_iter, certify, f_d0, f_d_final, ramp_iters,
                seed, stall_iters, lengths, cg_mode=0, f_s=0, ann_budget=0, fd_rule=0, fd_tau=0.0, eq14=0):
    nx, ny, nz = (n_el, n_el, n_el) if np.isscalar(n_el) else n_el
    mesh = dd_mesh(nx, ny, nz, *lengths)
    L = _load(load)
    ii = None if init_idx is None else np.ascontiguousarray(init_idx, dtype=np.int32)
    opts = dd_solve_opts(int(mode), int(certify), float(f_d0), float(f_d_final), int(ramp_iters), int(max_iter),
                         float(cg_rtol), int(cg_max_iter), int(seed), _ptr(ii), int(stall_iters), int(cg_mode),
                         int(f_s), int(ann_budget), int(fd_rule), float(fd_tau), int(eq14))
    return mesh, L, opts, ii


def dd_solver_create(ds, ctx, n_el, load, mode: int = DD_SEARCH_EXACT_FP32, init_idx=None, max_iter: int = 100,
                     cg_rtol: float = 1e-12, cg_max_iter: int = 20000, certify: bool = True, f_d0: float = 0.0,
                     f_d_final: float = 0.0, ramp_iters: int = 20, seed: int = 0, stall_iters: int = 3,
                     lengths=(1.0, 1.0, 1.0), cg_mode: int = 0, f_s: int = 0, ann_budget: int = 0,
                     fd_rule: int = 0, fd_tau: float = 0.0, eq14: int = 0):
    mesh, L, opts, ii = _solve_args(n_el, load, mode, init_idx, max_iter, cg_rtol, cg_max_iter, certify, f_d0,
                                    f_d_final, ramp_iters, seed, stall_iters, lengths, cg_mode, f_s, ann_budget,
                                    fd_rule, fd_tau, eq14)
    sv = c_void_p()
    _check(ctx, lib().dd_solver_create(ds, ctypes.byref(mesh), ctypes.byref(L), ctypes.byref(opts),
                                       ctypes.byref(sv)))
    return sv


def dd_solver_step(sv, ctx) -> dd_iter_info:
    info = dd_iter_info()
    _check(ctx, lib().dd_solver_step(sv, ctypes.byref(info)))
    return info


def dd_solver_done(sv) -> bool:
    return bool(lib().dd_solver_done(sv))


def dd_solver_result(sv, ctx) -> Result:
    r = dd_result()
    try:
        _check(ctx, lib().dd_solver_result(sv, ctypes.byref(r)))
        return Result(r)
    finally:
        lib().dd_result_free(ctypes.byref(r))


def dd_solver_free(sv) -> None:
    lib().dd_solver_free(sv)


def dd_launch_count(ctx) -> int:
    return int(lib().dd_launch_count(ctx))


def dd_dataset_ann_nlist(ds) -> int:
    return int(lib().dd_dataset_ann_nlist(ds))


def dd_dataset_ann_index(ds, ctx):
    """Host copy of the k-means partition: (cluster_of [N], centroids [L,12], radii [L])."""
    L = dd_dataset_ann_nlist(ds)
    N = dd_dataset_size(ds)
    cl = np.empty(N, np.int32)
    cent = np.empty((L, 12), np.float64)
    rad = np.empty(L, np.float64)
    _check(ctx, lib().dd_dataset_ann_index(ds, _ptr(cl), _ptr(cent), _ptr(rad)))
    return cl, cent, rad


def dd_dataset_ann_cells(ds, ctx):
    """Host copy of the cell level of a two-level partition: (L2, centroids
    [L1,12], radii [L1]); leaf l of dd_dataset_ann_index lies in cell l // L2."""
    L1, L2 = c_int32(0), c_int32(0)
    _check(ctx, lib().dd_dataset_ann_cells(ds, ctypes.byref(L1), ctypes.byref(L2), None, None))
    cent = np.empty((L1.value, 12), np.float64)
    rad = np.empty(L1.value, np.float64)
    _check(ctx, lib().dd_dataset_ann_cells(ds, None, None, _ptr(cent), _ptr(rad)))
    return L2.value, cent, rad


def dd_dataset_ann_build_fallback(ds) -> int:
    """Build rows the tensor-core nearest-centroid passes left to the ALU."""
    return int(lib().dd_dataset_ann_build_fallback(ds))


def dd_pca_metric(ctx, eps_sig) -> np.ndarray:
    """Data-derived metric (Sec. 3.1) of float32 [N, 12] data (numpy array or
    CUDA tensor): C = sym(A_sig A_eps^{-1}) of the six principal components."""
    out = (c_double * 36)()
    _check(ctx, lib().dd_pca_metric(ctx, _ptr(eps_sig), int(eps_sig.shape[0]), out))
    return np.array(out[:]).reshape(6, 6)


def dd_dataset_knn_k(ds) -> int:
    return int(lib().dd_dataset_knn_k(ds))


def dd_dataset_knn_graph(ds, ctx):
    """Host copy of the k-nearest-neighbour graph: int32 [N, k] data indices,
    nearest first, -1 where fewer than k neighbours were found."""
    k = dd_dataset_knn_k(ds)
    nbr = np.empty((dd_dataset_size(ds), k), np.int32)
    _check(ctx, lib().dd_dataset_knn_graph(ds, _ptr(nbr)))
    return nbr


def dd_project_nearest_noalloc(ds, ctx, y_dev, idx_dev, d2_dev, stream=None, wait: bool = False) -> None:
    """Exact projection that allocates no device memory (device buffers only;
    asynchronous on `stream` unless wait).  For callers that cannot allocate
    during a call, e.g. a loop whose device memory is reserved by another
    allocator.  wait=True synchronises and reports a device-side timeout."""
    _check(ctx, lib().dd_project_nearest_noalloc(ds, _ptr(y_dev), int(y_dev.shape[0]), _ptr(idx_dev),
                                                 _ptr(d2_dev), stream, int(bool(wait))))


def dd_solvers_step(svs, ctx):
    """One iteration of several solvers at once; returns their dd_iter_info."""
    n = len(svs)
    arr = (c_void_p * n)(*[sv.value for sv in svs])
    infos = (dd_iter_info * n)()
    _check(ctx, lib().dd_solvers_step(arr, n, infos))
    return list(infos)


def dd_solve_batch(ds, ctx, n_els, loads, mode: int = DD_SEARCH_EXACT_FP32, init_idx=None, max_iter: int = 100,
                   cg_rtol: float = 1e-12, cg_max_iter: int = 20000, certify: bool = True, f_d0: float = 0.0,
                   f_d_final: float = 0.0, ramp_iters: int = 20, seed: int = 0, stall_iters: int = 3,
                   cg_mode: int = 0, allow_not_converged: bool = True, f_s: int = 0, ann_budget: int = 0,
                   fd_rule: int = 0, fd_tau: float = 0.0, eq14: int = 0):
    """Solve several cube problems together; n_els[i] edge elements, loads[i]."""
    n = len(n_els)
    meshes = (dd_mesh * n)(*[dd_mesh(k, k, k, 1.0, 1.0, 1.0) for k in n_els])
    Ls = (dd_load * n)(*[_load(L)
                         for L in loads])
    _, _, opts, ii = _solve_args(n_els[0], loads[0], mode, init_idx, max_iter, cg_rtol, cg_max_iter, certify, f_d0,
                                 f_d_final, ramp_iters, seed, stall_iters, (1.0, 1.0, 1.0), cg_mode, f_s,
                                 ann_budget, fd_rule, fd_tau, eq14)
    outs = (dd_result * n)()
    st = lib().dd_solve_batch(ds, n, meshes, Ls, ctypes.byref(opts), outs)
    try:
        if st != DD_OK and not (allow_not_converged and st == DD_ERR_NOT_CONVERGED):
            _check(ctx, st)
        return [Result(r) for r in outs]
    finally:
        for r in outs:
            lib().dd_result_free(ctypes.byref(r))


def dd_server_start(ds, ctx, mode: int = DD_SEARCH_EXACT_FP32, state_budget: int = 0, max_batch: int = 0,
                    max_iter: int = 100, cg_rtol: float = 1e-12, cg_max_iter: int = 20000, certify: bool = True,
                    f_d0: float = 0.0, f_d_final: float = 0.0, ramp_iters: int = 20, stall_iters: int = 3,
                    cg_mode: int = 0, f_s: int = 0, ann_budget: int = 0, fd_rule: int = 0, fd_tau: float = 0.0,
                    eq14: int = 0):
    so = dd_solve_opts(int(mode), int(certify), float(f_d0), float(f_d_final), int(ramp_iters), int(max_iter),
                       float(cg_rtol), int(cg_max_iter), 0, None, int(stall_iters), int(cg_mode), int(f_s),
                       int(ann_budget), int(fd_rule), float(fd_tau), int(eq14))
    o = dd_server_opts(so, int(state_budget), int(max_batch))
    srv = c_void_p()
    _check(ctx, lib().dd_server_start(ds, ctypes.byref(o), ctypes.byref(srv)))
    return srv


def dd_server_submit(srv, n_el, load, seed: int = 0, lengths=(1.0, 1.0, 1.0)) -> int:
    nx, ny, nz = (n_el, n_el, n_el) if np.isscalar(n_el) else n_el
    mesh = dd_mesh(nx, ny, nz, *lengths)
    L = _load(load)
    t = c_int64()
    st = lib().dd_server_submit(srv, ctypes.byref(mesh), ctypes.byref(L), int(seed), ctypes.byref(t))
    if st != DD_OK:
        raise DDError(st, "dd_server_submit")
    return int(t.value)


def dd_server_poll(srv, ctx, ticket: int, timeout_s: float = 0.0):
    """(Result, latency_ms) once finished; None if not finished yet."""
    r = dd_result()
    lat = c_double()
    st = lib().dd_server_poll(srv, int(ticket), float(timeout_s), ctypes.byref(r), ctypes.byref(lat))
    if st == DD_ERR_TIMEOUT:
        return None
    try:
        if st not in (DD_OK, DD_ERR_NOT_CONVERGED):
            raise DDError(st, f"served request {ticket} failed")
        return Result(r), float(lat.value)
    finally:
        lib().dd_result_free(ctypes.byref(r))


def dd_server_get_stats(srv) -> dd_server_stats:
    s = dd_server_stats()
    lib().dd_server_get_stats(srv, ctypes.byref(s))
    return s


def dd_server_stop(srv) -> None:
    lib().dd_server_stop(srv)
