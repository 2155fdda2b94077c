"""ctypes front end of the oracle's brute-force nearest-neighbour scan (nn.c).

Exact P_D of Eq. (7): for each mapped query the data point with the smallest
squared Euclidean distance in the map of Sec. 3.2 (which equals d_e^2 / 2 of
Eq. 3).  TEST INFRASTRUCTURE ONLY.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_build", "liboracle_nn.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile nn.c with gcc (OpenMP, no FP contraction) into oracle/_build."""
    src = os.path.join(_HERE, "nn.c")
    gen_src = os.path.join(os.path.dirname(_HERE), "dd_inputs", "gen.c")
    newest = max(os.path.getmtime(src), os.path.getmtime(gen_src))
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < newest:
        os.makedirs(os.path.dirname(_SO), exist_ok=True)
        tmp = _SO + f".{os.getpid()}.tmp"
        gen = os.path.join(os.path.dirname(_HERE), "dd_inputs", "gen.c")
        subprocess.run(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
                        src, gen, "-o", tmp, "-lm"], check=True)
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int64)
            lib.oracle_nn_top2.argtypes = [dp, ctypes.c_int64, dp, ctypes.c_int64, ctypes.c_int,
                                           ip, dp, ip, dp]
            lib.oracle_nn_top2.restype = None
            lib.oracle_nn_threads.restype = ctypes.c_int
            vp = ctypes.c_void_p
            lib.oracle_nn_stream.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                             ctypes.c_double, vp, ctypes.c_uint64, ctypes.c_int64, vp, vp, vp,
                                             ctypes.c_int64, vp, vp]
            lib.oracle_nn_stream.restype = None
            _lib = lib
    return _lib


def threads() -> int:
    return int(_load().oracle_nn_threads())


def nn_top2(zd: np.ndarray, zq: np.ndarray):
    """Exact nearest and second-nearest data rows for every query row.

    Returns (i1, d1, i2, d2): int64 indices and float64 squared distances
    |z_j - q|^2 in the mapped coordinates.
    """
    lib = _load()
    zd = np.ascontiguousarray(zd, dtype=np.float64)
    zq = np.ascontiguousarray(zq, dtype=np.float64)
    n, dim = zd.shape
    m = zq.shape[0]
    assert zq.shape[1] == dim
    i1 = np.empty(m, np.int64)
    i2 = np.empty(m, np.int64)
    d1 = np.empty(m, np.float64)
    d2 = np.empty(m, np.float64)
    dp = ctypes.POINTER(ctypes.c_double)
    ip = ctypes.POINTER(ctypes.c_int64)
    lib.oracle_nn_top2(zd.ctypes.data_as(dp), n, zq.ctypes.data_as(dp), m, dim,
                       i1.ctypes.data_as(ip), d1.ctypes.data_as(dp),
                       i2.ctypes.data_as(ip), d2.ctypes.data_as(dp))
    return i1, d1, i2, d2


def nn_stream(law, seed: int, N: int, C, zq):
    """Exact nearest point of every mapped query over the seeded data set of
    N points (law: dd_inputs.DataLaw, generated chunk by chunk in C with the
    law's own stiffness), mapped with the metric C.
    Returns (index int64, squared mapped distance)."""
    from . import metric
    import dd_inputs
    lib = _load()
    C = np.ascontiguousarray(C, dtype=np.float64)
    Ch, Cmh = metric.metric_roots(C)
    C_law = np.ascontiguousarray(dd_inputs.isotropic_C(law.E, law.nu))
    Ch = np.ascontiguousarray(Ch)
    Cmh = np.ascontiguousarray(Cmh)
    zq = np.ascontiguousarray(zq, dtype=np.float64)
    m = len(zq)
    i1 = np.empty(m, np.int64)
    d1 = np.empty(m)
    lib.oracle_nn_stream(law.code, law.eps_lo, law.eps_hi, law.noise_std, law.beta, C_law.ctypes.data, seed, N,
                         Ch.ctypes.data, Cmh.ctypes.data, zq.ctypes.data, m, i1.ctypes.data, d1.ctypes.data)
    return i1, d1


def nn_topk(zd: np.ndarray, zq: np.ndarray, k: int, chunk: int = 256):
    """The k nearest data rows of every query row (Eq. 7 extended to the k
    best): indices int64 [m x k] and squared distances [m x k] in the mapped
    coordinates, nearest first, ties to the lower index; -1 and +inf past the
    N-th.  Plain numpy: full distance rows, then a stable sort."""
    zd = np.asarray(zd, dtype=np.float64)
    zq = np.asarray(zq, dtype=np.float64)
    n, m = len(zd), len(zq)
    idx = np.full((m, k), -1, np.int64)
    dist = np.full((m, k), np.inf)
    kk = min(k, n)
    for a in range(0, m, chunk):
        d = ((zq[a:a + chunk, None, :] - zd[None, :, :]) ** 2).sum(-1)
        order = np.argsort(d, axis=1, kind="stable")[:, :kk]    # stable: equal distances keep index order
        idx[a:a + chunk, :kk] = order
        dist[a:a + chunk, :kk] = np.take_along_axis(d, order, axis=1)
    return idx, dist
