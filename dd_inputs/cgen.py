"""ctypes front end of dd_inputs/gen.c (the C copy of the data-set generator)."""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

from . import DataLaw, isotropic_C

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_build", "libddinputs.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    src = os.path.join(_HERE, "gen.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        os.makedirs(os.path.dirname(_SO), exist_ok=True)
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.run(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared", src, "-o", tmp, "-lm"],
                       check=True)
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            L.ddi_make_dataset.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                           ctypes.c_double, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int64,
                                           ctypes.c_int64, ctypes.c_void_p]
            L.ddi_make_dataset.restype = None
            _lib = L
    return _lib


def make_dataset(N: int, law: DataLaw, seed: int = 0, start: int = 0) -> np.ndarray:
    """Same values as dd_inputs.make_dataset, generated in C."""
    out = np.empty((N, 12), np.float32)
    C = np.ascontiguousarray(isotropic_C(law.E, law.nu))
    _load().ddi_make_dataset(law.code, law.eps_lo, law.eps_hi, law.noise_std, law.beta, C.ctypes.data, seed,
                             start, N, out.ctypes.data)
    return out
