"""Helpers shared by the GPU parity tests (comparison rules of the tests)."""
import numpy as np

from oracle import metric, nn


def oracle_nn(data, y, C):
    """FP64 oracle: nearest index, d_e^2 (Eq. 3) of it, and second-best d_e^2."""
    i1, d1, i2, d2 = nn.nn_top2(metric.to_z(data.astype(np.float64), C), metric.to_z(y, C))
    return i1, 2.0 * d1, 2.0 * d2


def assert_nn_parity(idx, d2, data, y, C, rel_gap=1e-6, rtol=1e-5):
    """Indices bit-exact where the FP64 gap between best and second best
    exceeds rel_gap (relative); elsewhere the GPU's point must be as near as
    the oracle's within rel_gap.  Distances within rtol relative."""
    i1, b1, b2 = oracle_nn(data, y, C)
    idx = np.asarray(idx).astype(np.int64)
    d2 = np.asarray(d2)
    gap_ok = (b2 - b1) > rel_gap * np.maximum(b1, 1e-300)
    bad = np.nonzero(gap_ok & (idx != i1))[0]
    assert bad.size == 0, f"{bad.size} indices differ where the gap is clear, e.g. q={bad[:5]} gpu={idx[bad[:5]]} oracle={i1[bad[:5]]}"
    amb = np.nonzero(~gap_ok & (idx != i1))[0]
    if amb.size:
        dg = metric.local_d2(y[amb], data[idx[amb]].astype(np.float64), C)
        assert np.all(dg <= b1[amb] * (1 + rel_gap) + 1e-300)
    assert np.allclose(d2, b1, rtol=rtol, atol=1e-300)
    return i1, b1
