"""Pins of the oracle's brute-force nearest-neighbour projection (Eq. 7)."""
import numpy as np

import dd_inputs as I
from oracle import metric as M
from oracle import nn


def test_hand_case_on_a_line():
    zd = np.zeros((4, 12)); zd[:, 0] = [0.0, 1.0, 2.0, 3.0]
    zq = np.zeros((2, 12)); zq[0, 0] = 1.4; zq[1, 0] = -5.0
    i1, d1, i2, d2 = nn.nn_top2(zd, zq)
    assert i1.tolist() == [1, 0] and i2.tolist() == [2, 1]
    assert np.allclose(d1, [0.16, 25.0]) and np.allclose(d2, [0.36, 36.0])


def test_planted_queries_and_ties():
    rng = np.random.default_rng(2)
    zd = rng.standard_normal((300, 12))
    zd[250] = zd[17]                      # duplicate: lowest index must win
    i1, d1, i2, d2 = nn.nn_top2(zd, zd[[5, 17, 250, 299]])
    assert i1.tolist() == [5, 17, 17, 299]
    assert np.all(d1 == 0.0)
    assert i2[1] == 250 and d2[1] == 0.0


def test_matches_exhaustive_eq3_in_state_space():
    """Brute force over Eq. (3) itself, in (eps, sig) space, pure Python."""
    law = I.LINEAR
    C = I.isotropic_C()
    data = I.make_dataset(400, law, seed=11).astype(np.float64)
    ys = I.make_states(40, law, seed=12, spread=0.3)
    i1, d1, _, _ = nn.nn_top2(M.to_z(data, C), M.to_z(ys, C))
    for q in range(len(ys)):
        best, bj = np.inf, -1
        for j in range(len(data)):
            d = M.local_d2(ys[q:q + 1], data[j:j + 1], C)[0]
            if d < best:
                best, bj = d, j
        assert np.isclose(2 * d1[q], best, rtol=1e-10)
        if bj != i1[q]:   # only a numerical tie may differ
            dj = M.local_d2(ys[q:q + 1], data[i1[q]:i1[q] + 1], C)[0]
            assert abs(dj - best) <= 1e-12 * best


def test_min_and_second_min_property():
    rng = np.random.default_rng(3)
    zd = rng.standard_normal((3000, 12))
    zq = rng.standard_normal((64, 12)) * 1.5
    i1, d1, i2, d2 = nn.nn_top2(zd, zq)
    full = ((zq[:, None, :] - zd[None, :, :]) ** 2).sum(-1)
    s = np.sort(full, axis=1)
    assert np.allclose(d1, s[:, 0], rtol=1e-13) and np.allclose(d2, s[:, 1], rtol=1e-13)
    assert np.array_equal(i1, full.argmin(1))


def test_streaming_scan_equals_in_memory_scan():
    """The chunked scan over generated data equals the in-memory scan."""
    law = I.NONLINEAR
    C = I.isotropic_C()
    N = (1 << 20) + 4321                    # more than one chunk, ragged tail
    data = I.make_dataset(N, law, seed=6)
    zq = M.to_z(I.make_states(24, law, seed=7, spread=0.1), C)
    i1, d1, _, _ = nn.nn_top2(M.to_z(data, C), zq)
    j1, e1 = nn.nn_stream(law, 6, N, C, zq)
    assert np.array_equal(i1, j1) and np.allclose(d1, e1, rtol=1e-12)


def test_topk_by_hand_and_against_top2():
    zd = np.zeros((5, 12)); zd[:, 0] = [0.0, 1.0, 2.0, 3.0, 1.0]
    zq = np.zeros((1, 12)); zq[0, 0] = 1.4
    i, d = nn.nn_topk(zd, zq, 4)
    # distances 1.96, 0.16, 0.36, 2.56, 0.16: the tie 1 / 4 goes to the lower index
    assert i.tolist() == [[1, 4, 2, 0]] and np.allclose(d, [[0.16, 0.16, 0.36, 1.96]])
    i, d = nn.nn_topk(zd[:2], zq, 4)          # fewer points than k: padded
    assert i.tolist() == [[1, 0, -1, -1]] and np.isinf(d[0, 2:]).all()
    C = I.isotropic_C()
    data = I.make_dataset(3000, I.NONLINEAR, seed=4).astype(np.float64)
    Z, zq = M.to_z(data, C), M.to_z(I.make_states(300, I.NONLINEAR, seed=5, spread=0.2), C)
    i, d = nn.nn_topk(Z, zq, 6)
    i1, d1, i2, d2 = nn.nn_top2(Z, zq)
    assert np.array_equal(i[:, 0], i1) and np.array_equal(i[:, 1], i2)
    assert np.allclose(d[:, 0], d1, rtol=1e-12) and np.allclose(d[:, 1], d2, rtol=1e-12)
    assert np.all(np.diff(d, axis=1) >= 0)
    # every point left out is at least as far as the k-th
    for q in range(0, 300, 37):
        rest = np.setdiff1d(np.arange(len(Z)), i[q])
        assert (((Z[rest] - zq[q]) ** 2).sum(1) >= d[q, -1]).all()
