"""Pins of the oracle's approximate search rules (Sec. 4.2-4.5, Eq. 13)."""
import numpy as np

import dd_inputs as I
from oracle import ann, metric, nn


def setup(N=3000, L=24, seed=0):
    C = I.isotropic_C()
    data = I.make_dataset(N, I.NONLINEAR, seed=seed).astype(np.float64)
    Z = metric.to_z(data, C)
    cent, rad, cl = ann.kmeans_partition(Z, L, seed=seed)
    y = I.make_states(80, I.NONLINEAR, seed=seed + 1, spread=0.3)
    return Z, metric.to_z(y, C), cent, rad, cl


def test_fd_one_is_exact():
    Z, zq, cent, rad, cl = setup()
    i, d = ann.ann_search(Z, zq, cent, rad, cl, f_d=1.0, n_cand=24)
    j, e, _, _ = nn.nn_top2(Z, zq)
    assert np.array_equal(i, j) and np.allclose(d, e)


def test_fd_one_exact_with_short_candidate_list():
    # the completeness test sends uncovered queries to the exhaustive search
    Z, zq, cent, rad, cl = setup()
    i, d = ann.ann_search(Z, zq, cent, rad, cl, f_d=1.0, n_cand=3)
    j, e, _, _ = nn.nn_top2(Z, zq)
    assert np.array_equal(i, j)


def test_warm_start_never_worse_and_fd_monotone_on_average():
    Z, zq, cent, rad, cl = setup(seed=3)
    prev = np.random.default_rng(0).integers(0, len(Z), len(zq))
    i0, d0 = ann.ann_search(Z, zq, cent, rad, cl, f_d=0.0, prev_idx=prev)
    dprev = ((Z[prev] - zq) ** 2).sum(1)
    assert np.all(d0 <= dprev)
    _, d4 = ann.ann_search(Z, zq, cent, rad, cl, f_d=0.6, prev_idx=prev)
    _, e, _, _ = nn.nn_top2(Z, zq)
    assert np.all(d4 <= d0) and np.all(e <= d4 * (1 + 1e-12))


def test_fd_zero_single_descent_on_separated_clusters():
    """Well separated clusters: f_d = 0 searches only the nearest-centroid
    cluster, whose best point is then the answer."""
    rng = np.random.default_rng(5)
    centres = rng.standard_normal((6, 12)) * 100
    Z = np.concatenate([c + rng.standard_normal((50, 12)) for c in centres])
    cl = np.repeat(np.arange(6), 50)
    cent = np.array([Z[cl == l].mean(0) for l in range(6)])
    rad = np.array([np.sqrt(((Z[cl == l] - cent[l]) ** 2).sum(1).max()) for l in range(6)])
    zq = centres[[1, 4]] + rng.standard_normal((2, 12)) * 3
    i, d = ann.ann_search(Z, zq, cent, rad, cl, f_d=0.0)
    for qi, q in enumerate(zq):
        l = int(np.argmin(((cent - q) ** 2).sum(1)))
        mem = np.nonzero(cl == l)[0]
        jj = mem[np.argmin(((Z[mem] - q) ** 2).sum(1))]
        assert i[qi] == jj
