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


def setup2(N=2500, L1=6, L2=10, seed=0):
    C = I.isotropic_C()
    data = I.make_dataset(N, I.NONLINEAR, seed=seed).astype(np.float64)
    Z = metric.to_z(data, C)
    part = ann.tree2_partition(Z, L1, L2, seed=seed)
    y = I.make_states(60, I.NONLINEAR, seed=seed + 1, spread=0.3)
    return Z, metric.to_z(y, C), part


def test_tree2_partition_is_valid():
    Z, zq, (cc, cr, lc, lr, leaf) = setup2()
    L2 = 10
    assert leaf.min() >= 0 and leaf.max() < len(lc)
    for l in np.unique(leaf):
        m = leaf == l
        assert np.sqrt(((Z[m] - lc[l]) ** 2).sum(1)).max() <= lr[l] * (1 + 1e-12)
        assert np.sqrt(((Z[m] - cc[l // L2]) ** 2).sum(1)).max() <= cr[l // L2] * (1 + 1e-12)


def test_tree2_one_leaf_per_cell_is_the_flat_search():
    """With one leaf per cell (the leaf is the cell) the two-level rules are
    the flat rules of ann_search, answer for answer."""
    Z, zq, cent, rad, cl = setup(seed=2)
    prev = np.random.default_rng(1).integers(0, len(Z), len(zq))
    for f_d in (0.0, 0.4, 1.0):
        for pv in (None, prev):
            a = ann.ann_search(Z, zq, cent, rad, cl, f_d, prev_idx=pv, n_cand=8)
            b = ann.tree2_search(Z, zq, cent, rad, cent, rad, cl, 1, f_d, prev_idx=pv, n_cand=8)
            assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_tree2_fd_one_is_exact_with_short_lists():
    """f_d = 1 with 3 of 6 cells and 3 of 10 leaves per cell as candidates:
    the completeness tests send uncovered queries to the exhaustive search,
    so every answer is the brute-force nearest point."""
    Z, zq, (cc, cr, lc, lr, leaf) = setup2(seed=4)
    prev = np.random.default_rng(2).integers(0, len(Z), len(zq))
    j, e, _, _ = nn.nn_top2(Z, zq)
    for pv in (None, prev):
        i, d = ann.tree2_search(Z, zq, cc, cr, lc, lr, leaf, 10, 1.0, prev_idx=pv, n_cand=3, k_fine=3)
        assert np.array_equal(i, j) and np.allclose(d, e, rtol=1e-12, atol=0)


def test_tree2_fd_zero_is_the_descent():
    """f_d = 0 on well separated cells and leaves: only the nearest cell's
    nearest leaf is searched, whose best point is the answer; a warm start
    in another cell is kept only when it is nearer."""
    rng = np.random.default_rng(7)
    cells = rng.standard_normal((4, 12)) * 1000
    leaf_off = rng.standard_normal((3, 12)) * 50
    Z, leaf = [], []
    for c in range(4):
        for f in range(3):
            Z.append(cells[c] + leaf_off[f] + rng.standard_normal((20, 12)))
            leaf += [c * 3 + f] * 20
    Z = np.concatenate(Z)
    leaf = np.array(leaf)
    lc = np.array([Z[leaf == l].mean(0) for l in range(12)])
    lr = np.array([np.sqrt(((Z[leaf == l] - lc[l]) ** 2).sum(1).max()) for l in range(12)])
    cell_of = leaf // 3
    cc = np.array([Z[cell_of == c].mean(0) for c in range(4)])
    cr = np.array([np.sqrt(((Z[cell_of == c] - cc[c]) ** 2).sum(1).max()) for c in range(4)])
    zq = np.stack([cells[2] + leaf_off[1] + rng.standard_normal(12) * 2, cells[0] + leaf_off[2]])
    i, d = ann.tree2_search(Z, zq, cc, cr, lc, lr, leaf, 3, 0.0)
    for qi, l in enumerate((7, 2)):
        mem = np.nonzero(leaf == l)[0]
        assert i[qi] == mem[np.argmin(((Z[mem] - zq[qi]) ** 2).sum(1))]
    # a warm start far away (another cell) loses to the descent's leaf
    far = np.array([np.nonzero(leaf == 0)[0][0], np.nonzero(leaf == 11)[0][0]])
    i2, _ = ann.tree2_search(Z, zq, cc, cr, lc, lr, leaf, 3, 0.0, prev_idx=far)
    assert np.array_equal(i2, i)


def test_tree2_handoff_never_farther_and_exact():
    """A budget of leaves searched at once, the rest after: the chosen leaves
    only grow, so no answer is farther than with every leaf at once, and some
    are nearer; f_d = 1 stays exact."""
    Z, zq, (cc, cr, lc, lr, leaf) = setup2(seed=6)
    prev = np.random.default_rng(3).integers(0, len(Z), len(zq))
    j, e, _, _ = nn.nn_top2(Z, zq)
    nearer = 0
    for pv in (None, prev):
        for f_d in (0.0, 0.4):
            _, d_all = ann.tree2_search(Z, zq, cc, cr, lc, lr, leaf, 10, f_d, prev_idx=pv, n_cand=3, k_fine=3)
            for b in (0, 1, 2, 4):
                _, d_b = ann.tree2_search(Z, zq, cc, cr, lc, lr, leaf, 10, f_d, prev_idx=pv, n_cand=3, k_fine=3,
                                          budget=b)
                assert np.all(d_b <= d_all) and np.all(e <= d_b * (1 + 1e-12))
                nearer += int(np.sum(d_b < d_all))
        for b in (0, 1, 2):
            i, _ = ann.tree2_search(Z, zq, cc, cr, lc, lr, leaf, 10, 1.0, prev_idx=pv, n_cand=3, k_fine=3, budget=b)
            assert np.array_equal(i, j)
    assert nearer > 0
