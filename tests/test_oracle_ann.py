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


# ---------------------------------------------------------------------------
# Eq. (14): the moving-query skip and the second bound it needs
# ---------------------------------------------------------------------------
def moved(zq, scale, seed):
    """Queries displaced by random steps of plain length scale * U(0, 1)."""
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(zq.shape)
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return zq + v * (scale * rng.random((len(zq), 1)))


def test_second_bound_below_brute_force_second_at_fd_one():
    """At f_d = 1 the second bound never exceeds the distance of the
    brute-force second-nearest point (C scan), flat and two-level, with
    short candidate lists, warm and cold; and it is not vacuous."""
    Z, zq, cent, rad, cl = setup(seed=8)
    Z2, zq2, part = setup2(seed=9)
    prev = np.random.default_rng(6).integers(0, len(Z), len(zq))
    j, e, _, e2 = nn.nn_top2(Z, zq)
    j2, f, _, f2 = nn.nn_top2(Z2, zq2)
    tight = 0
    for pv in (None, prev):
        for n_cand in (3, 8, 24):
            i, d, s = ann.ann_search(Z, zq, cent, rad, cl, 1.0, prev_idx=pv, n_cand=n_cand, with_second=True)
            assert np.array_equal(i, j) and np.all(s <= e2 * (1 + 1e-12))
            tight += int(np.sum(s > d))
        i, d, s = ann.tree2_search(Z2, zq2, *part, 10, 1.0, prev_idx=None if pv is None else pv % len(Z2),
                                   n_cand=3, k_fine=3, with_second=True)
        assert np.array_equal(i, j2) and np.all(s <= f2 * (1 + 1e-12))
        tight += int(np.sum(s > d))
    assert tight > 0


def test_kept_answers_equal_brute_force_at_fd_one():
    """A search at f_d = 1, then the queries moved by steps around the Eq. (14)
    radius: every query the record keeps gets the brute-force nearest point of
    its new position, flat and two-level."""
    Z, zq, cent, rad, cl = setup(N=4000, L=16, seed=10)
    Z2, zq2, part = setup2(seed=11)
    kept = 0
    for k, (search, ZZ, qq) in enumerate((
            (lambda q, **kw: ann.ann_search(Z, q, cent, rad, cl, 1.0, n_cand=4, **kw), Z, zq),
            (lambda q, **kw: ann.tree2_search(Z2, q, *part, 10, 1.0, n_cand=3, k_fine=3, **kw), Z2, zq2))):
        i1, d1, s1 = search(qq, with_second=True)
        delta = 0.5 * (np.sqrt(s1) - np.sqrt(d1))
        for scale in (0.5, 1.0, 2.0):
            q2 = moved(qq, scale * np.median(delta), seed=20 + k)
            keep = np.array([ann.moving_query_keeps(q2[t], qq[t], d1[t], s1[t])[0] for t in range(len(qq))])
            i2, d2, s2 = search(q2, prev_idx=i1, motion=(qq, d1, s1, 1.0), with_second=True)
            j, e, _, e2 = nn.nn_top2(ZZ, q2)
            assert np.array_equal(i2, j)
            assert np.all(s2 <= e2 * (1 + 1e-12))
            kept += int(keep.sum())
    assert kept > 0


def line_case():
    """Points on the first axis: cluster A = {0.1, 1.0}, cluster B =
    {-0.3, -5.0}; query at 0.  The nearest point is 0.1 (A); the second
    nearest is -0.3, in B, which Eq. (13) prunes at f_d = 1 (centroid -2.65,
    radius 2.35: 2.65 - 2.35 = 0.3 >= d_c = 0.1)."""
    x = np.array([0.1, 1.0, -0.3, -5.0])
    Z = np.zeros((4, 12))
    Z[:, 0] = x
    cl = np.array([0, 0, 1, 1])
    cent = np.zeros((2, 12))
    cent[:, 0] = [0.55, -2.65]
    rad = np.array([0.45, 2.35])
    q = np.zeros((1, 12))
    return Z, q, cent, rad, cl


def test_second_nearest_in_a_pruned_cluster():
    """The search reads only cluster A, so the second-best of the points read
    is 1.0 (radius (1.0 - 0.1)/2 = 0.45); a move to -0.25 (0.25 < 0.45) would
    keep 0.1 although -0.3 is then nearer (0.05 < 0.35).  The bound of the
    pruned cluster gives the second bound 0.3 (radius 0.1): the move is not
    kept and the search finds -0.3.  The same with B a leaf of one cell."""
    Z, q, cent, rad, cl = line_case()
    i, d, s = ann.ann_search(Z, q, cent, rad, cl, 1.0, with_second=True)
    assert i[0] == 0 and np.isclose(d[0], 0.01) and np.isclose(s[0], 0.09)
    q2 = q.copy()
    q2[0, 0] = -0.25
    # the rule on the points read would keep the stale answer
    assert ann.moving_query_keeps(q2[0], q[0], d[0], 1.0)[0]
    assert np.argmin(((Z - q2[0]) ** 2).sum(1)) == 2
    keep, mv = ann.moving_query_keeps(q2[0], q[0], d[0], s[0])
    assert not keep and np.isclose(mv, 0.25)
    i2, d2 = ann.ann_search(Z, q2, cent, rad, cl, 1.0, prev_idx=i, motion=(q, d, s, 1.0))
    assert i2[0] == 2 and np.isclose(d2[0], 0.05 ** 2)
    # two levels: one cell holding A and B as leaves
    cc = Z.mean(0, keepdims=True)
    cr = np.array([np.sqrt(((Z - cc) ** 2).sum(1)).max()])
    i, d, s = ann.tree2_search(Z, q, cc, cr, cent, rad, cl, 2, 1.0, with_second=True)
    assert i[0] == 0 and np.isclose(s[0], 0.09)
    i2, _ = ann.tree2_search(Z, q2, cc, cr, cent, rad, cl, 2, 1.0, prev_idx=i, motion=(q, d, s, 1.0))
    assert i2[0] == 2


def test_second_bound_scales_with_fd_and_records_are_not_used_above_their_fd():
    """At f_d = 0.5 cluster B counts with half its radius: bound
    2.65 - 1.175 = 1.475 > 1.0, so the second bound is the read 1.0.  That
    record keeps the move to -0.25 at f_d = 0.5 (the search at 0.5 from the
    warm start also prunes B and answers 0.1), but a search at f_d = 1 does
    not use it and finds the exact -0.3."""
    Z, q, cent, rad, cl = line_case()
    i, d, s = ann.ann_search(Z, q, cent, rad, cl, 0.5, with_second=True)
    assert i[0] == 0 and np.isclose(s[0], 1.0)
    _, _, s0 = ann.ann_search(Z, q, cent, rad, cl, 0.0, with_second=True)
    assert np.isclose(s0[0], 1.0)                           # B's bound 2.65
    q2 = q.copy()
    q2[0, 0] = -0.25
    rec = (q, d, s, 0.5)
    k5, d5, s5 = ann.ann_search(Z, q2, cent, rad, cl, 0.5, prev_idx=i, motion=rec, with_second=True)
    assert k5[0] == 0 and np.isclose(d5[0], 0.35 ** 2) and np.isclose(s5[0], (1.0 - 0.25) ** 2)
    assert ann.ann_search(Z, q2, cent, rad, cl, 0.5, prev_idx=i)[0][0] == 0
    assert ann.ann_search(Z, q2, cent, rad, cl, 1.0, prev_idx=i, motion=rec)[0][0] == 2


def test_one_leaf_per_cell_second_bound_is_the_flat_one():
    Z, zq, cent, rad, cl = setup(seed=12)
    prev = np.random.default_rng(2).integers(0, len(Z), len(zq))
    for f_d in (0.0, 0.5, 1.0):
        for pv in (None, prev):
            a = ann.ann_search(Z, zq, cent, rad, cl, f_d, prev_idx=pv, n_cand=8, with_second=True)
            b = ann.tree2_search(Z, zq, cent, rad, cent, rad, cl, 1, f_d, prev_idx=pv, n_cand=8, with_second=True)
            assert all(np.array_equal(x, y) for x, y in zip(a, b))


def test_found_second_is_the_papers_estimate_below_fd_one():
    """second="found" returns the second-closest point read (the paper's p2)
    below f_d = 1 and the certified bound at f_d = 1.  Line case at
    f_d = 0.9: cluster B's bound is 2.65 - 0.9 x 2.35 = 0.535, so the
    certified second is 0.535^2, the found one 1.0 (the point at 1.0)."""
    Z, q, cent, rad, cl = line_case()
    _, _, s = ann.ann_search(Z, q, cent, rad, cl, 0.9, with_second=True)
    assert np.isclose(s[0], 0.535 ** 2)
    _, _, s = ann.ann_search(Z, q, cent, rad, cl, 0.9, with_second=True, second="found")
    assert np.isclose(s[0], 1.0)
    _, _, s = ann.ann_search(Z, q, cent, rad, cl, 1.0, with_second=True, second="found")
    assert np.isclose(s[0], 0.09)
    cc = Z.mean(0, keepdims=True)
    cr = np.array([np.sqrt(((Z - cc) ** 2).sum(1)).max()])
    _, _, s = ann.tree2_search(Z, q, cc, cr, cent, rad, cl, 2, 0.9, with_second=True, second="found")
    assert np.isclose(s[0], 1.0)
    # the found second is never below the certified one
    Z2, zq2, part = setup2(seed=13)
    for f_d in (0.0, 0.5):
        a = ann.tree2_search(Z2, zq2, *part, 10, f_d, with_second=True)
        b = ann.tree2_search(Z2, zq2, *part, 10, f_d, with_second=True, second="found")
        assert np.array_equal(a[0], b[0]) and np.all(b[2] >= a[2])
