"""Pins of the oracle's k-NN graph and greedy walk (Sec. 4.4)."""
import numpy as np

import dd_inputs as I
from oracle import knng, metric, nn


def on_line(xs):
    """Points on the first axis of the 12-d mapped space."""
    Z = np.zeros((len(xs), 12))
    Z[:, 0] = xs
    return Z


def test_graph_by_hand():
    # x = 0, 1, 3, 7, 15 with k = 2, worked out by hand
    g = knng.knn_graph(on_line([0.0, 1.0, 3.0, 7.0, 15.0]), 2)
    assert g.tolist() == [[1, 2], [0, 2], [1, 0], [2, 1], [3, 2]]
    # equal distances go to the lower index; rows are padded when N - 1 < k
    g = knng.knn_graph(on_line([0.0, 1.0, -1.0]), 3)
    assert g.tolist() == [[1, 2, -1], [0, 2, -1], [0, 1, -1]]


def test_first_neighbour_is_brute_force_second_nearest():
    """The first neighbour of a point is its nearest other point, which the
    C brute-force scan reports as the second nearest of the point itself."""
    data = I.make_dataset(700, I.NONLINEAR, seed=3)
    Z = metric.to_z(data.astype(np.float64), I.isotropic_C())
    g = knng.knn_graph(Z, 4)
    i1, d1, i2, d2 = nn.nn_top2(Z, Z)
    assert np.array_equal(i1, np.arange(len(Z)))          # no duplicate points
    assert np.array_equal(g[:, 0], i2)
    # neighbours are sorted by distance
    dg = np.array([((Z[g[i]] - Z[i]) ** 2).sum(1) for i in range(len(Z))])
    assert np.all(np.diff(dg, axis=1) >= 0)
    assert np.allclose(dg[:, 0], d2, rtol=1e-13, atol=0)   # summation order differs


def test_walk_on_a_chain():
    """Points x = 0..9 with k = 2 form a chain; a query at 7.2 walked from 0
    moves 0 -> 2 -> 3 -> 4 -> 5 -> 6 -> 7 and stops (both neighbours of 7 are
    farther): 6 node changes, answer 7, second distance that of 8."""
    Z = on_line(np.arange(10.0))
    g = knng.knn_graph(Z, 2)
    q = on_line([7.2])[0]
    j, d, s, moves, evals = knng.greedy_walk(Z, g, q, 0)
    assert (j, moves, evals) == (7, 6, 1 + 2 * 7)
    assert np.isclose(d, 0.2 ** 2) and np.isclose(s, 0.8 ** 2)
    # bounded to 3 node changes: stops at 4, radius 0 (second = own distance)
    j, d, s, moves, evals = knng.greedy_walk(Z, g, q, 0, f_s=3)
    assert (j, moves) == (4, 3) and s == d and np.isclose(d, 3.2 ** 2)
    # a start at the answer evaluates one neighbourhood and stays
    j, d, s, moves, evals = knng.greedy_walk(Z, g, q, 7)
    assert (j, moves, evals) == (7, 0, 3)


def test_walk_on_complete_graph_is_exact():
    """With every point linked to all others one step reaches the nearest
    point from any start, and every point is evaluated, so the second
    distance is the exact second nearest (brute force in C)."""
    data = I.make_dataset(300, I.LINEAR, seed=5)
    Z = metric.to_z(data.astype(np.float64), I.isotropic_C())
    g = knng.knn_graph(Z, len(Z) - 1)
    y = I.make_states(40, I.LINEAR, seed=6, spread=0.3)
    zq = metric.to_z(y, I.isotropic_C())
    starts = np.random.default_rng(1).integers(0, len(Z), len(zq))
    j, d, s, moves, evals = knng.walk_all(Z, g, zq, starts)
    i1, d1, i2, d2 = nn.nn_top2(Z, zq)
    assert np.array_equal(j, i1)
    assert np.allclose(d, d1, rtol=1e-12) and np.allclose(s, d2, rtol=1e-12)
    assert np.all(moves <= 1)


def test_walk_ends_in_a_local_minimum_and_never_worse():
    """On a sparse graph the walk may stop short of the nearest point, but the
    answer is never farther than the start and, without a bound, none of its
    neighbours is nearer."""
    data = I.make_dataset(1500, I.NONLINEAR, seed=8)
    Z = metric.to_z(data.astype(np.float64), I.isotropic_C())
    g = knng.knn_graph(Z, 6)
    y = I.make_states(200, I.NONLINEAR, seed=9, spread=0.1)
    zq = metric.to_z(y, I.isotropic_C())
    starts = np.random.default_rng(2).integers(0, len(Z), len(zq))
    j, d, s, moves, evals = knng.walk_all(Z, g, zq, starts)
    d_start = ((Z[starts] - zq) ** 2).sum(1)
    assert np.all(d <= d_start)
    for i in range(len(zq)):
        dn = ((Z[g[j[i]]] - zq[i]) ** 2).sum(1)
        assert np.all(dn >= d[i])
        assert s[i] >= d[i]
    assert np.all(evals == 1 + 6 * (moves + 1))
    # a denser graph reaches the nearest point more often (Sec. 4.4)
    i1, _, _, _ = nn.nn_top2(Z, zq)
    g16 = knng.knn_graph(Z, 16)
    j16 = knng.walk_all(Z, g16, zq, starts)[0]
    assert 0.05 < np.mean(j == i1) < np.mean(j16 == i1) < 1.0


def test_eq14_keep_reproduces_the_walk_from_the_warm_start():
    """A walk that ended at a local minimum p1 evaluated every neighbour of
    p1, so its second distance s bounds them from below.  A query that then
    moves by less than (sqrt(s) - sqrt(d1)) / 2 (Eq. 14) is still strictly
    nearer to p1 than to any neighbour of p1, so the walk from the warm start
    p1 stays there: the skip returns what the walk would.  Moves just beyond
    the radius do change some answers (the radius is not vacuous)."""
    data = I.make_dataset(1200, I.NONLINEAR, seed=10)
    Z = metric.to_z(data.astype(np.float64), I.isotropic_C())
    g = knng.knn_graph(Z, 6)
    y = I.make_states(150, I.NONLINEAR, seed=11, spread=0.1)
    zq = metric.to_z(y, I.isotropic_C())
    starts = np.random.default_rng(3).integers(0, len(Z), len(zq))
    rng = np.random.default_rng(4)
    kept = changed = 0
    for i in range(len(zq)):
        j, d, s, moves, _ = knng.greedy_walk(Z, g, zq[i], int(starts[i]))
        delta = 0.5 * (np.sqrt(s) - np.sqrt(d))
        if not delta > 0:
            continue
        for scale in (0.3, 0.999):
            v = rng.standard_normal(12)
            q2 = zq[i] + v / np.linalg.norm(v) * delta * scale
            j2, _, _, m2, _ = knng.greedy_walk(Z, g, q2, j)
            assert j2 == j and m2 == 0
            kept += 1
        # the nearest other point at 3 delta: moving towards it can flip the answer
        nb = [int(t) for t in g[j]]
        dn = ((Z[nb] - zq[i]) ** 2).sum(1)
        far = nb[int(np.argmin(dn))]
        u = (Z[far] - zq[i]) / np.linalg.norm(Z[far] - zq[i])
        changed += int(knng.greedy_walk(Z, g, zq[i] + u * 3 * delta, j)[0] != j)
    assert kept > 0 and changed > 0
