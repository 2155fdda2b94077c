"""Approximate nearest-data search of Sec. 4.2-4.5 (FP64 oracle).

TEST INFRASTRUCTURE ONLY.  Restates, on a given partition of the data into
clusters (centroid c_l, radius d_r = largest centroid-member distance), the
rules of the paper's k-means search with the warm start of Sec. 4.3:

  * descent: the cluster whose centroid is nearest to the query is searched;
  * warm start: the previous nearest point is the first current best, with
    d_c its distance, and its cluster is searched first;
  * backtracking (Eq. 13): a further cluster, taken in order of increasing
    centroid distance d(x, q), is searched when d(x, q) - f_d d_r < d_c;
    f_d = 1 gives the exact search by the triangle inequality;
  * only the `n_cand` nearest centroids are candidates for backtracking; for
    an exact request (f_d = 1), when a cluster beyond them could still pass
    Eq. (13) (tested with the largest radius), the query is answered by the
    exhaustive search instead, so f_d = 1 stays exact.

Moving queries (Eq. 14, Sec. 4.4).  The paper keeps the previous nearest
point p1 without a search when the query moved by less than half the gap
between the distances of the nearest and second-nearest points.  The
printed difference d(q, p1) - d(q, p2) is <= 0; the reading taken is
delta = (d2 - d1) / 2 with plain (not squared) distances and a strict test.
The triangle inequality makes the skip exact when d2 is a *lower bound* on
the distance of every other data point.  The second-best of the points a
search read is not one: a point of a cluster that Eq. (13) pruned can lie
nearer.  So every search here also returns

    s = min( second-smallest distance among the points read (the answer
             excluded),
             (d(x, q) - f_d d_r)^2 for every cluster not searched,
             with d(x, q) - f_d d_r clipped at 0 ),

where clusters beyond the candidate list count with the last candidate's
centroid distance and the largest radius.  At f_d = 1 this bounds the true
second-nearest distance from below, so a kept answer is the exact nearest
point.  Below 1 it is the bound under the cluster model that Eq. (13) itself
uses (the points of a cluster within f_d d_r of its centroid), so a kept
answer carries the same certificate as a search at that f_d.  A record made
at one f_d is used only by a search at the same or a lower f_d (the bound is
weaker for a larger f_d).  After a keep, the new second bound is
(sqrt(s) - |q_new - q_old|)^2 (triangle inequality again).

The paper's own wording takes p2 as the second-closest point "from the
search" and calls the relation an estimate.  `second="found"` returns that
instead (the second-smallest distance among the points read) below f_d = 1;
a search at f_d = 1 always returns the certified bound, so that an exact
search stays exact.  A "found" record serves any f_d below 1.

Distances are plain Euclidean distances in the mapped coordinates of
Sec. 3.2 (|dq|^2 = d_e^2 / 2).  Ties go to the lowest data index.
Pinned by tests/test_oracle_ann.py (f_d = 1 equals brute force; warm start
never worse than the previous point; f_d = 0 on a partition that isolates
points reproduces the nearest-centroid answer; the second bound never
exceeds the brute-force second distance at f_d = 1; a kept answer equals
brute force; a hand-built case whose second-nearest point lies in a pruned
cluster).

`tree2_search` applies the same rules on a two-level partition (cells, each
split into L2 leaves; leaf l lies in cell l // L2): Eq. (13) first chooses
the cells among the `n_cand` nearest, then, inside a chosen cell, the leaves
among its `k_fine` nearest, each leaf tested with its own radius and the
d_c reached so far.  The nearest cell and its nearest leaf are always
searched (the descent).  For f_d = 1 a leaf beyond the `k_fine` nearest of
a visited cell, or a cell beyond the `n_cand` nearest, that could still pass
Eq. (13) sends the query to the exhaustive search.  The second bound takes,
for a cell not visited, its own centroid distance and radius, and for a
visited cell every leaf of it not searched with the leaf's centroid distance
and radius.  The candidate-list lengths and the hand-off `budget` restate
the GPU design's limits, not the paper's (which searches a deep tree);
tests pin the paper-level facts (f_d = 1 exact for any of them, a budget
never farther).  Pinned by tests/test_oracle_ann.py (one leaf per cell
reproduces `ann_search` answer for answer, second bound included; f_d = 1
equals brute force).
"""
from __future__ import annotations

import math

import numpy as np


def moving_query_keeps(q, q_prev, d1_prev, d2_prev):
    """Eq. (14) with the sign read as delta = (d2 - d1)/2: True when the query
    moved (plain distance |q - q_prev|) strictly less than delta.  d1_prev and
    d2_prev are squared distances (the answer's and the second bound)."""
    mv = math.sqrt(float(((np.asarray(q, np.float64) - np.asarray(q_prev, np.float64)) ** 2).sum()))
    return mv < 0.5 * (math.sqrt(d2_prev) - math.sqrt(d1_prev)), mv


def second_rule_certified(second_rule, f_d):
    """True when the second distance is the certified bound: always for
    "certified", and for "found" (the paper's estimate) at f_d = 1."""
    if second_rule not in ("certified", "found"):
        raise ValueError(second_rule)
    return second_rule == "certified" or f_d >= 1.0


def _bound_sq(b):
    """Squared lower bound from a plain one that may be negative."""
    return max(b, 0.0) ** 2


def _kept(Z, q, qi, prev_idx, motion, f_d):
    """Eq. (14) test of query qi against its motion record; returns
    (answer, squared distance, second bound) when it is kept, else None."""
    if motion is None or prev_idx is None:
        return None
    q_prev, d1p, d2p, fdp = motion
    fd_rec = fdp if np.isscalar(fdp) else fdp[qi]
    if f_d > fd_rec:
        return None
    keep, mv = moving_query_keeps(q, q_prev[qi], d1p[qi], d2p[qi])
    if not keep:
        return None
    j0 = int(prev_idx[qi])
    return j0, float(((Z[j0] - q) ** 2).sum()), _bound_sq(math.sqrt(d2p[qi]) - mv)


def ann_search(Z, zq, cent, rad, cluster_of, f_d, prev_idx=None, n_cand=8, motion=None, with_second=False,
               second="certified"):
    """Returns (idx, squared distance) for every query row of zq, and with
    with_second=True also the squared second bound s (module docstring).

    motion: None, or (previous queries [m x 12], their squared answer
    distances [m], their squared second bounds [m], the f_d the record was
    made at (scalar or [m])); with prev_idx it enables the Eq. (14) skip."""
    second_kind = second
    Z = np.asarray(Z, dtype=np.float64)
    zq = np.asarray(zq, dtype=np.float64)
    cent = np.asarray(cent, dtype=np.float64)
    rad = np.asarray(rad, dtype=np.float64)
    L = len(cent)
    members = [np.nonzero(cluster_of == l)[0] for l in range(L)]
    rmax = rad.max()
    out_i = np.empty(len(zq), np.int64)
    out_d = np.empty(len(zq))
    out_s = np.empty(len(zq))
    for qi, q in enumerate(zq):
        kept = _kept(Z, q, qi, prev_idx, motion, f_d)
        if kept is not None:
            out_i[qi], out_d[qi], out_s[qi] = kept
            continue
        dcent = np.sqrt(((cent - q) ** 2).sum(1))
        order = np.lexsort((np.arange(L), dcent))[:n_cand]
        best_d, best_j = np.inf, -1
        read = {}            # data index -> squared distance, every point read

        def scan(l):
            nonlocal best_d, best_j
            for j in members[l]:
                d = float(((Z[j] - q) ** 2).sum())
                read[int(j)] = d
                if d < best_d or (d == best_d and j < best_j):
                    best_d, best_j = d, int(j)

        cl0 = -1
        if prev_idx is not None:
            j0 = int(prev_idx[qi])
            best_d, best_j = float(((Z[j0] - q) ** 2).sum()), j0
            read[j0] = best_d
            cl0 = int(cluster_of[j0])
            scan(cl0)
        dc = np.sqrt(best_d)
        bound = np.inf       # plain lower bound on the points of clusters not searched
        for k, l in enumerate(order):
            if l == cl0:
                continue
            if k == 0 or dcent[l] - f_d * rad[l] < dc:
                scan(l)
                dc = np.sqrt(best_d)
            else:
                bound = min(bound, dcent[l] - f_d * rad[l])
        if L > n_cand:
            bound = min(bound, dcent[order[-1]] - f_d * rmax)
        if f_d >= 1.0 and L > n_cand and dcent[order[-1]] - f_d * rmax < dc:
            d = ((Z - q) ** 2).sum(1)
            best_j = int(np.argmin(d))
            best_d = float(d[best_j])
            second = float(np.min(np.delete(d, best_j))) if len(d) > 1 else np.inf
        else:
            second = min([v for j, v in read.items() if j != best_j], default=np.inf)
            if second_rule_certified(second_rule=second_kind, f_d=f_d):
                second = min(second, _bound_sq(bound))
        out_i[qi], out_d[qi], out_s[qi] = best_j, best_d, second
    return (out_i, out_d, out_s) if with_second else (out_i, out_d)


def tree2_search(Z, zq, cell_cent, cell_rad, leaf_cent, leaf_rad, leaf_of, L2, f_d, prev_idx=None, n_cand=8,
                 k_fine=8, budget=None, motion=None, with_second=False, second="certified"):
    """Returns (idx, squared distance) for every query row of zq on the
    two-level partition: cells (centroids, radii) and their leaves (leaf l
    in cell l // L2; centroids, radii, leaf of every data point); with
    with_second=True also the squared second bound (module docstring).

    budget: None searches every chosen leaf at once, d_c shrinking after
    each.  An integer b searches only the first b chosen leaves at once (the
    warm-start leaf first).  Every later leaf that passes Eq. (13) with the
    d_c reached then is searched at the end, without shrinking d_c: the
    chosen set can only grow, so the answer is never farther.
    motion: as in ann_search (the Eq. 14 skip)."""
    second_kind = second
    Z = np.asarray(Z, dtype=np.float64)
    zq = np.asarray(zq, dtype=np.float64)
    cell_cent = np.asarray(cell_cent, dtype=np.float64)
    cell_rad = np.asarray(cell_rad, dtype=np.float64)
    leaf_cent = np.asarray(leaf_cent, dtype=np.float64)
    leaf_rad = np.asarray(leaf_rad, dtype=np.float64)
    L1, L = len(cell_cent), len(leaf_cent)
    members = [np.nonzero(leaf_of == l)[0] for l in range(L)]
    r1max, rmax = cell_rad.max(), leaf_rad.max()
    out_i = np.empty(len(zq), np.int64)
    out_d = np.empty(len(zq))
    out_s = np.empty(len(zq))
    for qi, q in enumerate(zq):
        kept = _kept(Z, q, qi, prev_idx, motion, f_d)
        if kept is not None:
            out_i[qi], out_d[qi], out_s[qi] = kept
            continue
        dcell = np.sqrt(((cell_cent - q) ** 2).sum(1))
        cells = np.lexsort((np.arange(L1), dcell))[:n_cand]
        best_d, best_j = np.inf, -1
        read = {}            # data index -> squared distance, every point read

        def scan(l):
            # every member's distance; the first minimum is the lowest index
            nonlocal best_d, best_j
            mem = members[l]
            if len(mem) == 0:
                return
            d = ((Z[mem] - q) ** 2).sum(1)
            for j, v in zip(mem, d):
                read[int(j)] = float(v)
            t = int(np.argmin(d))
            if d[t] < best_d or (d[t] == best_d and mem[t] < best_j):
                best_d, best_j = float(d[t]), int(mem[t])

        nscan, deferred = 0, []

        def take(l):
            nonlocal nscan, dc
            if budget is None or nscan < budget:
                scan(l)
                nscan += 1
                dc = np.sqrt(best_d)
            else:
                deferred.append(l)

        l0 = -1
        dc = np.inf
        if prev_idx is not None:
            j0 = int(prev_idx[qi])
            best_d, best_j = float(((Z[j0] - q) ** 2).sum()), j0
            read[j0] = best_d
            dc = np.sqrt(best_d)
            l0 = int(leaf_of[j0])
            take(l0)
        incomplete = False
        bound = np.inf       # plain lower bound on the points of cells and leaves not searched
        for k1, c in enumerate(cells):
            if not (k1 == 0 or dcell[c] - f_d * cell_rad[c] < dc):
                # the warm-start leaf is the one leaf searched outside a
                # visited cell: a cell made of it alone needs no bound
                if not (L2 == 1 and c == l0):
                    bound = min(bound, dcell[c] - f_d * cell_rad[c])
                continue
            leaves = np.arange(c * L2, (c + 1) * L2)
            dleaf = np.sqrt(((leaf_cent[leaves] - q) ** 2).sum(1))
            order = np.lexsort((leaves, dleaf))
            passed = set()
            for k2, o in enumerate(order[:k_fine]):
                l = int(leaves[o])
                if (k1 == 0 and k2 == 0) or dleaf[o] - f_d * leaf_rad[l] < dc:
                    passed.add(l)
                    if l != l0:
                        take(l)
            for o in range(L2):
                l = int(leaves[o])
                if l not in passed and l != l0:
                    bound = min(bound, dleaf[o] - f_d * leaf_rad[l])
            if f_d >= 1.0 and L2 > k_fine and dleaf[order[k_fine:]].min() - f_d * rmax < dc:
                incomplete = True
        if L1 > n_cand:
            bound = min(bound, dcell[cells[-1]] - f_d * r1max)
        if f_d >= 1.0 and L1 > n_cand and dcell[cells[-1]] - f_d * r1max < dc:
            incomplete = True
        for l in deferred:
            scan(l)
        if incomplete:
            d = ((Z - q) ** 2).sum(1)
            best_j = int(np.argmin(d))
            best_d = float(d[best_j])
            second = float(np.min(np.delete(d, best_j))) if len(d) > 1 else np.inf
        else:
            second = min([v for j, v in read.items() if j != best_j], default=np.inf)
            if second_rule_certified(second_rule=second_kind, f_d=f_d):
                second = min(second, _bound_sq(bound))
        out_i[qi], out_d[qi], out_s[qi] = best_j, best_d, second
    return (out_i, out_d, out_s) if with_second else (out_i, out_d)


def kmeans_partition(Z, L, iters=10, seed=0):
    """A plain Lloyd partition (for tests that need one without the GPU):
    returns (centroids, radii, cluster_of)."""
    rng = np.random.default_rng(seed)
    cent = Z[rng.choice(len(Z), L, replace=False)].copy()
    for _ in range(iters):
        d = ((Z[:, None, :] - cent[None, :, :]) ** 2).sum(-1)
        a = d.argmin(1)
        for l in range(L):
            if np.any(a == l):
                cent[l] = Z[a == l].mean(0)
    d = ((Z[:, None, :] - cent[None, :, :]) ** 2).sum(-1)
    a = d.argmin(1)
    rad = np.array([np.sqrt(d[a == l, l].max()) if np.any(a == l) else 0.0 for l in range(L)])
    return cent, rad, a


def tree2_partition(Z, L1, L2, iters=10, seed=0):
    """A plain two-level partition (for tests that need one without the GPU):
    Lloyd cells, then Lloyd leaves inside every cell (leaf l in cell l // L2;
    a leaf left without members keeps its cell's centroid and radius 0).
    Returns (cell centroids, cell radii, leaf centroids, leaf radii,
    leaf of every point)."""
    Z = np.asarray(Z, dtype=np.float64)
    ccent, crad, cell_of = kmeans_partition(Z, L1, iters=iters, seed=seed)
    lcent = np.repeat(ccent, L2, axis=0)
    lrad = np.zeros(L1 * L2)
    leaf_of = np.empty(len(Z), np.int64)
    for c in range(L1):
        mem = np.nonzero(cell_of == c)[0]
        if len(mem) == 0:
            continue
        k = min(L2, len(mem))
        cent, rad, a = kmeans_partition(Z[mem], k, iters=iters, seed=seed + 1 + c)
        lcent[c * L2:c * L2 + k] = cent
        lrad[c * L2:c * L2 + k] = rad
        leaf_of[mem] = c * L2 + a
    return ccent, crad, lcent, lrad, leaf_of
