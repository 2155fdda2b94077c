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

Distances are plain Euclidean distances in the mapped coordinates of
Sec. 3.2 (|dq|^2 = d_e^2 / 2).  Ties go to the lowest data index.
Pinned by tests/test_oracle_ann.py (f_d = 1 equals brute force; warm start
never worse than the previous point; f_d = 0 on a partition that isolates
points reproduces the nearest-centroid answer).

`tree2_search` applies the same rules on a two-level partition (cells, each
split into L2 leaves; leaf l lies in cell l // L2): Eq. (13) first chooses
the cells among the `n_cand` nearest, then, inside a chosen cell, the leaves
among its `k_fine` nearest, each leaf tested with its own radius and the
d_c reached so far.  The nearest cell and its nearest leaf are always
searched (the descent).  For f_d = 1 a leaf beyond the `k_fine` nearest of
a visited cell, or a cell beyond the `n_cand` nearest, that could still pass
Eq. (13) sends the query to the exhaustive search.  Pinned by
tests/test_oracle_ann.py (one leaf per cell reproduces `ann_search`; f_d = 1
equals brute force).
"""
from __future__ import annotations

import numpy as np


def ann_search(Z, zq, cent, rad, cluster_of, f_d, prev_idx=None, n_cand=8):
    """Returns (idx, squared distance) for every query row of zq."""
    Z = np.asarray(Z, dtype=np.float64)
    zq = np.asarray(zq, dtype=np.float64)
    cent = np.asarray(cent, dtype=np.float64)
    rad = np.asarray(rad, dtype=np.float64)
    L = len(cent)
    members = [np.nonzero(cluster_of == l)[0] for l in range(L)]
    rmax = rad.max()
    out_i = np.empty(len(zq), np.int64)
    out_d = np.empty(len(zq))
    for qi, q in enumerate(zq):
        dcent = np.sqrt(((cent - q) ** 2).sum(1))
        order = np.lexsort((np.arange(L), dcent))[:n_cand]
        best_d, best_j = np.inf, -1

        def scan(l):
            nonlocal best_d, best_j
            for j in members[l]:
                d = float(((Z[j] - q) ** 2).sum())
                if d < best_d or (d == best_d and j < best_j):
                    best_d, best_j = d, int(j)

        cl0 = -1
        if prev_idx is not None:
            j0 = int(prev_idx[qi])
            best_d, best_j = float(((Z[j0] - q) ** 2).sum()), j0
            cl0 = int(cluster_of[j0])
            scan(cl0)
        dc = np.sqrt(best_d)
        for k, l in enumerate(order):
            if l == cl0:
                continue
            if k == 0 or dcent[l] - f_d * rad[l] < dc:
                scan(l)
                dc = np.sqrt(best_d)
        if f_d >= 1.0 and L > n_cand and dcent[order[-1]] - f_d * rmax < dc:
            d = ((Z - q) ** 2).sum(1)
            best_j = int(np.argmin(d))
            best_d = float(d[best_j])
        out_i[qi], out_d[qi] = best_j, best_d
    return out_i, out_d


def tree2_search(Z, zq, cell_cent, cell_rad, leaf_cent, leaf_rad, leaf_of, L2, f_d, prev_idx=None, n_cand=8,
                 k_fine=8, budget=None):
    """Returns (idx, squared distance) for every query row of zq on the
    two-level partition: cells (centroids, radii) and their leaves (leaf l
    in cell l // L2; centroids, radii, leaf of every data point).

    budget: None searches every chosen leaf at once, d_c shrinking after
    each.  An integer b searches only the first b chosen leaves at once (the
    warm-start leaf first).  Every later leaf that passes Eq. (13) with the
    d_c reached then is searched at the end, without shrinking d_c: the
    chosen set can only grow, so the answer is never farther."""
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
    for qi, q in enumerate(zq):
        dcell = np.sqrt(((cell_cent - q) ** 2).sum(1))
        cells = np.lexsort((np.arange(L1), dcell))[:n_cand]
        best_d, best_j = np.inf, -1

        def scan(l):
            # every member's distance; the first minimum is the lowest index
            nonlocal best_d, best_j
            mem = members[l]
            if len(mem) == 0:
                return
            d = ((Z[mem] - q) ** 2).sum(1)
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
            dc = np.sqrt(best_d)
            l0 = int(leaf_of[j0])
            take(l0)
        incomplete = False
        for k1, c in enumerate(cells):
            if not (k1 == 0 or dcell[c] - f_d * cell_rad[c] < dc):
                continue
            leaves = np.arange(c * L2, (c + 1) * L2)
            dleaf = np.sqrt(((leaf_cent[leaves] - q) ** 2).sum(1))
            order = np.lexsort((leaves, dleaf))
            for k2, o in enumerate(order[:k_fine]):
                l = int(leaves[o])
                if (k1 == 0 and k2 == 0) or dleaf[o] - f_d * leaf_rad[l] < dc:
                    if l != l0:
                        take(l)
            if f_d >= 1.0 and L2 > k_fine and dleaf[order[k_fine:]].min() - f_d * rmax < dc:
                incomplete = True
        if f_d >= 1.0 and L1 > n_cand and dcell[cells[-1]] - f_d * r1max < dc:
            incomplete = True
        for l in deferred:
            scan(l)
        if incomplete:
            d = ((Z - q) ** 2).sum(1)
            best_j = int(np.argmin(d))
            best_d = float(d[best_j])
        out_i[qi], out_d[qi] = best_j, best_d
    return out_i, out_d


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
