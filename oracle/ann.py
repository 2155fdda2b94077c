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
