"""k-nearest-neighbour graph and its greedy walk, Sec. 4.4.

TEST INFRASTRUCTURE ONLY: imported by tests/ and nothing else.

Distances are squared Euclidean distances in the mapped coordinates of
Sec. 3.2 (|z_i - z_j|^2 = d_e^2 / 2 of Eq. 3), in FP64.

knn_graph    every data point linked to its k nearest *other* points, nearest
             first, ties to the lower index: the definition, one row of the
             distance matrix at a time (small N only).
greedy_walk  the greedy search of Sec. 4.4: from a start point, the distances
             of all graph neighbours of the current point to the query are
             evaluated and the nearest of them becomes the current point if it
             is strictly nearer than the current point; the walk ends at a
             point none of whose neighbours is nearer (a local minimum of the
             graph) or after f_s node changes (the bound of Sec. 4.4; f_s = 0
             means no bound).  In the DD iteration the start is the previous
             nearest neighbour (warm start, Sec. 4.4).

Readings (the paper is silent): among neighbours at equal distance the lower
data index is taken; the second distance reported for the moving-query radius
of Eq. (14) is the smallest distance of any evaluated point other than the
answer, and a walk stopped by f_s reports the answer's own distance there
(radius 0: its answer is not a local minimum, so it is not kept unsearched).
A walk that ended at a local minimum p1 evaluated every neighbour of p1, so
that second distance bounds them from below; a query that moves by less than
the Eq. (14) radius is then still strictly nearer to p1 than to any of them,
and the walk from the warm start p1 would stay at p1.  The skip therefore
returns exactly what the walk would (not the exact nearest point, which the
walk does not promise either); tests/test_oracle_knng.py pins this.
"""
from __future__ import annotations

import math

import numpy as np


def knn_graph(Z: np.ndarray, k: int) -> np.ndarray:
    """int64 [N x k]: row i holds the k nearest points j != i of Z (rows of
    mapped coordinates), nearest first, ties to the lower index; -1 pads rows
    when N - 1 < k."""
    Z = np.asarray(Z, dtype=np.float64)
    N = len(Z)
    out = np.full((N, k), -1, dtype=np.int64)
    idx = np.arange(N)
    for i in range(N):
        d = ((Z - Z[i]) ** 2).sum(axis=1)
        d[i] = math.inf
        order = np.lexsort((idx, d))          # by distance, then index
        n = min(k, N - 1)
        out[i, :n] = order[:n]
    return out


def greedy_walk(Z: np.ndarray, nbr: np.ndarray, q: np.ndarray, start: int, f_s: int = 0):
    """One greedy walk of Sec. 4.4 for the mapped query q.

    Returns (answer index, its squared distance, second squared distance,
    node changes, distances evaluated)."""
    Z = np.asarray(Z, dtype=np.float64)
    q = np.asarray(q, dtype=np.float64)

    def dist(j):
        return float(((Z[j] - q) ** 2).sum())

    cur, dcur = int(start), dist(start)
    second = math.inf
    moves, evals = 0, 1
    bounded = False
    while True:
        if f_s > 0 and moves >= f_s:
            bounded = True
            break
        cand = [int(j) for j in nbr[cur] if j >= 0]
        if not cand:
            break
        ds = [dist(j) for j in cand]
        evals += len(cand)
        b = min(range(len(cand)), key=lambda t: (ds[t], cand[t]))
        rest = min((ds[t] for t in range(len(cand)) if t != b), default=math.inf)
        if ds[b] < dcur:
            second = min(second, dcur, rest)
            cur, dcur = cand[b], ds[b]
            moves += 1
        else:
            second = min(second, ds[b])
            break
    if bounded:
        second = dcur
    return cur, dcur, second, moves, evals


def walk_all(Z: np.ndarray, nbr: np.ndarray, zq: np.ndarray, starts: np.ndarray, f_s: int = 0):
    """greedy_walk for every query row of zq from starts[i]; arrays of the
    answers, distances, second distances, node changes and evaluations."""
    res = [greedy_walk(Z, nbr, zq[i], int(starts[i]), f_s) for i in range(len(zq))]
    cols = list(zip(*res)) if res else [[]] * 5
    return (np.array(cols[0], dtype=np.int64), np.array(cols[1], dtype=np.float64),
            np.array(cols[2], dtype=np.float64), np.array(cols[3], dtype=np.int64),
            np.array(cols[4], dtype=np.int64))
