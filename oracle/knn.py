"""Oracle for the kNN graph construction of Sec. 5.1 (FP64, CPU, brute force).  Test
infrastructure only: nothing in the product path imports it.

The paper builds its input graphs from Euclidean distances between samples (kNN graphs of
the JAFFE and AT&T images, Sec. 5.1) and gives no further detail.  The readings used:
  * exact k nearest neighbours of every point by Euclidean distance, the point itself
    excluded; equal distances are ordered by the lower index;
  * the squared distance of points p, q in R^d is the sum over coordinates c = 0 .. d-1,
    in that order, of (p_c - q_c)^2, each product and sum rounded to FP64 (no fused
    multiply-add): neighbours are chosen by that value, so both implementations take the
    same decision on near-ties;
  * the graph is the union of the directed kNN relations (i ~ j when j is among the k
    nearest of i, or i among the k nearest of j);
  * weights are Gaussian, w_ij = exp(-d_ij^2 / sigma^2), with sigma the mean of the N k
    directed nearest-neighbour distances d = sqrt(d^2).

Brute force: the full row of squared distances from each point to every other point, a
stable sort of it (which keeps the lower index first among equal values), the first k.
"""
from __future__ import annotations

import numpy as np


def squared_distances(points: np.ndarray, rows: np.ndarray) -> np.ndarray:
    """d2[r, j] for query rows `rows` against all points, coordinates summed in order."""
    P = np.asarray(points, dtype=np.float64)
    d2 = np.zeros((rows.shape[0], P.shape[0]))
    for c in range(P.shape[1]):
        diff = P[rows, c][:, None] - P[None, :, c]
        d2 = d2 + diff * diff
    return d2


def knn_lists(points: np.ndarray, k: int, block: int = 512, rows=None):
    """Directed kNN: (nbr int64 [len(rows), k], d2 float64 [len(rows), k]) ordered by
    (d2, index), for the query points `rows` (all points when None)."""
    P = np.asarray(points, dtype=np.float64)
    n = P.shape[0]
    if not (1 <= k < n):
        raise ValueError("need 1 <= k < n")
    rows = np.arange(n) if rows is None else np.asarray(rows, dtype=np.int64)
    nbr = np.empty((rows.shape[0], k), dtype=np.int64)
    dd = np.empty((rows.shape[0], k))
    for r0 in range(0, rows.shape[0], block):
        sel = np.arange(r0, min(rows.shape[0], r0 + block))
        q = rows[sel]
        d2 = squared_distances(P, q)
        d2[np.arange(q.shape[0]), q] = np.inf                 # not its own neighbour
        order = np.argsort(d2, axis=1, kind="stable")[:, :k]
        nbr[sel] = order
        dd[sel] = np.take_along_axis(d2, order, axis=1)
    return nbr, dd


def knn_graph(points: np.ndarray, k: int):
    """The symmetric (union) kNN graph with Gaussian weights, canonical CSR.

    Returns (row_ptr int64 [n+1], col int32 ascending per row, w float64, sigma)."""
    P = np.asarray(points, dtype=np.float64)
    n = P.shape[0]
    nbr, d2 = knn_lists(P, k)
    sigma = float(np.mean(np.sqrt(d2)))
    rows = np.repeat(np.arange(n, dtype=np.int64), k)
    cols = nbr.reshape(-1)
    # union of both directions, one entry per unordered pair and direction
    i = np.concatenate([rows, cols])
    j = np.concatenate([cols, rows])
    key = np.unique(i * n + j)
    i, j = key // n, key % n
    # squared distance of each edge, from its own two end points in the order (row, col)
    d2e = np.zeros(i.shape[0])
    for c in range(P.shape[1]):
        diff = P[i, c] - P[j, c]
        d2e = d2e + diff * diff
    w = np.exp(-d2e / (sigma * sigma))
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(i, minlength=n), out=row_ptr[1:])
    return row_ptr, j.astype(np.int32), w, sigma
