"""Oracle for betweenness centrality and its variance, VBC (Sec. 3.3, Table 1).  Test
infrastructure only: nothing in the product path imports it.

Sec. 3.3 defines C_B(i) = sum over s, t != i of sigma_st(i) / sigma_st, with sigma_st the
number of shortest paths from s to t and sigma_st(i) those through i, and qualifies a graph
as a manifold graph by the variance of C_B over its nodes (VBC).  Readings:
  * shortest paths count hops (the graph's weights are similarities, not lengths);
  * the sum runs over ordered pairs (s, t), s != t, both different from i, as printed
    (each unordered pair counts twice); pairs with no path contribute nothing;
  * VBC is the population variance (1/N) sum_i (C_B(i) - mean C_B)^2.
Computed by Brandes' accumulation (Brandes 2001): for every source s a breadth-first search
counts shortest paths sigma_s, then the dependencies delta_s(v) = sum over successors w of
(sigma_s(v) / sigma_s(w)) (1 + delta_s(w)) are accumulated in reverse BFS order, and
C_B(v) = sum over s != v of delta_s(v).
"""
from __future__ import annotations

from collections import deque

import numpy as np


def betweenness(n: int, row_ptr: np.ndarray, col: np.ndarray) -> np.ndarray:
    """C_B over ordered pairs, hop-count shortest paths, FP64 (Brandes)."""
    rp = np.asarray(row_ptr, dtype=np.int64)
    cl = np.asarray(col, dtype=np.int64)
    cb = np.zeros(n)
    for s in range(n):
        dist = np.full(n, -1, dtype=np.int64)
        sigma = np.zeros(n)
        dist[s] = 0
        sigma[s] = 1.0
        order = []
        q = deque([s])
        while q:
            v = q.popleft()
            order.append(v)
            for w in cl[rp[v]:rp[v + 1]]:
                if dist[w] < 0:
                    dist[w] = dist[v] + 1
                    q.append(w)
                if dist[w] == dist[v] + 1:
                    sigma[w] += sigma[v]
        delta = np.zeros(n)
        for w in reversed(order):
            for v in cl[rp[w]:rp[w + 1]]:
                if dist[v] == dist[w] - 1:
                    delta[v] += sigma[v] / sigma[w] * (1.0 + delta[w])
            if w != s:
                cb[w] += delta[w]
    return cb


def vbc(cb: np.ndarray) -> float:
    """Population variance of the betweenness centralities."""
    cb = np.asarray(cb, dtype=np.float64)
    return float(np.mean((cb - np.mean(cb)) ** 2))
