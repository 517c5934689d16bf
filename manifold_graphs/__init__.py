"""Seeded synthetic manifold graphs: the inputs shared by the oracle and the CUDA path.

This module holds no arithmetic of the embedding method itself (no two-hop sets, no
Q, mu, epsilon, b, no eigensolver).  It only produces the input graph G(V, E, W) of
Sec. 3.1: points sampled on a manifold, an exact k-nearest-neighbour graph built from
Euclidean distances (the graph construction of Sec. 5.1), and a handful of small
named graphs used as test inputs (the ring and line of Fig. 2, the triangle mesh of
Fig. 3, paths, complete graphs, random graphs).

Every graph is returned in canonical CSR form: ``row_ptr`` int64[N+1], ``col`` int32
(ascending within each row, no duplicates, no diagonal) and ``w`` float64 (positive),
symmetric.

Choices the paper leaves open (it names none of them), fixed here once for both sides:
  * kNN is exact, by Euclidean distance; a point is not its own neighbour.
  * Symmetrisation is by union: i ~ j if j is among the k nearest of i or vice versa.
  * Weights are Gaussian, w_ij = exp(-d_ij^2 / sigma^2), with sigma the mean of all
    N*k directed k-nearest-neighbour distances.
  * Within a row, neighbours with equal distance are ordered by lower index.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

__all__ = [
    "Graph", "sample_points", "knn_graph", "manifold_graph", "from_edges",
    "ring", "path", "complete", "triangle_mesh", "erdos_renyi", "two_components",
    "SHAPES",
]

SHAPES = ("square", "swiss_roll", "sphere", "torus")


@dataclass
class Graph:
    """Symmetric weighted graph in canonical CSR form."""
    n: int
    row_ptr: np.ndarray   # int64[n+1]
    col: np.ndarray       # int32[nnz]
    w: np.ndarray         # float64[nnz]
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.col.shape[0])

    def degrees(self) -> np.ndarray:
        return np.diff(self.row_ptr)


# ----------------------------------------------------------------------------------
# point samplers (seeded PCG64 streams)
# ----------------------------------------------------------------------------------

def sample_points(shape: str, n: int, seed: int) -> np.ndarray:
    """Draw n seeded points on a manifold.

    square      uniform in the unit square [0,1]^2
    swiss_roll  t ~ U[1.5 pi, 4.5 pi], h ~ U[0, 20], point (t cos t, h, t sin t)
    sphere      uniform on the unit 2-sphere (normalised standard Gaussians)
    torus       uniform (by area) on the torus surface with R = 1, r = 0.4
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    if shape == "square":
        return rng.random((n, 2))
    if shape == "swiss_roll":
        t = rng.uniform(1.5 * math.pi, 4.5 * math.pi, n)
        h = rng.uniform(0.0, 20.0, n)
        return np.stack([t * np.cos(t), h, t * np.sin(t)], axis=1)
    if shape == "sphere":
        g = rng.standard_normal((n, 3))
        return g / np.linalg.norm(g, axis=1, keepdims=True)
    if shape == "torus":
        R, r = 1.0, 0.4
        # tube angle v has area density proportional to (R + r cos v): rejection sampling
        out_v = np.empty(0)
        while out_v.shape[0] < n:
            m = 2 * (n - out_v.shape[0]) + 16
            v = rng.uniform(0.0, 2.0 * math.pi, m)
            acc = rng.uniform(0.0, R + r, m) < (R + r * np.cos(v))
            out_v = np.concatenate([out_v, v[acc]])
        v = out_v[:n]
        u = rng.uniform(0.0, 2.0 * math.pi, n)
        return np.stack([(R + r * np.cos(v)) * np.cos(u),
                         (R + r * np.cos(v)) * np.sin(u),
                         r * np.sin(v)], axis=1)
    raise ValueError(f"unknown shape {shape!r}; expected one of {SHAPES}")


# ----------------------------------------------------------------------------------
# graph assembly helpers
# ----------------------------------------------------------------------------------

def from_edges(n: int, i: np.ndarray, j: np.ndarray, w: np.ndarray, name: str = "") -> Graph:
    """Canonical symmetric CSR from an undirected edge list (each edge listed once or twice).

    Duplicate (i, j) pairs must carry equal weights; self loops are rejected.
    """
    i = np.asarray(i, dtype=np.int64)
    j = np.asarray(j, dtype=np.int64)
    w = np.asarray(w, dtype=np.float64)
    if np.any(i == j):
        raise ValueError("self loops are not allowed")
    ii = np.concatenate([i, j])
    jj = np.concatenate([j, i])
    ww = np.concatenate([w, w])
    key = ii * n + jj
    order = np.argsort(key, kind="stable")
    key, ii, jj, ww = key[order], ii[order], jj[order], ww[order]
    first = np.ones(key.shape[0], dtype=bool)
    first[1:] = key[1:] != key[:-1]
    ii, jj, ww = ii[first], jj[first], ww[first]
    counts = np.bincount(ii, minlength=n)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    return Graph(n, row_ptr, jj.astype(np.int32), ww.copy(), name)


def knn_graph(points: np.ndarray, k: int, name: str = "") -> Graph:
    """Exact symmetric (union) kNN graph with Gaussian weights (see module docstring)."""
    from scipy.spatial import cKDTree

    pts = np.ascontiguousarray(points, dtype=np.float64)
    n = pts.shape[0]
    if n <= k:
        raise ValueError("need more than k points")
    tree = cKDTree(pts)
    d, idx = tree.query(pts, k=k + 1, workers=-1)
    idx = idx.astype(np.int64)
    # drop the point itself; order by (distance, index) for a deterministic tie rule
    rows = np.repeat(np.arange(n, dtype=np.int64), k + 1)
    dd = d.reshape(-1)
    jj = idx.reshape(-1)
    keep = jj != rows
    order = np.lexsort((jj, dd, rows))
    rows, dd, jj, keep = rows[order], dd[order], jj[order], keep[order]
    rows, dd, jj = rows[keep], dd[keep], jj[keep]
    # a row that did not contain itself (duplicate points) keeps k+1 entries: trim to k
    cnt = np.bincount(rows, minlength=n)
    if np.any(cnt != k):
        start = np.zeros(n + 1, dtype=np.int64)
        np.cumsum(cnt, out=start[1:])
        rank = np.arange(rows.shape[0]) - start[rows]
        sel = rank < k
        rows, dd, jj = rows[sel], dd[sel], jj[sel]
    sigma = float(np.mean(dd))
    diff = pts[rows] - pts[jj]
    d2 = np.einsum("ij,ij->i", diff, diff)
    w = np.exp(-d2 / (sigma * sigma))
    g = from_edges(n, rows, jj, w, name or f"knn{k}")
    return g


def manifold_graph(shape: str, n: int, k: int, seed: int) -> Graph:
    """Points of `shape` (seeded) joined into the symmetric k-NN graph."""
    return knn_graph(sample_points(shape, n, seed), k, name=f"{shape}-n{n}-k{k}-s{seed}")


# ----------------------------------------------------------------------------------
# small named graphs (unit weights unless stated)
# ----------------------------------------------------------------------------------

def ring(n: int, weight: float = 1.0) -> Graph:
    """Cycle C_n (the ring of Fig. 2(b) for n = 5)."""
    i = np.arange(n)
    return from_edges(n, i, (i + 1) % n, np.full(n, weight), f"ring{n}")


def path(n: int, weight: float = 1.0) -> Graph:
    """Path P_n (the line of Fig. 2(a) for n = 5)."""
    i = np.arange(n - 1)
    return from_edges(n, i, i + 1, np.full(n - 1, weight), f"path{n}")


def complete(n: int) -> Graph:
    i, j = np.triu_indices(n, 1)
    return from_edges(n, i, j, np.ones(i.shape[0]), f"complete{n}")


def triangle_mesh(rows: int = 4) -> Graph:
    """Triangular mesh with 1, 2, ..., `rows` nodes per row and unit edges.

    rows = 4 gives the 10-node, 18-edge mesh of Fig. 3.
    """
    ids = {}
    for r in range(rows):
        for c in range(r + 1):
            ids[(r, c)] = len(ids)
    ei, ej = [], []
    for (r, c), a in ids.items():
        if (r, c + 1) in ids:
            ei.append(a); ej.append(ids[(r, c + 1)])
        if (r + 1, c) in ids:
            ei.append(a); ej.append(ids[(r + 1, c)])
        if (r + 1, c + 1) in ids:
            ei.append(a); ej.append(ids[(r + 1, c + 1)])
    return from_edges(len(ids), np.array(ei), np.array(ej), np.ones(len(ei)), f"mesh{rows}")


def erdos_renyi(n: int, p: float, seed: int, weighted: bool = True) -> Graph:
    """G(n, p) with seeded uniform(0.5, 1.5) weights (or unit weights)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    i, j = np.triu_indices(n, 1)
    keep = rng.random(i.shape[0]) < p
    i, j = i[keep], j[keep]
    w = rng.uniform(0.5, 1.5, i.shape[0]) if weighted else np.ones(i.shape[0])
    return from_edges(n, i, j, w, f"er{n}-{p}-s{seed}")


def two_components(a: Graph, b: Graph) -> Graph:
    """Disjoint union of two graphs (the second relabelled after the first)."""
    n = a.n + b.n
    ia = np.repeat(np.arange(a.n), np.diff(a.row_ptr))
    ib = np.repeat(np.arange(b.n), np.diff(b.row_ptr)) + a.n
    i = np.concatenate([ia, ib])
    j = np.concatenate([a.col.astype(np.int64), b.col.astype(np.int64) + a.n])
    w = np.concatenate([a.w, b.w])
    return from_edges(n, i, j, w, f"{a.name}+{b.name}")
