"""Pins for the oracle's betweenness centrality and VBC (Sec. 3.3): closed forms on paths,
stars, complete graphs and odd rings, networkx's Brandes implementation, and a brute-force
enumeration of all shortest paths on a small graph."""
import itertools

import numpy as np
import pytest

import manifold_graphs as mg
from oracle import betweenness as ob


def test_path_closed_form():
    # on P_n node i lies on every path between its i left and n-1-i right neighbours:
    # 2 i (n-1-i) ordered pairs; VBC from those values
    n = 9
    g = mg.path(n)
    cb = ob.betweenness(g.n, g.row_ptr, g.col)
    want = np.array([2.0 * i * (n - 1 - i) for i in range(n)])
    np.testing.assert_array_equal(cb, want)
    assert ob.vbc(cb) == pytest.approx(float(np.var(want)), rel=1e-15)


def test_star_complete_and_odd_ring():
    n = 7
    i = np.zeros(n - 1, dtype=np.int64)
    j = np.arange(1, n)
    star = mg.from_edges(n, i, j, np.ones(n - 1))
    cb = ob.betweenness(star.n, star.row_ptr, star.col)
    assert cb[0] == (n - 1) * (n - 2) and np.all(cb[1:] == 0)   # every ordered leaf pair
    k = mg.complete(6)
    assert np.all(ob.betweenness(k.n, k.row_ptr, k.col) == 0)
    # odd ring C_(2r+1): unique shortest paths; node 0 is interior to the paths between
    # a at distance p on one side and b at distance q on the other with p + q <= r:
    # r (r - 1) / 2 unordered pairs per side pairing -> (n-1)(n-3)/4 ordered
    for n in (5, 9, 15):
        g = mg.ring(n)
        cb = ob.betweenness(g.n, g.row_ptr, g.col)
        np.testing.assert_allclose(cb, (n - 1) * (n - 3) / 4.0)
        assert ob.vbc(cb) == pytest.approx(0.0, abs=1e-20)


def test_matches_networkx():
    nx = pytest.importorskip("networkx")
    for g in (mg.erdos_renyi(60, 0.08, 3), mg.manifold_graph("square", 150, 6, 2), mg.triangle_mesh(5),
              mg.ring(10)):
        cb = ob.betweenness(g.n, g.row_ptr, g.col)
        G = nx.Graph()
        G.add_nodes_from(range(g.n))
        rows = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
        G.add_edges_from(zip(rows.tolist(), g.col.tolist()))
        ref = nx.betweenness_centrality(G, normalized=False)
        np.testing.assert_allclose(cb, [2.0 * ref[v] for v in range(g.n)], rtol=1e-12, atol=1e-12)


def test_brute_force_path_enumeration():
    """All shortest paths of every ordered pair listed explicitly on a small graph."""
    g = mg.erdos_renyi(11, 0.3, 7, weighted=False)
    n = g.n
    adj = [set(g.col[g.row_ptr[v]:g.row_ptr[v + 1]].tolist()) for v in range(n)]
    # hop distances by Floyd-Warshall on the 0/1 adjacency
    D = np.full((n, n), np.inf)
    for v in range(n):
        D[v, v] = 0
        for w in adj[v]:
            D[v, w] = 1
    for m in range(n):
        D = np.minimum(D, D[:, [m]] + D[[m], :])

    def paths(s, t):
        if s == t:
            return [[s]]
        return [[s] + p for w in adj[s] if D[w, t] == D[s, t] - 1 for p in paths(w, t)]

    cb = np.zeros(n)
    for s, t in itertools.permutations(range(n), 2):
        if not np.isfinite(D[s, t]):
            continue
        ps = paths(s, t)
        for v in range(n):
            if v not in (s, t):
                cb[v] += sum(v in p for p in ps) / len(ps)
    np.testing.assert_allclose(ob.betweenness(n, g.row_ptr, g.col), cb, rtol=1e-13, atol=1e-13)
