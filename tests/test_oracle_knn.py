"""Pins for the oracle's kNN graph construction (Sec. 5.1): hand-worked examples, the tie
rule, an independent k-d tree and the structural invariants of a union kNN graph."""
import math

import numpy as np
import pytest
from scipy.spatial import cKDTree

import manifold_graphs as mg
from oracle import knn as ok


def test_points_on_a_line_by_hand():
    # x = 0, 1, 3, 6, 10 (y = 0), k = 1: nearest of 0 is 1 (d 1), of 1 is 0 (d 1 < 2),
    # of 3 is 1 (d 2 < 3), of 6 is 3 (d 3 < 4), of 10 is 6 (d 4): the union is the path
    # 0-1-3-6-10; sigma = (1 + 1 + 2 + 3 + 4) / 5 = 2.2
    P = np.array([[0.0, 0.0], [1.0, 0.0], [3.0, 0.0], [6.0, 0.0], [10.0, 0.0]])
    nbr, d2 = ok.knn_lists(P, 1)
    assert nbr[:, 0].tolist() == [1, 0, 1, 2, 3]
    assert d2[:, 0].tolist() == [1.0, 1.0, 4.0, 9.0, 16.0]
    rp, col, w, sigma = ok.knn_graph(P, 1)
    assert sigma == pytest.approx(2.2, rel=1e-15)
    assert rp.tolist() == [0, 1, 3, 5, 7, 8]
    assert col.tolist() == [1, 0, 2, 1, 3, 2, 4, 3]
    want = [math.exp(-d * d / (2.2 * 2.2)) for d in (1, 1, 2, 2, 3, 3, 4, 4)]
    np.testing.assert_allclose(w, want, rtol=1e-15)


def test_ties_go_to_the_lower_index():
    # unit square corners: (0,0) has (1,0) [index 1] and (0,1) [index 2] at distance 1
    P = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0], [1.0, 1.0]])
    nbr, d2 = ok.knn_lists(P, 1)
    assert nbr[:, 0].tolist() == [1, 0, 0, 1]
    nbr2, _ = ok.knn_lists(P, 2)
    assert nbr2.tolist() == [[1, 2], [0, 3], [0, 3], [1, 2]]


@pytest.mark.parametrize("dim,n,k", [(2, 700, 8), (3, 900, 10), (3, 500, 12)])
def test_matches_kd_tree(dim, n, k):
    P = np.random.default_rng(dim * 100 + k).random((n, dim))
    nbr, d2 = ok.knn_lists(P, k)
    dist, idx = cKDTree(P).query(P, k=k + 1)
    assert np.array_equal(nbr, idx[:, 1:])                     # no ties in random data
    np.testing.assert_allclose(np.sqrt(d2), dist[:, 1:], rtol=1e-13)


def test_union_graph_invariants_and_generator_agreement():
    P = mg.sample_points("swiss_roll", 1500, 4)
    k = 10
    rp, col, w, sigma = ok.knn_graph(P, k)
    n = P.shape[0]
    # symmetric, ascending columns, no diagonal, every row holds its own k nearest
    rows = np.repeat(np.arange(n), np.diff(rp))
    A = {(int(a), int(b)): x for a, b, x in zip(rows, col, w)}
    assert all(A[(b, a)] == x for (a, b), x in A.items())
    assert all(np.all(np.diff(col[rp[i]:rp[i + 1]]) > 0) for i in range(n))
    assert not np.any(rows == col)
    nbr, _ = ok.knn_lists(P, k)
    assert all((i, int(j)) in A for i in range(n) for j in nbr[i])
    assert np.all((w > 0) & (w <= 1))
    # the shared input generator (k-d tree) builds the same graph; weights to rounding
    g = mg.knn_graph(P, k)
    assert np.array_equal(g.row_ptr, rp) and np.array_equal(g.col, col)
    np.testing.assert_allclose(g.w, w, rtol=1e-13)


def test_planted_error_in_sigma_is_detected():
    """sigma from squared distances instead of distances changes every weight."""
    P = mg.sample_points("square", 400, 2)
    rp, col, w, sigma = ok.knn_graph(P, 8)
    _, d2 = ok.knn_lists(P, 8)
    wrong = float(np.mean(d2))
    assert abs(wrong - sigma) > 1e-3 * sigma
