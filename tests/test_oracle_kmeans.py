"""Pins for the oracle's k-means (Sec. 5.2): a hand-worked run, the tie rule, scikit-learn's
Lloyd iteration from the same initial centres, and the monotone decrease of the inertia."""
import numpy as np
import pytest

from oracle import kmeans as okm


def test_hand_worked_run():
    # points 0, 1, 10, 11 on a line; centres start at 0 and 1.
    # step 1: 0 -> c0; 1, 10, 11 -> c1 (10: 81 < 100); centres 0 and 22/3
    # step 2: 0, 1 -> c0 (1 < 40.1); 10, 11 -> c1; centres 0.5 and 10.5
    # step 3: no change -> stop
    X = np.array([[0.0, 0.0], [1.0, 0.0], [10.0, 0.0], [11.0, 0.0]])
    a, C, steps = okm.kmeans(X, np.array([[0.0, 0.0], [1.0, 0.0]]), 10)
    assert a.tolist() == [0, 0, 1, 1]
    assert C.tolist() == [[0.5, 0.0], [10.5, 0.0]]
    assert steps == 3
    a1, C1, s1 = okm.kmeans(X, np.array([[0.0, 0.0], [1.0, 0.0]]), 1)
    assert a1.tolist() == [0, 1, 1, 1] and s1 == 1
    assert C1[1, 0] == pytest.approx(22.0 / 3.0, rel=1e-15)


def test_ties_go_to_the_lower_centre():
    X = np.array([[0.5, 0.0], [2.0, 0.0]])
    a = okm.assign(X, np.array([[1.0, 0.0], [0.0, 0.0]]))
    assert a.tolist() == [0, 0]                 # 0.5 is equidistant: lower index wins
    a = okm.assign(X, np.array([[0.0, 0.0], [1.0, 0.0]]))
    assert a.tolist() == [0, 1]


def test_empty_cluster_keeps_its_centre():
    X = np.array([[0.0, 0.0], [0.1, 0.0]])
    C0 = np.array([[0.0, 0.0], [100.0, 100.0]])
    a, C, _ = okm.kmeans(X, C0, 5)
    assert a.tolist() == [0, 0]
    assert C[1].tolist() == [100.0, 100.0]
    assert C[0].tolist() == [0.05, 0.0]


def test_matches_scikit_learn_lloyd():
    sk = pytest.importorskip("sklearn.cluster")
    rng = np.random.default_rng(3)
    X = np.concatenate([rng.normal(m, 0.3, (300, 4)) for m in (-2.0, 0.0, 2.0, 4.0)])
    C0 = X[rng.choice(X.shape[0], 4, replace=False)]
    a, C, steps = okm.kmeans(X, C0, 50)
    km = sk.KMeans(n_clusters=4, init=C0, n_init=1, max_iter=50, tol=0.0, algorithm="lloyd").fit(X)
    assert np.array_equal(a, km.labels_)
    np.testing.assert_allclose(C, km.cluster_centers_, rtol=1e-12, atol=1e-14)


def test_inertia_never_increases():
    rng = np.random.default_rng(8)
    X = rng.random((500, 3))
    C = X[:6].copy()
    prev = np.inf
    for _ in range(15):
        a = okm.assign(X, C)
        val = okm.inertia(X, a, C)
        assert val <= prev * (1 + 1e-12)
        prev = val
        C = okm.update(X, a, C)


def test_planted_wrong_count_is_detected():
    X = np.array([[0.0], [2.0], [10.0]])
    a = np.array([0, 0, 1], dtype=np.int32)
    C = okm.update(X, a, np.zeros((2, 1)))
    assert C[:, 0].tolist() == [1.0, 10.0]
    assert C[0, 0] != 2.0 / 3.0                  # a divisor off by one would give 2/3
