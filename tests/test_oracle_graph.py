"""Pins for the oracle's operator build (Sec. 3-4) against brute force, closed forms and invariants.

Each test checks the oracle against something other than itself: a pure-Python
breadth-first enumeration, the closed form of the odd ring, the Gershgorin definition
of mu (Eq. 7) rather than its solved form (Eq. 9), the GLR identity (Eq. 1), or a
structural invariant.  Planted mistakes at the end show the pins catch plausible bugs.
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp

import manifold_graphs as mg
from oracle import graph_ops as go
from oracle import eigen as ge


def brute_two_hop(g):
    """T_i by walking adjacency lists in plain Python."""
    adj = [set(g.col[g.row_ptr[i]:g.row_ptr[i + 1]].tolist()) for i in range(g.n)]
    out = []
    for i in range(g.n):
        s = set()
        for m in adj[i]:
            s |= adj[m]
        s.discard(i)
        s -= adj[i]
        out.append(sorted(s))
    return out


SMALL = [mg.ring(5), mg.ring(6), mg.ring(11), mg.path(5), mg.path(9), mg.triangle_mesh(),
         mg.complete(6), mg.erdos_renyi(30, 0.1, 1), mg.erdos_renyi(40, 0.2, 2),
         mg.erdos_renyi(25, 0.05, 3), mg.two_components(mg.ring(7), mg.path(6)),
         mg.manifold_graph("square", 60, 4, 7)]


@pytest.mark.parametrize("g", SMALL, ids=lambda g: g.name)
def test_two_hop_matches_brute_force(g):
    t_ptr, t_col, T = go.two_hop_sets(g.n, g.row_ptr, g.col)
    ref = brute_two_hop(g)
    for i in range(g.n):
        assert t_col[t_ptr[i]:t_ptr[i + 1]].tolist() == ref[i]
    assert T.tolist() == [len(r) for r in ref]


@pytest.mark.parametrize("g", SMALL, ids=lambda g: g.name)
def test_two_hop_symmetric_and_disjoint_from_edges(g):
    t_ptr, t_col, _ = go.two_hop_sets(g.n, g.row_ptr, g.col)
    Tm = sp.csr_matrix((np.ones(t_col.shape[0]), t_col, t_ptr), shape=(g.n, g.n))
    assert (Tm - Tm.T).nnz == 0
    S = go.pattern(g.n, g.row_ptr, g.col)
    assert Tm.multiply(S).nnz == 0
    assert np.all(Tm.diagonal() == 0)


def test_mesh_two_hop_sets_by_hand():
    # rows of the Fig. 3 mesh: 0 | 1 2 | 3 4 5 | 6 7 8 9
    g = mg.triangle_mesh()
    t_ptr, t_col, T = go.two_hop_sets(g.n, g.row_ptr, g.col)
    assert g.nnz == 36  # 18 undirected edges
    assert t_col[t_ptr[0]:t_ptr[1]].tolist() == [3, 4, 5]
    assert t_col[t_ptr[6]:t_ptr[7]].tolist() == [1, 4, 8]
    assert t_col[t_ptr[4]:t_ptr[5]].tolist() == [0, 6, 9]


@pytest.mark.parametrize("g", SMALL, ids=lambda g: g.name)
def test_q_quadratic_form_is_scaled_two_hop_distance(g):
    """x^T Q x = sum_i (1/T_i) sum_{j in T_i} (x_i - x_j)^2 (Laplacian reading of Eq. 5)."""
    ref = brute_two_hop(g)
    Q = go.q_matrix(g.n, *go.two_hop_sets(g.n, g.row_ptr, g.col)[:2])
    rng = np.random.default_rng(0)
    for _ in range(3):
        x = rng.standard_normal(g.n)
        direct = sum(sum((x[i] - x[j]) ** 2 for j in ref[i]) / len(ref[i])
                     for i in range(g.n) if ref[i])
        assert x @ (Q @ x) == pytest.approx(direct, rel=1e-12, abs=1e-12)


@pytest.mark.parametrize("g", SMALL, ids=lambda g: g.name)
def test_q_is_a_laplacian(g):
    t_ptr, t_col, T = go.two_hop_sets(g.n, g.row_ptr, g.col)
    Q = go.q_matrix(g.n, t_ptr, t_col)
    assert abs(Q - Q.T).max() == 0 if Q.nnz else True
    assert np.max(np.abs(Q @ np.ones(g.n))) < 1e-13
    ev = np.linalg.eigvalsh(Q.toarray())
    assert ev[0] > -1e-12
    # off-diagonal entries are -(1/T_i + 1/T_j), diagonal = 1 + sum_{j in T_i} 1/T_j
    Qc = Q.tocoo()
    for i, j, v in zip(Qc.row, Qc.col, Qc.data):
        if i != j:
            assert v == pytest.approx(-(1.0 / T[i] + 1.0 / T[j]), rel=1e-15)
        else:
            js = t_col[t_ptr[i]:t_ptr[i + 1]]
            assert v == pytest.approx(1.0 + np.sum(1.0 / T[js]), rel=1e-14)


@pytest.mark.parametrize("g", SMALL, ids=lambda g: g.name)
def test_laplacian_glr_identity(g):
    """Eq. 1: x^T L x = sum over edges W_ij (x_i - x_j)^2, each edge once."""
    L = go.laplacian(g.n, g.row_ptr, g.col, g.w)
    x = np.random.default_rng(1).standard_normal(g.n)
    rows = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
    once = rows < g.col
    direct = np.sum(g.w[once] * (x[rows[once]] - x[g.col[once]]) ** 2)
    assert x @ (L @ x) == pytest.approx(direct, rel=1e-12)


@pytest.mark.parametrize("n", [5, 7, 9, 13, 21, 101])
def test_odd_ring_closed_form(n):
    """Whole pipeline on C_n, n odd: T_i = {i +- 2}, Q = step-2 cycle Laplacian,
    eps = 2 - 2 cos(2 pi / n), mu = eps / 4, b = 1, and
    lambda_k = (2 - 2 cos t_k) - mu (2 - 2 cos 2 t_k) + eps with t_k = 2 pi k / n."""
    ops = go.from_graph(mg.ring(n))
    for i in range(n):
        assert ops.t_col[ops.t_ptr[i]:ops.t_ptr[i + 1]].tolist() == sorted({(i + 2) % n, (i - 2) % n})
    eps = 2 - 2 * math.cos(2 * math.pi / n)
    assert ops.eps == pytest.approx(eps, rel=1e-12)
    assert ops.mu == pytest.approx(eps / 4, rel=1e-12)
    assert np.allclose(ops.b, 1.0, rtol=0, atol=1e-14)
    t = 2 * np.pi * np.arange(n) / n
    lam = np.sort((2 - 2 * np.cos(t)) - ops.mu * (2 - 2 * np.cos(2 * t)) + ops.eps)
    res = ge.dense_geneig(ops.A, ops.b)
    assert np.max(np.abs(res.lam - lam)) < 1e-13
    # the first generalized eigenvector is constant with eigenvalue eps (b = 1)
    assert res.lam[0] == pytest.approx(eps, rel=1e-12)
    assert np.ptp(res.V[:, 0]) < 1e-12


@pytest.mark.parametrize("n", [6, 8, 12])
def test_even_ring_is_degenerate(n):
    ops = go.from_graph(mg.ring(n))
    assert ops.degenerate and ops.eps == 0.0 and ops.mu == 0.0
    assert abs(ops.A - ops.L).max() == 0


def test_complete_graph_has_no_two_hop_sets():
    ops = go.from_graph(mg.complete(7))
    assert np.all(ops.T == 0) and ops.Q.nnz == 0
    assert ops.eps == 0.0 and ops.mu == 0.0 and ops.degenerate


@pytest.mark.parametrize("n", [5, 10, 33])
def test_path_laplacian_spectrum(n):
    """mu = eps = 0, B = I: the textbook path spectrum 2 - 2 cos(pi k / n)."""
    ops = go.from_graph(mg.path(n), eps_override=0.0, mu_override=0.0)
    res = ge.dense_geneig(ops.A, np.ones(n))
    ref = 2 - 2 * np.cos(np.pi * np.arange(n) / n)
    assert np.max(np.abs(res.lam - ref)) < 1e-13


@pytest.mark.parametrize("n", [7, 10])
def test_ring_laplacian_spectrum_with_overrides(n):
    ops = go.from_graph(mg.ring(n), eps_override=0.0, mu_override=0.0)
    res = ge.dense_geneig(ops.A, ops.b)
    ref = np.sort(2 - 2 * np.cos(2 * np.pi * np.arange(n) / n))
    assert np.max(np.abs(res.lam - ref)) < 1e-13


MANIFOLD = [mg.triangle_mesh(), mg.manifold_graph("square", 300, 8, 1),
            mg.manifold_graph("swiss_roll", 400, 10, 2), mg.manifold_graph("sphere", 300, 10, 3),
            mg.manifold_graph("torus", 300, 8, 4), mg.erdos_renyi(60, 0.15, 5)]


@pytest.mark.parametrize("g", MANIFOLD, ids=lambda g: g.name)
def test_operator_invariants(g):
    ops = go.from_graph(g)
    A = ops.A
    assert abs(A - A.T).max() < 1e-15
    # A 1 = eps 1 (L 1 = Q 1 = 0)
    assert np.max(np.abs(A @ np.ones(g.n) - ops.eps)) < 1e-12
    # Gershgorin left ends are >= 0 and touch 0 at the row that sets mu (Eq. 7)
    left = A.diagonal() - ops.r
    assert np.min(left) > -1e-12
    if ops.eps > 0:
        assert np.min(left) < 1e-12
    # r_i / b_i is the same for every node and prod b_i = 1 (Sec. 4.3)
    ratio = ops.r / ops.b
    assert np.ptp(ratio) < 1e-12 * ratio.max()
    assert abs(np.sum(np.log(ops.b))) < 1e-10
    # supports of L and Q are disjoint off the diagonal (Sec. 4.2)
    Loff = ops.L - sp.diags(ops.L.diagonal())
    Qoff = ops.Q - sp.diags(ops.Q.diagonal())
    assert abs(Loff).multiply(abs(Qoff)).nnz == 0 or abs(Loff).multiply(abs(Qoff)).max() == 0
    # eps is the Fiedler value: Q's spectrum has one zero and eps next
    ev = np.linalg.eigvalsh(ops.Q.toarray())
    assert ev[1] == pytest.approx(ops.eps, rel=1e-10)


@pytest.mark.parametrize("g", MANIFOLD[:4], ids=lambda g: g.name)
def test_a_quadratic_form_by_brute_force(g):
    """Eq. 6 with the per-node split of Eq. 12: x^T A x = sum over edges w_ij (x_i - x_j)^2
    - mu sum_i (1/T_i) sum_{j in T_i} (x_i - x_j)^2 + eps |x|^2, the sums taken in plain
    Python over the adjacency lists and brute-force two-hop sets (the Laplacian reading of
    Eq. 5), against the oracle's assembled A."""
    ops = go.from_graph(g)
    ref = brute_two_hop(g)
    x = np.random.default_rng(5).standard_normal(g.n)
    glr = 0.0
    for i in range(g.n):
        for p in range(g.row_ptr[i], g.row_ptr[i + 1]):
            j = int(g.col[p])
            if i < j:
                glr += g.w[p] * (x[i] - x[j]) ** 2
    two_hop = sum(sum((x[i] - x[j]) ** 2 for j in ref[i]) / len(ref[i]) for i in range(g.n) if ref[i])
    direct = glr - ops.mu * two_hop + ops.eps * float(x @ x)
    assert x @ (ops.A @ x) == pytest.approx(direct, rel=1e-11)


@pytest.mark.parametrize("g", MANIFOLD, ids=lambda g: g.name)
def test_mu_is_largest_value_keeping_discs_nonnegative(g):
    """Eq. 7 directly: every disc left end of L - mu Q + eps I is >= 0 at mu, and some
    goes negative just above mu."""
    ops = go.from_graph(g)
    n = g.n

    def min_left_end(mu):
        A = (ops.L - mu * ops.Q + ops.eps * sp.identity(n)).toarray()
        d = np.diag(A)
        r = np.sum(np.abs(A), axis=1) - np.abs(d)
        return np.min(d - r)

    assert min_left_end(ops.mu) > -1e-12
    assert min_left_end(ops.mu * (1 + 1e-6)) < 0


def test_structure_of_a_is_diag_edges_two_hop():
    g = mg.manifold_graph("square", 200, 8, 3)
    ops = go.from_graph(g)
    ref = brute_two_hop(g)
    for i in range(g.n):
        nb = set(g.col[g.row_ptr[i]:g.row_ptr[i + 1]].tolist())
        want = sorted(nb | set(ref[i]) | {i})
        assert ops.a_col[ops.a_ptr[i]:ops.a_ptr[i + 1]].tolist() == want


def test_isolated_node_is_an_error():
    g = mg.from_edges(4, np.array([0, 1]), np.array([1, 2]), np.ones(2))   # node 3 isolated
    with pytest.raises(ValueError):
        go.from_graph(g)


def test_fiedler_by_lobpcg_matches_dense(monkeypatch):
    g = mg.manifold_graph("square", 700, 8, 11)
    ops = go.from_graph(g)
    monkeypatch.setattr(go, "DENSE_MAX", 100)
    ops2 = go.from_graph(g, eps_tol=1e-13)
    assert ops2.eps == pytest.approx(ops.eps, rel=1e-8)


# ---- planted mistakes: each must break at least one pin above ------------------------

def test_planted_literal_theta_breaks_ring_closed_form():
    ops = go.from_graph(mg.ring(9), reading="literal")
    eps = 2 - 2 * math.cos(2 * math.pi / 9)
    assert not np.isclose(ops.eps, eps, rtol=1e-6)


def test_planted_dropped_eps_term_breaks_invariant():
    g = mg.manifold_graph("square", 300, 8, 1)
    ops = go.from_graph(g)
    A_bad = ops.L - ops.mu * ops.Q          # forgot + eps I
    assert np.max(np.abs(A_bad @ np.ones(g.n) - ops.eps)) > 1e-6


def test_planted_transposed_two_hop_rule_breaks_brute_force():
    g = mg.erdos_renyi(30, 0.1, 1)
    S = go.pattern(g.n, g.row_ptr, g.col)
    bad = (S @ S).tocsr()          # forgot to remove 1-hop neighbours and the diagonal
    bad.sort_indices()
    ref = brute_two_hop(g)
    assert any(bad.indices[bad.indptr[i]:bad.indptr[i + 1]].tolist() != ref[i] for i in range(g.n))


def test_planted_sign_of_mu_q_breaks_quadratic_form_pin():
    """A = L + mu Q + eps I (wrong sign of the two-hop term) keeps A 1 = eps 1 and symmetry,
    but the brute-force quadratic form of Eq. 6 / Eq. 12 catches it."""
    g = mg.manifold_graph("square", 300, 8, 1)
    ops = go.from_graph(g)
    ref = brute_two_hop(g)
    A_bad = (ops.L + ops.mu * ops.Q + ops.eps * sp.identity(g.n)).tocsr()
    assert np.max(np.abs(A_bad @ np.ones(g.n) - ops.eps)) < 1e-12
    x = np.random.default_rng(5).standard_normal(g.n)
    rows = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
    once = rows < g.col
    glr = float(np.sum(g.w[once] * (x[rows[once]] - x[g.col[once]]) ** 2))
    two_hop = sum(sum((x[i] - x[j]) ** 2 for j in ref[i]) / len(ref[i]) for i in range(g.n) if ref[i])
    direct = glr - ops.mu * two_hop + ops.eps * float(x @ x)
    assert x @ (A_bad @ x) != pytest.approx(direct, rel=1e-6)
