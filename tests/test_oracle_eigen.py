"""Pins for the oracle's generalized eigensolvers (Eq. 10-11) and its residual measure.

The dense solver is pinned to closed-form spectra (in test_oracle_graph.py) and to an
independent LAPACK generalized routine here; the oracle's textbook LOBPCG is pinned to
the dense solver and to ARPACK shift-invert on larger graphs.
"""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse.linalg as spla

import manifold_graphs as mg
from oracle import graph_ops as go
from oracle import eigen as ge


@pytest.fixture(scope="module")
def square1k():
    return go.from_graph(mg.manifold_graph("square", 1000, 8, 1))


@pytest.fixture(scope="module")
def swiss2k():
    return go.from_graph(mg.manifold_graph("swiss_roll", 2000, 10, 2))


def test_dense_geneig_properties(square1k):
    ops = square1k
    res = ge.dense_geneig(ops.A, ops.b, 8)
    V, lam = res.V, res.lam
    A = ops.A.toarray()
    assert np.allclose(V.T @ (ops.b[:, None] * V), np.eye(8), atol=1e-12)
    assert np.allclose(V.T @ A @ V, np.diag(lam), atol=1e-12)
    eta = ge.backward_errors(ops.A, ops.b, lam, V)
    assert np.all(eta < 1e-13)
    assert np.all(np.diff(lam) >= 0)


def test_dense_geneig_matches_lapack_generalized(square1k):
    ops = square1k
    res = ge.dense_geneig(ops.A, ops.b, 6)
    lam_ref, V_ref = sla.eigh(ops.A.toarray(), np.diag(ops.b), subset_by_index=[0, 5])
    assert np.allclose(res.lam, lam_ref, rtol=1e-12, atol=0)
    for k in range(6):   # separated eigenvalues: vectors agree up to sign
        c = abs(res.V[:, k] @ (ops.b * V_ref[:, k]))
        assert c == pytest.approx(1.0, abs=1e-9)


def test_sign_convention():
    V = np.array([[1.0, -3.0], [-2.0, 3.0], [0.5, 1.0]])
    F = ge.fix_signs(V)
    assert F[1, 0] == 2.0          # largest magnitude positive
    assert F[0, 1] == 3.0          # tie -> lowest index positive


@pytest.mark.parametrize("K,guard", [(2, 2), (4, 0), (8, 4)])
def test_lobpcg_matches_dense(square1k, K, guard):
    ops = square1k
    d = ge.dense_geneig(ops.A, ops.b, K + 1)
    r = ge.lobpcg(ops.A, ops.b, K, guard=guard, tol=1e-12, seed=3)
    assert r.converged
    assert np.max(np.abs(r.lam - d.lam[:K]) / d.lam[:K]) < 1e-10
    assert ge.subspace_angle(r.V, d.V[:, :K]) < 1e-7


def test_lobpcg_swiss_roll_matches_dense(swiss2k):
    ops = swiss2k
    d = ge.dense_geneig(ops.A, ops.b, 9)
    r = ge.lobpcg(ops.A, ops.b, 8, guard=2, tol=1e-12, seed=1)
    assert r.converged
    assert np.max(np.abs(r.lam - d.lam[:8]) / d.lam[:8]) < 1e-9
    assert ge.subspace_angle(r.V, d.V[:, :8]) < 1e-6


def test_lobpcg_with_constraint_gives_fiedler_value(square1k):
    ops = square1k
    n = ops.n
    Y = np.ones((n, 1)) / np.sqrt(n)
    r = ge.lobpcg(ops.Q, np.ones(n), 1, guard=3, Y=Y, tol=1e-13, seed=2)
    assert r.lam[0] == pytest.approx(ops.eps, rel=1e-9)


@pytest.mark.slow
def test_lobpcg_matches_arpack_shift_invert():
    ops = go.from_graph(mg.manifold_graph("swiss_roll", 6000, 10, 5))
    import scipy.sparse as sp
    B = sp.diags(ops.b).tocsc()
    lam_ref = np.sort(spla.eigsh(ops.A.tocsc(), k=6, M=B, sigma=0.0, which="LM",
                                 return_eigenvectors=False))
    r = ge.lobpcg(ops.A, ops.b, 6, guard=2, tol=1e-11, seed=4)
    assert r.converged
    assert np.max(np.abs(r.lam - lam_ref) / lam_ref) < 1e-8


def test_backward_error_detects_perturbation(square1k):
    ops = square1k
    d = ge.dense_geneig(ops.A, ops.b, 3)
    V = d.V.copy()
    V[:, 1] += 1e-4 * np.random.default_rng(0).standard_normal(ops.n)
    eta = ge.backward_errors(ops.A, ops.b, d.lam, V)
    assert eta[0] < 1e-13 and eta[1] > 1e-7


def test_gershgorin_norm_bounds_spectral_norm(square1k):
    ops = square1k
    nA = ge.gershgorin_norm(ops.A)
    top = np.linalg.eigvalsh(ops.A.toarray())[-1]
    assert top <= nA * (1 + 1e-14)


def test_subspace_angle_basic():
    rng = np.random.default_rng(0)
    U = rng.standard_normal((50, 3))
    assert ge.subspace_angle(U, U @ rng.standard_normal((3, 3))) < 1e-12
    e = np.zeros((50, 1)); e[0] = 1
    f = np.zeros((50, 1)); f[0] = np.cos(0.01); f[1] = np.sin(0.01)
    assert ge.subspace_angle(e, f) == pytest.approx(0.01, rel=1e-9)


def test_planted_wrong_b_scaling_breaks_generalized_residual(square1k):
    """Using B^{-1} where B^{-1/2} is needed gives vectors that are not eigenvectors."""
    ops = square1k
    s = 1.0 / ops.b
    C = (ops.A.toarray() * np.sqrt(s)[:, None]) * np.sqrt(s)[None, :]
    lam, U = np.linalg.eigh(C)
    V_bad = U[:, :3] * s[:, None]
    eta = ge.backward_errors(ops.A, ops.b, lam[:3], V_bad)
    assert np.max(eta) > 1e-6


def test_gershgorin_norm_exact_on_hand_computed_matrices():
    """||A||_G = max_i (A_ii + sum_{j != i} |A_ij|), worked by hand:
    rows of [[4,-1,0],[-1,5,-2],[0,-2,3]] give 4+1, 5+3, 3+2 -> 8 (the middle row);
    [[2,0.5,-0.25],[0.5,1,0],[-0.25,0,6]] gives 2.75, 1.5, 6.25 -> 6.25 (the last row,
    so a norm taken from the first row, or doubled, or without the diagonal, fails)."""
    A = np.array([[4.0, -1.0, 0.0], [-1.0, 5.0, -2.0], [0.0, -2.0, 3.0]])
    assert ge.gershgorin_norm(A) == 8.0
    A2 = np.array([[2.0, 0.5, -0.25], [0.5, 1.0, 0.0], [-0.25, 0.0, 6.0]])
    assert ge.gershgorin_norm(A2) == 6.25


def test_sparse_geneig_matches_dense_definition():
    """Shift-invert Lanczos against the dense eigendecomposition of B^-1/2 A B^-1/2."""
    ops = go.from_graph(mg.manifold_graph("swiss_roll", 1500, 10, 9))
    d = ge.dense_geneig(ops.A, ops.b, 6)
    s = ge.sparse_geneig(ops.A, ops.b, 6)
    np.testing.assert_allclose(s.lam, d.lam, rtol=1e-10)
    for j in range(6):
        assert ge.subspace_angle(s.V[:, [j]], d.V[:, [j]]) < 1e-7
    VBV = s.V.T @ (ops.b[:, None] * s.V)
    assert np.max(np.abs(VBV - np.eye(6))) < 1e-10
    assert np.max(ge.backward_errors(ops.A, ops.b, s.lam, s.V)) < 1e-13


def test_sparse_geneig_odd_ring_closed_form():
    """Odd ring C_N (b = 1): lambda_k = (2 - 2cos t) - mu (2 - 2cos 2t) + eps, t = 2 pi k / N,
    eps = 2 - 2cos(2 pi / N) and mu = eps / 4 (the closed form of Sec. 4 on the ring)."""
    N = 4001
    ops = go.build_graph_ops(*_ring_csr(N), eps_override=2 - 2 * np.cos(2 * np.pi / N))
    eps = ops.eps
    mu = eps / 4
    t = 2 * np.pi * np.arange(N) / N
    lam_all = np.sort((2 - 2 * np.cos(t)) - mu * (2 - 2 * np.cos(2 * t)) + eps)
    s = ge.sparse_geneig(ops.A, ops.b, 5)
    np.testing.assert_allclose(s.lam, lam_all[:5], rtol=1e-9)
    assert ops.mu == pytest.approx(mu, rel=1e-12)


def test_fiedler_value_sparse_odd_ring_and_dense():
    N = 4001
    g = mg.ring(N)
    t_ptr, t_col, T = go.two_hop_sets(g.n, g.row_ptr, g.col)
    Q = go.q_matrix(g.n, t_ptr, t_col)
    eps, res = go.fiedler_value_sparse(Q, 1)
    assert eps == pytest.approx(2 - 2 * np.cos(2 * np.pi / N), rel=1e-9)
    assert res < 1e-12
    g2 = mg.manifold_graph("square", 1200, 8, 4)
    t_ptr, t_col, T = go.two_hop_sets(g2.n, g2.row_ptr, g2.col)
    Q2 = go.q_matrix(g2.n, t_ptr, t_col)
    eps2, _ = go.fiedler_value_sparse(Q2, 1)
    assert eps2 == pytest.approx(np.linalg.eigvalsh(Q2.toarray())[1], rel=1e-10)
    assert go.fiedler_value_sparse(Q2, 2) == (0.0, 0.0)


def _ring_csr(N):
    g = mg.ring(N)
    return g.n, g.row_ptr, g.col, g.w


def test_relative_residual_zero_for_exact_pairs_and_scale_invariant(swiss2k):
    ops = swiss2k
    d = ge.dense_geneig(ops.A, ops.b, 5)
    rho = ge.relative_residuals(ops.A, ops.b, d.lam, d.V)
    assert np.max(rho) < 1e-9
    # a perturbation of size delta along another eigenvector gives
    # rho = delta |lam_j - lam_k| / (lam_k sqrt(1 + delta^2)) exactly (B-orthonormal pairs)
    delta = 1e-3
    v = d.V[:, 1] + delta * d.V[:, 3]
    rq = float(v @ (ops.A @ v)) / float(v @ (ops.b * v))
    rho1 = ge.relative_residuals(ops.A, ops.b, np.array([rq]), v[:, None])[0]
    # exact value from the two-term expansion: r = (lam1 - rq) B v1 + delta (lam3 - rq) B v3
    l1, l3 = d.lam[1], d.lam[3]
    rn = np.sqrt((l1 - rq) ** 2 + (delta * (l3 - rq)) ** 2)
    want = rn / ((abs(rq) + 2.0 ** -53 * ge.gershgorin_norm(ops.A)) * np.sqrt(1 + delta ** 2))
    assert rho1 == pytest.approx(want, rel=1e-6)
    # scaling A and lambda together leaves rho unchanged; scaling V leaves it unchanged
    rho2 = ge.relative_residuals(3.0 * ops.A, ops.b, np.array([3.0 * rq]), 7.0 * v[:, None])[0]
    assert rho2 == pytest.approx(rho1, rel=1e-9)


def test_lobpcg_relative_measure_converges_to_the_dense_pairs(swiss2k):
    ops = swiss2k
    d = ge.dense_geneig(ops.A, ops.b, 5)
    r = ge.lobpcg(ops.A, ops.b, 4, guard=2, tol=1e-9, seed=3, measure="relative")
    assert r.converged
    np.testing.assert_allclose(r.lam, d.lam[:4], rtol=1e-12)
    assert np.max(ge.relative_residuals(ops.A, ops.b, r.lam, r.V)) <= 1e-9
