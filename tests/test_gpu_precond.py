"""The LOBPCG preconditioner (Chebyshev polynomial in the Jacobi-scaled L + eps I).

The preconditioner changes how fast LOBPCG converges, never what it converges to: every
degree must give the K smallest generalized eigenpairs of (A, B) within the same tolerances
as the plain Jacobi form (eigenvalues against the oracle's dense solve, subspace angles per
cluster, backward errors recomputed by the oracle), and higher degrees must need fewer
iterations.  Degree 1 is the Jacobi preconditioner.
"""
import numpy as np
import pytest

import manifold_graphs as mg
from oracle import eigen as oe
from oracle import graph_ops as og

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(gpu_lib):
    c = gpu_lib.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def square(ctx):
    g = mg.manifold_graph("square", 2000, 8, 11)
    ref = og.from_graph(g)
    dense = oe.dense_geneig(ref.A, ref.b, 9)
    ops = ctx.build(g, precision="fp64")
    yield g, ref, dense, ops
    ops.close()


def check(lam, V, ref, dense, K, lam_tol, angle_tol, eta_tol):
    rel = np.abs(lam - dense.lam[:K]) / dense.lam[:K]
    assert np.max(rel) <= lam_tol, rel
    ang = oe.subspace_angle(V[:, :K], dense.V[:, :K])
    assert ang <= angle_tol, ang
    eta = oe.backward_errors(ref.A, ref.b, lam, V)
    assert np.all(eta <= eta_tol), eta


@pytest.mark.parametrize("degree", [1, 4, 24])
def test_fp32_same_pairs_at_every_degree(ctx, square, degree):
    g, ref, dense, ops = square
    lam, V, info, s = ctx.embed(ops, 8, 1e-5, precision="fp32", guard=4, precond_degree=degree)
    assert s == 0
    # the 9th eigenvalue is well separated on this graph, so the first 8 span is defined
    check(lam, V, ref, dense, 8, 1e-4, 2e-3, 2e-6)


@pytest.mark.parametrize("degree", [1, 24])
def test_fp64_same_pairs(ctx, square, degree):
    g, ref, dense, ops = square
    lam, V, info, s = ctx.embed(ops, 4, 1e-9, precision="fp64", guard=4, precond_degree=degree)
    assert s == 0
    check(lam, V, ref, dense, 4, 1e-6, 1e-5, 2e-9)


def test_higher_degree_needs_fewer_iterations(ctx, square):
    g, ref, dense, ops = square
    iters = []
    for degree in (1, 8, 24):
        lam, V, info, s = ctx.embed(ops, 8, 1e-5, precision="fp32", guard=4, precond_degree=degree)
        assert s == 0
        iters.append(info.iters)
    assert iters[0] > iters[1] > iters[2], iters


def test_degree_is_clamped_at_64(ctx, square):
    g, ref, dense, ops = square
    lam, V, info, s = ctx.embed(ops, 4, 1e-5, precision="fp32", guard=4, precond_degree=1000)
    assert s == 0
    check(lam, V, ref, dense, 4, 1e-4, 2e-3, 2e-6)


def test_eps_solve_degree(ctx):
    g = mg.manifold_graph("swiss_roll", 4000, 10, 3)
    ref = og.from_graph(g)
    its = []
    for degree in (1, 24):
        ops = ctx.build(g, precision="fp32", eps_precond_degree=degree)
        info = ops.info()
        assert info.eps == pytest.approx(ref.eps, rel=2e-5)
        its.append(info.eps_iters)
        ops.close()
    assert its[1] < its[0], its
