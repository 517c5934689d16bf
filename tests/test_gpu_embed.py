"""GPU LOBPCG embedding (Sec. 4.3, Eq. 10-11) against the oracle's dense generalized eigensolver.

Tolerances (the required accuracy of this build): eigenvalues within 1e-6 relative in the
FP64 form and 1e-4 in the FP32 form; eigenvectors within 1e-3 in subspace angle, compared
per cluster of eigenvalues (relative gap < 1e-6 groups a cluster; a cluster that straddles
K is not compared, since only its span inside the first K is defined).
"""
import math

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


def clusters(lam, rel=1e-6):
    groups, cur = [], [0]
    for k in range(1, len(lam)):
        if abs(lam[k] - lam[k - 1]) <= rel * max(abs(lam[k]), 1e-300):
            cur.append(k)
        else:
            groups.append(cur)
            cur = [k]
    groups.append(cur)
    return groups


def compare(lam, V, ref_lam, ref_V, K, lam_tol, angle_tol=1e-3):
    """lam/V from the GPU vs the oracle's first K + 1 pairs."""
    rel = np.abs(lam - ref_lam[:K]) / np.abs(ref_lam[:K])
    assert np.max(rel) <= lam_tol, rel
    for grp in clusters(ref_lam[:K + 1]):
        if grp[-1] >= K:
            continue
        ang = oe.subspace_angle(V[:, grp], ref_V[:, grp])
        assert ang <= angle_tol, (grp, ang)


def test_config_plain_fp64_square_1000(ctx):
    """Plain method, FP64: 1,000 points in the unit square, 8-NN, K = 2, tol 1e-8."""
    g = mg.manifold_graph("square", 1000, 8, 1)
    ref = og.from_graph(g)
    d = oe.dense_geneig(ref.A, ref.b, 3)
    ops = ctx.build(g, precision="fp64")
    lam, V, info, s = ctx.embed(ops, 2, 1e-8, precision="fp64", guard=2)
    assert s == 0
    compare(lam, V, d.lam, d.V, 2, 1e-6)
    eta = oe.backward_errors(ref.A, ref.b, lam, V)
    assert np.all(eta <= 2e-8)
    assert np.allclose(V.T @ (ref.b[:, None] * V), np.eye(2), atol=1e-10)


@pytest.mark.parametrize("shape,n,k,K,guard", [("square", 1000, 8, 2, 2), ("square", 1000, 8, 8, 4),
                                               ("swiss_roll", 3000, 10, 8, 4), ("sphere", 2500, 10, 16, 8),
                                               ("torus", 2000, 12, 4, 4)])
@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_reduced_precision_matches_dense_oracle(ctx, shape, n, k, K, guard, prec):
    """FP32 blocks, and the BF16 form (the preconditioner's blocks in BF16): the same
    tolerances against the oracle's dense generalized eigendecomposition."""
    g = mg.manifold_graph(shape, n, k, 3)
    ref = og.from_graph(g)
    d = oe.dense_geneig(ref.A, ref.b, K + 1)
    ops = ctx.build(g, precision=prec)
    lam, V, info, s = ctx.embed(ops, K, 1e-5, precision=prec, guard=guard)
    assert s == 0, s
    compare(lam, V, d.lam, d.V, K, 1e-4)
    VBV = V.T @ (ref.b[:, None] * V)
    assert np.max(np.abs(VBV - np.eye(K))) < 1e-4


@pytest.mark.parametrize("n", [101, 301])
def test_odd_ring_closed_form(ctx, n):
    ops = ctx.build(mg.ring(n), precision="fp64")
    eps = 2 - 2 * math.cos(2 * math.pi / n)
    assert ops.info().eps == pytest.approx(eps, rel=1e-10)
    lam, V, info, s = ctx.embed(ops, 5, 1e-11, precision="fp64", guard=3)
    t = 2 * np.pi * np.arange(n) / n
    mu = eps / 4
    ref = np.sort((2 - 2 * np.cos(t)) - mu * (2 - 2 * np.cos(2 * t)) + eps)[:5]
    assert np.max(np.abs(lam - ref) / ref) < 1e-8
    # the first vector is the constant (b = 1, eigenvalue eps)
    assert np.ptp(V[:, 0]) < 1e-6 * np.max(np.abs(V[:, 0]))


def test_degenerate_graph_still_embeds(ctx):
    """eps = 0 (even ring): A = L, B = I; the spectrum is the cycle's 2 - 2 cos(2 pi k / n)."""
    n = 200
    ops = ctx.build(mg.ring(n), precision="fp32")
    lam, V, info, s = ctx.embed(ops, 3, 1e-5, precision="fp32", guard=1)
    ref = np.sort(2 - 2 * np.cos(2 * np.pi * np.arange(n) / n))[:3]
    assert abs(lam[0]) < 1e-6
    assert np.max(np.abs(lam[1:] - ref[1:]) / ref[1:]) < 1e-4


def test_laplacian_eigenmaps_special_case(ctx):
    """mu = eps = 0 on a path: (L, B) with b_i proportional to the degree."""
    g = mg.path(400)
    ops = ctx.build(g, precision="fp64", eps=0.0, mu=0.0)
    ref = og.from_graph(g, eps_override=0.0, mu_override=0.0)
    d = oe.dense_geneig(ref.A, ref.b, 5)
    lam, V, info, s = ctx.embed(ops, 4, 1e-11, precision="fp64", guard=4)
    assert abs(lam[0]) < 1e-9
    assert np.max(np.abs(lam[1:] - d.lam[1:4]) / d.lam[1:4]) < 1e-6


def test_sign_convention_and_determinism(ctx):
    g = mg.manifold_graph("square", 1500, 8, 5)
    ops = ctx.build(g, precision="fp32")
    lam1, V1, _, _ = ctx.embed(ops, 4, 1e-5, precision="fp32", guard=4, seed=9)
    lam2, V2, _, _ = ctx.embed(ops, 4, 1e-5, precision="fp32", guard=4, seed=9)
    assert np.array_equal(lam1, lam2) and np.array_equal(V1, V2)
    for k in range(4):
        i = int(np.argmax(np.abs(V1[:, k])))
        assert V1[i, k] > 0


def test_initial_block_is_honoured(ctx):
    """Starting from the converged vectors converges at once to the same pairs."""
    g = mg.manifold_graph("square", 1200, 8, 6)
    ops = ctx.build(g, precision="fp64")
    lam, V, info, s = ctx.embed(ops, 4, 1e-10, precision="fp64", guard=4)
    x0 = np.ascontiguousarray(V.T)                   # [K, n] = column-major n x K
    lam2, V2, info2, s2 = ctx.embed(ops, 4, 1e-9, precision="fp64", guard=4, x0=x0)
    assert info2.iters <= 3
    assert np.allclose(lam2, lam, rtol=1e-9)


def test_not_converged_returns_partial_results(ctx):
    from paper_2112_07862_gb300 import mge
    g = mg.manifold_graph("square", 2000, 8, 7)
    ops = ctx.build(g, precision="fp32")
    lam, V, info, s = ctx.embed(ops, 4, 1e-12, precision="fp32", guard=4, maxiter=5)
    assert s == mge.MGE_ENOTCONVERGED
    assert info.iters == 5
    assert np.all(np.isfinite(lam)) and np.all(np.isfinite(V))


def test_tolerance_below_the_fp32_floor_ends_as_not_converged(ctx):
    """A relative residual of 1e-10 is out of FP32's reach: the solve ends (stagnation or
    maxiter) with MGE_ENOTCONVERGED and its current pairs, which are still accurate."""
    from paper_2112_07862_gb300 import mge
    g = mg.manifold_graph("square", 2000, 8, 7)
    ref = og.from_graph(g)
    d = oe.dense_geneig(ref.A, ref.b, 5)
    ops = ctx.build(g, precision="fp32")
    lam, V, info, s = ctx.embed(ops, 4, 1e-10, precision="fp32", maxiter=3000)
    assert s == mge.MGE_ENOTCONVERGED
    assert np.all(np.isfinite(lam)) and np.all(np.isfinite(V))
    assert np.max(np.abs(lam - d.lam[:4]) / d.lam[:4]) < 1e-4


def test_invalid_embed_arguments(ctx):
    from paper_2112_07862_gb300 import mge
    ops = ctx.build(mg.ring(41), precision="fp64")
    for K, guard in [(0, 0), (20, 8), (30, 0)]:
        with pytest.raises(mge.MgeError) as e:
            ctx.embed(ops, K, 1e-6, guard=guard)
        assert e.value.status == mge.MGE_EINVAL
    small = ctx.build(mg.ring(9), precision="fp64")
    with pytest.raises(mge.MgeError):
        ctx.embed(small, 8, 1e-6)       # n < 2 m
    with pytest.raises(mge.MgeError):
        ctx.embed(ops, 2, -1.0)
