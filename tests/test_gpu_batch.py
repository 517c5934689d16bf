"""Batched embedding (mge_embed_batch): several graphs of uneven size and K solved as branches
of one CUDA graph launch.  Each result must be the one mge_embed gives for that graph alone
(eigenvalues to 1e-10 relative, vectors to 1e-8: only the order of floating-point atomics
differs), and one member of the batch is checked against the oracle's dense generalized
eigensolver (Sec. 4.3, Eq. 10-11) with the FP32 tolerances of the single-solve tests."""
import numpy as np
import pytest

import manifold_graphs as mg
from oracle import eigen as oe
from oracle import graph_ops as og

pytestmark = pytest.mark.gpu

GRAPHS = [("square", 3000, 8, 4), ("swiss_roll", 8000, 10, 8), ("torus", 2000, 12, 4),
          ("sphere", 5000, 10, 16), ("square", 1200, 10, 2), ("swiss_roll", 2500, 8, 8)]


@pytest.fixture(scope="module")
def ctx(gpu_lib):
    c = gpu_lib.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("precision,tol", [("fp32", 1e-5), ("bf16", 1e-5), ("fp64", 1e-9)])
def test_batch_equals_alone(ctx, precision, tol):
    graphs = [(mg.manifold_graph(s, n, k, 20 + i), K) for i, (s, n, k, K) in enumerate(GRAPHS)]
    ops = [ctx.build(g, precision=precision) for g, _ in graphs]
    alone = [ctx.embed(o, K, tol, precision=precision, guard=2) for o, (_, K) in zip(ops, graphs)]
    lams, Vs, infos, s = ctx.embed_batch(ops, [K for _, K in graphs], tol, precision=precision, guard=2)
    assert s == 0
    for (g, K), (lam0, V0, i0, s0), lam, V, info in zip(graphs, alone, lams, Vs, infos):
        assert s0 == 0 and info.status == 0
        assert V.shape == (g.n, K)
        assert np.allclose(lam, lam0, rtol=1e-10, atol=0), (lam, lam0)
        assert np.max(np.abs(V - V0)) < 1e-8
        assert abs(info.iters - i0.iters) <= 1
        assert np.all(np.asarray(info.resid[:K]) <= tol)
    for o in ops:
        o.close()


def test_batch_member_matches_dense_oracle(ctx):
    g = mg.manifold_graph("square", 1500, 8, 7)
    ref = og.from_graph(g)
    d = oe.dense_geneig(ref.A, ref.b, 5)
    big = mg.manifold_graph("swiss_roll", 6000, 10, 8)
    ops = [ctx.build(big, precision="fp32"), ctx.build(g, precision="fp32")]
    lams, Vs, infos, s = ctx.embed_batch(ops, [8, 4], 1e-5, precision="fp32", guard=4)
    assert s == 0
    lam, V = lams[1], Vs[1]
    assert np.max(np.abs(lam - d.lam[:4]) / d.lam[:4]) <= 1e-4
    assert oe.subspace_angle(V, d.V[:, :4]) <= 1e-3
    eta = oe.backward_errors(ref.A, ref.b, lam, V)
    assert np.all(eta <= 1e-6)
    for o in ops:
        o.close()


def test_batch_rejects_bad_arguments(ctx, gpu_lib):
    mge = gpu_lib
    g = mg.manifold_graph("square", 1000, 8, 3)
    ops = ctx.build(g, precision="fp32")
    with pytest.raises(mge.MgeError) as e:
        mge.mge_embed_batch(ctx.h, [ops.h], [40], 1e-6, mge.embed_opts("fp32"))
    assert e.value.status == mge.MGE_EINVAL
    x0 = np.zeros((2, g.n))
    with pytest.raises(mge.MgeError) as e:
        mge.mge_embed_batch(ctx.h, [ops.h], [2], 1e-6, mge.embed_opts("fp32", x0=x0))
    assert e.value.status == mge.MGE_EINVAL
    assert mge.load().mge_embed_batch(ctx.h, 0, None, None, 1e-6, None, None, None, None) == mge.MGE_EINVAL
    ops.close()


def test_batch_build_equals_single_builds(ctx):
    """mge_build_graph_ops_batch (builds on several host threads and streams at once) gives
    each graph the operators mge_build_graph_ops gives it alone: the integer structure and
    T bit for bit, eps and the values up to the order of the eps solve's atomics."""
    graphs = [mg.manifold_graph(s, n, k, 40 + i) for i, (s, n, k, _) in enumerate(GRAPHS)]
    graphs.append(mg.ring(10))                       # even ring: two-hop graph disconnected
    single = [ctx.build(g, precision="fp32") for g in graphs]
    batch = ctx.build_batch(graphs, workers=3, precision="fp32")
    for g, a, b in zip(graphs, single, batch):
        assert b.h is not None and b.status == a.status
        ea, eb = a.export(), b.export()
        for key in ("a_ptr", "a_col", "T"):
            assert np.array_equal(ea[key], eb[key]), key
        ia, ib = a.info(), b.info()
        assert ib.eps == pytest.approx(ia.eps, rel=1e-9, abs=1e-300)
        assert ib.mu == pytest.approx(ia.mu, rel=1e-9, abs=1e-300)
        assert np.allclose(eb["a_val"], ea["a_val"], rtol=1e-9, atol=1e-15)
        assert np.allclose(eb["b"], ea["b"], rtol=1e-9, atol=0)
    for o in single + batch:
        o.close()
