"""GPU operator build (Sec. 4) against the oracle: structure bit-exact, values within rounding.

Tolerances: CSR structure (row pointers, ascending columns, explicit diagonal) and the
two-hop counts T_i are compared bit for bit.  FP64 values are sums of at most a row's worth
of terms in a different order than the oracle's assembly, so they agree to a few ulp times
the row length; the tests use 1e-13 relative.  eps comes from two different eigensolvers
(dense in the oracle, LOBPCG on the GPU): 1e-9 relative in FP64, 2e-5 in FP32 (the default
relative-residual tolerances, 1e-10 and 1e-5, bound eps's error far below these).  mu, A's two-hop values and b
inherit eps's relative error.
"""
import numpy as np
import pytest
import torch

import manifold_graphs as mg
from oracle import graph_ops as og

pytestmark = pytest.mark.gpu

GRAPHS = [mg.triangle_mesh(), mg.ring(9), mg.ring(31), mg.path(12), mg.erdos_renyi(60, 0.15, 5),
          mg.erdos_renyi(200, 0.05, 6), mg.manifold_graph("square", 600, 8, 1),
          mg.manifold_graph("swiss_roll", 1500, 10, 2), mg.manifold_graph("sphere", 1200, 10, 3),
          mg.manifold_graph("torus", 1000, 12, 4)]


def hub_graph(n=1300):
    """Every row's candidate list exceeds a warp's buffer: exercises the bitmap path."""
    i = np.arange(n - 1)
    gi = np.concatenate([i, i[:-1]])
    gj = np.concatenate([np.full(n - 1, n - 1), i[1:]])
    return mg.from_edges(n, gi, gj, np.ones(gi.shape[0]), "hub")


@pytest.fixture(scope="module")
def ctx(gpu_lib):
    c = gpu_lib.Context(0)
    yield c
    c.close()


def check_structure(ex, ref):
    assert np.array_equal(ex["a_ptr"], ref.a_ptr)
    assert np.array_equal(ex["a_col"], ref.a_col)
    assert np.array_equal(ex["T"], ref.T)
    qp = np.zeros(ref.n + 1, np.int64)
    np.cumsum(1 + ref.T, out=qp[1:])
    assert np.array_equal(ex["q_ptr"], qp)
    for i in range(0, ref.n, max(1, ref.n // 50)):
        cols = ex["q_col"][ex["q_ptr"][i]:ex["q_ptr"][i + 1]]
        want = sorted(set(ref.t_col[ref.t_ptr[i]:ref.t_ptr[i + 1]].tolist()) | {i})
        assert cols.tolist() == want


@pytest.mark.parametrize("g", GRAPHS, ids=lambda g: g.name)
def test_fp64_build_matches_oracle(ctx, g):
    ref = og.from_graph(g)
    ops = ctx.build(g, precision="fp64")
    ex = ops.export()
    info = ops.info()
    check_structure(ex, ref)
    assert info.degenerate == int(ref.degenerate)
    assert info.eps == pytest.approx(ref.eps, rel=1e-9, abs=1e-14)
    assert info.mu == pytest.approx(ref.mu, rel=1e-9, abs=1e-14)
    # values: with the oracle's eps the comparison is at rounding level
    ops2 = ctx.build(g, precision="fp64", eps=ref.eps)
    ex2 = ops2.export()
    np.testing.assert_allclose(ex2["a_val"], ref.a_val, rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(ex2["b"], ref.b, rtol=1e-12)
    Q = ref.Q.tocsr()
    qv = np.array([Q[i, j] for i, j in zip(np.repeat(np.arange(g.n), np.diff(ex2["q_ptr"])), ex2["q_col"])])
    np.testing.assert_allclose(ex2["q_val"], qv, rtol=1e-13, atol=1e-15)
    ops.close()
    ops2.close()


def test_bitmap_path_and_degenerate_status(ctx):
    from paper_2112_07862_gb300 import mge
    g = hub_graph()
    ref = og.from_graph(g)
    ops = ctx.build(g, precision="fp64")
    assert ops.status == mge.MGE_EDEGENERATE
    check_structure(ops.export(), ref)


@pytest.mark.parametrize("n", [6, 8, 20])
def test_even_ring_is_degenerate(ctx, n):
    from paper_2112_07862_gb300 import mge
    ops = ctx.build(mg.ring(n), precision="fp32")
    info = ops.info()
    assert ops.status == mge.MGE_EDEGENERATE and info.degenerate == 1
    assert info.eps == 0.0 and info.mu == 0.0 and info.two_hop_components == 2


def test_complete_graph_is_degenerate(ctx):
    from paper_2112_07862_gb300 import mge
    ops = ctx.build(mg.complete(9), precision="fp64")
    info = ops.info()
    assert ops.status == mge.MGE_EDEGENERATE and info.eps == 0.0 and info.two_hop_components == 9
    assert np.all(ops.export()["T"] == 0)


@pytest.mark.parametrize("shape,n,k", [("square", 3000, 8), ("swiss_roll", 4000, 10)])
def test_fp32_eps_within_tolerance(ctx, shape, n, k):
    g = mg.manifold_graph(shape, n, k, 7)
    ref = og.from_graph(g)
    ops = ctx.build(g, precision="fp32")
    info = ops.info()
    check_structure(ops.export(), ref)
    assert info.eps == pytest.approx(ref.eps, rel=2e-5)
    assert info.mu == pytest.approx(ref.mu, rel=2e-5)


def test_device_inputs_give_the_same_operators(ctx):
    from paper_2112_07862_gb300 import mge
    g = mg.manifold_graph("square", 800, 8, 2)
    rp = torch.from_numpy(g.row_ptr).cuda()
    col = torch.from_numpy(g.col).cuda()
    w = torch.from_numpy(g.w).cuda()
    h, s = mge.mge_build_graph_ops(ctx.h, g.n, rp, col, w, True, mge.ops_opts("fp64"))
    dev = mge.Ops(h, s)
    host = ctx.build(g, precision="fp64")
    a, b = dev.export(), host.export()
    for k in a:
        assert np.array_equal(a[k], b[k]), k


def test_malformed_inputs_are_rejected(ctx):
    from paper_2112_07862_gb300 import mge
    g = mg.ring(10)
    bad = g.col.copy()
    bad[0], bad[1] = bad[1], bad[0]               # unsorted row
    with pytest.raises(mge.MgeError) as e:
        mge.mge_build_graph_ops(ctx.h, g.n, g.row_ptr, bad, g.w)
    assert e.value.status == mge.MGE_EINVAL
    w = g.w.copy()
    w[0] = 2.0                                      # W_01 != W_10
    with pytest.raises(mge.MgeError) as e:
        mge.mge_build_graph_ops(ctx.h, g.n, g.row_ptr, g.col, w)
    assert e.value.status == mge.MGE_ENOTSYM
    w = g.w.copy()
    w[3] = -1.0
    with pytest.raises(mge.MgeError) as e:
        mge.mge_build_graph_ops(ctx.h, g.n, g.row_ptr, g.col, w)
    assert e.value.status == mge.MGE_EINVAL
    rp = g.row_ptr.copy()
    rp[5] = rp[6] + 3                               # non-monotone row pointers
    with pytest.raises(mge.MgeError) as e:
        mge.mge_build_graph_ops(ctx.h, g.n, rp, g.col, g.w)
    assert e.value.status == mge.MGE_EINVAL


def test_isolated_node_is_an_error(ctx):
    from paper_2112_07862_gb300 import mge
    g = mg.from_edges(6, np.array([0, 1, 2, 3]), np.array([1, 2, 3, 4]), np.ones(4))   # node 5 isolated
    with pytest.raises(mge.MgeError) as e:
        mge.mge_build_graph_ops(ctx.h, g.n, g.row_ptr, g.col, g.w, False, mge.ops_opts("fp64"))
    assert e.value.status == mge.MGE_EISOLATED


def test_empty_graph_and_tiny_inputs(ctx):
    from paper_2112_07862_gb300 import mge
    with pytest.raises(mge.MgeError) as e:
        mge.mge_build_graph_ops(ctx.h, 0, np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0))
    assert e.value.status == mge.MGE_EINVAL
    # one edge: both nodes have r_i > 0, no two-hop sets, eps forced to 0
    g = mg.path(2)
    ops = ctx.build(g, precision="fp64")
    assert ops.status == mge.MGE_EDEGENERATE
    assert ops.info().nnz_a == 4


def test_ops_handle_may_outlive_its_context(gpu_lib):
    c = gpu_lib.Context(0)
    ops = c.build(mg.ring(31), precision="fp64")
    c.close()
    ex = ops.export()                 # still readable after the context is gone
    assert ex["a_ptr"][-1] == ops.info().nnz_a
    ops.close()                       # releases its device memory and the context's host object
