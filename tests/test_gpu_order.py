"""The library's node order (locality renumbering at build time).

The operators are renumbered so that SpMM tiles hold compact patches of the graph; the
numbering is an internal layout and must not show at the API: exported operators, products
and eigenvectors are in the caller's order and agree with a build that keeps that order
(keep_order=1), and both agree with the oracle.  The order itself must be a permutation,
deterministic, and must cut the distinct neighbour rows per 128-row tile.
"""
import numpy as np
import pytest
import torch

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
def roll():
    return mg.manifold_graph("swiss_roll", 20000, 10, 2)


def tile_distinct(g, order):
    """Distinct column indices per 128-row tile, over the nonzeros, for rows in `order`."""
    rank = np.empty(g.n, np.int64)
    rank[order] = np.arange(g.n)
    rows = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
    key = (rank[rows] // 128) * g.n + rank[g.col]
    return len(np.unique(key)) / g.col.size


def test_order_is_a_deterministic_permutation_with_locality(ctx, roll):
    a = ctx.build(roll, precision="fp32")
    b = ctx.build(roll, precision="fp32")
    oa, ob = a.node_order(), b.node_order()
    assert np.array_equal(np.sort(oa), np.arange(roll.n))
    assert np.array_equal(oa, ob)
    assert tile_distinct(roll, np.arange(roll.n)) > 0.9       # the generator's order is random
    assert tile_distinct(roll, oa) < 0.35
    k = ctx.build(roll, precision="fp32", keep_order=True)
    assert np.array_equal(k.node_order(), np.arange(roll.n))
    for o in (a, b, k):
        o.close()


def test_exported_operators_do_not_depend_on_the_order(ctx):
    g = mg.manifold_graph("square", 3000, 8, 5)
    ref = og.from_graph(g)
    # eps and mu fixed, so that both builds define A identically
    kw = dict(precision="fp64", eps=ref.eps, mu=ref.mu)
    a = ctx.build(g, **kw)
    k = ctx.build(g, keep_order=True, **kw)
    ea, ek = a.export(), k.export()
    for name in ("a_ptr", "a_col", "q_ptr", "q_col", "T"):
        assert np.array_equal(ea[name], ek[name]), name
    for name in ("a_val", "q_val", "b"):
        np.testing.assert_allclose(ea[name], ek[name], rtol=1e-13, atol=1e-15, err_msg=name)
    assert not np.array_equal(a.node_order(), np.arange(g.n))
    a.close()
    k.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_products_are_in_the_callers_order(gpu_lib, ctx, prec):
    mge = gpu_lib
    g = mg.manifold_graph("square", 3000, 8, 5)
    ref = og.from_graph(g)
    kw = dict(precision="fp64", eps=ref.eps, mu=ref.mu)
    a = ctx.build(g, **kw)
    k = ctx.build(g, keep_order=True, **kw)
    dt = torch.float64 if prec == "fp64" else torch.float32
    X = torch.randn(g.n, 8, generator=torch.Generator().manual_seed(3), dtype=torch.float64).to("cuda", dt)
    torch.cuda.synchronize()      # the library works on its own stream: X must be complete
    tol = dict(rtol=1e-12, atol=1e-12) if prec == "fp64" else dict(rtol=2e-5, atol=2e-5)
    for which in (0, 1):
        Ya, Yk = torch.empty_like(X), torch.empty_like(X)
        mge.mge_ops_apply(ctx.h, a.h, which, mge.PRECISION[prec], 8, X, Ya)
        mge.mge_ops_apply(ctx.h, k.h, which, mge.PRECISION[prec], 8, X, Yk)
        torch.cuda.synchronize()
        torch.testing.assert_close(Ya, Yk, **tol)
        # and the same through the in-place entry point
        XY = X.clone()
        torch.cuda.synchronize()
        mge.mge_ops_apply_inplace(ctx.h, a.h, which, mge.PRECISION[prec], 8, XY)
        torch.cuda.synchronize()
        torch.testing.assert_close(XY, Ya, rtol=0.0, atol=0.0)
    a.close()
    k.close()


def test_eigenpairs_do_not_depend_on_the_order(ctx):
    g = mg.manifold_graph("square", 2000, 8, 11)
    ref = og.from_graph(g)
    dense = oe.dense_geneig(ref.A, ref.b, 9)
    res = []
    for keep in (False, True):
        ops = ctx.build(g, precision="fp64", keep_order=keep)
        lam, V, info, s = ctx.embed(ops, 8, 1e-9, precision="fp64", guard=4)
        assert s == 0
        rel = np.abs(lam - dense.lam[:8]) / dense.lam[:8]
        assert np.max(rel) <= 1e-6, rel
        assert oe.subspace_angle(V[:, :8], dense.V[:, :8]) <= 1e-5
        res.append((lam, V))
        ops.close()
    np.testing.assert_allclose(res[0][0], res[1][0], rtol=1e-8)


def test_initial_block_is_read_in_the_callers_order(ctx):
    # starting from the converged eigenvectors (caller's order), the solve stops at once
    g = mg.manifold_graph("square", 2000, 8, 11)
    ref = og.from_graph(g)
    dense = oe.dense_geneig(ref.A, ref.b, 9)
    ops = ctx.build(g, precision="fp64")
    assert not np.array_equal(ops.node_order(), np.arange(g.n))
    x0 = np.ascontiguousarray(dense.V[:, :4].T)                # [K, n] = column-major n x K
    lam, V, info, s = ctx.embed(ops, 4, 1e-8, precision="fp64", guard=-1, x0=x0)
    assert s == 0
    assert info.iters <= 2, info.iters
    np.testing.assert_allclose(lam, dense.lam[:4], rtol=1e-8)
    ops.close()


def _splitmix64(x):
    x = (x + np.uint64(0x9E3779B97F4A7C15)).astype(np.uint64)
    x = ((x ^ (x >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)).astype(np.uint64)
    x = ((x ^ (x >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)).astype(np.uint64)
    return x ^ (x >> np.uint64(31))


def _cell_order(g, cell=128):
    """The order the build defines, restated: seeds where splitmix64(i) % cell == 0, every node
    joins the nearest seed in hops (ties: smaller seed), sort by (cell, min(hops, 255), node)."""
    n = g.n
    idx = np.arange(n, dtype=np.uint64)
    inf = np.uint64(0xFFFFFFFFFFFFFFFF)
    s = np.where(_splitmix64(idx) % np.uint64(cell) == 0, idx, inf)
    rows = np.repeat(np.arange(n), np.diff(g.row_ptr))
    with np.errstate(over="ignore"):
        while True:
            v = s[g.col]
            cand = np.where(v == inf, inf, v + np.uint64(1 << 32))
            best = s.copy()
            np.minimum.at(best, rows, cand)
            if np.array_equal(best, s):
                break
            s = best
    head = (s == idx) | (s == inf)
    cell_of = np.cumsum(head) - head
    seed = np.where(s == inf, idx, s & np.uint64(0xFFFFFFFF)).astype(np.int64)
    dist = np.where(s == inf, 0, np.minimum(s >> np.uint64(32), np.uint64(255))).astype(np.int64)
    key = (cell_of[seed].astype(np.int64) << 8) | dist
    return np.argsort(key, kind="stable")


@pytest.mark.parametrize("graph", ["roll", "ring", "hub"])
def test_order_matches_its_definition(ctx, roll, graph):
    if graph == "roll":
        g = roll
    elif graph == "ring":
        g = mg.ring(3001)
    else:
        n_hub = 1300
        i = np.arange(n_hub - 1)
        g = mg.from_edges(n_hub, np.concatenate([i, i[:-1]]), np.concatenate([np.full(n_hub - 1, n_hub - 1), i[1:]]),
                          np.ones(2 * n_hub - 3), "hub")
    ops = ctx.build(g, precision="fp32", eps=1e-3)
    assert np.array_equal(ops.node_order(), _cell_order(g))
    ops.close()
