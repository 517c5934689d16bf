"""Serving: requests admitted by HBM footprint run concurrently; each result is the same as
when the request runs alone (eigenvalues to 1e-10 relative, vectors to 1e-8).  The mix holds
FP32 and BF16 requests side by side."""
import ctypes

import numpy as np
import pytest

import manifold_graphs as mg

pytestmark = pytest.mark.gpu


def request(mge, g, K, tol=1e-5, seed=0, precision="fp32", guard=4):
    r = mge.mge_request()
    r.n = g.n
    r.row_ptr = g.row_ptr.ctypes.data
    r.col = g.col.ctypes.data
    r.w = g.w.ctypes.data
    r.K = K
    r.tol = tol
    r.precision = mge.PRECISION[precision]
    r.guard = guard
    r.maxiter = 0
    r.seed = seed
    return r


def test_results_are_the_same_alone_and_in_the_mix(gpu_lib):
    mge = gpu_lib
    graphs = [(mg.manifold_graph("square", 3000, 8, 1), 4, "fp32"),
              (mg.manifold_graph("sphere", 5000, 10, 2), 8, "bf16"),
              (mg.manifold_graph("swiss_roll", 8000, 10, 3), 8, "fp32"),
              (mg.manifold_graph("torus", 2000, 12, 4), 2, "bf16"),
              (mg.manifold_graph("square", 12000, 10, 5), 16, "bf16"),
              (mg.manifold_graph("sphere", 1500, 10, 6), 4, "fp32")]
    with mge.Context(0) as ctx:
        alone = []
        for g, K, p in graphs:
            ops = ctx.build(g, precision=p)
            lam, V, info, s = ctx.embed(ops, K, 1e-5, precision=p, guard=4)
            alone.append((lam, V))
            ops.close()
    with mge.Context(0) as ctx:
        tickets = [mge.mge_submit(ctx.h, request(mge, g, K, precision=p)) for g, K, p in graphs]
        for (g, K, p), t, (lam0, V0) in zip(graphs, tickets, alone):
            s, r = mge.mge_poll(ctx.h, t, -1)
            assert s == 0 and r.status == 0, (s, r.status)
            lam = np.ctypeslib.as_array(r.lambda_, shape=(K,)).copy()
            V = np.ctypeslib.as_array(r.V, shape=(K, g.n)).T.copy()
            assert np.allclose(lam, lam0, rtol=1e-10, atol=0)
            assert np.max(np.abs(V - V0)) < 1e-8
            assert r.latency_ms >= r.queue_ms >= 0
            assert mge.mge_release(ctx.h, t) == 0


def test_poll_and_release_errors(gpu_lib):
    mge = gpu_lib
    with mge.Context(0) as ctx:
        s, r = mge.mge_poll(ctx.h, 12345, 0)
        assert s == mge.MGE_ENOTFOUND
        assert mge.mge_release(ctx.h, 999) == mge.MGE_ENOTFOUND


def test_budget_admission_rejects_oversized_request(gpu_lib):
    mge = gpu_lib
    g = mg.manifold_graph("square", 20000, 10, 9)
    with mge.Context(0, hbm_budget_bytes=1 << 20) as ctx:
        with pytest.raises(mge.MgeError) as e:
            mge.mge_submit(ctx.h, request(mge, g, 8))
        assert e.value.status == mge.MGE_ENOMEM


def test_budget_serialises_but_completes(gpu_lib):
    """A budget that fits one request at a time still serves them all, in order."""
    mge = gpu_lib
    gs = [mg.manifold_graph("square", 4000, 8, s) for s in range(4)]
    with mge.Context(0, hbm_budget_bytes=64 << 20) as ctx:
        ts = [mge.mge_submit(ctx.h, request(mge, g, 4)) for g in gs]
        for t in ts:
            s, r = mge.mge_poll(ctx.h, t, -1)
            assert s == 0 and r.status == 0
            mge.mge_release(ctx.h, t)


def test_eight_slots_every_request_matches_alone(gpu_lib, monkeypatch):
    """Eight slots: the builds, graph captures and handle releases of different requests
    interleave on eight host threads, and every request still converges to its result
    alone (a device-wide synchronisation in one slot would break another slot's capture)."""
    mge = gpu_lib
    specs = [("square", 1500, 4), ("sphere", 2500, 8), ("swiss_roll", 3000, 8), ("torus", 2000, 2),
             ("square", 4000, 16), ("sphere", 1200, 4), ("swiss_roll", 5000, 4), ("torus", 3500, 8)] * 2
    graphs = [(mg.manifold_graph(shape, n, 10, 60 + i), K) for i, (shape, n, K) in enumerate(specs)]
    with mge.Context(0) as ctx:
        alone = []
        for g, K in graphs:
            ops = ctx.build(g, precision="fp32")
            lam, V, info, s = ctx.embed(ops, K, 1e-5, precision="fp32", guard=4)
            alone.append((lam, V))
            ops.close()
    monkeypatch.setenv("MGE_SERVE_SLOTS", "8")
    with mge.Context(0) as ctx:
        tickets = [mge.mge_submit(ctx.h, request(mge, g, K)) for g, K in graphs]
        for (g, K), t, (lam0, V0) in zip(graphs, tickets, alone):
            s, r = mge.mge_poll(ctx.h, t, -1)
            assert s == 0 and r.status == 0, (s, r.status, mge.mge_ctx_last_error(ctx.h))
            lam = np.ctypeslib.as_array(r.lambda_, shape=(K,)).copy()
            V = np.ctypeslib.as_array(r.V, shape=(K, g.n)).T.copy()
            assert np.allclose(lam, lam0, rtol=1e-10, atol=0)
            assert np.max(np.abs(V - V0)) < 1e-8
            assert mge.mge_release(ctx.h, t) == 0


def test_requests_given_as_points(gpu_lib):
    """A request given as points runs kNN graph, operators and embedding on the device; its
    result equals the graph built by mge_knn_graph and embedded alone."""
    mge = gpu_lib
    sets = [(mg.sample_points("sphere", 4000, 31), 10, 8, "fp32"),
            (mg.sample_points("square", 3000, 32), 8, 4, "fp32"),
            (mg.sample_points("swiss_roll", 6000, 33), 10, 8, "bf16")]
    with mge.Context(0) as ctx:
        alone = []
        for P, k, K, p in sets:
            g = mge.mge_knn_graph(ctx.h, P, k)
            rp, col, w = mge.mge_graph_csr(g)
            n, _, _ = mge.mge_graph_info(g)
            h, s = mge.mge_build_graph_ops(ctx.h, n, rp, col, w, True, mge.ops_opts(p))
            mge.mge_graph_destroy(g)
            lam, V, info, s2 = mge.mge_embed(ctx.h, h, K, 1e-5, mge.embed_opts(p, guard=4))
            mge.mge_ops_destroy(h)
            alone.append((lam, V.T))
    with mge.Context(0) as ctx:
        tickets = []
        for P, k, K, p in sets:
            r = mge.mge_request()
            r.n, r.K, r.tol, r.precision, r.guard = P.shape[0], K, 1e-5, mge.PRECISION[p], 4
            Pc = np.ascontiguousarray(P)
            r.points, r.dim, r.knn = Pc.ctypes.data, P.shape[1], k
            tickets.append(mge.mge_submit(ctx.h, r))
        for (P, k, K, p), t, (lam0, V0) in zip(sets, tickets, alone):
            s, r = mge.mge_poll(ctx.h, t, -1)
            assert s == 0 and r.status == 0, (s, r.status)
            lam = np.ctypeslib.as_array(r.lambda_, shape=(K,)).copy()
            V = np.ctypeslib.as_array(r.V, shape=(K, P.shape[0])).T.copy()
            assert np.allclose(lam, lam0, rtol=1e-10, atol=0)
            assert np.max(np.abs(V - V0)) < 1e-8
            mge.mge_release(ctx.h, t)
