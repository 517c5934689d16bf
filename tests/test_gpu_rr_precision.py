"""Rayleigh-Ritz precision of FP32 solves: the inverse-pencil FP32 form, the FP64 Jacobi form,
and the default that starts in FP32 and moves to FP64 when the residuals stop falling.

Every form must give the oracle's pairs (eigenvalues 1e-4 relative, vectors 1e-3 rad per
cluster: the reduced-precision bar); `info.rr_fp64_from` must say which form ran.  A
tolerance out of reach makes the default switch once the FP32 form stalls.
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
def case(ctx):
    g = mg.manifold_graph("swiss_roll", 20000, 10, 31)
    t_ptr, t_col, _ = og.two_hop_sets(g.n, g.row_ptr, g.col)
    eps, _ = og.fiedler_value_sparse(og.q_matrix(g.n, t_ptr, t_col), og.two_hop_components(g.n, t_ptr, t_col))
    ref = og.build_graph_ops(g.n, g.row_ptr, g.col, g.w, eps_override=eps)
    d = oe.sparse_geneig(ref.A, ref.b, 9)
    ops = ctx.build(g, precision="fp32")
    yield g, d, ops
    ops.close()


def check_pairs(lam, V, d, K):
    rel = np.abs(lam - d.lam[:K]) / d.lam[:K]
    assert np.max(rel) <= 1e-4, rel
    gaps = np.abs(np.diff(d.lam[:K + 1])) / d.lam[1:K + 1]
    start = 0
    for j in range(K):
        if gaps[j] > 1e-6:            # cluster [start, j] closed off from the next eigenvalue
            assert oe.subspace_angle(V[:, start:j + 1], d.V[:, start:j + 1]) <= 1e-3, (start, j)
            start = j + 1


@pytest.mark.parametrize("mode", [-1, 0, 1])
def test_every_form_gives_the_oracle_pairs(ctx, case, mode):
    from paper_2112_07862_gb300 import mge
    g, d, ops = case
    K = 8
    lam, V, info, s = ctx.embed(ops, K, 1e-5, precision="fp32", rr_fp64=mode)
    assert s == mge.MGE_OK
    check_pairs(lam, V, d, K)
    assert max(info.resid[k] for k in range(K)) <= 1e-5
    if mode == -1:
        assert info.rr_fp64_from == -1
    elif mode == 1:
        assert info.rr_fp64_from == 0
    else:
        assert info.rr_fp64_from == -1 or 0 < info.rr_fp64_from < info.iters


def test_stalled_fp32_moves_to_fp64(ctx, case):
    """A tolerance below what FP32 blocks reach (measured on this graph, one GB300: largest
    relative residual 0.7e-6 .. 1.1e-6 from iteration 20 on, in either Rayleigh-Ritz form)
    stalls the FP32 form within 1000x of the tolerance: the default then switches, and the
    solve ends as not converged with the oracle's pairs."""
    from paper_2112_07862_gb300 import mge
    g, d, ops = case
    K = 8
    lam, V, info, s = ctx.embed(ops, K, 1e-8, precision="fp32", rr_fp64=0, maxiter=150)
    assert s == mge.MGE_ENOTCONVERGED
    assert 0 < info.rr_fp64_from < info.iters
    check_pairs(lam, V, d, K)
    lam2, V2, info2, s2 = ctx.embed(ops, K, 1e-8, precision="fp32", rr_fp64=-1, maxiter=150)
    assert s2 == mge.MGE_ENOTCONVERGED and info2.rr_fp64_from == -1
    check_pairs(lam2, V2, d, K)
