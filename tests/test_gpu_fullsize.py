"""The benchmark workload at full size (200,000 swiss-roll points, 10-NN, K = 8, FP32,
tol 1e-5), checked against the oracle where it can be computed at this size:
  * the whole A / Q structure and the two-hop counts, bit-exact (oracle sparse build);
  * eps against the oracle's FP64 LOBPCG value (2e-5 relative, the FP32 form's tolerance);
  * the returned pairs' backward errors, recomputed in FP64 by the oracle with its own A, B;
  * B-orthonormality V^T B V = I and the ascending order.
"""
import numpy as np
import pytest

import manifold_graphs as mg
from oracle import eigen as oe
from oracle import graph_ops as og

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def test_config_swiss_roll_200k_fp32(gpu_lib):
    g = mg.manifold_graph("swiss_roll", 200_000, 10, 2)
    with gpu_lib.Context(0) as ctx:
        ops = ctx.build(g, precision="fp32")
        info = ops.info()
        ex = ops.export()
        lam, V, ei, s = ctx.embed(ops, 8, 1e-5, precision="fp32")
        ops.close()
    assert s == 0
    t_ptr, t_col, T = og.two_hop_sets(g.n, g.row_ptr, g.col)
    assert np.array_equal(ex["T"], T)
    a_ptr, a_col = og.a_structure(g.n, g.row_ptr, g.col, t_ptr, t_col)
    assert np.array_equal(ex["a_ptr"], a_ptr) and np.array_equal(ex["a_col"], a_col)
    # the oracle's operators built with the GPU's eps: residuals of the returned pairs
    ref = og.build_graph_ops(g.n, g.row_ptr, g.col, g.w, eps_override=info.eps)
    np.testing.assert_allclose(ex["a_val"], ref.a_val, rtol=1e-12, atol=1e-16)
    eta = oe.backward_errors(ref.A, ref.b, lam, V)
    assert np.all(eta <= 2e-5), eta
    assert np.all(np.diff(lam) > 0)
    VBV = V.T @ (ref.b[:, None] * V)
    assert np.max(np.abs(VBV - np.eye(8))) < 1e-4
    # eps against the oracle's FP64 value (deflated LOBPCG on Q)
    Y = np.ones((g.n, 1)) / np.sqrt(g.n)
    r = oe.lobpcg(ref.Q, np.ones(g.n), 1, guard=3, Y=Y, tol=1e-8, seed=1, maxiter=4000)
    assert info.eps == pytest.approx(r.lam[0], rel=2e-5)
