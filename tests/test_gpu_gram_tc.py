"""Rayleigh-Ritz Grams on the tensor cores (tcgen05, TF32 with split operands) against the
CUDA-core Grams (compensated FP32) and the oracle's dense generalized eigendecomposition.

The Grams only steer the iteration: a solve with either must converge to the same pairs, so
both are compared with the oracle (eigenvalues 1e-4 relative, vectors 1e-3 rad per cluster)
and with each other (eigenvalues 1e-5 relative).  Block widths 12, 16 and 24 take the
tensor-core path (the width of the basis [X W P] is 36, 48 and 72) on graphs of at least
65,536 nodes; the oracle's reference is its shift-invert Lanczos (machine precision).
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


def clusters(lam, rel=1e-6):
    out, cur = [], [0]
    for j in range(1, len(lam)):
        if abs(lam[j] - lam[j - 1]) <= rel * abs(lam[j]):
            cur.append(j)
        else:
            out.append(cur)
            cur = [j]
    out.append(cur)
    return out


@pytest.mark.parametrize("shape,n,K,guard", [("swiss_roll", 70000, 8, 4), ("square", 66000, 8, 8),
                                             ("sphere", 80000, 16, 8), ("torus", 70000, 12, 12)])
def test_tensor_core_grams_give_the_oracle_pairs(ctx, shape, n, K, guard):
    g = mg.manifold_graph(shape, n, 10, 21)
    t_ptr, t_col, _ = og.two_hop_sets(g.n, g.row_ptr, g.col)
    eps, _ = og.fiedler_value_sparse(og.q_matrix(g.n, t_ptr, t_col), og.two_hop_components(g.n, t_ptr, t_col))
    ref = og.build_graph_ops(g.n, g.row_ptr, g.col, g.w, eps_override=eps)
    d = oe.sparse_geneig(ref.A, ref.b, K + 1)
    ops = ctx.build(g, precision="fp32")
    res = {}
    for cc in (False, True):
        lam, V, info, s = ctx.embed(ops, K, 1e-5, precision="fp32", guard=guard, gram_cuda_cores=cc)
        assert s == 0, (cc, s)
        assert info.m in (12, 16, 24)
        rel = np.abs(lam - d.lam[:K]) / d.lam[:K]
        assert np.max(rel) <= 1e-4, (cc, rel)
        for grp in clusters(d.lam[:K + 1]):
            if grp[-1] < K:
                assert oe.subspace_angle(V[:, grp], d.V[:, grp]) <= 1e-3, (cc, grp)
        res[cc] = (lam, info.iters)
    np.testing.assert_allclose(res[False][0], res[True][0], rtol=1e-5)
    assert abs(res[False][1] - res[True][1]) <= max(3, res[True][1] // 5)
    ops.close()
