"""GPU kNN graph construction (Sec. 5.1) against the oracle's brute force.

The neighbour selection is integer work decided by FP64 squared distances that both sides
compute the same way (coordinates summed in order, no fused multiply-add), so the CSR
structure must match bit for bit -- including point sets full of exact ties (integer
lattices), where the lower index must win.  sigma and the weights are FP64 sums and
exponentials in a different order than the oracle's: 1e-13 relative.
At the benchmark's size (200,000 swiss-roll points) the oracle checks sampled rows one by
one: each row must hold the row's own k nearest and, for every other entry j, i must be
among j's k nearest.
"""
import numpy as np
import pytest

import manifold_graphs as mg
from oracle import knn as ok
from oracle import eigen as oe
from oracle import graph_ops as og

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(gpu_lib):
    c = gpu_lib.Context(0)
    yield c
    c.close()


def lattice(shape):
    axes = [np.arange(s, dtype=np.float64) for s in shape]
    return np.stack(np.meshgrid(*axes, indexing="ij"), axis=-1).reshape(-1, len(shape))


CASES = [
    ("square", mg.sample_points("square", 3000, 1), 8),
    ("swiss_roll", mg.sample_points("swiss_roll", 4000, 2), 10),
    ("sphere", mg.sample_points("sphere", 3000, 3), 10),
    ("torus", mg.sample_points("torus", 2500, 4), 12),
    ("cube32", np.random.default_rng(5).random((2000, 3)), 32),
    ("k1", mg.sample_points("square", 500, 6), 1),
    ("tiny", mg.sample_points("sphere", 40, 7), 5),
    ("lattice2d", lattice((30, 30)), 8),
    ("lattice3d", lattice((12, 12, 12)), 6),
    ("lattice_shifted", lattice((20, 25)) * 0.5 + 1e3, 12),
    ("duplicates", np.repeat(mg.sample_points("square", 300, 8), 2, axis=0), 4),
]


@pytest.mark.parametrize("name,P,k", CASES, ids=[c[0] for c in CASES])
def test_knn_graph_matches_brute_force(ctx, name, P, k):
    from paper_2112_07862_gb300 import mge
    g = mge.mge_knn_graph(ctx.h, P, k)
    try:
        rp, col, w = mge.mge_graph_export(g)
        n, nnz, sigma = mge.mge_graph_info(g)
    finally:
        mge.mge_graph_destroy(g)
    rp0, col0, w0, sigma0 = ok.knn_graph(P, k)
    assert n == P.shape[0] and nnz == col0.shape[0]
    assert np.array_equal(rp, rp0)
    assert np.array_equal(col, col0)
    assert sigma == pytest.approx(sigma0, rel=1e-13)
    np.testing.assert_allclose(w, w0, rtol=1e-13, atol=0)


def test_device_points_and_errors(ctx):
    import torch
    from paper_2112_07862_gb300 import mge
    P = mg.sample_points("swiss_roll", 2000, 9)
    Pd = torch.from_numpy(P).cuda()
    torch.cuda.synchronize()
    g = mge.mge_knn_graph(ctx.h, Pd, 10)
    rp, col, w = mge.mge_graph_export(g)
    mge.mge_graph_destroy(g)
    rp0, col0, w0, _ = ok.knn_graph(P, 10)
    assert np.array_equal(rp, rp0) and np.array_equal(col, col0)
    for bad, k in [(np.zeros((10, 4)), 3), (P[:5], 5), (np.zeros((10, 3)), 2)]:
        with pytest.raises(mge.MgeError) as e:
            mge.mge_knn_graph(ctx.h, bad, k)
        assert e.value.status == mge.MGE_EINVAL
    Pn = P.copy()
    Pn[7, 1] = np.nan
    with pytest.raises(mge.MgeError) as e:
        mge.mge_knn_graph(ctx.h, Pn, 10)
    assert e.value.status == mge.MGE_EINVAL


def test_points_to_embedding_matches_the_oracle(ctx):
    """Points -> kNN graph -> operators -> embedding, all on the GPU, against the oracle's
    own brute-force graph, operators and dense generalized eigendecomposition."""
    from paper_2112_07862_gb300 import mge
    P = mg.sample_points("sphere", 2000, 11)
    g = mge.mge_knn_graph(ctx.h, P, 10)
    rp_d, col_d, w_d = mge.mge_graph_csr(g)
    n, nnz, _ = mge.mge_graph_info(g)
    h, s = mge.mge_build_graph_ops(ctx.h, n, rp_d, col_d, w_d, True, mge.ops_opts("fp64"))
    lam, V, info, s2 = mge.mge_embed(ctx.h, h, 4, 1e-9, mge.embed_opts("fp64"))
    mge.mge_ops_destroy(h)
    mge.mge_graph_destroy(g)
    rp0, col0, w0, _ = ok.knn_graph(P, 10)
    ref = og.build_graph_ops(n, rp0, col0, w0)
    d = oe.dense_geneig(ref.A, ref.b, 5)
    assert s2 == 0
    np.testing.assert_allclose(lam, d.lam[:4], rtol=1e-6)
    assert oe.subspace_angle(V.T, d.V[:, :4]) < 1e-4


@pytest.mark.slow
def test_full_size_rows_against_brute_force(ctx):
    from paper_2112_07862_gb300 import mge
    P = mg.sample_points("swiss_roll", 200_000, 2)
    k = 10
    g = mge.mge_knn_graph(ctx.h, P, k)
    rp, col, w = mge.mge_graph_export(g)
    _, _, sigma = mge.mge_graph_info(g)
    mge.mge_graph_destroy(g)
    rows = np.random.default_rng(0).choice(P.shape[0], 300, replace=False)
    nbr, d2 = ok.knn_lists(P, k, rows=rows)
    for r, i in enumerate(rows):
        row = col[rp[i]:rp[i + 1]]
        assert np.all(np.diff(row) > 0)
        assert set(nbr[r].tolist()) <= set(row.tolist())
        others = [j for j in row.tolist() if j not in set(nbr[r].tolist())]
        if others:
            nj, _ = ok.knn_lists(P, k, rows=np.array(others))
            assert all(i in set(nj[t].tolist()) for t in range(len(others)))
        wi = w[rp[i]:rp[i + 1]]
        d2i = ((P[row] - P[i]) ** 2).sum(axis=1)
        np.testing.assert_allclose(wi, np.exp(-d2i / sigma ** 2), rtol=1e-12)
    # sigma: the mean of all n k directed distances, against the oracle's kd-tree-free value
    # on a subsample of rows (an estimate: the full mean is checked on smaller graphs)
    assert sigma == pytest.approx(float(np.mean(np.sqrt(d2))), rel=0.05)
