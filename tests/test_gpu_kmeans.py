"""GPU k-means of the embedding (Sec. 5.2) against the oracle's Lloyd iteration.

Assignments are integer results decided by FP64 distances that both sides compute the same
way (coordinates in order, no fused multiply-add, ties to the lower centre), from centres
that are exactly rounded means on both sides: assignments, centres and the number of steps
must agree bit for bit.
"""
import numpy as np
import pytest

import manifold_graphs as mg
from oracle import kmeans as okm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(gpu_lib):
    c = gpu_lib.Context(0)
    yield c
    c.close()


def blobs(n, K, C, seed):
    rng = np.random.default_rng(seed)
    means = rng.normal(0, 3, (C, K))
    return means[rng.integers(0, C, n)] + rng.normal(0, 1, (n, K))


def check(mge, ctx, X, C0, iters):
    a, C, steps = mge.mge_kmeans(ctx.h, X, C0, iters)
    a0, C_0, steps0 = okm.kmeans(X, C0, iters)
    assert steps == steps0
    assert np.array_equal(a, a0)
    assert np.array_equal(C, C_0)
    return a, C, steps


@pytest.mark.parametrize("n,K,C,iters", [(20000, 4, 6, 100), (5000, 8, 16, 30), (3000, 2, 3, 5),
                                         (1000, 24, 40, 50), (257, 64, 64, 20)])
def test_matches_oracle_on_blobs(ctx, n, K, C, iters):
    from paper_2112_07862_gb300 import mge
    X = blobs(n, K, C, n + K)
    C0 = X[np.random.default_rng(1).choice(n, C, replace=False)]
    check(mge, ctx, X, C0, iters)


def test_ties_empty_clusters_and_small_cases(ctx):
    from paper_2112_07862_gb300 import mge
    # integer lattice points with centres at half-integers: many exact ties
    g = np.stack(np.meshgrid(np.arange(20.0), np.arange(20.0), indexing="ij"), -1).reshape(-1, 2)
    C0 = np.array([[4.5, 4.5], [9.5, 4.5], [4.5, 9.5], [9.5, 9.5], [500.0, 500.0]])
    a, C, _ = check(mge, ctx, g, C0, 20)
    assert C[4].tolist() == [500.0, 500.0]              # empty cluster kept its centre
    check(mge, ctx, g, C0[:1], 3)                       # one cluster
    check(mge, ctx, g[:1], C0[:2], 3)                   # one point
    check(mge, ctx, blobs(500, 3, 4, 2), blobs(4, 3, 4, 3), 1)      # a single step


def test_device_path_on_a_gpu_embedding(ctx):
    """Embedding -> k-means on the device: V as mge_embed leaves it (column-major)."""
    import torch
    from paper_2112_07862_gb300 import mge
    g = mg.manifold_graph("swiss_roll", 6000, 10, 12)
    ops = ctx.build(g, precision="fp32")
    Vd = torch.empty((8, g.n), dtype=torch.float64, device="cuda")
    lam, V, info, s = mge.mge_embed(ctx.h, ops.h, 8, 1e-5, mge.embed_opts("fp32", v_on_device=True), Vd)
    ops.close()
    assert s == 0
    idx = np.random.default_rng(4).choice(g.n, 10, replace=False)
    Vh = Vd.cpu().numpy().T.copy()                      # [n, K]
    C0h = Vh[idx]
    C0d = torch.from_numpy(C0h).cuda()
    torch.cuda.synchronize()
    a, C, steps = mge.mge_kmeans(ctx.h, Vd, C0d, 60)
    a0, C_0, steps0 = okm.kmeans(Vh, C0h, 60)
    assert steps == steps0
    assert np.array_equal(a.cpu().numpy(), a0)
    assert np.array_equal(C.cpu().numpy(), C_0)


def test_invalid_arguments(ctx):
    from paper_2112_07862_gb300 import mge
    X = blobs(100, 4, 2, 1)
    for C0, it in [(X[:2], 0), (np.zeros((2000, 4)), 5)]:
        with pytest.raises(mge.MgeError) as e:
            mge.mge_kmeans(ctx.h, X, C0, it)
        assert e.value.status == mge.MGE_EINVAL


@pytest.mark.slow
def test_full_size_embedding_shape(ctx):
    """200,000 points in 8 dimensions (the benchmark embedding's shape), 16 clusters."""
    from paper_2112_07862_gb300 import mge
    X = blobs(200_000, 8, 16, 77)
    C0 = X[np.random.default_rng(5).choice(X.shape[0], 16, replace=False)]
    check(mge, ctx, X, C0, 25)
