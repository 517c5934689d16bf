"""GPU betweenness centrality and VBC (Sec. 3.3) against the oracle's Brandes accumulation.

C_B sums path-count ratios in FP64 in a different order than the oracle (dependencies pulled
in CSR order per level, partials summed per CTA), so values agree to rounding: 1e-10
relative to the largest C_B (path counts on manifold graphs reach far beyond 2^53, so the
ratios themselves carry rounding).  Closed forms are checked exactly where they are small
integers.
"""
import numpy as np
import pytest

import manifold_graphs as mg
from oracle import betweenness as ob

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(gpu_lib):
    c = gpu_lib.Context(0)
    yield c
    c.close()


GRAPHS = [mg.path(50), mg.ring(31), mg.ring(40), mg.complete(12), mg.triangle_mesh(6),
          mg.erdos_renyi(300, 0.02, 5), mg.two_components(mg.ring(9), mg.path(7)),
          mg.manifold_graph("square", 600, 8, 1), mg.manifold_graph("swiss_roll", 1000, 10, 2),
          mg.manifold_graph("sphere", 800, 10, 3)]


@pytest.mark.parametrize("g", GRAPHS, ids=[g.name for g in GRAPHS])
def test_matches_oracle(ctx, g):
    from paper_2112_07862_gb300 import mge
    cb, vbc = mge.mge_betweenness(ctx.h, g.n, g.row_ptr, g.col)
    ref = ob.betweenness(g.n, g.row_ptr, g.col)
    scale = max(1.0, float(np.max(np.abs(ref))))
    np.testing.assert_allclose(cb, ref, rtol=0, atol=1e-10 * scale)
    assert vbc == pytest.approx(ob.vbc(ref), rel=1e-9, abs=1e-9 * scale * scale)


def test_closed_forms_and_device_path(ctx):
    import torch
    from paper_2112_07862_gb300 import mge
    n = 64
    g = mg.path(n)
    rp = torch.from_numpy(g.row_ptr).cuda()
    col = torch.from_numpy(g.col).cuda()
    torch.cuda.synchronize()
    cb, vbc = mge.mge_betweenness(ctx.h, n, rp, col)
    want = np.array([2.0 * i * (n - 1 - i) for i in range(n)])
    assert np.array_equal(cb.cpu().numpy(), want)
    assert vbc == pytest.approx(float(np.var(want)), rel=1e-14)
    r = mg.ring(101)
    cb, vbc = mge.mge_betweenness(ctx.h, r.n, r.row_ptr, r.col)
    assert np.all(cb == 100 * 98 / 4.0) and vbc == 0.0


def test_malformed_csr_rejected(ctx):
    from paper_2112_07862_gb300 import mge
    g = mg.ring(10)
    bad = g.col.copy()
    bad[3] = 99
    with pytest.raises(mge.MgeError) as e:
        mge.mge_betweenness(ctx.h, g.n, g.row_ptr, bad)
    assert e.value.status == mge.MGE_EINVAL
