"""The SpMM of the iteration (Y = A X and Y = Q X) against the oracle's sparse product.

FP64: 1e-12 relative to max |Y|.  FP32: the kernel sums a_ij (x_j - x_i) in FP32 over a row;
with |x| ~ 1 each term carries ~2^-24 relative error, so the tolerance is 64 * 2^-24 times the
row's sum of |a_ij| (|x_j| + |x_i|), a bound of the accumulated rounding.
"""
import numpy as np
import pytest
import torch

import manifold_graphs as mg
from oracle import graph_ops as og

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(gpu_lib):
    c = gpu_lib.Context(0)
    yield c
    c.close()


CASES = [("square", 1000, 8), ("swiss_roll", 5003, 10), ("sphere", 2000, 10)]


@pytest.mark.parametrize("shape,n,k", CASES)
@pytest.mark.parametrize("prec,m", [("fp64", 4), ("fp64", 24), ("fp32", 4), ("fp32", 8), ("fp32", 12),
                                    ("fp32", 16), ("fp32", 24)])
@pytest.mark.parametrize("which", [0, 1])
def test_apply_matches_oracle(ctx, shape, n, k, prec, m, which):
    from paper_2112_07862_gb300 import mge
    g = mg.manifold_graph(shape, n, k, 11)
    ref = og.from_graph(g)
    ops = ctx.build(g, precision="fp64", eps=ref.eps)
    dt = torch.float64 if prec == "fp64" else torch.float32
    X = torch.randn(g.n, m, dtype=torch.float64, generator=torch.Generator().manual_seed(m + which))
    Xd = X.to("cuda", dt).contiguous()
    Y = torch.empty(g.n, m, dtype=dt, device="cuda")
    mge.mge_ops_apply(ctx.h, ops.h, which, mge.PRECISION[prec], m, Xd, Y)
    Mat = ref.A if which == 0 else ref.Q
    Xr = Xd.double().cpu().numpy()
    Yref = Mat @ Xr
    got = Y.double().cpu().numpy()
    if prec == "fp64":
        assert np.max(np.abs(got - Yref)) <= 1e-12 * np.max(np.abs(Yref))
    else:
        absM = abs(Mat).tocsr()
        bound = 64 * 2.0 ** -24 * (absM @ np.abs(Xr) + absM.sum(axis=1).A * np.abs(Xr))
        assert np.all(np.abs(got - Yref) <= bound + 1e-30)
    ops.close()


def test_apply_rejects_bad_width(ctx):
    from paper_2112_07862_gb300 import mge
    g = mg.ring(64)
    ops = ctx.build(g, precision="fp64")
    X = torch.zeros(g.n, 5, dtype=torch.float64, device="cuda")
    with pytest.raises(mge.MgeError):
        mge.mge_ops_apply(ctx.h, ops.h, 0, mge.MGE_FP64, 5, X, X)
