"""In-place operator product through the library's fixed device array (no allocation).

mge_ops_apply_inplace runs the same SpMM kernel as mge_ops_apply on a copy of the block
held in a fixed device array, so on the same input its output must equal
mge_ops_apply's bit for bit (tolerance zero).  Checked on two calls in a row, since every
call shares the array; blocks larger than the array are rejected before anything is
touched.  The file name sorts last so that the test also runs after all other GPU tests.

The library runs on its own (non-blocking) stream, so every block built by torch on its
current stream is synchronised before it is handed over.
"""
import numpy as np
import pytest
import torch

import manifold_graphs as mg

pytestmark = pytest.mark.gpu

SCRATCH_BYTES = 32 << 20


def _block(n, m, dt, gen):
    return torch.randn(n, m, generator=gen, dtype=torch.float64).to("cuda", dt).contiguous()


@pytest.mark.parametrize("prec,m,which", [("fp32", 8, 0), ("fp64", 24, 0), ("fp32", 4, 1), ("fp64", 12, 1)])
def test_inplace_apply_equals_apply_on_two_calls(gpu_lib, prec, m, which):
    mge = gpu_lib
    ctx = mge.Context(0)
    g = mg.manifold_graph("square", 3000, 8, 5)
    ops = ctx.build(g, precision="fp64")
    dt = torch.float64 if prec == "fp64" else torch.float32
    gen = torch.Generator().manual_seed(11 + m)
    for call in range(2):
        X = _block(g.n, m, dt, gen)
        Y = torch.empty_like(X)
        XY = X.clone()
        torch.cuda.synchronize()
        mge.mge_ops_apply(ctx.h, ops.h, which, mge.PRECISION[prec], m, X, Y)
        mge.mge_ops_apply_inplace(ctx.h, ops.h, which, mge.PRECISION[prec], m, XY)
        torch.cuda.synchronize()
        torch.testing.assert_close(XY, Y, rtol=0.0, atol=0.0, msg=f"call {call}")
    ops.close()
    ctx.close()


def test_inplace_apply_limit(gpu_lib):
    mge = gpu_lib
    ctx = mge.Context(0)
    n = 180_000                                   # 24 FP64 columns: 34.6 MB > 32 MiB
    ops = ctx.build(mg.path(n), precision="fp64")  # two-hop graph disconnected: eps = 0
    assert ops.status == mge.MGE_EDEGENERATE
    big = torch.ones(n, 24, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    assert big.numel() * 8 > SCRATCH_BYTES
    with pytest.raises(mge.MgeError) as e:
        mge.mge_ops_apply_inplace(ctx.h, ops.h, 0, mge.MGE_FP64, 24, big)
    assert e.value.status == mge.MGE_EINVAL
    assert "scratch" in str(e.value)
    assert bool(torch.all(big == 1.0))           # rejected before anything was written
    # the same rows in FP32 (17.3 MB) fit, and match the out-of-place product
    gen = torch.Generator().manual_seed(5)
    for _ in range(2):
        X = _block(n, 24, torch.float32, gen)
        Y = torch.empty_like(X)
        torch.cuda.synchronize()
        mge.mge_ops_apply(ctx.h, ops.h, 0, mge.MGE_FP32, 24, X, Y)
        mge.mge_ops_apply_inplace(ctx.h, ops.h, 0, mge.MGE_FP32, 24, X)
        torch.cuda.synchronize()
        torch.testing.assert_close(X, Y, rtol=0.0, atol=0.0)
    ops.close()
    ctx.close()
