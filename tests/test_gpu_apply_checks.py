"""Argument checks of the operator-product entry points, called through the C ABI.

A block pointer that is not 16-byte aligned, that points to host memory, or a width the
kernel has no instantiation for must come back as MGE_EINVAL from a check on the host,
before any kernel runs: the output buffer is left untouched.  (The kernels read rows with
16-byte loads and bulk copies, so such a pointer would otherwise fault on the device.)
The Python wrappers add checks of dtype, shape and contiguity that the C side cannot see.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import manifold_graphs as mg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup(gpu_lib):
    mge = gpu_lib
    ctx = mge.Context(0)
    g = mg.manifold_graph("square", 1000, 8, 3)
    ops = ctx.build(g, precision="fp32")
    yield mge, ctx, ops, g.n
    ops.close()
    ctx.close()


def _raw(mge):
    return mge.load()


def test_misaligned_pointers_rejected(setup):
    mge, ctx, ops, n = setup
    lib = _raw(mge)
    X = torch.randn(n + 1, 8, dtype=torch.float32, device="cuda")
    Y = torch.full((n + 1, 8), 7.0, dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    s = lib.mge_ops_apply(ctx.h, ops.h, 0, mge.MGE_FP32, 8, X.data_ptr() + 4, Y.data_ptr(), None)
    assert s == mge.MGE_EINVAL
    assert "aligned" in mge.mge_ctx_last_error(ctx.h)
    s = lib.mge_ops_apply(ctx.h, ops.h, 0, mge.MGE_FP32, 8, X.data_ptr(), Y.data_ptr() + 8, None)
    assert s == mge.MGE_EINVAL
    s = lib.mge_ops_apply_inplace(ctx.h, ops.h, 0, mge.MGE_FP32, 8, Y.data_ptr() + 4, None)
    assert s == mge.MGE_EINVAL
    torch.cuda.synchronize()
    assert bool(torch.all(Y == 7.0))


def test_host_pointers_rejected(setup):
    mge, ctx, ops, n = setup
    lib = _raw(mge)
    Xh = np.ones((n, 8), np.float32)
    Yh = np.full((n, 8), 7.0, np.float32)
    Xd = torch.ones(n, 8, dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    s = lib.mge_ops_apply(ctx.h, ops.h, 0, mge.MGE_FP32, 8, Xh.ctypes.data, Yh.ctypes.data, None)
    assert s == mge.MGE_EINVAL
    assert "device memory" in mge.mge_ctx_last_error(ctx.h) or "CUDA pointer" in mge.mge_ctx_last_error(ctx.h)
    s = lib.mge_ops_apply(ctx.h, ops.h, 0, mge.MGE_FP32, 8, Xd.data_ptr(), Yh.ctypes.data, None)
    assert s == mge.MGE_EINVAL
    s = lib.mge_ops_apply_inplace(ctx.h, ops.h, 0, mge.MGE_FP32, 8, Yh.ctypes.data, None)
    assert s == mge.MGE_EINVAL
    # pinned host memory is a CUDA pointer too, but not device memory
    Yp = torch.full((n, 8), 7.0, dtype=torch.float32).pin_memory()
    s = lib.mge_ops_apply_inplace(ctx.h, ops.h, 0, mge.MGE_FP32, 8, Yp.data_ptr(), None)
    assert s == mge.MGE_EINVAL
    assert np.all(Yh == 7.0) and bool(torch.all(Yp == 7.0))


@pytest.mark.parametrize("m", [2, 32, 48])
def test_unsupported_width_rejected(setup, m):
    mge, ctx, ops, n = setup
    lib = _raw(mge)
    Y = torch.full((n, m), 7.0, dtype=torch.float32, device="cuda")
    X = torch.ones(n, m, dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    assert lib.mge_ops_apply(ctx.h, ops.h, 0, mge.MGE_FP32, m, X.data_ptr(), Y.data_ptr(), None) == mge.MGE_EINVAL
    assert lib.mge_ops_apply_inplace(ctx.h, ops.h, 0, mge.MGE_FP32, m, Y.data_ptr(), None) == mge.MGE_EINVAL
    assert "width" in mge.mge_ctx_last_error(ctx.h)
    torch.cuda.synchronize()
    assert bool(torch.all(Y == 7.0))


def test_python_wrapper_checks_dtype_and_shape(setup):
    mge, ctx, ops, n = setup
    X64 = torch.ones(n, 8, dtype=torch.float64, device="cuda")
    with pytest.raises(mge.MgeError):
        mge.mge_ops_apply_inplace(ctx.h, ops.h, 0, mge.MGE_FP32, 8, X64)
    Xs = torch.ones(n - 1, 8, dtype=torch.float32, device="cuda")
    with pytest.raises(mge.MgeError):
        mge.mge_ops_apply(ctx.h, ops.h, 0, mge.MGE_FP32, 8, Xs, Xs)
    Xt = torch.ones(8, n, dtype=torch.float32, device="cuda").t()
    with pytest.raises(mge.MgeError):
        mge.mge_ops_apply_inplace(ctx.h, ops.h, 0, mge.MGE_FP32, 8, Xt)
    assert bool(torch.all(X64 == 1.0))
