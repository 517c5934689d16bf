"""Python binding of libmge (include/mge.h): argument marshalling only.

Every function named ``mge_*`` here calls the C entry point of the same name; the
arithmetic runs in the library's CUDA kernels.  Host arrays are numpy arrays; device
arrays are torch CUDA tensors (their ``data_ptr()`` is passed).  Loading fails loudly when
libmge.so is missing: there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmge.so")

MGE_OK, MGE_EINVAL, MGE_ENOTSYM, MGE_EISOLATED, MGE_EDEGENERATE, MGE_ENOTCONVERGED = 0, 1, 2, 3, 4, 5
MGE_ENOMEM, MGE_EAGAIN, MGE_ETIMEOUT, MGE_EDEVICE, MGE_ECHOLESKY, MGE_ENOTFOUND = 6, 7, 8, 9, 10, 11
MGE_ENOTFINITE = 12
MGE_FP64, MGE_FP32, MGE_BF16 = 0, 1, 2
PRECISION = {"fp64": MGE_FP64, "fp32": MGE_FP32, "bf16": MGE_BF16}

# every symbol include/mge.h declares
EXPORTS = [
    "mge_create", "mge_destroy", "mge_strerror", "mge_ctx_last_error", "mge_ctx_stats",
    "mge_ctx_set_timing", "mge_ctx_reset_stats", "mge_ctx_set_autotune", "mge_build_graph_ops", "mge_build_graph_ops_batch", "mge_ops_destroy",
    "mge_ops_info", "mge_ops_export", "mge_ops_node_order", "mge_ops_apply", "mge_ops_apply_inplace", "mge_embed", "mge_embed_batch", "mge_submit", "mge_poll",
    "mge_release", "mge_betweenness", "mge_kmeans", "mge_knn_graph", "mge_graph_info", "mge_graph_csr", "mge_graph_export", "mge_graph_destroy",
]


class mge_stats(C.Structure):
    _fields_ = [("kernel_launches", C.c_uint64), ("spmm_launches", C.c_uint64),
                ("spmm_ms", C.c_double), ("spmm_bytes", C.c_uint64), ("hbm_in_use", C.c_size_t),
                ("tune_entries", C.c_uint64)]


class mge_ops_opts(C.Structure):
    _fields_ = [("precision", C.c_int), ("eps_override_set", C.c_int), ("eps_override", C.c_double),
                ("mu_override_set", C.c_int), ("mu_override", C.c_double), ("eps_tol", C.c_double),
                ("eps_guard", C.c_int), ("eps_maxiter", C.c_int), ("seed", C.c_uint64),
                ("stream", C.c_void_p), ("eps_precond_degree", C.c_int), ("keep_order", C.c_int)]


class mge_ops_info_t(C.Structure):
    _fields_ = [("n", C.c_int64), ("nnz_w", C.c_int64), ("nnz_a", C.c_int64), ("nnz_q", C.c_int64),
                ("eps", C.c_double), ("mu", C.c_double), ("norm_a", C.c_double), ("bmax", C.c_double),
                ("degenerate", C.c_int), ("two_hop_components", C.c_int), ("eps_iters", C.c_int),
                ("eps_resid", C.c_double), ("build_ms", C.c_double)]


class mge_embed_opts(C.Structure):
    _fields_ = [("precision", C.c_int), ("guard", C.c_int), ("maxiter", C.c_int), ("seed", C.c_uint64),
                ("check_every", C.c_int), ("use_graph", C.c_int), ("x0", C.c_void_p), ("x0_cols", C.c_int),
                ("x0_on_device", C.c_int), ("v_on_device", C.c_int), ("stream", C.c_void_p),
                ("precond_degree", C.c_int), ("rr_fp64", C.c_int),
                ("gram_cuda_cores", C.c_int)]


class mge_embed_info(C.Structure):
    _fields_ = [("status", C.c_int), ("iters", C.c_int), ("m", C.c_int), ("drops", C.c_int),
                ("resid", C.c_double * 64), ("solve_ms", C.c_double), ("rr_fp64_from", C.c_int)]


class mge_request(C.Structure):
    _fields_ = [("n", C.c_int64), ("row_ptr", C.c_void_p), ("col", C.c_void_p), ("w", C.c_void_p),
                ("K", C.c_int), ("tol", C.c_double), ("precision", C.c_int), ("guard", C.c_int),
                ("maxiter", C.c_int), ("seed", C.c_uint64), ("points", C.c_void_p), ("dim", C.c_int),
                ("knn", C.c_int)]


class mge_result(C.Structure):
    _fields_ = [("status", C.c_int), ("n", C.c_int64), ("K", C.c_int), ("eps", C.c_double),
                ("mu", C.c_double), ("iters", C.c_int), ("latency_ms", C.c_double),
                ("queue_ms", C.c_double), ("lambda_", C.POINTER(C.c_double)), ("V", C.POINTER(C.c_double))]


_lib = None


def load(path: str = LIB_PATH):
    """Loads libmge.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_2112_07862_gb300.build.build()")
    lib = C.CDLL(path)
    vp, i, i64, d, u64, sz = C.c_void_p, C.c_int, C.c_int64, C.c_double, C.c_uint64, C.c_size_t
    sig = {
        "mge_create": (i, [i, sz, C.POINTER(vp)]),
        "mge_destroy": (i, [vp]),
        "mge_strerror": (C.c_char_p, [i]),
        "mge_ctx_last_error": (C.c_char_p, [vp]),
        "mge_ctx_stats": (i, [vp, C.POINTER(mge_stats)]),
        "mge_ctx_set_timing": (i, [vp, i]),
        "mge_ctx_reset_stats": (i, [vp]),
        "mge_ctx_set_autotune": (i, [vp, i, C.c_char_p]),
        "mge_build_graph_ops": (i, [vp, i64, vp, vp, vp, i, C.POINTER(mge_ops_opts), C.POINTER(vp)]),
        "mge_build_graph_ops_batch": (i, [vp, i, vp, vp, vp, vp, i, C.POINTER(mge_ops_opts), i, vp, vp]),
        "mge_ops_destroy": (i, [vp]),
        "mge_ops_info": (i, [vp, C.POINTER(mge_ops_info_t)]),
        "mge_ops_export": (i, [vp, vp, vp, vp, vp, vp, vp, vp, vp, i]),
        "mge_ops_node_order": (i, [vp, vp, i]),
        "mge_ops_apply": (i, [vp, vp, i, i, i, vp, vp, vp]),
        "mge_ops_apply_inplace": (i, [vp, vp, i, i, i, vp, vp]),
        "mge_embed": (i, [vp, vp, i, d, C.POINTER(mge_embed_opts), vp, vp, C.POINTER(mge_embed_info)]),
        "mge_embed_batch": (i, [vp, i, vp, vp, d, C.POINTER(mge_embed_opts), vp, vp, vp]),
        "mge_submit": (i, [vp, C.POINTER(mge_request), C.POINTER(u64)]),
        "mge_poll": (i, [vp, u64, i, C.POINTER(mge_result)]),
        "mge_release": (i, [vp, u64]),
        "mge_knn_graph": (i, [vp, i64, i, vp, i, i, vp, C.POINTER(vp)]),
        "mge_kmeans": (i, [vp, i64, i, vp, i, vp, i, i, vp, vp, C.POINTER(i), vp]),
        "mge_betweenness": (i, [vp, i64, vp, vp, i, vp, C.POINTER(d), vp]),
        "mge_graph_info": (i, [vp, C.POINTER(i64), C.POINTER(i64), C.POINTER(d)]),
        "mge_graph_csr": (i, [vp, C.POINTER(vp), C.POINTER(vp), C.POINTER(vp)]),
        "mge_graph_export": (i, [vp, vp, vp, vp, i]),
        "mge_graph_destroy": (i, [vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


class MgeError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{msg} (status {status})")
        self.status = status


def _ptr(a):
    """Host numpy array, torch tensor or raw address (int) -> address (None passes NULL)."""
    if a is None:
        return None
    if isinstance(a, int):
        return a
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data


# ---- one wrapper per C entry point ------------------------------------------------------

def mge_strerror(s: int) -> str:
    return load().mge_strerror(s).decode()


def mge_create(device: int = 0, hbm_budget_bytes: int = 0):
    h = C.c_void_p()
    s = load().mge_create(device, hbm_budget_bytes, C.byref(h))
    if s != MGE_OK:
        raise MgeError(s, f"mge_create: {mge_strerror(s)}")
    return h


def mge_destroy(ctx) -> int:
    return load().mge_destroy(ctx)


def mge_ctx_last_error(ctx) -> str:
    return load().mge_ctx_last_error(ctx).decode()


def mge_ctx_stats(ctx) -> mge_stats:
    st = mge_stats()
    load().mge_ctx_stats(ctx, C.byref(st))
    return st


def mge_ctx_set_timing(ctx, on: bool) -> int:
    return load().mge_ctx_set_timing(ctx, 1 if on else 0)


def mge_ctx_set_autotune(ctx, mode: int, cache_path: str | None = None) -> None:
    """mode 0 fixed rules, 1 tune new shapes (default), 2 known shapes only; cache_path: JSON file."""
    s = load().mge_ctx_set_autotune(ctx, int(mode), cache_path.encode() if cache_path else None)
    _check(ctx, s, "mge_ctx_set_autotune")


def mge_ctx_reset_stats(ctx) -> int:
    return load().mge_ctx_reset_stats(ctx)


def _check(ctx, s, what, ok=(MGE_OK,)):
    if s not in ok:
        raise MgeError(s, f"{what}: {mge_strerror(s)}: {mge_ctx_last_error(ctx)}")
    return s


def mge_build_graph_ops(ctx, n, row_ptr, col, w, on_device: bool = False, opts: mge_ops_opts | None = None):
    """Returns (ops handle, status).  Host inputs are numpy int64/int32/float64 arrays; device
    inputs are torch tensors of the same dtypes."""
    h = C.c_void_p()
    if not on_device:
        row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
        col = np.ascontiguousarray(col, dtype=np.int32)
        w = np.ascontiguousarray(w, dtype=np.float64)
    s = load().mge_build_graph_ops(ctx, int(n), _ptr(row_ptr), _ptr(col), _ptr(w), 1 if on_device else 0,
                                   C.byref(opts) if opts is not None else None, C.byref(h))
    _check(ctx, s, "mge_build_graph_ops", ok=(MGE_OK, MGE_EDEGENERATE))
    return h, s


def mge_knn_graph(ctx, points, k: int, stream=None):
    """kNN graph of the points (numpy [n, dim] float64 on the host, or a torch CUDA tensor).
    Returns the graph handle."""
    on_device = hasattr(points, "data_ptr")
    if not on_device:
        points = np.ascontiguousarray(points, dtype=np.float64)
    n, dim = int(points.shape[0]), int(points.shape[1])
    h = C.c_void_p()
    s = load().mge_knn_graph(ctx, n, dim, _ptr(points), 1 if on_device else 0, int(k), stream, C.byref(h))
    _check(ctx, s, "mge_knn_graph")
    return h


def mge_betweenness(ctx, n, row_ptr, col, stream=None):
    """Betweenness centralities (numpy [n] on the host path, a torch tensor when row_ptr and
    col are torch CUDA tensors) and the VBC."""
    vbc = C.c_double()
    if hasattr(row_ptr, "data_ptr"):
        import torch
        cb = torch.empty(int(n), dtype=torch.float64, device=row_ptr.device)
        s = load().mge_betweenness(ctx, int(n), _ptr(row_ptr), _ptr(col), 1, _ptr(cb), C.byref(vbc), stream)
    else:
        rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
        cl = np.ascontiguousarray(col, dtype=np.int32)
        cb = np.empty(int(n), np.float64)
        s = load().mge_betweenness(ctx, int(n), _ptr(rp), _ptr(cl), 0, _ptr(cb), C.byref(vbc), stream)
    _check(ctx, s, "mge_betweenness")
    return cb, vbc.value


def mge_kmeans(ctx, X, centres0, max_iters: int, stream=None):
    """k-means of the rows of X (numpy [n, K] float64, or a torch CUDA tensor [K, n] -- the
    column-major layout mge_embed returns V in) from centres0 [C, K].  Returns (assign int32
    [n], centres [C, K], assignment steps) as numpy arrays on the host path, torch tensors on
    the device path."""
    iters = C.c_int()
    if hasattr(X, "data_ptr"):
        import torch
        K, n = int(X.shape[0]), int(X.shape[1])
        c0 = centres0.contiguous()
        a = torch.empty(n, dtype=torch.int32, device=X.device)
        cen = torch.empty_like(c0)
        s = load().mge_kmeans(ctx, n, K, _ptr(X), int(c0.shape[0]), _ptr(c0), int(max_iters), 1, _ptr(a),
                              _ptr(cen), C.byref(iters), stream)
    else:
        Xc = np.asfortranarray(X, dtype=np.float64)             # column-major [n x K]
        n, K = Xc.shape
        c0 = np.ascontiguousarray(centres0, dtype=np.float64)
        a = np.empty(n, np.int32)
        cen = np.empty_like(c0)
        s = load().mge_kmeans(ctx, n, K, Xc.ctypes.data, int(c0.shape[0]), _ptr(c0), int(max_iters), 0, _ptr(a),
                              _ptr(cen), C.byref(iters), stream)
    _check(ctx, s, "mge_kmeans")
    return a, cen, iters.value


def mge_graph_info(g):
    n, nnz, sigma = C.c_int64(), C.c_int64(), C.c_double()
    s = load().mge_graph_info(g, C.byref(n), C.byref(nnz), C.byref(sigma))
    if s != MGE_OK:
        raise MgeError(s, "mge_graph_info")
    return n.value, nnz.value, sigma.value


def mge_graph_csr(g):
    """Borrowed device pointers (row_ptr, col, w) of the graph."""
    rp, col, w = C.c_void_p(), C.c_void_p(), C.c_void_p()
    s = load().mge_graph_csr(g, C.byref(rp), C.byref(col), C.byref(w))
    if s != MGE_OK:
        raise MgeError(s, "mge_graph_csr")
    return rp.value, col.value, w.value


def mge_graph_export(g):
    """Host copies (row_ptr int64, col int32, w float64) of the graph's CSR."""
    n, nnz, _ = mge_graph_info(g)
    rp = np.empty(n + 1, np.int64)
    col = np.empty(nnz, np.int32)
    w = np.empty(nnz, np.float64)
    s = load().mge_graph_export(g, _ptr(rp), _ptr(col), _ptr(w), 0)
    if s != MGE_OK:
        raise MgeError(s, "mge_graph_export")
    return rp, col, w


def mge_graph_destroy(g) -> int:
    return load().mge_graph_destroy(g)


def mge_build_graph_ops_batch(ctx, graphs, on_device: bool = False, opts: mge_ops_opts | None = None,
                              workers: int = 0):
    """graphs: a list of (n, row_ptr, col, w) (numpy arrays, or torch CUDA tensors when
    on_device).  Returns (list of handles, None where a build failed; list of statuses;
    status)."""
    count = len(graphs)
    keep = []
    ns = (C.c_int64 * count)()
    rps, cols, ws = (C.c_void_p * count)(), (C.c_void_p * count)(), (C.c_void_p * count)()
    for i, (n, rp, col, w) in enumerate(graphs):
        if not on_device:
            rp = np.ascontiguousarray(rp, dtype=np.int64)
            col = np.ascontiguousarray(col, dtype=np.int32)
            w = np.ascontiguousarray(w, dtype=np.float64)
        keep.append((rp, col, w))
        ns[i], rps[i], cols[i], ws[i] = int(n), _ptr(rp), _ptr(col), _ptr(w)
    out = (C.c_void_p * count)()
    sts = (C.c_int * count)()
    s = load().mge_build_graph_ops_batch(ctx, count, ns, rps, cols, ws, 1 if on_device else 0,
                                         C.byref(opts) if opts is not None else None, int(workers), out, sts)
    _check(ctx, s, "mge_build_graph_ops_batch", ok=(MGE_OK, MGE_EDEGENERATE))
    return [C.c_void_p(h) if h else None for h in out], list(sts), s


def mge_ops_destroy(ops) -> int:
    return load().mge_ops_destroy(ops)


def mge_ops_info(ops) -> mge_ops_info_t:
    info = mge_ops_info_t()
    load().mge_ops_info(ops, C.byref(info))
    return info


def mge_ops_export(ops):
    """Host copies of A, Q (CSR, FP64), b and T as numpy arrays."""
    info = mge_ops_info(ops)
    n, na, nq = info.n, info.nnz_a, info.nnz_q
    a_ptr = np.empty(n + 1, np.int64); a_col = np.empty(na, np.int32); a_val = np.empty(na, np.float64)
    q_ptr = np.empty(n + 1, np.int64); q_col = np.empty(nq, np.int32); q_val = np.empty(nq, np.float64)
    b = np.empty(n, np.float64); T = np.empty(n, np.int32)
    s = load().mge_ops_export(ops, _ptr(a_ptr), _ptr(a_col), _ptr(a_val), _ptr(q_ptr), _ptr(q_col),
                              _ptr(q_val), _ptr(b), _ptr(T), 0)
    if s != MGE_OK:
        raise MgeError(s, "mge_ops_export")
    return dict(a_ptr=a_ptr, a_col=a_col, a_val=a_val, q_ptr=q_ptr, q_col=q_col, q_val=q_val, b=b, T=T)


def mge_ops_node_order(ops):
    """The library's node order: order[r] = the caller's node in row r of the operators."""
    n = mge_ops_info(ops).n
    order = np.empty(n, np.int32)
    s = load().mge_ops_node_order(ops, _ptr(order), 0)
    if s != MGE_OK:
        raise MgeError(s, "mge_ops_node_order")
    return order


def _check_block(ops, precision: int, m: int, t, name: str):
    """A block handed to an apply entry point: a contiguous CUDA tensor of shape (n, m)
    whose dtype is the precision's element type (the C entry point itself checks the
    pointer's alignment and memory type, but cannot see the tensor's size or dtype)."""
    import torch
    want = {MGE_FP64: torch.float64, MGE_FP32: torch.float32}.get(precision)
    n = mge_ops_info(ops).n
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.is_contiguous()):
        raise MgeError(MGE_EINVAL, f"{name} must be a contiguous CUDA tensor")
    if want is not None and t.dtype != want:
        raise MgeError(MGE_EINVAL, f"{name} has dtype {t.dtype}; precision {precision} needs {want}")
    if tuple(t.shape) != (n, m):
        raise MgeError(MGE_EINVAL, f"{name} has shape {tuple(t.shape)}; expected {(n, m)}")


def mge_ops_apply(ctx, ops, which: int, precision: int, m: int, X, Y, stream=None) -> int:
    """Y = A X (which=0) or Q X (which=1); X, Y torch CUDA tensors [n, m] row-major."""
    _check_block(ops, precision, m, X, "X")
    _check_block(ops, precision, m, Y, "Y")
    s = load().mge_ops_apply(ctx, ops, which, precision, m, _ptr(X), _ptr(Y), stream)
    return _check(ctx, s, "mge_ops_apply")


def mge_ops_apply_inplace(ctx, ops, which: int, precision: int, m: int, XY, stream=None) -> int:
    """XY <- A XY (which=0) or Q XY (which=1) in place; XY a torch CUDA tensor [n, m].  The
    library allocates nothing for it (a fixed 32 MiB device array holds the copy)."""
    _check_block(ops, precision, m, XY, "XY")
    s = load().mge_ops_apply_inplace(ctx, ops, which, precision, m, _ptr(XY), stream)
    return _check(ctx, s, "mge_ops_apply_inplace")


def mge_embed(ctx, ops, K: int, tol: float, opts: mge_embed_opts | None = None, V=None):
    """Returns (lambda[K] numpy, V, info, status).  V: a host numpy float64 array [K, n]
    (column-major n x K) or a device tensor when opts.v_on_device; allocated on the host
    when None."""
    info = mge_ops_info(ops)
    lam = np.empty(K, np.float64)
    if V is None and not (opts is not None and opts.v_on_device):
        V = np.empty((K, info.n), np.float64)
    ei = mge_embed_info()
    s = load().mge_embed(ctx, ops, K, float(tol), C.byref(opts) if opts is not None else None,
                         _ptr(lam), _ptr(V), C.byref(ei))
    _check(ctx, s, "mge_embed", ok=(MGE_OK, MGE_ENOTCONVERGED))
    return lam, V, ei, s


def mge_embed_batch(ctx, ops, K, tol: float, opts: mge_embed_opts | None = None, V=None):
    """Batched mge_embed over the handles `ops` with K[i] pairs each, in one graph launch.
    Returns (list of lambda arrays, list of V, list of mge_embed_info, status).  V: None
    (host arrays [K_i, n_i] are allocated unless opts.v_on_device), or a list of host numpy
    float64 arrays / device tensors [K_i, n_i] (column-major n_i x K_i), entries may be None."""
    count = len(ops)
    K = [int(k) for k in K]
    if len(K) != count:
        raise ValueError("ops and K differ in length")
    on_dev = opts is not None and opts.v_on_device
    lams = [np.empty(k, np.float64) for k in K]
    if V is None:
        V = [None] * count if on_dev else [np.empty((k, mge_ops_info(o).n), np.float64) for o, k in zip(ops, K)]
    handles = (C.c_void_p * count)(*[o.value if isinstance(o, C.c_void_p) else o for o in ops])
    ks = (C.c_int * count)(*K)
    lam_p = (C.c_void_p * count)(*[_ptr(a) for a in lams])
    v_p = (C.c_void_p * count)(*[_ptr(v) for v in V])
    infos = (mge_embed_info * count)()
    s = load().mge_embed_batch(ctx, count, handles, ks, float(tol), C.byref(opts) if opts is not None else None,
                               lam_p, v_p, infos)
    _check(ctx, s, "mge_embed_batch", ok=(MGE_OK, MGE_ENOTCONVERGED))
    return lams, V, list(infos), s


def mge_submit(ctx, req: mge_request) -> int:
    t = C.c_uint64()
    s = load().mge_submit(ctx, C.byref(req), C.byref(t))
    _check(ctx, s, "mge_submit")
    return t.value


def mge_poll(ctx, ticket: int, timeout_ms: int = -1):
    r = mge_result()
    s = load().mge_poll(ctx, ticket, timeout_ms, C.byref(r))
    return s, r


def mge_release(ctx, ticket: int) -> int:
    return load().mge_release(ctx, ticket)


# ---- conveniences ------------------------------------------------------------------------

def ops_opts(precision="fp32", eps=None, mu=None, eps_tol=0.0, seed=0, stream=None, eps_guard=0,
             eps_maxiter=0, eps_precond_degree=0, keep_order=False) -> mge_ops_opts:
    o = mge_ops_opts()
    o.precision = PRECISION[precision] if isinstance(precision, str) else int(precision)
    if eps is not None:
        o.eps_override_set, o.eps_override = 1, float(eps)
    if mu is not None:
        o.mu_override_set, o.mu_override = 1, float(mu)
    o.eps_tol = eps_tol
    o.eps_guard = eps_guard
    o.eps_maxiter = eps_maxiter
    o.seed = seed
    o.stream = stream
    o.eps_precond_degree = eps_precond_degree
    o.keep_order = 1 if keep_order else 0
    return o


def embed_opts(precision="fp32", guard=0, maxiter=0, seed=0, check_every=0, use_graph=True, x0=None,
               v_on_device=False, stream=None, precond_degree=0, rr_fp64=False,
               gram_cuda_cores=False) -> mge_embed_opts:
    o = mge_embed_opts()
    o.precision = PRECISION[precision] if isinstance(precision, str) else int(precision)
    o.guard = guard
    o.maxiter = maxiter
    o.seed = seed
    o.check_every = check_every
    o.use_graph = 1 if use_graph else 0
    if x0 is not None:
        o.x0 = _ptr(x0)
        o.x0_cols = x0.shape[0]
        o.x0_on_device = 1 if hasattr(x0, "data_ptr") else 0
    o.v_on_device = 1 if v_on_device else 0
    o.stream = stream
    o.precond_degree = precond_degree
    # True / 1: FP64 throughout; False / 0: automatic; -1: FP32 throughout
    o.rr_fp64 = int(rr_fp64)
    o.gram_cuda_cores = 1 if gram_cuda_cores else 0
    return o


class Context:
    """Owns an mge_ctx; closes it on exit."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0):
        self.h = mge_create(device, hbm_budget_bytes)

    def close(self):
        if self.h:
            mge_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def build(self, g, **kw):
        """Operators for a manifold_graphs.Graph-like object (n, row_ptr, col, w) on the host."""
        ops, s = mge_build_graph_ops(self.h, g.n, g.row_ptr, g.col, g.w, False, ops_opts(**kw))
        return Ops(ops, s)

    def embed(self, ops, K, tol, **kw):
        lam, V, info, s = mge_embed(self.h, ops.h, K, tol, embed_opts(**kw))
        return lam, V.T if isinstance(V, np.ndarray) else V, info, s

    def build_batch(self, graphs, workers=0, **kw):
        hs, sts, s = mge_build_graph_ops_batch(self.h, [(g.n, g.row_ptr, g.col, g.w) for g in graphs], False,
                                               ops_opts(**kw), workers)
        return [Ops(h, st) for h, st in zip(hs, sts)]

    def embed_batch(self, ops, K, tol, **kw):
        lams, Vs, infos, s = mge_embed_batch(self.h, [o.h for o in ops], K, tol, embed_opts(**kw))
        return lams, [v.T if isinstance(v, np.ndarray) else v for v in Vs], infos, s

    def stats(self):
        return mge_ctx_stats(self.h)


class Ops:
    def __init__(self, h, status):
        self.h = h
        self.status = status

    def info(self):
        return mge_ops_info(self.h)

    def export(self):
        return mge_ops_export(self.h)

    def node_order(self):
        return mge_ops_node_order(self.h)

    def close(self):
        if self.h:
            mge_ops_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
