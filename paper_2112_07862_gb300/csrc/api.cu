// C ABI entry points of libmge (declared in include/mge.h).
#include "mge_internal.cuh"

#include <algorithm>
#include <memory>
#include <thread>
#include <vector>

#include <cstdarg>
#include <cstring>

namespace mge {

mge_status build_graph_ops_impl(Ctx* ctx, cudaStream_t st, int64_t n, const int64_t* rp_in,
                                const int32_t* col_in, const double* w_in, int on_device,
                                const mge_ops_opts* opts, Ops* ops);
mge_status serve_submit(Ctx* ctx, const mge_request* req, uint64_t* ticket);
mge_status serve_poll(Ctx* ctx, uint64_t ticket, int timeout_ms, mge_result* out);
mge_status serve_release(Ctx* ctx, uint64_t ticket);
void serve_shutdown(Ctx* ctx);

void set_error(Ctx* ctx, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (ctx) {
    std::lock_guard<std::mutex> g(ctx->err_mu);
    ctx->last_error = buf;
  }
}

mge_status dev_alloc(Ctx* ctx, void** p, size_t bytes) {
  if (ctx->budget && ctx->in_use.load() + bytes > ctx->budget) {
    set_error(ctx, "HBM budget exceeded: %zu in use + %zu requested > %zu", ctx->in_use.load(), bytes,
              ctx->budget);
    return MGE_ENOMEM;
  }
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    set_error(ctx, "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
    *p = nullptr;
    return MGE_ENOMEM;
  }
  ctx->in_use += bytes;
  return MGE_OK;
}

void dev_free(Ctx* ctx, void* p, size_t bytes) {
  if (!p) return;
  cudaFree(p);
  if (ctx) ctx->in_use -= bytes;
}

PersistentPool& persistent_pool() {
  static thread_local PersistentPool p;
  return p;
}

mge_status dev_alloc_async(Ctx* ctx, void** p, size_t bytes, cudaStream_t st) {
  if (!ctx->pool) return dev_alloc(ctx, p, bytes);
  if (ctx->budget && ctx->in_use.load() + bytes > ctx->budget) {
    set_error(ctx, "HBM budget exceeded: %zu in use + %zu requested > %zu", ctx->in_use.load(), bytes,
              ctx->budget);
    return MGE_ENOMEM;
  }
  cudaError_t e = cudaMallocFromPoolAsync(p, bytes, ctx->pool, st);
  if (e != cudaSuccess) {
    set_error(ctx, "cudaMallocFromPoolAsync(%zu): %s", bytes, cudaGetErrorString(e));
    *p = nullptr;
    return MGE_ENOMEM;
  }
  ctx->in_use += bytes;
  return MGE_OK;
}

void dev_free_async(Ctx* ctx, void* p, size_t bytes, cudaStream_t st) {
  if (!p) return;
  if (!ctx || !ctx->pool) { dev_free(ctx, p, bytes); return; }
  cudaFreeAsync(p, st);
  ctx->in_use -= bytes;
}

static cudaStream_t pick_stream(Ctx* ctx, void* s) {
  return s ? static_cast<cudaStream_t>(s) : ctx->stream;
}

// Arithmetic of the Rayleigh-Ritz eigensolve and of W's Cholesky for reduced-precision
// blocks: FP64 when opts.rr_fp64 is set (FP64 blocks always)
static bool rr_fp64_for(const mge_embed_opts& e, int prec) {
  return prec == MGE_FP64 || e.rr_fp64 > 0;
}

// Extra LOBPCG columns beyond K: opts.guard > 0 as given, < 0 none, 0 the default of K more
// (block width 2K, at most the widest block, 24).  The K-th pair converges at a rate set by
// lambda_K / lambda_{m+1}; with no guard that ratio is the gap to the next eigenvalue, which
// on manifold graphs is about 1% (measured on a 200k-node swiss roll, K = 8: 100 iterations
// at m = 8, 27 at m = 16 for a relative residual of 1e-5).
static int guard_for(const mge_embed_opts& e, int K) {
  if (e.guard > 0) return e.guard;
  if (e.guard < 0) return 0;
  return std::max(0, std::min(K, 24 - K));
}

// Widths the operator-product entry points support (the SpMM kernel's instantiations).
static bool apply_width_ok(int m) { return m == 4 || m == 8 || m == 12 || m == 16 || m == 24; }

// A block pointer handed to mge_ops_apply[_inplace]: 16-byte aligned (the kernels read
// rows with 16-byte loads and bulk copies) and device memory of the context's device (a
// host or foreign pointer would fault inside the kernel).  Checked on the host before any
// launch, so a bad pointer returns MGE_EINVAL with the buffer untouched.
static mge_status check_block_ptr(Ctx* ctx, const void* p, const char* who, const char* name) {
  if (reinterpret_cast<uintptr_t>(p) & 15u) {
    set_error(ctx, "%s: %s is not 16-byte aligned", who, name);
    return MGE_EINVAL;
  }
  cudaPointerAttributes a{};
  cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error(ctx, "%s: %s is not a CUDA pointer", who, name);
    return MGE_EINVAL;
  }
  if ((a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged) || a.device != ctx->device) {
    set_error(ctx, "%s: %s is not device memory of device %d", who, name, ctx->device);
    return MGE_EINVAL;
  }
  return MGE_OK;
}

}  // namespace mge

using namespace mge;

extern "C" {

const char* mge_strerror(mge_status s) {
  switch (s) {
    case MGE_OK: return "ok";
    case MGE_EINVAL: return "invalid argument";
    case MGE_ENOTSYM: return "W is not symmetric";
    case MGE_EISOLATED: return "isolated node: B is singular";
    case MGE_EDEGENERATE: return "eps = 0: the two-hop graph is disconnected";
    case MGE_ENOTCONVERGED: return "not converged within maxiter";
    case MGE_ENOMEM: return "out of device memory or HBM budget";
    case MGE_EAGAIN: return "queue or budget full; retry";
    case MGE_ETIMEOUT: return "timed out";
    case MGE_EDEVICE: return "CUDA error";
    case MGE_ECHOLESKY: return "Rayleigh-Ritz basis collapsed";
    case MGE_ENOTFOUND: return "unknown ticket";
    case MGE_ENOTFINITE: return "non-finite value in the iteration";
  }
  return "unknown status";
}

mge_status mge_create(int device, size_t hbm_budget_bytes, mge_ctx** out) {
  if (!out) return MGE_EINVAL;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return MGE_EINVAL;
  if (cudaSetDevice(device) != cudaSuccess) return MGE_EDEVICE;
  mge_ctx* c = new mge_ctx();
  Ctx* ctx = &c->impl;
  ctx->device = device;
  ctx->budget = hbm_budget_bytes;
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) { delete c; return MGE_EDEVICE; }
  ctx->num_sms = prop.multiProcessorCount;
  ctx->self = c;
  if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) { delete c; return MGE_EDEVICE; }
  {
    // the scratch pool keeps what it is given back (release threshold: never)
    cudaMemPoolProps pp = {};
    pp.allocType = cudaMemAllocationTypePinned;
    pp.location.type = cudaMemLocationTypeDevice;
    pp.location.id = device;
    if (cudaMemPoolCreate(&ctx->pool, &pp) == cudaSuccess) {
      uint64_t keep = ~0ull;
      cudaMemPoolSetAttribute(ctx->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    } else {
      ctx->pool = nullptr;
      cudaGetLastError();
    }
  }
  *out = c;
  return MGE_OK;
}

// The context's host object lives until the last ops handle built from it is destroyed, so
// an ops handle may outlive mge_destroy (its device memory is released by mge_ops_destroy).
static void ctx_release(Ctx* ctx) {
  if (--ctx->refs == 0) {
    cudaSetDevice(ctx->device);
    if (ctx->pool) {
      cudaDeviceSynchronize();          // every scratch free has completed
      cudaMemPoolDestroy(ctx->pool);
    }
    for (void* h : ctx->state_host) cudaFreeHost(h);
    delete static_cast<mge_ctx*>(ctx->self);
  }
}

mge_status mge_destroy(mge_ctx* c) {
  if (!c) return MGE_EINVAL;
  Ctx* ctx = &c->impl;
  if (ctx->closed) return MGE_EINVAL;
  ctx->closed = true;
  cudaSetDevice(ctx->device);
  serve_shutdown(ctx);
  for (auto& e : ctx->ev_pool) { cudaEventDestroy(e.first); cudaEventDestroy(e.second); }
  ctx->ev_pool.clear();
  if (ctx->stream) cudaStreamDestroy(ctx->stream);
  ctx->stream = nullptr;
  ctx_release(ctx);
  return MGE_OK;
}

const char* mge_ctx_last_error(const mge_ctx* c) {
  if (!c) return "null context";
  return c->impl.last_error.c_str();
}

mge_status mge_ctx_stats(const mge_ctx* c, mge_stats* out) {
  if (!c || !out) return MGE_EINVAL;
  const Ctx* ctx = &c->impl;
  out->kernel_launches = ctx->kernel_launches.load();
  out->spmm_launches = ctx->spmm_launches;
  out->spmm_ms = ctx->spmm_ms;
  out->spmm_bytes = ctx->spmm_bytes;
  out->hbm_in_use = ctx->in_use.load();
  {
    std::lock_guard<std::mutex> lock(const_cast<Ctx*>(ctx)->tune_mu);
    out->tune_entries = ctx->tune.size();
  }
  return MGE_OK;
}

mge_status mge_ctx_set_autotune(mge_ctx* c, int mode, const char* cache_path) {
  if (!c) return MGE_EINVAL;
  return tune_set(&c->impl, mode, cache_path);
}

mge_status mge_ctx_set_timing(mge_ctx* c, int on) {
  if (!c) return MGE_EINVAL;
  c->impl.timing = on != 0;
  return MGE_OK;
}

mge_status mge_ctx_reset_stats(mge_ctx* c) {
  if (!c) return MGE_EINVAL;
  c->impl.kernel_launches = 0;
  c->impl.spmm_launches = 0;
  c->impl.spmm_ms = 0;
  c->impl.spmm_bytes = 0;
  return MGE_OK;
}

mge_status mge_build_graph_ops(mge_ctx* c, int64_t n, const int64_t* row_ptr, const int32_t* col,
                               const double* w, int on_device, const mge_ops_opts* opts, mge_ops** out) {
  if (!c || !out) return MGE_EINVAL;
  *out = nullptr;
  Ctx* ctx = &c->impl;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return MGE_EDEVICE;
  cudaStream_t st = pick_stream(ctx, opts ? opts->stream : nullptr);
  if (ctx->closed) return MGE_EINVAL;
  mge_ops* o = new mge_ops();
  ctx->refs++;
  mge_status s = build_graph_ops_impl(ctx, st, n, row_ptr, col, w, on_device, opts, &o->impl);
  if (s != MGE_OK && s != MGE_EDEGENERATE) {
    delete o;
    ctx_release(ctx);
    return s;
  }
  *out = o;
  return s;
}

mge_status mge_build_graph_ops_batch(mge_ctx* c, int count, const int64_t* n, const int64_t* const* row_ptr,
                                     const int32_t* const* col, const double* const* w, int on_device,
                                     const mge_ops_opts* opts, int workers, mge_ops** out, mge_status* status) {
  NvtxRange nvtx_range("mge.build_batch");
  if (!c || count < 1 || !n || !row_ptr || !col || !w || !out) return MGE_EINVAL;
  Ctx* ctx = &c->impl;
  if (ctx->closed) return MGE_EINVAL;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return MGE_EDEVICE;
  for (int i = 0; i < count; ++i) out[i] = nullptr;
  // device inputs may still be in flight on the caller's stream
  if (on_device) MGE_CUDA(ctx, cudaStreamSynchronize(pick_stream(ctx, opts ? opts->stream : nullptr)));
  mge_ops_opts oo{};
  oo.precision = MGE_FP32;
  if (opts) oo = *opts;
  // graph i is built by worker i % nw on that worker's stream, in both phases
  const int nw = std::max(1, std::min(workers > 0 ? workers : 8, count));
  std::vector<cudaStream_t> streams((size_t)nw, nullptr);
  for (int t = 0; t < nw; ++t) MGE_CUDA(ctx, cudaStreamCreateWithFlags(&streams[t], cudaStreamNonBlocking));
  std::vector<mge_status> sts((size_t)count, MGE_EDEVICE);    // stays so for a graph no worker took
  std::vector<std::unique_ptr<BuildState>> bss((size_t)count);
  std::vector<double> eps((size_t)count, 0.0);
  auto run_workers = [&](auto&& fn) {
    std::vector<std::thread> pool;
    auto work = [&](int t) {
      if (cudaSetDevice(ctx->device) != cudaSuccess) return;
      for (int i = t; i < count; i += nw) fn(i, streams[t]);
    };
    for (int t = 1; t < nw; ++t) {
      try {
        pool.emplace_back(work, t);
      } catch (...) {
        break;
      }
    }
    work(0);
    for (auto& th : pool) th.join();
    // a worker that could not be started leaves its graphs with MGE_EDEVICE
  };
  // phase 1: everything up to the eps solve
  run_workers([&](int i, cudaStream_t s) {
    mge_ops* o = new mge_ops();
    ctx->refs++;
    bss[i] = std::make_unique<BuildState>();
    mge_ops_opts local = oo;
    local.stream = s;
    sts[i] = build_phase1(ctx, s, n[i], row_ptr[i], col[i], w[i], on_device, &local, &o->impl, bss[i].get());
    if (sts[i] != MGE_OK) {
      bss[i].reset();
      delete o;
      ctx_release(ctx);
      return;
    }
    out[i] = o;
  });
  // phase 2: every eps solve as a branch of one CUDA graph launch
  std::vector<int> idx;
  for (int i = 0; i < count; ++i)
    if (sts[i] == MGE_OK && bss[i]->need_eps) idx.push_back(i);
  if (!idx.empty()) {
    const int ne = (int)idx.size();
    std::vector<LobOp> qops((size_t)ne);
    std::vector<int> Ks((size_t)ne, 1), ms((size_t)ne);
    std::vector<LobResult> res((size_t)ne);
    std::vector<mge_status> est((size_t)ne, MGE_OK);
    for (int e = 0; e < ne; ++e) { qops[e] = bss[idx[e]]->qop; ms[e] = bss[idx[e]]->eps_m; }
    const BuildState& b0 = *bss[idx[0]];
    double ms_batch = 0;
    mge_status s = lobpcg_solve_batch(ctx, streams[0], ne, qops.data(), b0.eps_precision, Ks.data(), ms.data(),
                                      b0.eps_tol, b0.eps_maxiter, b0.eps_seed, nullptr, res.data(), est.data(),
                                      &ms_batch);
    for (int e = 0; e < ne; ++e) {
      const int i = idx[e];
      const mge_status si = (s != MGE_OK && s != MGE_ENOTCONVERGED) ? s : est[e];
      if (si != MGE_OK && si != MGE_ENOTCONVERGED) { sts[i] = si; continue; }
      eps[i] = res[e].lambda.empty() ? 0.0 : res[e].lambda[0];
      out[i]->impl.eps_iters = res[e].iters;
      out[i]->impl.eps_resid = res[e].eta.empty() ? 0.0 : res[e].eta[0];
    }
  }
  // phase 3: mu, A, B and the preconditioner's operator
  run_workers([&](int i, cudaStream_t s) {
    (void)s;
    if (!out[i]) return;
    if (sts[i] == MGE_OK) sts[i] = build_phase3(bss[i].get(), &out[i]->impl, eps[i]);
    bss[i].reset();
    if (sts[i] != MGE_OK && sts[i] != MGE_EDEGENERATE) {
      out[i]->impl.each_buffer([](auto& b) { if (b.pooled) b.st = cudaStreamPerThread; });
      delete out[i];
      out[i] = nullptr;
      ctx_release(ctx);
    }
  });
  for (auto s : streams) {
    cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
  }
  mge_status first = MGE_OK;
  for (int i = 0; i < count; ++i) {
    if (status) status[i] = sts[i];
    if (first == MGE_OK && sts[i] != MGE_OK && sts[i] != MGE_EDEGENERATE) first = sts[i];
  }
  return first;
}

mge_status mge_ops_destroy(mge_ops* o) {
  if (!o) return MGE_EINVAL;
  Ctx* ctx = o->impl.ctx;
  if (ctx) cudaSetDevice(ctx->device);
  // Every call that uses the handle has finished its device work when it returns (each one
  // synchronises its stream), so the pooled arrays go back to the pool at once, ordered on
  // this thread's per-thread default stream (the stream of the build may be gone).  No
  // device-wide synchronisation: that would invalidate a graph capture another host thread
  // (a serving slot) has in progress.
  o->impl.each_buffer([](auto& b) { if (b.pooled) b.st = cudaStreamPerThread; });
  delete o;
  if (ctx) ctx_release(ctx);
  return MGE_OK;
}

mge_status mge_ops_info(const mge_ops* o, mge_ops_info_t* out) {
  if (!o || !out) return MGE_EINVAL;
  const Ops& op = o->impl;
  out->n = op.n; out->nnz_w = op.nnz_w; out->nnz_a = op.nnz_a; out->nnz_q = op.nnz_q;
  out->eps = op.eps; out->mu = op.mu; out->norm_a = op.norm_a; out->bmax = op.bmax;
  out->degenerate = op.degenerate; out->two_hop_components = op.ncomp;
  out->eps_iters = op.eps_iters; out->eps_resid = op.eps_resid; out->build_ms = op.build_ms;
  return MGE_OK;
}

// CSR of an operator in the library's node order -> the caller's order (host arrays): row i
// is internal row rank[i], columns renamed by order and sorted ascending
static void csr_to_caller(int64_t n, const std::vector<int64_t>& rp, const std::vector<int32_t>& col,
                          const std::vector<double>& val, const std::vector<int32_t>& order,
                          const std::vector<int32_t>& rank, std::vector<int64_t>& rp2, std::vector<int32_t>& col2,
                          std::vector<double>& val2) {
  rp2.assign(n + 1, 0);
  for (int64_t i = 0; i < n; ++i) rp2[i + 1] = rp2[i] + (rp[rank[i] + 1] - rp[rank[i]]);
  col2.resize(col.size());
  val2.resize(val.size());
  std::vector<std::pair<int32_t, double>> row;
  for (int64_t i = 0; i < n; ++i) {
    const int64_t s = rp[rank[i]], e = rp[rank[i] + 1];
    row.clear();
    for (int64_t p = s; p < e; ++p) row.emplace_back(order[col[p]], val.empty() ? 0.0 : val[p]);
    std::sort(row.begin(), row.end(), [](const auto& a, const auto& b) { return a.first < b.first; });
    for (size_t k = 0; k < row.size(); ++k) {
      col2[rp2[i] + k] = row[k].first;
      if (!val2.empty()) val2[rp2[i] + k] = row[k].second;
    }
  }
}

mge_status mge_ops_export(const mge_ops* o, int64_t* a_ptr, int32_t* a_col, double* a_val, int64_t* q_ptr,
                          int32_t* q_col, double* q_val, double* b, int32_t* T, int on_device) {
  if (!o) return MGE_EINVAL;
  const Ops& op = o->impl;
  Ctx* ctx = op.ctx;
  cudaSetDevice(ctx->device);
  cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  cudaStream_t st = ctx->closed ? nullptr : ctx->stream;
  if (!op.order.p) {
    if (a_ptr) MGE_CUDA(ctx, cudaMemcpyAsync(a_ptr, op.a_ptr.p, (op.n + 1) * sizeof(int64_t), k, st));
    if (a_col && op.nnz_a) MGE_CUDA(ctx, cudaMemcpyAsync(a_col, op.a_col.p, op.nnz_a * sizeof(int32_t), k, st));
    if (a_val && op.nnz_a) MGE_CUDA(ctx, cudaMemcpyAsync(a_val, op.a_val.p, op.nnz_a * sizeof(double), k, st));
    if (q_ptr) MGE_CUDA(ctx, cudaMemcpyAsync(q_ptr, op.q_ptr.p, (op.n + 1) * sizeof(int64_t), k, st));
    if (q_col && op.nnz_q) MGE_CUDA(ctx, cudaMemcpyAsync(q_col, op.q_col.p, op.nnz_q * sizeof(int32_t), k, st));
    if (q_val && op.nnz_q) MGE_CUDA(ctx, cudaMemcpyAsync(q_val, op.q_val.p, op.nnz_q * sizeof(double), k, st));
    if (b) MGE_CUDA(ctx, cudaMemcpyAsync(b, op.b.p, op.n * sizeof(double), k, st));
    if (T) MGE_CUDA(ctx, cudaMemcpyAsync(T, op.T.p, op.n * sizeof(int32_t), k, st));
    MGE_CUDA(ctx, cudaStreamSynchronize(st));
    return MGE_OK;
  }
  // renumbered operators: bring them to the host and rename them into the caller's order
  const int64_t n = op.n;
  std::vector<int32_t> order(n), rank(n);
  MGE_CUDA(ctx, cudaMemcpyAsync(order.data(), op.order.p, n * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  MGE_CUDA(ctx, cudaMemcpyAsync(rank.data(), op.rank.p, n * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  auto fetch = [&](const int64_t* dp, const int32_t* dc, const double* dv, int64_t nnz, std::vector<int64_t>& rp,
                   std::vector<int32_t>& c, std::vector<double>& v) -> mge_status {
    rp.resize(n + 1); c.resize(nnz); v.resize(nnz);
    MGE_CUDA(ctx, cudaMemcpyAsync(rp.data(), dp, (n + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    if (nnz) {
      MGE_CUDA(ctx, cudaMemcpyAsync(c.data(), dc, nnz * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
      MGE_CUDA(ctx, cudaMemcpyAsync(v.data(), dv, nnz * sizeof(double), cudaMemcpyDeviceToHost, st));
    }
    MGE_CUDA(ctx, cudaStreamSynchronize(st));
    return MGE_OK;
  };
  auto put = [&](void* dst, const void* src, size_t bytes) -> mge_status {
    if (!dst || !bytes) return MGE_OK;
    MGE_CUDA(ctx, cudaMemcpyAsync(dst, src, bytes, on_device ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost, st));
    return MGE_OK;
  };
  std::vector<int64_t> rp, rp2;
  std::vector<int32_t> c, c2;
  std::vector<double> v, v2;
  if (a_ptr || a_col || a_val) {
    MGE_TRY(fetch(op.a_ptr.p, op.a_col.p, op.a_val.p, op.nnz_a, rp, c, v));
    csr_to_caller(n, rp, c, v, order, rank, rp2, c2, v2);
    MGE_TRY(put(a_ptr, rp2.data(), (n + 1) * sizeof(int64_t)));
    MGE_TRY(put(a_col, c2.data(), op.nnz_a * sizeof(int32_t)));
    MGE_TRY(put(a_val, v2.data(), op.nnz_a * sizeof(double)));
    MGE_CUDA(ctx, cudaStreamSynchronize(st));
  }
  if (q_ptr || q_col || q_val) {
    MGE_TRY(fetch(op.q_ptr.p, op.q_col.p, op.q_val.p, op.nnz_q, rp, c, v));
    csr_to_caller(n, rp, c, v, order, rank, rp2, c2, v2);
    MGE_TRY(put(q_ptr, rp2.data(), (n + 1) * sizeof(int64_t)));
    MGE_TRY(put(q_col, c2.data(), op.nnz_q * sizeof(int32_t)));
    MGE_TRY(put(q_val, v2.data(), op.nnz_q * sizeof(double)));
    MGE_CUDA(ctx, cudaStreamSynchronize(st));
  }
  if (b) {
    std::vector<double> bi(n), bo(n);
    MGE_CUDA(ctx, cudaMemcpyAsync(bi.data(), op.b.p, n * sizeof(double), cudaMemcpyDeviceToHost, st));
    MGE_CUDA(ctx, cudaStreamSynchronize(st));
    for (int64_t i = 0; i < n; ++i) bo[i] = bi[rank[i]];
    MGE_TRY(put(b, bo.data(), n * sizeof(double)));
    MGE_CUDA(ctx, cudaStreamSynchronize(st));
  }
  if (T) {
    std::vector<int32_t> ti(n), to(n);
    MGE_CUDA(ctx, cudaMemcpyAsync(ti.data(), op.T.p, n * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    MGE_CUDA(ctx, cudaStreamSynchronize(st));
    for (int64_t i = 0; i < n; ++i) to[i] = ti[rank[i]];
    MGE_TRY(put(T, to.data(), n * sizeof(int32_t)));
    MGE_CUDA(ctx, cudaStreamSynchronize(st));
  }
  return MGE_OK;
}

mge_status mge_ops_node_order(const mge_ops* o, int32_t* order, int on_device) {
  if (!o || !order) return MGE_EINVAL;
  const Ops& op = o->impl;
  Ctx* ctx = op.ctx;
  cudaSetDevice(ctx->device);
  cudaStream_t st = ctx->closed ? nullptr : ctx->stream;
  if (op.order.p) {
    MGE_CUDA(ctx, cudaMemcpyAsync(order, op.order.p, op.n * sizeof(int32_t),
                                  on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
    MGE_CUDA(ctx, cudaStreamSynchronize(st));
    return MGE_OK;
  }
  std::vector<int32_t> id(op.n);
  for (int64_t i = 0; i < op.n; ++i) id[i] = (int32_t)i;
  MGE_CUDA(ctx, cudaMemcpyAsync(order, id.data(), op.n * sizeof(int32_t),
                                on_device ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost, st));
  MGE_CUDA(ctx, cudaStreamSynchronize(st));
  return MGE_OK;
}

// ---- kNN graph from points -------------------------------------------------------------

mge_status mge_knn_graph(mge_ctx* c, int64_t n, int dim, const double* points, int on_device, int k,
                         void* stream, mge_graph** out) {
  NvtxRange nvtx_range("mge.knn_graph");
  if (!c || !out || !points) return MGE_EINVAL;
  *out = nullptr;
  Ctx* ctx = &c->impl;
  if (ctx->closed) return MGE_EINVAL;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return MGE_EDEVICE;
  if (n < 2 || dim < 2 || dim > 3 || k < 1 || k > 32 || k >= n) {
    set_error(ctx, "knn_graph: need dim in {2, 3}, 1 <= k <= 32 and k < n");
    return MGE_EINVAL;
  }
  cudaStream_t st = pick_stream(ctx, stream);
  if (on_device) MGE_TRY(check_block_ptr(ctx, points, "knn_graph", "points"));
  mge_graph* g = new mge_graph();
  g->impl.ctx = ctx;
  ctx->refs++;
  mge_status s;
  {
    PersistentPoolScope pool_scope(st);      // the graph's arrays come from the context's pool
    DevBuf<double> pd;
    const double* P = points;
    s = MGE_OK;
    if (!on_device) {
      s = pd.scratch(ctx, (size_t)n * dim, st);
      if (s == MGE_OK) {
        cudaError_t e = cudaMemcpyAsync(pd.p, points, (size_t)n * dim * sizeof(double), cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) { set_error(ctx, "knn_graph: copy of the points: %s", cudaGetErrorString(e)); s = MGE_EDEVICE; }
      }
      P = pd.p;
    }
    if (s == MGE_OK) s = knn_graph_build(ctx, st, n, dim, P, k, &g->impl);
    if (s == MGE_OK && cudaStreamSynchronize(st) != cudaSuccess) s = MGE_EDEVICE;
  }
  if (s != MGE_OK) {
    g->impl.each_buffer([](auto& b) { if (b.pooled) b.st = cudaStreamPerThread; });
    delete g;
    ctx_release(ctx);
    return s;
  }
  *out = g;
  return MGE_OK;
}

mge_status mge_graph_info(const mge_graph* g, int64_t* n, int64_t* nnz, double* sigma) {
  if (!g) return MGE_EINVAL;
  if (n) *n = g->impl.n;
  if (nnz) *nnz = g->impl.nnz;
  if (sigma) *sigma = g->impl.sigma;
  return MGE_OK;
}

mge_status mge_graph_csr(const mge_graph* g, const int64_t** row_ptr, const int32_t** col, const double** w) {
  if (!g) return MGE_EINVAL;
  if (row_ptr) *row_ptr = g->impl.row_ptr.p;
  if (col) *col = g->impl.col.p;
  if (w) *w = g->impl.w.p;
  return MGE_OK;
}

mge_status mge_graph_export(const mge_graph* g, int64_t* row_ptr, int32_t* col, double* w, int on_device) {
  if (!g) return MGE_EINVAL;
  const Graph& gr = g->impl;
  Ctx* ctx = gr.ctx;
  cudaSetDevice(ctx->device);
  cudaStream_t st = ctx->closed ? nullptr : ctx->stream;
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (row_ptr) MGE_CUDA(ctx, cudaMemcpyAsync(row_ptr, gr.row_ptr.p, (gr.n + 1) * sizeof(int64_t), kind, st));
  if (col) MGE_CUDA(ctx, cudaMemcpyAsync(col, gr.col.p, gr.nnz * sizeof(int32_t), kind, st));
  if (w) MGE_CUDA(ctx, cudaMemcpyAsync(w, gr.w.p, gr.nnz * sizeof(double), kind, st));
  MGE_CUDA(ctx, cudaStreamSynchronize(st));
  return MGE_OK;
}

mge_status mge_graph_destroy(mge_graph* g) {
  if (!g) return MGE_EINVAL;
  Ctx* ctx = g->impl.ctx;
  if (ctx) cudaSetDevice(ctx->device);
  // as mge_ops_destroy: the pooled arrays go back on this thread's per-thread default stream
  g->impl.each_buffer([](auto& b) { if (b.pooled) b.st = cudaStreamPerThread; });
  delete g;
  if (ctx) ctx_release(ctx);
  return MGE_OK;
}

// ---- betweenness centrality and VBC ----------------------------------------------------------

mge_status mge_betweenness(mge_ctx* c, int64_t n, const int64_t* row_ptr, const int32_t* col, int on_device,
                           double* cb, double* vbc, void* stream) {
  NvtxRange nvtx_range("mge.betweenness");
  if (!c || !row_ptr || !cb || n < 1) return MGE_EINVAL;
  Ctx* ctx = &c->impl;
  if (ctx->closed) return MGE_EINVAL;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return MGE_EDEVICE;
  cudaStream_t st = pick_stream(ctx, stream);
  DevBuf<int64_t> rpd;
  DevBuf<int32_t> cold;
  DevBuf<double> cbd;
  const int64_t* rp = row_ptr;
  const int32_t* cl = col;
  double* out = cb;
  if (on_device) {
    MGE_TRY(check_block_ptr(ctx, row_ptr, "betweenness", "row_ptr"));
    MGE_TRY(check_block_ptr(ctx, cb, "betweenness", "cb"));
  } else {
    const int64_t nnz = row_ptr[n];
    if (row_ptr[0] != 0 || nnz < 0 || (nnz > 0 && !col)) { set_error(ctx, "betweenness: malformed CSR"); return MGE_EINVAL; }
    MGE_TRY(rpd.scratch(ctx, (size_t)n + 1, st));
    MGE_TRY(cold.scratch(ctx, (size_t)std::max<int64_t>(nnz, 1), st));
    MGE_TRY(cbd.scratch(ctx, (size_t)n, st));
    MGE_CUDA(ctx, cudaMemcpyAsync(rpd.p, row_ptr, (n + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, st));
    if (nnz > 0) MGE_CUDA(ctx, cudaMemcpyAsync(cold.p, col, nnz * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    rp = rpd.p; cl = cold.p; out = cbd.p;
  }
  MGE_TRY(betweenness_run(ctx, st, n, rp, cl, out, vbc));
  if (!on_device) {
    MGE_CUDA(ctx, cudaMemcpyAsync(cb, cbd.p, n * sizeof(double), cudaMemcpyDeviceToHost, st));
    MGE_CUDA(ctx, cudaStreamSynchronize(st));
  }
  return MGE_OK;
}

// ---- k-means of the embedding --------------------------------------------------------------

mge_status mge_kmeans(mge_ctx* c, int64_t n, int K, const double* X, int C, const double* centres0, int max_iters,
                      int on_device, int32_t* assign, double* centres, int* iters, void* stream) {
  NvtxRange nvtx_range("mge.kmeans");
  if (!c || !X || !centres0 || !assign || !centres) return MGE_EINVAL;
  Ctx* ctx = &c->impl;
  if (ctx->closed) return MGE_EINVAL;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return MGE_EDEVICE;
  if (n < 1 || K < 1 || K > 64 || C < 1 || (int64_t)C * K > 4096 || max_iters < 1) {
    set_error(ctx, "kmeans: need n >= 1, 1 <= K <= 64, C >= 1, C K <= 4096, max_iters >= 1");
    return MGE_EINVAL;
  }
  cudaStream_t st = pick_stream(ctx, stream);
  const size_t cb = (size_t)C * K * sizeof(double);
  DevBuf<double> xd, cd;
  DevBuf<int32_t> ad;
  const double* Xd = X;
  double* Cd = centres;
  int32_t* Ad = assign;
  if (on_device) {
    for (const void* p : {(const void*)X, (const void*)centres0, (const void*)assign, (const void*)centres})
      MGE_TRY(check_block_ptr(ctx, p, "kmeans", "a buffer"));
    if (centres != centres0) MGE_CUDA(ctx, cudaMemcpyAsync(centres, centres0, cb, cudaMemcpyDeviceToDevice, st));
  } else {
    MGE_TRY(xd.scratch(ctx, (size_t)n * K, st));
    MGE_TRY(cd.scratch(ctx, (size_t)C * K, st));
    MGE_TRY(ad.scratch(ctx, (size_t)n, st));
    MGE_CUDA(ctx, cudaMemcpyAsync(xd.p, X, (size_t)n * K * sizeof(double), cudaMemcpyHostToDevice, st));
    MGE_CUDA(ctx, cudaMemcpyAsync(cd.p, centres0, cb, cudaMemcpyHostToDevice, st));
    Xd = xd.p; Cd = cd.p; Ad = ad.p;
  }
  int steps = 0;
  MGE_TRY(kmeans_run(ctx, st, n, K, Xd, C, Cd, max_iters, Ad, &steps));
  if (!on_device) {
    MGE_CUDA(ctx, cudaMemcpyAsync(assign, ad.p, (size_t)n * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    MGE_CUDA(ctx, cudaMemcpyAsync(centres, cd.p, cb, cudaMemcpyDeviceToHost, st));
  }
  MGE_CUDA(ctx, cudaStreamSynchronize(st));
  if (iters) *iters = steps;
  return MGE_OK;
}

static LobOp make_op(const Ops& op, int which, int precision) {
  LobOp l;
  l.n = op.n;
  l.row_order = op.order.p;
  l.row_rank = op.rank.p;
  bool dbl = precision == MGE_FP64;
  if (which == 0) {
    l.ptr = op.a_ptr.p; l.col = op.a_col.p;
    l.val = dbl ? (const void*)op.a_val.p : (const void*)op.a_val32.p;
    l.shift = op.eps;
    l.b = dbl ? (const void*)op.b.p : (const void*)op.b32.p;
    l.dinv = dbl ? (const void*)op.dinv_a.p : (const void*)op.dinv_a32.p;
    l.norm = op.norm_a; l.bmax = op.bmax; l.deflate = false; l.beta = op.beta_a;
    l.nnz = op.nnz_a;
    // the preconditioner approximates A^-1 through L + eps I: mu Q moves only the bottom of
    // the spectrum, by O(eps), and W has far fewer nonzeros than A
    if (op.l_val.p) {
      l.pc_ptr = op.w_ptr.p; l.pc_col = op.w_col.p;
      l.pc_val = dbl ? (const void*)op.l_val.p : (const void*)op.l_val32.p;
      l.pc_shift = op.eps;
      l.pc_dinv = dbl ? (const void*)op.l_dinv.p : (const void*)op.l_dinv32.p;
      l.pc_beta = op.beta_l;
      l.pc_nnz = op.nnz_w;
      if (op.l_sl.built()) {
        l.sl_slp = op.l_sl.slp.p; l.sl_perm = op.l_sl.perm.p; l.sl_col = op.l_sl.col.p;
        l.sl_val = dbl ? (const void*)op.l_sl.val.p : (const void*)op.l_sl.val32.p;
        l.sl_max_tile_slots = op.l_sl.max_tile_slots;
      }
    }
  } else {
    l.ptr = op.q_ptr.p; l.col = op.q_col.p;
    l.val = dbl ? (const void*)op.q_val.p : (const void*)op.q_val32.p;
    l.shift = 0.0; l.b = nullptr;
    l.dinv = dbl ? (const void*)op.dinv_q.p : (const void*)op.dinv_q32.p;
    l.norm = op.norm_q; l.bmax = 1.0; l.deflate = true; l.beta = op.beta_q;
    l.nnz = op.nnz_q;
    if (op.q_sl.built()) {
      l.sl_slp = op.q_sl.slp.p; l.sl_perm = op.q_sl.perm.p; l.sl_col = op.q_sl.col.p;
      l.sl_val = dbl ? (const void*)op.q_sl.val.p : (const void*)op.q_sl.val32.p;
      l.sl_max_tile_slots = op.q_sl.max_tile_slots;
    }
  }
  return l;
}

mge_status mge_ops_apply(mge_ctx* c, const mge_ops* o, int which, int precision, int m, const void* X, void* Y,
                         void* stream) {
  if (!c || !o || !X || !Y || (which != 0 && which != 1)) return MGE_EINVAL;
  if (c->impl.closed) return MGE_EINVAL;
  Ctx* ctx = &c->impl;
  cudaSetDevice(ctx->device);
  if (precision != MGE_FP64 && precision != MGE_FP32) {
    set_error(ctx, "apply: precision %d not supported", precision);
    return MGE_EINVAL;
  }
  if (!apply_width_ok(m)) { set_error(ctx, "apply: unsupported width %d (4, 8, 12, 16 or 24)", m); return MGE_EINVAL; }
  MGE_TRY(check_block_ptr(ctx, X, "apply", "X"));
  MGE_TRY(check_block_ptr(ctx, Y, "apply", "Y"));
  cudaStream_t st = pick_stream(ctx, stream);
  LobOp l = make_op(o->impl, which, precision);
  MGE_TRY(spmm_apply(ctx, st, l, precision, m, X, Y));
  MGE_CUDA(ctx, cudaStreamSynchronize(st));
  return MGE_OK;
}

mge_status mge_ops_apply_inplace(mge_ctx* c, const mge_ops* o, int which, int precision, int m, void* XY,
                                 void* stream) {
  if (!c || !o || !XY || (which != 0 && which != 1)) return MGE_EINVAL;
  if (c->impl.closed) return MGE_EINVAL;
  Ctx* ctx = &c->impl;
  cudaSetDevice(ctx->device);
  if (precision != MGE_FP64 && precision != MGE_FP32) {
    set_error(ctx, "apply_inplace: precision %d not supported", precision);
    return MGE_EINVAL;
  }
  if (!apply_width_ok(m)) {
    set_error(ctx, "apply_inplace: unsupported width %d (4, 8, 12, 16 or 24)", m);
    return MGE_EINVAL;
  }
  MGE_TRY(check_block_ptr(ctx, XY, "apply_inplace", "XY"));
  cudaStream_t st = pick_stream(ctx, stream);
  LobOp l = make_op(o->impl, which, precision);
  MGE_TRY(spmm_apply_inplace(ctx, st, l, precision, m, XY));
  MGE_CUDA(ctx, cudaStreamSynchronize(st));
  return MGE_OK;
}

mge_status mge_embed(mge_ctx* c, const mge_ops* o, int K, double tol, const mge_embed_opts* opts,
                     double* lambda, void* V, mge_embed_info* info) {
  NvtxRange nvtx_range("mge.embed");
  if (!c || !o || !lambda) return MGE_EINVAL;
  if (c->impl.closed) return MGE_EINVAL;
  Ctx* ctx = &c->impl;
  cudaSetDevice(ctx->device);
  mge_embed_opts e{};
  e.precision = MGE_FP32;
  e.maxiter = 20000;
  e.check_every = 16;
  e.use_graph = 1;
  if (opts) e = *opts;
  if (e.maxiter <= 0) e.maxiter = 20000;
  if (e.check_every <= 0) e.check_every = 16;
  if (!(tol > 0)) { set_error(ctx, "tol must be > 0"); return MGE_EINVAL; }
  if (K < 1) { set_error(ctx, "K must be >= 1"); return MGE_EINVAL; }
  const int guard = guard_for(e, K);
  int m = round_block_width(K + guard);
  if (m < 0 || m > 24) { set_error(ctx, "K + guard = %d exceeds the widest block (24)", K + guard); return MGE_EINVAL; }
  const Ops& op = o->impl;
  if (op.n < 2 * m) { set_error(ctx, "graph has %lld nodes; need at least %d", (long long)op.n, 2 * m); return MGE_EINVAL; }
  if (e.precision != MGE_FP64 && e.precision != MGE_FP32 && e.precision != MGE_BF16) {
    set_error(ctx, "bad precision");
    return MGE_EINVAL;
  }
  // MGE_BF16: FP32 blocks and values, the preconditioner's blocks in BF16
  const bool bf16 = e.precision == MGE_BF16;
  int prec = bf16 ? MGE_FP32 : e.precision;
  cudaStream_t st = pick_stream(ctx, e.stream);
  LobOp l = make_op(op, 0, prec);
  l.pc_bf16 = bf16;
  // optional initial block
  DevBuf<double> x0d;
  const double* x0 = nullptr;
  int x0c = 0;
  if (e.x0 && e.x0_cols > 0) {
    x0c = std::min(e.x0_cols, m);
    if (e.x0_on_device) x0 = e.x0;
    else {
      MGE_TRY(x0d.scratch(ctx, (size_t)op.n * x0c, st));
      MGE_CUDA(ctx, cudaMemcpyAsync(x0d.p, e.x0, (size_t)op.n * x0c * sizeof(double), cudaMemcpyHostToDevice, st));
      x0 = x0d.p;
    }
  }
  DevBuf<double> vd;
  double* vout = nullptr;
  if (V) {
    if (e.v_on_device) vout = static_cast<double*>(V);
    else { MGE_TRY(vd.scratch(ctx, (size_t)op.n * K, st)); vout = vd.p; }
  }
  LobResult r;
  l.precond_degree = e.precond_degree > 0 ? std::min(e.precond_degree, kMaxPrecondDegree) : default_precond_degree(op.n);
  if (bf16) l.precond_degree = std::min(l.precond_degree, kBf16MaxPrecondDegree);
  l.rr_fp64 = rr_fp64_for(e, prec);
  l.rr_switch = e.rr_fp64 == 0;
  l.gram_cuda_cores = e.gram_cuda_cores != 0;
  mge_status s = lobpcg_solve(ctx, st, l, prec, K, m, tol, e.maxiter, e.seed, e.check_every, e.use_graph != 0,
                              x0, x0c, vout, &r);
  if (s != MGE_OK && s != MGE_ENOTCONVERGED) {
    if (info) { info->status = s; info->iters = r.iters; }
    return s;
  }
  for (int k = 0; k < K; ++k) lambda[k] = r.lambda[k];
  if (V && !e.v_on_device) {
    MGE_CUDA(ctx, cudaMemcpyAsync(V, vd.p, (size_t)op.n * K * sizeof(double), cudaMemcpyDeviceToHost, st));
    MGE_CUDA(ctx, cudaStreamSynchronize(st));
  }
  if (info) {
    info->status = s;
    info->iters = r.iters;
    info->m = m;
    info->drops = r.drops;
    info->rr_fp64_from = r.rr64_from;
    for (int k = 0; k < 64; ++k) info->resid[k] = k < K ? r.eta[k] : 0.0;
    info->solve_ms = r.ms;
  }
  return s;
}

mge_status mge_embed_batch(mge_ctx* c, int count, const mge_ops* const* ops, const int* K, double tol,
                           const mge_embed_opts* opts, double* const* lambda, void* const* V,
                           mge_embed_info* info) {
  NvtxRange nvtx_range("mge.embed_batch");
  if (!c || count < 1 || !ops || !K || !lambda) return MGE_EINVAL;
  if (c->impl.closed) return MGE_EINVAL;
  Ctx* ctx = &c->impl;
  cudaSetDevice(ctx->device);
  mge_embed_opts e{};
  e.precision = MGE_FP32;
  if (opts) e = *opts;
  if (e.maxiter <= 0) e.maxiter = 20000;
  if (!(tol > 0)) { set_error(ctx, "tol must be > 0"); return MGE_EINVAL; }
  if (e.x0 && e.x0_cols > 0) { set_error(ctx, "embed_batch: x0 is not supported"); return MGE_EINVAL; }
  if (e.precision != MGE_FP64 && e.precision != MGE_FP32 && e.precision != MGE_BF16) {
    set_error(ctx, "bad precision");
    return MGE_EINVAL;
  }
  const bool bf16 = e.precision == MGE_BF16;
  const int prec = bf16 ? MGE_FP32 : e.precision;
  std::vector<LobOp> lops((size_t)count);
  std::vector<int> ms((size_t)count);
  for (int i = 0; i < count; ++i) {
    if (!ops[i] || !lambda[i]) { set_error(ctx, "embed_batch: NULL handle or lambda at %d", i); return MGE_EINVAL; }
    if (K[i] < 1) { set_error(ctx, "embed_batch: K[%d] = %d", i, K[i]); return MGE_EINVAL; }
    const int guard = guard_for(e, K[i]);
    const int m = round_block_width(K[i] + guard);
    if (m < 0 || m > 24) { set_error(ctx, "embed_batch: K + guard = %d exceeds the widest block (24)", K[i] + guard); return MGE_EINVAL; }
    const Ops& op = ops[i]->impl;
    if (op.n < 2 * m) { set_error(ctx, "embed_batch: graph %d has %lld nodes; need at least %d", i, (long long)op.n, 2 * m); return MGE_EINVAL; }
    ms[i] = m;
    lops[i] = make_op(op, 0, prec);
    lops[i].precond_degree = e.precond_degree > 0 ? std::min(e.precond_degree, kMaxPrecondDegree) : default_precond_degree(op.n);
    if (bf16) lops[i].precond_degree = std::min(lops[i].precond_degree, kBf16MaxPrecondDegree);
    lops[i].rr_fp64 = rr_fp64_for(e, prec);
    lops[i].rr_switch = e.rr_fp64 == 0;
    lops[i].pc_bf16 = bf16;
    lops[i].gram_cuda_cores = e.gram_cuda_cores != 0;
  }
  cudaStream_t st = pick_stream(ctx, e.stream);
  // V buffers: the caller's device arrays, or scratch copied to the caller's host arrays
  std::vector<DevBuf<double>> vd((size_t)count);
  std::vector<double*> vout((size_t)count, nullptr);
  for (int i = 0; i < count && V; ++i) {
    if (!V[i]) continue;
    if (e.v_on_device) vout[i] = static_cast<double*>(V[i]);
    else { MGE_TRY(vd[i].scratch(ctx, (size_t)lops[i].n * K[i], st)); vout[i] = vd[i].p; }
  }
  std::vector<LobResult> res((size_t)count);
  std::vector<mge_status> sts((size_t)count, MGE_OK);
  double ms_batch = 0;
  MGE_TRY(lobpcg_solve_batch(ctx, st, count, lops.data(), prec, K, ms.data(), tol, e.maxiter, e.seed,
                             vout.data(), res.data(), sts.data(), &ms_batch));
  mge_status first = MGE_OK;
  for (int i = 0; i < count; ++i) {
    const mge_status s = sts[i];
    if (s == MGE_OK || s == MGE_ENOTCONVERGED)
      for (int k = 0; k < K[i]; ++k) lambda[i][k] = res[i].lambda[k];
    if (V && V[i] && !e.v_on_device && (s == MGE_OK || s == MGE_ENOTCONVERGED))
      MGE_CUDA(ctx, cudaMemcpyAsync(V[i], vd[i].p, (size_t)lops[i].n * K[i] * sizeof(double), cudaMemcpyDeviceToHost, st));
    if (info) {
      info[i].status = s;
      info[i].iters = res[i].iters;
      info[i].m = ms[i];
      info[i].drops = res[i].drops;
      info[i].rr_fp64_from = res[i].rr64_from;
      for (int k = 0; k < 64; ++k) info[i].resid[k] = (k < K[i] && k < (int)res[i].eta.size()) ? res[i].eta[k] : 0.0;
      info[i].solve_ms = ms_batch;
    }
    if (first == MGE_OK && s != MGE_OK) first = s;
  }
  MGE_CUDA(ctx, cudaStreamSynchronize(st));
  return first;
}

mge_status mge_submit(mge_ctx* c, const mge_request* req, uint64_t* ticket) {
  if (!c || !req || !ticket) return MGE_EINVAL;
  return serve_submit(&c->impl, req, ticket);
}

mge_status mge_poll(mge_ctx* c, uint64_t ticket, int timeout_ms, mge_result* out) {
  if (!c || !out) return MGE_EINVAL;
  return serve_poll(&c->impl, ticket, timeout_ms, out);
}

mge_status mge_release(mge_ctx* c, uint64_t ticket) {
  if (!c) return MGE_EINVAL;
  return serve_release(&c->impl, ticket);
}

}  // extern "C"
