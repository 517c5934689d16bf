// Serving: a request queue with HBM-footprint admission and concurrent slots.
//
// mge_submit copies the request's graph and enqueues it.  A fixed set of slot threads, each
// with its own CUDA stream, takes requests in arrival order as soon as the request's device
// footprint fits the context's budget next to the requests already running; the requests
// on the device overlap (their kernels share the GPU through the streams).  Each result is
// independent of what runs beside it: a solve touches only its own buffers.
#include "mge_internal.cuh"

#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <thread>

namespace mge {

namespace {

using Clock = std::chrono::steady_clock;

struct Entry {
  mge_request req{};
  std::vector<int64_t> rp;
  std::vector<int32_t> col;
  std::vector<double> w;
  std::vector<double> points;  // a request given as points: its kNN graph is built on the device
  size_t footprint = 0;
  Clock::time_point t_submit, t_admit, t_done;
  bool done = false;
  mge_status status = MGE_OK;
  double eps = 0, mu = 0;
  int iters = 0;
  std::vector<double> lambda, V;
};

struct Serve {
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<uint64_t> queue;
  std::map<uint64_t, Entry> entries;
  uint64_t next_ticket = 1;
  size_t reserved = 0;       // footprint of running requests
  size_t budget = 0;
  bool stop = false;
  std::vector<std::thread> slots;
  size_t max_queue = 4096;
};

// Device bytes one request holds at its peak: W and its two-hop scratch, Q and A (FP64 and
// FP32 values), and the seven LOBPCG blocks of its FP32 or FP64 iteration.
size_t footprint(const mge_request& r) {
  int64_t n = r.n;
  // a request given as points: the union kNN graph holds between k and about 1.5 k entries
  // per row; the kNN construction's own scratch is below the build's
  int64_t nnz = r.points ? (int64_t)(1.5 * r.knn * n) : (r.row_ptr ? r.row_ptr[r.n] : 0);
  double deg = n > 0 ? (double)nnz / n : 0;
  double cand = (double)nnz * deg;                 // sum of candidate counts
  double nnz_t = std::min(cand, (double)nnz * 2.5);
  double nnz_a = n + nnz + nnz_t, nnz_q = n + nnz_t;
  const int guard = r.guard > 0 ? r.guard : r.guard < 0 ? 0 : std::max(0, std::min(r.K, 24 - r.K));
  int m = round_block_width(r.K + guard);
  if (m < 0) m = 24;
  size_t es = r.precision == MGE_FP64 ? 8 : 4;
  double bytes = nnz * 12.0 + cand * 4.0 + nnz_a * 16.0 + nnz_q * 16.0 + n * 80.0 +
                 7.0 * n * m * es + (double)n * r.K * 8.0 + (1 << 20);
  return (size_t)bytes;
}

void run_one(Ctx* ctx, cudaStream_t st, Entry& e) {
  mge_ops* ops = nullptr;
  mge_ops_opts oo{};
  oo.precision = (e.req.precision == MGE_FP64 || e.req.precision == MGE_BF16) ? e.req.precision : MGE_FP32;
  oo.seed = e.req.seed;
  oo.stream = st;
  mge_ctx* c = static_cast<mge_ctx*>(ctx->self);
  mge_status s;
  if (!e.points.empty()) {
    // points -> kNN graph (Sec. 5.1) -> operators, all on the slot's stream
    mge_graph* g = nullptr;
    s = mge_knn_graph(c, e.req.n, e.req.dim, e.points.data(), 0, e.req.knn, st, &g);
    if (s != MGE_OK) { e.status = s; return; }
    const int64_t* rp = nullptr;
    const int32_t* col = nullptr;
    const double* w = nullptr;
    mge_graph_csr(g, &rp, &col, &w);
    s = mge_build_graph_ops(c, e.req.n, rp, col, w, 1, &oo, &ops);
    mge_graph_destroy(g);
  } else {
    s = mge_build_graph_ops(c, e.req.n, e.rp.data(), e.col.data(), e.w.data(), 0, &oo, &ops);
  }
  if (s != MGE_OK && s != MGE_EDEGENERATE) { e.status = s; return; }
  mge_ops_info_t info{};
  mge_ops_info(ops, &info);
  e.eps = info.eps;
  e.mu = info.mu;
  mge_embed_opts eo{};
  eo.precision = oo.precision;
  eo.guard = e.req.guard;
  eo.maxiter = e.req.maxiter;
  eo.seed = e.req.seed;
  eo.stream = st;
  eo.use_graph = 1;
  e.lambda.assign(e.req.K, 0.0);
  e.V.assign((size_t)e.req.n * e.req.K, 0.0);
  mge_embed_info ei{};
  mge_status s2 = mge_embed(c, ops, e.req.K, e.req.tol, &eo, e.lambda.data(), e.V.data(), &ei);
  e.iters = ei.iters;
  mge_ops_destroy(ops);
  e.status = (s2 != MGE_OK) ? s2 : s;
}

void slot_loop(Ctx* ctx, Serve* sv) {
  cudaSetDevice(ctx->device);
  cudaStream_t st;
  cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  for (;;) {
    uint64_t t = 0;
    Entry* e = nullptr;
    {
      std::unique_lock<std::mutex> lk(sv->mu);
      sv->cv_work.wait(lk, [&] {
        if (sv->stop) return true;
        if (sv->queue.empty()) return false;
        Entry& head = sv->entries[sv->queue.front()];
        return sv->budget == 0 || sv->reserved == 0 || sv->reserved + head.footprint <= sv->budget;
      });
      if (sv->stop) break;
      t = sv->queue.front();
      sv->queue.pop_front();
      e = &sv->entries[t];
      sv->reserved += e->footprint;
      e->t_admit = Clock::now();
    }
    run_one(ctx, st, *e);
    {
      std::lock_guard<std::mutex> lk(sv->mu);
      e->t_done = Clock::now();
      e->done = true;
      sv->reserved -= e->footprint;
      e->rp.clear(); e->rp.shrink_to_fit();
      e->col.clear(); e->col.shrink_to_fit();
      e->w.clear(); e->w.shrink_to_fit();
    }
    sv->cv_done.notify_all();
    sv->cv_work.notify_all();
  }
  cudaStreamDestroy(st);
}

Serve* get_serve(Ctx* ctx) {
  static std::mutex init_mu;
  std::lock_guard<std::mutex> g(init_mu);
  if (!ctx->serve) {
    Serve* sv = new Serve();
    sv->budget = ctx->budget;
    int slots = 4;
    if (const char* s = getenv("MGE_SERVE_SLOTS")) slots = std::max(1, atoi(s));
    for (int i = 0; i < slots; ++i) sv->slots.emplace_back(slot_loop, ctx, sv);
    ctx->serve = sv;
  }
  return static_cast<Serve*>(ctx->serve);
}

}  // namespace

mge_status serve_submit(Ctx* ctx, const mge_request* req, uint64_t* ticket) {
  const bool pts = req->points != nullptr;
  if (req->n < 1 || req->K < 1 || !(req->tol > 0) ||
      (pts && (req->dim < 2 || req->dim > 3 || req->knn < 1 || req->knn > 32 || req->knn >= req->n)) ||
      (!pts && (!req->row_ptr || !req->col || !req->w))) {
    set_error(ctx, "submit: invalid request");
    return MGE_EINVAL;
  }
  Serve* sv = get_serve(ctx);
  Entry e;
  e.req = *req;
  if (pts) {
    e.points.assign(req->points, req->points + (size_t)req->n * req->dim);
  } else {
    int64_t nnz = req->row_ptr[req->n];
    if (nnz < 0) { set_error(ctx, "submit: bad row_ptr"); return MGE_EINVAL; }
    e.rp.assign(req->row_ptr, req->row_ptr + req->n + 1);
    e.col.assign(req->col, req->col + nnz);
    e.w.assign(req->w, req->w + nnz);
  }
  e.footprint = footprint(*req);
  e.t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    if (sv->budget && e.footprint > sv->budget) {
      set_error(ctx, "submit: request needs %zu bytes, budget is %zu", e.footprint, sv->budget);
      return MGE_ENOMEM;
    }
    if (sv->queue.size() >= sv->max_queue) return MGE_EAGAIN;
    uint64_t t = sv->next_ticket++;
    e.req.row_ptr = nullptr; e.req.col = nullptr; e.req.w = nullptr; e.req.points = nullptr;
    sv->entries.emplace(t, std::move(e));
    sv->queue.push_back(t);
    *ticket = t;
  }
  sv->cv_work.notify_all();
  return MGE_OK;
}

mge_status serve_poll(Ctx* ctx, uint64_t ticket, int timeout_ms, mge_result* out) {
  Serve* sv = get_serve(ctx);
  std::unique_lock<std::mutex> lk(sv->mu);
  auto it = sv->entries.find(ticket);
  if (it == sv->entries.end()) return MGE_ENOTFOUND;
  auto ready = [&] { return it->second.done; };
  if (timeout_ms < 0) sv->cv_done.wait(lk, ready);
  else if (!sv->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready)) return MGE_ETIMEOUT;
  Entry& e = it->second;
  out->status = e.status;
  out->n = e.req.n;
  out->K = e.req.K;
  out->eps = e.eps;
  out->mu = e.mu;
  out->iters = e.iters;
  out->latency_ms = std::chrono::duration<double, std::milli>(e.t_done - e.t_submit).count();
  out->queue_ms = std::chrono::duration<double, std::milli>(e.t_admit - e.t_submit).count();
  out->lambda = e.lambda.data();
  out->V = e.V.data();
  return MGE_OK;
}

mge_status serve_release(Ctx* ctx, uint64_t ticket) {
  Serve* sv = get_serve(ctx);
  std::lock_guard<std::mutex> lk(sv->mu);
  auto it = sv->entries.find(ticket);
  if (it == sv->entries.end()) return MGE_ENOTFOUND;
  if (!it->second.done) return MGE_EAGAIN;
  sv->entries.erase(it);
  return MGE_OK;
}

void serve_shutdown(Ctx* ctx) {
  if (!ctx->serve) return;
  Serve* sv = static_cast<Serve*>(ctx->serve);
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stop = true;
  }
  sv->cv_work.notify_all();
  for (auto& t : sv->slots) t.join();
  delete sv;
  ctx->serve = nullptr;
}

}  // namespace mge
