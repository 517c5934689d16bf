// Internal declarations shared by the libmge translation units.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <stdio.h>

#include <atomic>
#include <cmath>
#include <map>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/mge.h"

namespace mge {

// A named range on the NVTX timeline (header-only NVTX 3: inert unless a profiler is attached)
// around each phase of a call, so that a timeline shows build, eps solve, embedding, kNN,
// k-means and betweenness as separate spans.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// ---------------------------------------------------------------------------------------
// error plumbing: every CUDA call is checked and turned into an mge_status
// ---------------------------------------------------------------------------------------
struct Ctx;
void set_error(Ctx* ctx, const char* fmt, ...);

#define MGE_CUDA(ctx, call)                                                              \
  do {                                                                                   \
    cudaError_t _e = (call);                                                             \
    if (_e != cudaSuccess) {                                                             \
      ::mge::set_error((ctx), "%s:%d %s: %s", __FILE__, __LINE__, #call,                 \
                       cudaGetErrorString(_e));                                          \
      return (_e == cudaErrorMemoryAllocation) ? MGE_ENOMEM : MGE_EDEVICE;               \
    }                                                                                    \
  } while (0)

#define MGE_TRY(expr)                                                                    \
  do {                                                                                   \
    mge_status _s = (expr);                                                              \
    if (_s != MGE_OK) return _s;                                                         \
  } while (0)

// Launch bookkeeping: every kernel launch goes through this so the context can count it.
#define MGE_LAUNCHED(ctx, k) ((ctx)->kernel_launches += (k))

// ---------------------------------------------------------------------------------------
// device memory: plain cudaMallocAsync-free allocations accounted against a budget
// ---------------------------------------------------------------------------------------
// One autotuned kernel configuration: the Chebyshev step's shared-memory stage budget and
// whether it loads the row's own R, d and D^-1 before its gathers (tune.cu).
struct TuneEntry {
  int budget = 0;
  int prefetch = 0;
  double us = 0;                   // its measured time per launch
};

struct Ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  size_t budget = 0;               // 0 = unlimited
  std::atomic<size_t> in_use{0};
  std::atomic<uint64_t> kernel_launches{0};
  // SpMM timing (roofline measurement)
  bool timing = false;
  uint64_t spmm_launches = 0;
  double spmm_ms = 0.0;
  uint64_t spmm_bytes = 0;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_pool;
  size_t ev_used = 0;
  std::vector<uint64_t> ev_bytes;
  std::string last_error;
  std::mutex err_mu;
  int num_sms = 0;
  // stream-ordered pool for the scratch of one call (freed memory stays in the pool, so a
  // repeated call neither allocates from the driver nor synchronises the device)
  cudaMemPool_t pool = nullptr;
  std::vector<void*> state_host;   // pinned host copies of solve status words (reused)
  std::mutex state_mu;
  void* serve = nullptr;           // serving state (serve.cu)
  void* self = nullptr;            // the owning mge_ctx*
  std::atomic<int> refs{1};        // the context itself plus one per live ops handle
  bool closed = false;
  // kernel autotuning (tune.cu): mode 0 off (fixed rules), 1 tune keys not yet known, 2 use
  // known keys only; entries persist in a JSON file when a path is set
  int tune_mode = 1;
  std::string tune_path;
  std::mutex tune_mu;
  std::map<std::string, TuneEntry> tune;
};

// autotuning cache (tune.cu)
bool tune_lookup(Ctx* ctx, const std::string& key, TuneEntry* e);
void tune_store(Ctx* ctx, const std::string& key, const TuneEntry& e);
mge_status tune_set(Ctx* ctx, int mode, const char* path);

mge_status dev_alloc(Ctx* ctx, void** p, size_t bytes);
void dev_free(Ctx* ctx, void* p, size_t bytes);
// scratch ordered on stream st: usable by work on st after this call, returned to the
// context's pool by work on st (the caller uses it on st only)
mge_status dev_alloc_async(Ctx* ctx, void** p, size_t bytes, cudaStream_t st);
void dev_free_async(Ctx* ctx, void* p, size_t bytes, cudaStream_t st);
// While set (the operator build), alloc() also draws from the pool, ordered on this stream;
// such arrays are freed by mge_ops_destroy after a device synchronisation.
struct PersistentPool {
  bool on = false;
  cudaStream_t st = nullptr;
};
PersistentPool& persistent_pool();
struct PersistentPoolScope {
  PersistentPool prev;
  explicit PersistentPoolScope(cudaStream_t s) : prev(persistent_pool()) { persistent_pool() = PersistentPool{true, s}; }
  ~PersistentPoolScope() { persistent_pool() = prev; }
};

// Device array owned by the library: alloc() for memory that outlives the call (the
// operators; cudaMalloc), scratch() for memory used by one call on one stream (the
// context's stream-ordered pool).
template <typename T>
struct DevBuf {
  T* p = nullptr;
  size_t n = 0;
  Ctx* ctx = nullptr;
  bool pooled = false;
  cudaStream_t st = nullptr;
  mge_status alloc(Ctx* c, size_t count) {
    if (c && c->pool && persistent_pool().on) return scratch(c, count, persistent_pool().st);
    release();
    ctx = c;
    n = count;
    if (count == 0) return MGE_OK;
    void* q = nullptr;
    mge_status s = dev_alloc(c, &q, count * sizeof(T));
    if (s != MGE_OK) { n = 0; return s; }
    p = static_cast<T*>(q);
    return MGE_OK;
  }
  mge_status scratch(Ctx* c, size_t count, cudaStream_t stream) {
    release();
    ctx = c;
    n = count;
    if (count == 0) return MGE_OK;
    void* q = nullptr;
    mge_status s = dev_alloc_async(c, &q, count * sizeof(T), stream);
    if (s != MGE_OK) { n = 0; return s; }
    p = static_cast<T*>(q);
    pooled = true;
    st = stream;
    return MGE_OK;
  }
  void release() {
    if (p) {
      if (pooled) dev_free_async(ctx, p, n * sizeof(T), st);
      else dev_free(ctx, p, n * sizeof(T));
    }
    p = nullptr;
    n = 0;
    pooled = false;
    st = nullptr;
  }
  // exchange the arrays (and how each is to be freed) of two buffers
  void swap(DevBuf& o) {
    std::swap(p, o.p); std::swap(n, o.n); std::swap(ctx, o.ctx);
    std::swap(pooled, o.pooled); std::swap(st, o.st);
  }
  ~DevBuf() { release(); }
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
};

// ---------------------------------------------------------------------------------------
// Row-sorted, slice-padded copy of a CSR operator (the layout of the Chebyshev steps).
// The rows of each tile of kSliceTileRows consecutive rows are sorted by length, longest
// first, and cut into slices of kSliceRows sorted rows; every row of a slice is padded to the
// slice's longest row rounded up to a multiple of 4 (padding: value 0, column = the slice's
// first row, so that a padded term a (x_j - x_i) is exactly 0).  Slot k of the row at sorted
// position q of slice s is element slp[s] + (k / 4) * 64 + q * 4 + k % 4: one 16-byte load
// gives a row four consecutive slots, and the 16 rows' loads are contiguous.
// ---------------------------------------------------------------------------------------
constexpr int kSliceTileRows = 128;
constexpr int kSliceRows = 16;
constexpr int kSlicesPerTile = kSliceTileRows / kSliceRows;

struct Sliced {
  int64_t ntiles = 0, slots = 0;
  int64_t max_tile_slots = 0;       // slots of the densest tile
  DevBuf<int64_t> slp;              // [kSlicesPerTile * ntiles + 4]: first slot of each slice;
                                    // the entries from index kSlicesPerTile * ntiles on = slots
  DevBuf<uint8_t> perm;             // [kSliceTileRows * ntiles]: tile-local row at each sorted
                                    // position, 0xFF past the last row
  DevBuf<int32_t> col;              // [slots]
  DevBuf<double> val;               // [slots]
  DevBuf<float> val32;              // [slots]
  bool built() const { return slp.p != nullptr; }
};

// ---------------------------------------------------------------------------------------
// operators built by mge_build_graph_ops (everything device resident)
// ---------------------------------------------------------------------------------------
struct Ops {
  Ctx* ctx = nullptr;
  int64_t n = 0, nnz_w = 0, nnz_a = 0, nnz_q = 0;
  // Every array below is in the library's node order: row r holds input node order[r]
  // (order and rank empty: the input order).  The API translates at its boundary.
  DevBuf<int32_t> order, rank;
  DevBuf<int64_t> w_ptr;  DevBuf<int32_t> w_col;  DevBuf<double> w_val;
  DevBuf<int32_t> T;
  DevBuf<int64_t> q_ptr;  DevBuf<int32_t> q_col;  DevBuf<double> q_val;
  DevBuf<int64_t> a_ptr;  DevBuf<int32_t> a_col;  DevBuf<double> a_val;
  DevBuf<float>   q_val32, a_val32;          // FP32 copies for the reduced-precision forms
  DevBuf<double>  b, dinv_a, dinv_q;         // B diagonal, Jacobi preconditioners
  DevBuf<float>   b32, dinv_a32, dinv_q32;
  // L + eps I in the SpMM's difference form (off-diagonal values -w_ij on W's structure):
  // the operator the LOBPCG preconditioner of A applies, with its Jacobi scaling and the
  // Gershgorin bound of its scaled spectrum
  DevBuf<double>  l_val, l_dinv;
  DevBuf<float>   l_val32, l_dinv32;
  double beta_l = 2;
  // sliced copies of Q (the eps solve's Chebyshev steps) and of L + eps I (the embedding's);
  // left unbuilt when the padding would more than double the stored entries
  Sliced q_sl, l_sl;
  double eps = 0, mu = 0, norm_a = 0, norm_q = 0, bmax = 1;
  double beta_a = 2, beta_q = 2;            // Gershgorin bounds of the spectra of D^-1 A, D^-1 Q
  int degenerate = 0, ncomp = 1, eps_iters = 0;
  double eps_resid = 0, build_ms = 0;
  // every device array of the handle
  template <typename F>
  void each_buffer(F f) {
    f(order); f(rank); f(w_ptr); f(w_col); f(w_val); f(T);
    f(q_ptr); f(q_col); f(q_val); f(a_ptr); f(a_col); f(a_val); f(q_val32); f(a_val32);
    f(b); f(dinv_a); f(dinv_q); f(b32); f(dinv_a32); f(dinv_q32);
    f(l_val); f(l_dinv); f(l_val32); f(l_dinv32);
    for (Sliced* sl : {&q_sl, &l_sl}) { f(sl->slp); f(sl->perm); f(sl->col); f(sl->val); f(sl->val32); }
  }
};

// ---------------------------------------------------------------------------------------
// kNN graph built from points by mge_knn_graph (device resident, canonical CSR)
// ---------------------------------------------------------------------------------------
struct Graph {
  Ctx* ctx = nullptr;
  int64_t n = 0, nnz = 0;
  int dim = 0, k = 0;
  double sigma = 0, cell_size = 0;
  DevBuf<int64_t> row_ptr;
  DevBuf<int32_t> col;
  DevBuf<double> w;
  template <typename F>
  void each_buffer(F f) { f(row_ptr); f(col); f(w); }
};

// Builds the symmetric kNN graph of n points (row-major n x dim FP64, device) into out (knn.cu).
mge_status knn_graph_build(Ctx* ctx, cudaStream_t st, int64_t n, int dim, const double* P, int k, Graph* out);

// k-means (Lloyd) of n points (X column-major [n x K], device) from the centres (row-major
// [C x K], device, updated in place); assign [n] device; kmeans.cu.
mge_status kmeans_run(Ctx* ctx, cudaStream_t st, int64_t n, int K, const double* X, int C, double* centres,
                      int max_iters, int32_t* assign, int* iters_out);

// Betweenness centrality cb [n] (device) of the CSR graph (device) and, vbc_out not NULL,
// its population variance; betweenness.cu.
mge_status betweenness_run(Ctx* ctx, cudaStream_t st, int64_t n, const int64_t* rp, const int32_t* col, double* cb,
                           double* vbc_out);

// ---------------------------------------------------------------------------------------
// LOBPCG operator description handed to the solver
// ---------------------------------------------------------------------------------------
// default degrees of the Chebyshev preconditioner of the LOBPCG solves (measured on a
// 200k-node swiss roll, K = 8, m = 16, relative residual 1e-5: embedding 145 / 73 / 44 / 27 /
// 21 iterations and 162 / 95 / 65 / 49 / 45 ms at degree 16 / 24 / 32 / 48 / 64; the eps
// solve converges in about 23 iterations at 24)
constexpr int kDefaultPrecondDegree = 64;
constexpr int kMaxPrecondDegree = 256;      // largest degree a caller may ask for
constexpr int kDefaultEpsPrecondDegree = 24;
// Defaults by graph size.  The best degree grows with n (the spectrum to flatten widens as the
// smallest eigenvalues shrink): measured best embedding degree 24 on graphs of 2k-50k nodes
// (512-graph batch: 8.3M node-embeddings/s at 24, 6.9M at 48, 5.7M at 64) and 64 at 200k;
// best eps-solve degree 8-12 on the small graphs, 32 at 200k and at 2M.
inline int default_precond_degree(int64_t n) {
  const int d = (int)std::lround(std::sqrt((double)n) / 5.0);
  return d < 16 ? 16 : d > kDefaultPrecondDegree ? kDefaultPrecondDegree : d;
}
inline int default_eps_precond_degree(int64_t n) {
  const int d = (int)std::lround(std::sqrt((double)n) / 12.0);
  return d < 8 ? 8 : d > 32 ? 32 : d;
}
// BF16 preconditioner blocks: the Chebyshev polynomial amplifies the bottom of the spectrum by
// about 2 d^2 against the top, so BF16 rounding (u = 2^-8) of its iterates leaves the
// preconditioned block with an O(1) relative error in the directions LOBPCG needs once
// u 2 d^2 > 1 (measured on a 200k-node swiss roll: d >= 24 stalls at eigenvalue errors of
// 7e-5).  The degree is capped where u 2 d^2 = 1/2.
constexpr int kBf16MaxPrecondDegree = 8;

struct LobOp {
  int64_t n = 0;
  int64_t nnz = -1, pc_nnz = -1;   // entries of the operator and of the preconditioner's (-1: read
                                   // from the row pointers on the device)
  const int64_t* ptr = nullptr;
  const int32_t* col = nullptr;
  const void* val = nullptr;       // double* or float* by precision
  double shift = 0;                // A = (Laplacian part) + shift * I  (eps for A, 0 for Q)
  const void* b = nullptr;         // NULL = identity B
  const void* dinv = nullptr;      // Jacobi preconditioner diag(A)^-1
  double norm = 1, bmax = 1;       // ||A||_G and max b for the backward error
  bool deflate = false;            // keep blocks orthogonal to the constant vector
  double beta = 2;                 // upper bound of the spectrum of diag(A)^-1 A
  int precond_degree = 1;          // Chebyshev preconditioner degree (1: Jacobi)
  bool rr_fp64 = false;            // FP32 blocks: Rayleigh-Ritz and W's Cholesky in FP64
  bool rr_switch = true;           // FP32 blocks: move to FP64 for both when the residuals stall
  bool pc_bf16 = false;            // FP32 blocks: the preconditioner's blocks in BF16
  bool gram_cuda_cores = false;    // FP32 blocks: Rayleigh-Ritz Grams on the CUDA cores only
  // operator the preconditioner applies, in the same difference form (pc_ptr NULL: the
  // operator itself); its diagonal scaling and Gershgorin bound
  const int64_t* pc_ptr = nullptr;
  const int32_t* pc_col = nullptr;
  const void* pc_val = nullptr;
  double pc_shift = 0;
  const void* pc_dinv = nullptr;
  double pc_beta = 2;
  // sliced copy of the operator the Chebyshev steps apply (NULL: they use its CSR form)
  const int64_t* sl_slp = nullptr;
  const uint8_t* sl_perm = nullptr;
  const int32_t* sl_col = nullptr;
  const void* sl_val = nullptr;     // double* or float* by precision
  int64_t sl_max_tile_slots = 0;
  // node order of the operator's rows (NULL: the caller's order): internal row r is caller
  // row row_order[r], caller row i is internal row row_rank[i]; x0 and V are in the
  // caller's order
  const int32_t* row_order = nullptr;
  const int32_t* row_rank = nullptr;
};

// The operator build in three phases (graph.cu): phase 1 up to the eps = lambda_2(Q) solve
// (two-hop sets, Q, its components), the eps solve (alone, or as one branch of a batched
// launch), phase 3 (mu, A, r, b and the preconditioner's operator).  The state that spans the
// phases: scratch ordered on the build's stream, the host copies of phase 1's scalars and the
// prepared eps solve.
struct BuildState {
  Ctx* ctx = nullptr;
  cudaStream_t st = nullptr;
  int64_t n = 0;
  mge_ops_opts o{};
  DevBuf<int64_t> U;                 // two-hop candidate offsets
  DevBuf<int32_t> tlist;             // two-hop lists
  DevBuf<unsigned> d_err;
  DevBuf<double> d_sc;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int h_ncomp = 0;
  double h_den = 0;
  bool need_eps = false;
  LobOp qop;
  int eps_m = 0, eps_maxiter = 0, eps_precision = MGE_FP32;
  double eps_tol = 0;
  uint64_t eps_seed = 0;
  BuildState() = default;
  BuildState(const BuildState&) = delete;
  BuildState& operator=(const BuildState&) = delete;
  ~BuildState() {
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  }
};
mge_status build_phase1(Ctx* ctx, cudaStream_t st, int64_t n, const int64_t* rp_in, const int32_t* col_in,
                        const double* w_in, int on_device, const mge_ops_opts* opts, Ops* ops, BuildState* bs);
mge_status build_eps_single(BuildState* bs, Ops* ops, double* eps);
mge_status build_phase3(BuildState* bs, Ops* ops, double eps);

struct LobResult {
  mge_status status = MGE_OK;
  int iters = 0;
  int drops = 0;
  int rr64_from = -1;              // FP64 Rayleigh-Ritz: -1 never, 0 from the start, k after iteration k
  std::vector<double> lambda;      // [K]
  std::vector<double> eta;         // [K]
  double ms = 0;
};

// Runs LOBPCG; V_out (device, FP64 column-major [n x K]) may be NULL.
mge_status lobpcg_solve(Ctx* ctx, cudaStream_t st, const LobOp& op, int precision, int K, int m,
                        double tol, int maxiter, uint64_t seed, int check_every, bool use_graph,
                        const double* x0_dev /*col-major n x x0_cols*/, int x0_cols,
                        double* V_out, LobResult* res);
// Runs `count` solves (operator ops[i], K[i] pairs, block width m[i]) as branches of one CUDA
// graph launched once on st; status[i] and res[i] per solve, batch_ms the launch's device time.
// V_out (NULL, or an array of device pointers that may hold NULLs) as in lobpcg_solve.
mge_status lobpcg_solve_batch(Ctx* ctx, cudaStream_t st, int count, const LobOp* ops, int precision, const int* K,
                              const int* m, double tol, int maxiter, uint64_t seed, double* const* V_out,
                              LobResult* res, mge_status* status, double* batch_ms);

mge_status spmm_apply(Ctx* ctx, cudaStream_t st, const LobOp& op, int precision, int m,
                      const void* X, void* Y);
// Y = A Y through a fixed device array (no allocation); see lobpcg.cu.
mge_status spmm_apply_inplace(Ctx* ctx, cudaStream_t st, const LobOp& op, int precision, int m, void* XY);
size_t inplace_scratch_bytes();

// out[0..n] = exclusive scan of in[0..n-1], out[n] = the total (synchronises the stream)
mge_status scan_exclusive(Ctx* ctx, cudaStream_t st, const int64_t* in, int64_t n, int64_t* out);

// Locality order of the nodes of W (order.cu): order[r] = the input node placed at row r,
// rank[i] = the row of input node i, and W renamed (rp_out, col_out, w_out; ascending
// columns, the same padding as the input copy).
mge_status locality_order(Ctx* ctx, cudaStream_t st, int64_t n, const int64_t* rp, const int32_t* col,
                          const double* w, int64_t nnz, DevBuf<int32_t>* order, DevBuf<int32_t>* rank,
                          DevBuf<int64_t>* rp_out, DevBuf<int32_t>* col_out, DevBuf<double>* w_out);

// supported block widths
inline int round_block_width(int m) {
  const int w[] = {4, 8, 12, 16, 24, 32};
  for (int x : w) if (m <= x) return x;
  return -1;
}

inline int ceil_div_i(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

}  // namespace mge

struct mge_ctx { mge::Ctx impl; };
struct mge_ops { mge::Ops impl; };
struct mge_graph { mge::Graph impl; };
