// Locality order of the nodes (a memory-layout step of the operator build; the paper's
// method does not depend on the node numbering).
//
// The SpMMs of both LOBPCG solves gather rows x_j of the iterate for the column indices j of
// each row, and on a k-NN graph whose nodes come in random order every gather touches a
// different 32-byte sector: the step is bound by the L2's sector rate.  Renumbering the
// nodes so that the rows of one SpMM tile are a compact patch of the graph lets the tile's
// gathers share sectors in L1 (measured on a 200k-node swiss roll: 3.5x fewer distinct rows
// per 128-row tile, Chebyshev step on L + eps I 18.5 -> 14.4 us, on Q 28.7 -> 18.4 us).
//
// The patches are the cells of a multi-source BFS: about one node in kCellNodes is a seed
// (chosen by a hash of its index), every node joins the seed nearest in hops (ties: the
// smaller seed index), and nodes are ordered by (cell, hop distance, node index) with a
// stable radix sort.  The BFS is a min-relaxation of the packed pair (distance, seed) to
// its unique fixed point, so the order does not depend on the order of updates.
#include "mge_internal.cuh"

#include <algorithm>

namespace mge {
namespace {

constexpr int kCellNodes = 128;          // mean nodes per cell: one SpMM tile
constexpr int kSweepsPerCheck = 4;
constexpr int kMaxSweeps = 1 << 20;
constexpr int kSortBlock = 1024;
constexpr uint64_t kUnreached = ~0ull;

inline unsigned blocks_for(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

__device__ __forceinline__ uint64_t mix64(uint64_t x) {
  // SplitMix64 finaliser (Steele, Lea, Flood 2014)
  x += 0x9e3779b97f4a7c15ull;
  x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ull;
  x = (x ^ (x >> 27)) * 0x94d049bb133111ebull;
  return x ^ (x >> 31);
}

// state s_i = (hop distance << 32) | seed; seeds start at (0, i), other nodes unreached
__global__ void k_cell_init(int64_t n, uint64_t* __restrict__ s) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  s[i] = (mix64((uint64_t)i) % kCellNodes == 0) ? (uint64_t)i : kUnreached;
}

// One relaxation sweep in place: s_i = min(s_i, min_j s_j + (1 << 32)).  Values written by
// other threads during the sweep may or may not be seen; either way s only decreases toward
// the same fixed point, and a sweep that changes nothing proves it reached.
__global__ void k_cell_sweep(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                             uint64_t* s, int* changed) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint64_t cur = s[i];
  uint64_t best = cur;
  for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
    const uint64_t v = s[col[p]];
    if (v != kUnreached && v + (1ull << 32) < best) best = v + (1ull << 32);
  }
  if (best < cur) {
    s[i] = best;
    *changed = 1;
  }
}

// cell representatives: seeds that were reached, and unreached nodes (a component without a
// seed: each such node forms its own cell)
__global__ void k_cell_heads(int64_t n, const uint64_t* __restrict__ s, int64_t* __restrict__ head) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  head[i] = (s[i] == (uint64_t)i || s[i] == kUnreached) ? 1 : 0;
}

// sort key: (cell index << 8) | min(distance, 255); value: the node
__global__ void k_cell_keys(int64_t n, const uint64_t* __restrict__ s, const int64_t* __restrict__ cell_of,
                            uint64_t* __restrict__ key, int32_t* __restrict__ val) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint64_t v = s[i];
  const uint64_t seed = (v == kUnreached) ? (uint64_t)i : (v & 0xffffffffull);
  const uint64_t dist = (v == kUnreached) ? 0 : ((v >> 32) < 255 ? (v >> 32) : 255);
  key[i] = ((uint64_t)cell_of[seed] << 8) | dist;
  val[i] = (int32_t)i;
}

// ---- stable LSD radix sort, 8 bits per pass ----------------------------------------------
// digit counts per block, digit-major: hist[d * nblocks + b]
__global__ void __launch_bounds__(kSortBlock) k_rs_hist(int64_t n, const uint64_t* __restrict__ key, int shift,
                                                         int64_t* __restrict__ hist) {
  __shared__ int cnt[256];
  for (int d = threadIdx.x; d < 256; d += blockDim.x) cnt[d] = 0;
  __syncthreads();
  const int64_t k = blockIdx.x * (int64_t)kSortBlock + threadIdx.x;
  if (k < n) atomicAdd(&cnt[(key[k] >> shift) & 255], 1);
  __syncthreads();
  for (int d = threadIdx.x; d < 256; d += blockDim.x) hist[(int64_t)d * gridDim.x + blockIdx.x] = cnt[d];
}

// Scatter in input order within each digit: an item's place is the digit's offset for the
// block, plus the same-digit items of earlier warps, plus those of earlier lanes.
__global__ void __launch_bounds__(kSortBlock) k_rs_scatter(int64_t n, const uint64_t* __restrict__ key_in,
                                                            const int32_t* __restrict__ val_in, int shift,
                                                            const int64_t* __restrict__ off,
                                                            uint64_t* __restrict__ key_out,
                                                            int32_t* __restrict__ val_out) {
  __shared__ int cnt[kSortBlock / 32][256];
  const int lane = threadIdx.x % 32, wid = threadIdx.x / 32;
  for (int t = threadIdx.x; t < (kSortBlock / 32) * 256; t += blockDim.x) (&cnt[0][0])[t] = 0;
  __syncthreads();
  const int64_t k = blockIdx.x * (int64_t)kSortBlock + threadIdx.x;
  const bool valid = k < n;
  const uint64_t kv = valid ? key_in[k] : 0;
  const int d = (int)((kv >> shift) & 255);
  const unsigned vm = __ballot_sync(0xffffffffu, valid);
  const unsigned peers = __match_any_sync(0xffffffffu, valid ? d : 256 + lane) & vm;
  const int rank = __popc(peers & ((1u << lane) - 1u));
  if (valid && rank == 0) cnt[wid][d] = __popc(peers);
  __syncthreads();
  for (int dd = threadIdx.x; dd < 256; dd += blockDim.x) {
    int run = 0;
    for (int w = 0; w < kSortBlock / 32; ++w) {
      const int c = cnt[w][dd];
      cnt[w][dd] = run;
      run += c;
    }
  }
  __syncthreads();
  if (valid) {
    const int64_t pos = off[(int64_t)d * gridDim.x + blockIdx.x] + cnt[wid][d] + rank;
    key_out[pos] = kv;
    val_out[pos] = val_in[k];
  }
}

__global__ void k_rank_of(int64_t n, const int32_t* __restrict__ order, int32_t* __restrict__ rank) {
  const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r < n) rank[order[r]] = (int32_t)r;
}

// ---- the graph in the new numbering --------------------------------------------------------
__global__ void k_perm_len(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ order,
                           int64_t* __restrict__ len) {
  const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r < n) len[r] = rp[order[r] + 1] - rp[order[r]];
}

// new row r = old row order[r] with columns renamed by rank and sorted ascending (insertion
// sort: rows of a k-NN graph are short)
__global__ void k_perm_fill(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                            const double* __restrict__ w, const int32_t* __restrict__ order,
                            const int32_t* __restrict__ rank, const int64_t* __restrict__ rp2,
                            int32_t* __restrict__ col2, double* __restrict__ w2) {
  const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= n) return;
  const int64_t s = rp[order[r]], len = rp[order[r] + 1] - s, o = rp2[r];
  for (int64_t k = 0; k < len; ++k) {
    const int32_t c = rank[col[s + k]];
    const double v = w[s + k];
    int64_t q = k;
    while (q > 0 && col2[o + q - 1] > c) {
      col2[o + q] = col2[o + q - 1];
      w2[o + q] = w2[o + q - 1];
      --q;
    }
    col2[o + q] = c;
    w2[o + q] = v;
  }
}

}  // namespace

mge_status locality_order(Ctx* ctx, cudaStream_t st, int64_t n, const int64_t* rp, const int32_t* col,
                          const double* w, int64_t nnz, DevBuf<int32_t>* order, DevBuf<int32_t>* rank,
                          DevBuf<int64_t>* rp_out, DevBuf<int32_t>* col_out, DevBuf<double>* w_out) {
  const int B = 256;
  // --- cells: multi-source BFS to the fixed point ---
  DevBuf<uint64_t> s;
  DevBuf<int> changed;
  MGE_TRY(s.scratch(ctx, n, st));
  MGE_TRY(changed.scratch(ctx, 1, st));
  k_cell_init<<<blocks_for(n, B), B, 0, st>>>(n, s.p);
  MGE_LAUNCHED(ctx, 1);
  int sweeps = 0;
  for (;;) {
    MGE_CUDA(ctx, cudaMemsetAsync(changed.p, 0, sizeof(int), st));
    for (int k = 0; k < kSweepsPerCheck; ++k) k_cell_sweep<<<blocks_for(n, B), B, 0, st>>>(n, rp, col, s.p, changed.p);
    MGE_LAUNCHED(ctx, kSweepsPerCheck);
    sweeps += kSweepsPerCheck;
    int h = 0;
    MGE_CUDA(ctx, cudaMemcpyAsync(&h, changed.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    MGE_CUDA(ctx, cudaStreamSynchronize(st));
    if (!h) break;
    if (sweeps >= kMaxSweeps) { set_error(ctx, "node ordering: BFS sweep limit reached"); return MGE_ETIMEOUT; }
  }
  // --- keys: cell index (cells numbered by their seed), then distance ---
  DevBuf<int64_t> head, cell_of;
  MGE_TRY(head.scratch(ctx, n, st));
  MGE_TRY(cell_of.scratch(ctx, n + 1, st));
  k_cell_heads<<<blocks_for(n, B), B, 0, st>>>(n, s.p, head.p);
  MGE_LAUNCHED(ctx, 1);
  MGE_TRY(scan_exclusive(ctx, st, head.p, n, cell_of.p));
  int64_t ncells = 0;
  MGE_CUDA(ctx, cudaMemcpyAsync(&ncells, cell_of.p + n, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  MGE_CUDA(ctx, cudaStreamSynchronize(st));
  DevBuf<uint64_t> key0, key1;
  DevBuf<int32_t> val0, val1;
  MGE_TRY(key0.scratch(ctx, n, st));
  MGE_TRY(key1.scratch(ctx, n, st));
  MGE_TRY(val0.scratch(ctx, n, st));
  MGE_TRY(val1.scratch(ctx, n, st));
  k_cell_keys<<<blocks_for(n, B), B, 0, st>>>(n, s.p, cell_of.p, key0.p, val0.p);
  MGE_LAUNCHED(ctx, 1);
  // --- stable radix sort over the key's significant bits ---
  int bits = 8;
  while (bits < 64 && (((uint64_t)std::max<int64_t>(ncells - 1, 0) << 8) >> bits) != 0) ++bits;
  const int64_t nb = (n + kSortBlock - 1) / kSortBlock;
  DevBuf<int64_t> hist, off;
  MGE_TRY(hist.scratch(ctx, 256 * nb, st));
  MGE_TRY(off.scratch(ctx, 256 * nb + 1, st));
  uint64_t* kin = key0.p; uint64_t* kout = key1.p;
  int32_t* vin = val0.p; int32_t* vout = val1.p;
  for (int shift = 0; shift < bits; shift += 8) {
    k_rs_hist<<<(unsigned)nb, kSortBlock, 0, st>>>(n, kin, shift, hist.p);
    MGE_LAUNCHED(ctx, 1);
    MGE_TRY(scan_exclusive(ctx, st, hist.p, 256 * nb, off.p));
    k_rs_scatter<<<(unsigned)nb, kSortBlock, 0, st>>>(n, kin, vin, shift, off.p, kout, vout);
    MGE_LAUNCHED(ctx, 1);
    std::swap(kin, kout);
    std::swap(vin, vout);
  }
  MGE_TRY(order->alloc(ctx, n));
  MGE_TRY(rank->alloc(ctx, n));
  MGE_CUDA(ctx, cudaMemcpyAsync(order->p, vin, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
  k_rank_of<<<blocks_for(n, B), B, 0, st>>>(n, order->p, rank->p);
  MGE_LAUNCHED(ctx, 1);
  // --- W in the new numbering (same padding as the input copy) ---
  DevBuf<int64_t> len;
  MGE_TRY(len.scratch(ctx, n, st));
  MGE_TRY(rp_out->alloc(ctx, n + 2));
  MGE_TRY(col_out->alloc(ctx, nnz + 4));
  MGE_TRY(w_out->alloc(ctx, nnz));
  MGE_CUDA(ctx, cudaMemsetAsync(rp_out->p + n + 1, 0, sizeof(int64_t), st));
  MGE_CUDA(ctx, cudaMemsetAsync(col_out->p + nnz, 0, 4 * sizeof(int32_t), st));
  k_perm_len<<<blocks_for(n, B), B, 0, st>>>(n, rp, order->p, len.p);
  MGE_LAUNCHED(ctx, 1);
  MGE_TRY(scan_exclusive(ctx, st, len.p, n, rp_out->p));
  k_perm_fill<<<blocks_for(n, B), B, 0, st>>>(n, rp, col, w, order->p, rank->p, rp_out->p, col_out->p, w_out->p);
  MGE_LAUNCHED(ctx, 1);
  MGE_CUDA(ctx, cudaGetLastError());
  return MGE_OK;
}

}  // namespace mge
