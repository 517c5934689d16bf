// kNN graph construction from points (Sec. 5.1: the input graphs are kNN graphs built from
// Euclidean distances between samples).  The paper leaves the details open; the library
// builds:
//   * the exact k nearest neighbours of every point (itself excluded) by Euclidean distance,
//     equal distances ordered by the lower index.  The squared distance is summed over the
//     coordinates in order, each product and sum rounded separately (no fused multiply-add),
//     so that the selection is a function of the inputs alone;
//   * the union of the directed relations (i ~ j if either is among the other's k nearest);
//   * Gaussian weights w_ij = exp(-d_ij^2 / sigma^2), sigma the mean of the n k directed
//     nearest-neighbour distances.
//
// Search: the points are binned into a uniform grid of cubic cells (counting sort by cell);
// one thread per point, in cell order so that a warp's queries visit the same cells, scans
// the cells in rings of growing Chebyshev radius around its own cell and keeps its k best
// (distance, index) pairs in registers.  After ring r every point within the distance from
// the query to the faces of the (2r+1)^d block of cells has been seen, so the search stops
// once the k-th best distance is below it.  The cell size comes from the points' occupancy:
// a first binning with about one cell per point, then cells grown or shrunk so that occupied
// cells hold about two points (points on a surface in 3-D occupy few of the cells).
//
// Symmetrisation: in-degrees by atomics, each row's candidates (its k nearest and the points
// that chose it) gathered into one list, sorted and deduplicated by one warp per row.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <vector>

#include "mge_internal.cuh"

namespace mge {
namespace knn {
namespace {

constexpr int kBlock = 256;
constexpr int kMaxRow = 1024;              // candidates of one row for the warp sort
constexpr int64_t kMaxCells = 1LL << 24;

__device__ __forceinline__ long long ord_key(double x) {
  // order-preserving map of doubles to signed 64-bit integers (for atomicMin / atomicMax)
  long long k = __double_as_longlong(x);
  return k >= 0 ? k : (k ^ 0x7fffffffffffffffLL);
}

__global__ void k_bbox(int64_t n, int dim, const double* __restrict__ P, long long* __restrict__ lohi) {
  __shared__ long long slo[3], shi[3];
  if (threadIdx.x < 3) { slo[threadIdx.x] = LLONG_MAX; shi[threadIdx.x] = LLONG_MIN; }
  __syncthreads();
  long long lo[3] = {LLONG_MAX, LLONG_MAX, LLONG_MAX}, hi[3] = {LLONG_MIN, LLONG_MIN, LLONG_MIN};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    for (int c = 0; c < dim; ++c) {
      const long long k = ord_key(P[i * dim + c]);
      lo[c] = min(lo[c], k);
      hi[c] = max(hi[c], k);
    }
  for (int c = 0; c < dim; ++c) { atomicMin(&slo[c], lo[c]); atomicMax(&shi[c], hi[c]); }
  __syncthreads();
  if (threadIdx.x < dim) {
    atomicMin(&lohi[threadIdx.x], slo[threadIdx.x]);
    atomicMax(&lohi[3 + threadIdx.x], shi[threadIdx.x]);
  }
}

struct Grid {
  double lo[3];
  double h, inv_h;
  double slack;          // rounding allowance of the cell faces (absolute)
  int g[3];
  int dim;
};

__device__ __forceinline__ int cell_coord(const Grid& gr, double x, int c) {
  int v = (int)floor((x - gr.lo[c]) * gr.inv_h);
  return min(max(v, 0), gr.g[c] - 1);
}

__device__ __forceinline__ int64_t cell_of(const Grid& gr, const double* p) {
  int64_t id = 0;
  for (int c = gr.dim - 1; c >= 0; --c) id = id * gr.g[c] + cell_coord(gr, p[c], c);
  return id;
}

__global__ void k_cell_count(int64_t n, Grid gr, const double* __restrict__ P, int64_t* __restrict__ cnt,
                             int32_t* __restrict__ cell) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = cell_of(gr, P + i * gr.dim);
    cell[i] = (int32_t)c;
    atomicAdd(reinterpret_cast<unsigned long long*>(cnt + c), 1ull);
  }
}

__global__ void k_count_nonzero(int64_t m, const int64_t* __restrict__ cnt, unsigned long long* __restrict__ occ) {
  unsigned long long local = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
    local += cnt[i] != 0;
  for (int o = 16; o > 0; o >>= 1) local += __shfl_xor_sync(0xffffffffu, local, o);
  if ((threadIdx.x & 31) == 0 && local) atomicAdd(occ, local);
}

// points in cell order: coordinates (structure of arrays) and their input indices
__global__ void k_scatter(int64_t n, int dim, const double* __restrict__ P, const int32_t* __restrict__ cell,
                          const int64_t* __restrict__ start, unsigned int* __restrict__ fill,
                          double* __restrict__ sp, int32_t* __restrict__ sidx) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t c = cell[i];
    const int64_t pos = start[c] + atomicAdd(fill + c, 1u);
    sidx[pos] = (int32_t)i;
    for (int d = 0; d < dim; ++d) sp[(int64_t)d * n + pos] = P[i * dim + d];
  }
}

// squared distance, coordinates in order, no contraction into fused multiply-adds
template <int D>
__device__ __forceinline__ double dist2(const double* q, const double* __restrict__ sp, int64_t n, int64_t j) {
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < D; ++c) {
    const double t = __dsub_rn(q[c], sp[(int64_t)c * n + j]);
    s = __dadd_rn(s, __dmul_rn(t, t));
  }
  return s;
}

// the k best (d2, index) pairs, ascending, in the last k of KB slots (the first KB - k hold
// sentinels that compare below every candidate, so the worst kept pair is always slot KB-1)
template <int KB>
struct TopK {
  double d[KB];
  int32_t j[KB];
  __device__ __forceinline__ void init(int k) {
#pragma unroll
    for (int s = 0; s < KB; ++s) {
      const bool sent = s < KB - k;
      d[s] = sent ? -1.0 : INFINITY;
      j[s] = sent ? -1 : INT_MAX;
    }
  }
  __device__ __forceinline__ static bool less(double da, int32_t ja, double db, int32_t jb) {
    return da < db || (da == db && ja < jb);
  }
  __device__ __forceinline__ void offer(double dn, int32_t jn) {
    if (!less(dn, jn, d[KB - 1], j[KB - 1])) return;
    d[KB - 1] = dn;
    j[KB - 1] = jn;
#pragma unroll
    for (int s = KB - 1; s > 0; --s) {
      if (less(d[s], j[s], d[s - 1], j[s - 1])) {
        const double td = d[s]; d[s] = d[s - 1]; d[s - 1] = td;
        const int32_t tj = j[s]; j[s] = j[s - 1]; j[s - 1] = tj;
      }
    }
  }
};

template <int D, int KB>
__global__ void __launch_bounds__(kBlock) k_query(int64_t n, int k, Grid gr, const double* __restrict__ sp,
                                                  const int32_t* __restrict__ sidx,
                                                  const int64_t* __restrict__ start, int32_t* __restrict__ nbr,
                                                  double* __restrict__ nd2, int* __restrict__ err) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n) return;
  double q[D];
  int qc[D];
#pragma unroll
  for (int c = 0; c < D; ++c) {
    q[c] = sp[(int64_t)c * n + t];
    qc[c] = cell_coord(gr, q[c], c);
  }
  const int32_t self = sidx[t];
  TopK<KB> best;
  best.init(k);
  int maxr = 0;
#pragma unroll
  for (int c = 0; c < D; ++c) maxr = max(maxr, max(qc[c], gr.g[c] - 1 - qc[c]));
  const int q1 = qc[1];
  int q2 = 0, g2 = 1;
  if constexpr (D > 2) { q2 = qc[2]; g2 = gr.g[2]; }
  auto scan_cell = [&](int c0, int c1, int c2) {
    const int64_t cid = ((int64_t)c2 * gr.g[1] + c1) * gr.g[0] + c0;
    const int64_t b = start[cid], e = start[cid + 1];
    for (int64_t p = b; p < e; ++p) {
      const int32_t jj = sidx[p];
      if (jj == self) continue;
      best.offer(dist2<D>(q, sp, n, p), jj);
    }
  };
  for (int r = 0; r <= maxr; ++r) {
    // the cells at Chebyshev distance exactly r from the query's cell: whole rows along axis 0
    // where axis 1 or 2 is at distance r, else the two end cells of the row
    const int lo0 = max(qc[0] - r, 0), hi0 = min(qc[0] + r, gr.g[0] - 1);
    const int lo1 = max(q1 - r, 0), hi1 = min(q1 + r, gr.g[1] - 1);
    const int lo2 = max(q2 - r, 0), hi2 = min(q2 + r, g2 - 1);
    for (int c2 = lo2; c2 <= hi2; ++c2)
      for (int c1 = lo1; c1 <= hi1; ++c1) {
        const bool edge = r == 0 || abs(c1 - q1) == r || (D > 2 && abs(c2 - q2) == r);
        if (edge) {
          for (int c0 = lo0; c0 <= hi0; ++c0) scan_cell(c0, c1, c2);
        } else {
          if (qc[0] - r >= 0) scan_cell(qc[0] - r, c1, c2);
          if (qc[0] + r <= gr.g[0] - 1) scan_cell(qc[0] + r, c1, c2);
        }
      }
    // distance from the query to the faces of the scanned block (grid borders excepted)
    double bd = INFINITY;
#pragma unroll
    for (int c = 0; c < D; ++c) {
      if (qc[c] - r > 0) bd = fmin(bd, q[c] - (gr.lo[c] + (double)(qc[c] - r) * gr.h));
      if (qc[c] + r < gr.g[c] - 1) bd = fmin(bd, (gr.lo[c] + (double)(qc[c] + r + 1) * gr.h) - q[c]);
    }
    const double worst = best.d[KB - 1];
    if (bd == INFINITY) break;                                     // every cell scanned
    bd -= gr.slack;
    if (bd > 0 && worst * (1.0 + 1e-9) < bd * bd) break;
  }
  if (best.j[KB - 1] == INT_MAX) atomicExch(err, 1);               // fewer than k points found
  const int64_t o = (int64_t)self * k;
#pragma unroll
  for (int s = 0; s < KB; ++s) {
    if (s >= KB - k) {
      nbr[o + s - (KB - k)] = best.j[s];
      nd2[o + s - (KB - k)] = best.d[s];
    }
  }
}

// deterministic sum of sqrt(d2) over all directed pairs: per-block partials, then in order
__global__ void k_sqrt_partial(int64_t m, const double* __restrict__ d2, double* __restrict__ part) {
  __shared__ double sh[kBlock];
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
    s += sqrt(d2[i]);
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = kBlock / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void k_indeg(int64_t m, const int32_t* __restrict__ nbr, int64_t* __restrict__ indeg) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(reinterpret_cast<unsigned long long*>(indeg + nbr[i]), 1ull);
}

__global__ void k_cand_len(int64_t n, int k, const int64_t* __restrict__ indeg, int64_t* __restrict__ len) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    len[i] = k + indeg[i];
}

__global__ void k_cand_fill(int64_t n, int k, const int32_t* __restrict__ nbr, const int64_t* __restrict__ cptr,
                            unsigned int* __restrict__ cursor, int32_t* __restrict__ cand) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * k; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / k;
    const int32_t j = nbr[e];
    cand[cptr[i] + (e - i * k)] = j;                                  // i's own choice
    cand[cptr[j] + k + atomicAdd(cursor + j, 1u)] = (int32_t)i;       // i chose j
  }
}

// one warp per row: sort the row's candidates, drop duplicates, write the unique ones back
// to the front of the row's range and the count to len
__global__ void k_row_unique(int64_t n, const int64_t* __restrict__ cptr, int32_t* __restrict__ cand,
                             int64_t* __restrict__ len, int* __restrict__ err) {
  __shared__ int32_t buf[kBlock / 32][kMaxRow];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int32_t* b = buf[w];
  for (int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; i < n;
       i += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const int64_t p0 = cptr[i];
    const int L = (int)(cptr[i + 1] - p0);
    if (L > kMaxRow) {
      if (lane == 0) { atomicExch(err, 2); len[i] = 0; }
      continue;
    }
    int P2 = 32;
    while (P2 < L) P2 <<= 1;
    for (int t = lane; t < P2; t += 32) b[t] = t < L ? cand[p0 + t] : INT_MAX;
    __syncwarp();
    // bitonic sort of P2 entries in shared memory
    for (int size = 2; size <= P2; size <<= 1)
      for (int stride = size >> 1; stride > 0; stride >>= 1) {
        for (int t = lane; t < P2; t += 32) {
          const int u = t ^ stride;
          if (u > t) {
            const bool up = (t & size) == 0;
            const int32_t x = b[t], y = b[u];
            if ((x > y) == up) { b[t] = y; b[u] = x; }
          }
        }
        __syncwarp();
      }
    // unique: compact the first occurrence of each value, in order
    int base = 0;
    for (int t0 = 0; t0 < L; t0 += 32) {
      const int t = t0 + lane;
      const bool first = t < L && (t == 0 || b[t] != b[t - 1]);
      const unsigned m = __ballot_sync(0xffffffffu, first);
      const int pos = base + __popc(m & ((1u << lane) - 1u));
      const int32_t v = t < L ? b[t] : 0;
      __syncwarp();
      if (first) cand[p0 + pos] = v;
      base += __popc(m);
    }
    if (lane == 0) len[i] = base;
    __syncwarp();
  }
}

__global__ void k_emit(int64_t n, int dim, const double* __restrict__ P, const int64_t* __restrict__ cptr,
                       const int32_t* __restrict__ cand, const int64_t* __restrict__ rp, double s2,
                       int32_t* __restrict__ col, double* __restrict__ w) {
  for (int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; i < n;
       i += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const int lane = threadIdx.x & 31;
    const int64_t o = rp[i], L = rp[i + 1] - o, c0 = cptr[i];
    for (int64_t t = lane; t < L; t += 32) {
      const int32_t j = cand[c0 + t];
      double s = 0.0;
      for (int c = 0; c < dim; ++c) {
        const double d = __dsub_rn(P[i * dim + c], P[(int64_t)j * dim + c]);
        s = __dadd_rn(s, __dmul_rn(d, d));
      }
      col[o + t] = j;
      w[o + t] = exp(-(s / s2));
    }
  }
}

inline unsigned grid_for(const Ctx* ctx, int64_t work) {
  const int64_t g = (work + kBlock - 1) / kBlock;
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(g, (int64_t)ctx->num_sms * 8));
}

template <int D, int KB>
void launch_query(cudaStream_t st, int64_t n, int k, const Grid& gr, const double* sp, const int32_t* sidx,
                  const int64_t* start, int32_t* nbr, double* nd2, int* err) {
  k_query<D, KB><<<(unsigned)((n + kBlock - 1) / kBlock), kBlock, 0, st>>>(n, k, gr, sp, sidx, start, nbr, nd2, err);
}

template <int D>
void launch_query_k(cudaStream_t st, int64_t n, int k, const Grid& gr, const double* sp, const int32_t* sidx,
                    const int64_t* start, int32_t* nbr, double* nd2, int* err) {
  if (k <= 8) launch_query<D, 8>(st, n, k, gr, sp, sidx, start, nbr, nd2, err);
  else if (k <= 16) launch_query<D, 16>(st, n, k, gr, sp, sidx, start, nbr, nd2, err);
  else launch_query<D, 32>(st, n, k, gr, sp, sidx, start, nbr, nd2, err);
}

// grid of cubic cells of side h over the bounding box (at least one cell per axis)
Grid make_grid(int dim, const double* lo, const double* hi, double h) {
  Grid g{};
  g.dim = dim;
  g.h = h;
  g.inv_h = 1.0 / h;
  double amax = 0.0;
  for (int c = 0; c < dim; ++c) amax = std::max(amax, std::max(std::fabs(lo[c]), std::fabs(hi[c])));
  g.slack = 1e-12 * h + 64.0 * 2.220446049250313e-16 * amax;
  for (int c = 0; c < 3; ++c) {
    g.lo[c] = c < dim ? lo[c] : 0.0;
    const double ext = c < dim ? hi[c] - lo[c] : 0.0;
    g.g[c] = c < dim ? (int)std::max<double>(1.0, std::min<double>(std::ceil(ext / h), 1 << 22)) : 1;
  }
  return g;
}

int64_t cells_of(const Grid& g) { return (int64_t)g.g[0] * g.g[1] * g.g[2]; }

}  // namespace
}  // namespace knn

mge_status knn_graph_build(Ctx* ctx, cudaStream_t st, int64_t n, int dim, const double* P, int k, Graph* out) {
  using namespace knn;
  if (n < 2 || dim < 2 || dim > 3 || k < 1 || k > 32 || k >= n || n > INT32_MAX - 1) {
    set_error(ctx, "knn: need dim in {2, 3}, 1 <= k <= 32, k < n < 2^31 (n = %lld, dim = %d, k = %d)",
              (long long)n, dim, k);
    return MGE_EINVAL;
  }
  // --- bounding box ---
  DevBuf<long long> lohi;
  MGE_TRY(lohi.scratch(ctx, 6, st));
  long long init[6] = {LLONG_MAX, LLONG_MAX, LLONG_MAX, LLONG_MIN, LLONG_MIN, LLONG_MIN};
  MGE_CUDA(ctx, cudaMemcpyAsync(lohi.p, init, sizeof(init), cudaMemcpyHostToDevice, st));
  k_bbox<<<grid_for(ctx, n), kBlock, 0, st>>>(n, dim, P, lohi.p);
  MGE_LAUNCHED(ctx, 1);
  long long hk[6];
  MGE_CUDA(ctx, cudaMemcpyAsync(hk, lohi.p, sizeof(hk), cudaMemcpyDeviceToHost, st));
  MGE_CUDA(ctx, cudaStreamSynchronize(st));
  double lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
  double vol = 1.0, maxext = 0.0;
  for (int c = 0; c < dim; ++c) {
    const long long a = hk[c], b = hk[3 + c];
    const long long ua = a >= 0 ? a : (a ^ 0x7fffffffffffffffLL), ub = b >= 0 ? b : (b ^ 0x7fffffffffffffffLL);
    std::memcpy(&lo[c], &ua, sizeof(double));
    std::memcpy(&hi[c], &ub, sizeof(double));
    if (!std::isfinite(lo[c]) || !std::isfinite(hi[c])) {
      set_error(ctx, "knn: non-finite coordinates");
      return MGE_EINVAL;
    }
    maxext = std::max(maxext, hi[c] - lo[c]);
  }
  if (!(maxext > 0)) {
    set_error(ctx, "knn: all points coincide");
    return MGE_EINVAL;
  }
  for (int c = 0; c < dim; ++c) vol *= std::max(hi[c] - lo[c], maxext * 1e-6);
  // --- cell size: about one cell per point, then resized so occupied cells hold ~2 points ---
  DevBuf<int64_t> cnt, start;
  DevBuf<int32_t> cell;
  MGE_TRY(cell.scratch(ctx, (size_t)n, st));
  DevBuf<unsigned long long> occ;
  MGE_TRY(occ.scratch(ctx, 1, st));
  double h = std::pow(vol / (double)n, 1.0 / dim);
  Grid gr = make_grid(dim, lo, hi, h);
  while (cells_of(gr) > kMaxCells) { h *= 1.25; gr = make_grid(dim, lo, hi, h); }
  for (int pass = 0; pass < 2; ++pass) {
    const int64_t nc = cells_of(gr);
    MGE_TRY(cnt.scratch(ctx, (size_t)nc + 1, st));
    MGE_CUDA(ctx, cudaMemsetAsync(cnt.p, 0, (nc + 1) * sizeof(int64_t), st));
    k_cell_count<<<grid_for(ctx, n), kBlock, 0, st>>>(n, gr, P, cnt.p, cell.p);
    MGE_LAUNCHED(ctx, 1);
    if (pass == 1) break;
    MGE_CUDA(ctx, cudaMemsetAsync(occ.p, 0, sizeof(unsigned long long), st));
    k_count_nonzero<<<grid_for(ctx, nc), kBlock, 0, st>>>(nc, cnt.p, occ.p);
    MGE_LAUNCHED(ctx, 1);
    unsigned long long hocc = 0;
    MGE_CUDA(ctx, cudaMemcpyAsync(&hocc, occ.p, sizeof(hocc), cudaMemcpyDeviceToHost, st));
    MGE_CUDA(ctx, cudaStreamSynchronize(st));
    const double per = (double)n / (double)std::max<unsigned long long>(1, hocc);
    // occupied cells scale as h^e with e the points' intrinsic dimension; estimate e from the
    // occupancy (a full d-dimensional cloud fills about n cells at this size)
    const double fill = (double)hocc / (double)std::min<int64_t>(n, nc);
    const double e = fill > 0.5 ? dim : (dim == 3 ? 2.0 : 1.0);
    const double target = 2.0;
    if (per > 2 * target || per < 0.5 * target) {
      double h2 = h * std::pow(target / per, 1.0 / e);
      Grid g2 = make_grid(dim, lo, hi, h2);
      while (cells_of(g2) > kMaxCells) { h2 *= 1.25; g2 = make_grid(dim, lo, hi, h2); }
      h = h2;
      gr = g2;
    } else {
      // keep this binning: count again only to reuse the same code path
    }
  }
  const int64_t nc = cells_of(gr);
  MGE_TRY(start.scratch(ctx, (size_t)nc + 1, st));
  MGE_TRY(scan_exclusive(ctx, st, cnt.p, nc, start.p));        // synchronises the stream
  // --- points in cell order ---
  DevBuf<unsigned int> fill;
  MGE_TRY(fill.scratch(ctx, (size_t)nc, st));
  MGE_CUDA(ctx, cudaMemsetAsync(fill.p, 0, nc * sizeof(unsigned int), st));
  DevBuf<double> sp;
  DevBuf<int32_t> sidx;
  MGE_TRY(sp.scratch(ctx, (size_t)n * dim, st));
  MGE_TRY(sidx.scratch(ctx, (size_t)n, st));
  k_scatter<<<grid_for(ctx, n), kBlock, 0, st>>>(n, dim, P, cell.p, start.p, fill.p, sp.p, sidx.p);
  MGE_LAUNCHED(ctx, 1);
  // --- k nearest of every point ---
  DevBuf<int32_t> nbr;
  DevBuf<double> nd2;
  DevBuf<int> err;
  MGE_TRY(nbr.scratch(ctx, (size_t)n * k, st));
  MGE_TRY(nd2.scratch(ctx, (size_t)n * k, st));
  MGE_TRY(err.scratch(ctx, 1, st));
  MGE_CUDA(ctx, cudaMemsetAsync(err.p, 0, sizeof(int), st));
  if (dim == 2) launch_query_k<2>(st, n, k, gr, sp.p, sidx.p, start.p, nbr.p, nd2.p, err.p);
  else launch_query_k<3>(st, n, k, gr, sp.p, sidx.p, start.p, nbr.p, nd2.p, err.p);
  MGE_LAUNCHED(ctx, 1);
  MGE_CUDA(ctx, cudaGetLastError());
  // --- sigma: mean of the n k directed distances ---
  const int64_t m = n * k;
  const unsigned nb = grid_for(ctx, m);
  DevBuf<double> part;
  MGE_TRY(part.scratch(ctx, nb, st));
  k_sqrt_partial<<<nb, kBlock, 0, st>>>(m, nd2.p, part.p);
  MGE_LAUNCHED(ctx, 1);
  std::vector<double> hpart(nb);
  MGE_CUDA(ctx, cudaMemcpyAsync(hpart.data(), part.p, nb * sizeof(double), cudaMemcpyDeviceToHost, st));
  int herr = 0;
  MGE_CUDA(ctx, cudaMemcpyAsync(&herr, err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  MGE_CUDA(ctx, cudaStreamSynchronize(st));
  if (herr) {
    set_error(ctx, "knn: a point found fewer than k neighbours");
    return MGE_EDEVICE;
  }
  double ssum = 0.0;
  for (double v : hpart) ssum += v;
  const double sigma = ssum / (double)m;
  if (!(sigma > 0)) {
    set_error(ctx, "knn: the mean neighbour distance is zero (coincident points)");
    return MGE_EINVAL;
  }
  // --- union symmetrisation ---
  DevBuf<int64_t> indeg, len, cptr;
  MGE_TRY(indeg.scratch(ctx, (size_t)n + 1, st));
  MGE_CUDA(ctx, cudaMemsetAsync(indeg.p, 0, (n + 1) * sizeof(int64_t), st));
  k_indeg<<<grid_for(ctx, m), kBlock, 0, st>>>(m, nbr.p, indeg.p);
  MGE_TRY(len.scratch(ctx, (size_t)n + 1, st));
  k_cand_len<<<grid_for(ctx, n), kBlock, 0, st>>>(n, k, indeg.p, len.p);
  MGE_LAUNCHED(ctx, 2);
  MGE_TRY(cptr.scratch(ctx, (size_t)n + 1, st));
  MGE_TRY(scan_exclusive(ctx, st, len.p, n, cptr.p));
  int64_t ncand = 0;
  MGE_CUDA(ctx, cudaMemcpyAsync(&ncand, cptr.p + n, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  MGE_CUDA(ctx, cudaStreamSynchronize(st));
  DevBuf<int32_t> cand;
  DevBuf<unsigned int> cursor;
  MGE_TRY(cand.scratch(ctx, (size_t)ncand, st));
  MGE_TRY(cursor.scratch(ctx, (size_t)n, st));
  MGE_CUDA(ctx, cudaMemsetAsync(cursor.p, 0, n * sizeof(unsigned int), st));
  k_cand_fill<<<grid_for(ctx, m), kBlock, 0, st>>>(n, k, nbr.p, cptr.p, cursor.p, cand.p);
  k_row_unique<<<grid_for(ctx, n * 32), kBlock, 0, st>>>(n, cptr.p, cand.p, len.p, err.p);
  MGE_LAUNCHED(ctx, 2);
  MGE_CUDA(ctx, cudaMemcpyAsync(&herr, err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  MGE_CUDA(ctx, cudaStreamSynchronize(st));
  if (herr) {
    set_error(ctx, "knn: a row has more than %d candidate neighbours (many coincident points)", kMaxRow);
    return MGE_EINVAL;
  }
  // --- the CSR and the weights ---
  MGE_TRY(out->row_ptr.alloc(ctx, (size_t)n + 1));
  MGE_TRY(scan_exclusive(ctx, st, len.p, n, out->row_ptr.p));
  int64_t nnz = 0;
  MGE_CUDA(ctx, cudaMemcpyAsync(&nnz, out->row_ptr.p + n, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  MGE_CUDA(ctx, cudaStreamSynchronize(st));
  MGE_TRY(out->col.alloc(ctx, (size_t)nnz));
  MGE_TRY(out->w.alloc(ctx, (size_t)nnz));
  k_emit<<<grid_for(ctx, n * 32), kBlock, 0, st>>>(n, dim, P, cptr.p, cand.p, out->row_ptr.p,
                                                   sigma * sigma, out->col.p, out->w.p);
  MGE_LAUNCHED(ctx, 1);
  MGE_CUDA(ctx, cudaGetLastError());
  MGE_CUDA(ctx, cudaStreamSynchronize(st));
  out->n = n;
  out->nnz = nnz;
  out->sigma = sigma;
  out->dim = dim;
  out->k = k;
  out->cell_size = h;
  return MGE_OK;
}

}  // namespace mge
