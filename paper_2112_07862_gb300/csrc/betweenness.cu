// Betweenness centrality and its variance, VBC (Sec. 3.3, Table 1: the paper qualifies its
// input graphs as manifold graphs by the variance of C_B over the nodes).
//   C_B(i) = sum over ordered pairs (s, t), s != t, both != i, of sigma_st(i) / sigma_st
// with shortest paths counted in hops, computed by Brandes' accumulation: for each source a
// breadth-first search that counts shortest paths, then the dependencies
//   delta_s(v) = sum over successors w of (sigma_s(v) / sigma_s(w)) (1 + delta_s(w))
// in reverse level order; C_B(v) = sum over sources s != v of delta_s(v).
//
// One CTA per source (sources blockIdx.x, blockIdx.x + gridDim.x, ...), level-synchronous:
// the frontier's threads claim undiscovered neighbours with an atomic compare-and-swap on
// the distance and append them to the CTA's BFS order; path counts and dependencies are
// then pulled by each vertex from its neighbours on the adjacent level, in CSR order, so the
// arithmetic does not depend on the order of discovery.  Each CTA accumulates its sources'
// dependencies into its own row of partials, summed afterwards in CTA order.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "mge_internal.cuh"

namespace mge {
namespace bc {
namespace {

constexpr int kThreads = 512;

__global__ void k_check_csr(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                            int* __restrict__ bad) {
  const int64_t nnz = rp[n];
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v <= n; v += (int64_t)gridDim.x * blockDim.x) {
    if (v == 0 && rp[0] != 0) atomicExch(bad, 1);
    if (v < n && rp[v] > rp[v + 1]) atomicExch(bad, 1);
  }
  if (nnz < 0) { atomicExch(bad, 1); return; }
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x)
    if (col[e] < 0 || col[e] >= n) atomicExch(bad, 1);
}

struct Work {
  int32_t* dist;      // [grid][n]
  double* sigma;      // [grid][n]
  double* delta;      // [grid][n]
  int32_t* order;     // [grid][n]   BFS order
  int32_t* lvl;       // [grid][n+2] level boundaries in the BFS order
  double* part;       // [grid][n]   C_B partials
};

__global__ void __launch_bounds__(kThreads) k_brandes(int64_t n, const int64_t* __restrict__ rp,
                                                      const int32_t* __restrict__ col, Work wk) {
  const size_t base = (size_t)blockIdx.x * n;
  int32_t* dist = wk.dist + base;
  double* sigma = wk.sigma + base;
  double* delta = wk.delta + base;
  int32_t* order = wk.order + base;
  int32_t* lvl = wk.lvl + (size_t)blockIdx.x * (n + 2);
  double* part = wk.part + base;
  __shared__ int s_tail;
  for (int64_t v = threadIdx.x; v < n; v += blockDim.x) part[v] = 0.0;
  for (int64_t s = blockIdx.x; s < n; s += gridDim.x) {
    for (int64_t v = threadIdx.x; v < n; v += blockDim.x) { dist[v] = -1; sigma[v] = 0.0; delta[v] = 0.0; }
    __syncthreads();
    if (threadIdx.x == 0) {
      dist[s] = 0; sigma[s] = 1.0; order[0] = (int32_t)s;
      lvl[0] = 0; lvl[1] = 1;
      s_tail = 1;
    }
    __syncthreads();
    // breadth-first levels: level L is order[lvl[L] .. lvl[L+1])
    int L = 0;
    for (;;) {
      const int lo = lvl[L], hi = lvl[L + 1];
      if (lo == hi) break;
      for (int f = lo + threadIdx.x; f < hi; f += blockDim.x) {
        const int32_t v = order[f];
        for (int64_t e = rp[v]; e < rp[v + 1]; ++e) {
          const int32_t w = col[e];
          if (atomicCAS(&dist[w], -1, L + 1) == -1) order[atomicAdd(&s_tail, 1)] = w;
        }
      }
      __syncthreads();
      const int nhi = s_tail;
      for (int f = hi + threadIdx.x; f < nhi; f += blockDim.x) {
        const int32_t w = order[f];
        double sg = 0.0;
        for (int64_t e = rp[w]; e < rp[w + 1]; ++e) {
          const int32_t v = col[e];
          if (dist[v] == L) sg += sigma[v];
        }
        sigma[w] = sg;
      }
      if (threadIdx.x == 0) lvl[L + 2] = nhi;
      __syncthreads();
      ++L;
    }
    // dependencies, deepest level first
    for (int l = L - 1; l >= 0; --l) {
      const int lo = lvl[l], hi = lvl[l + 1];
      for (int f = lo + threadIdx.x; f < hi; f += blockDim.x) {
        const int32_t v = order[f];
        double d = 0.0;
        const double sv = sigma[v];
        for (int64_t e = rp[v]; e < rp[v + 1]; ++e) {
          const int32_t w = col[e];
          if (dist[w] == l + 1) d += sv / sigma[w] * (1.0 + delta[w]);
        }
        delta[v] = d;
        if (v != s) part[v] += d;
      }
      __syncthreads();
    }
  }
}

__global__ void k_reduce_parts(int64_t n, int parts, const double* __restrict__ part, double* __restrict__ cb) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < parts; ++b) s += part[(size_t)b * n + v];
    cb[v] = s;
  }
}

// block partials of sum (x - shift)^p, p = 1 or 2, in a fixed order
__global__ void k_moment(int64_t n, const double* __restrict__ x, double shift, int p, double* __restrict__ out) {
  __shared__ double sh[256];
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double d = x[i] - shift;
    s += p == 1 ? d : d * d;
  }
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[blockIdx.x] = sh[0];
}

}  // namespace
}  // namespace bc

mge_status betweenness_run(Ctx* ctx, cudaStream_t st, int64_t n, const int64_t* rp, const int32_t* col, double* cb,
                           double* vbc_out) {
  using namespace bc;
  if (n < 1 || n > INT32_MAX - 2) { set_error(ctx, "betweenness: need 1 <= n < 2^31"); return MGE_EINVAL; }
  DevBuf<int> bad;
  MGE_TRY(bad.scratch(ctx, 1, st));
  MGE_CUDA(ctx, cudaMemsetAsync(bad.p, 0, sizeof(int), st));
  const unsigned gchk = (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 4 * ctx->num_sms));
  k_check_csr<<<gchk, 256, 0, st>>>(n, rp, col, bad.p);
  MGE_LAUNCHED(ctx, 1);
  int hbad = 0;
  MGE_CUDA(ctx, cudaMemcpyAsync(&hbad, bad.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  MGE_CUDA(ctx, cudaStreamSynchronize(st));
  if (hbad) { set_error(ctx, "betweenness: malformed CSR"); return MGE_EINVAL; }
  // one CTA per source, at most two per SM (the per-CTA workspace is 36 n bytes)
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(n, 2 * ctx->num_sms));
  Work wk{};
  DevBuf<int32_t> dist, order, lvl;
  DevBuf<double> sigma, delta, part;
  MGE_TRY(dist.scratch(ctx, (size_t)grid * n, st));
  MGE_TRY(order.scratch(ctx, (size_t)grid * n, st));
  MGE_TRY(lvl.scratch(ctx, (size_t)grid * (n + 2), st));
  MGE_TRY(sigma.scratch(ctx, (size_t)grid * n, st));
  MGE_TRY(delta.scratch(ctx, (size_t)grid * n, st));
  MGE_TRY(part.scratch(ctx, (size_t)grid * n, st));
  wk.dist = dist.p; wk.order = order.p; wk.lvl = lvl.p; wk.sigma = sigma.p; wk.delta = delta.p; wk.part = part.p;
  k_brandes<<<grid, kThreads, 0, st>>>(n, rp, col, wk);
  const unsigned gr = (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 4 * ctx->num_sms));
  k_reduce_parts<<<gr, 256, 0, st>>>(n, grid, part.p, cb);
  MGE_LAUNCHED(ctx, 2);
  if (vbc_out) {
    // population variance: the mean first, then the mean squared deviation (fixed orders)
    const unsigned gm = (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 256));
    DevBuf<double> mom;
    MGE_TRY(mom.scratch(ctx, gm, st));
    std::vector<double> h(gm);
    k_moment<<<gm, 256, 0, st>>>(n, cb, 0.0, 1, mom.p);
    MGE_LAUNCHED(ctx, 1);
    MGE_CUDA(ctx, cudaMemcpyAsync(h.data(), mom.p, gm * sizeof(double), cudaMemcpyDeviceToHost, st));
    MGE_CUDA(ctx, cudaStreamSynchronize(st));
    double s = 0.0;
    for (double v : h) s += v;
    const double mean = s / (double)n;
    k_moment<<<gm, 256, 0, st>>>(n, cb, mean, 2, mom.p);
    MGE_LAUNCHED(ctx, 1);
    MGE_CUDA(ctx, cudaMemcpyAsync(h.data(), mom.p, gm * sizeof(double), cudaMemcpyDeviceToHost, st));
    MGE_CUDA(ctx, cudaStreamSynchronize(st));
    double q = 0.0;
    for (double v : h) q += v;
    *vbc_out = q / (double)n;
  }
  MGE_CUDA(ctx, cudaGetLastError());
  MGE_CUDA(ctx, cudaStreamSynchronize(st));
  return MGE_OK;
}

}  // namespace mge
