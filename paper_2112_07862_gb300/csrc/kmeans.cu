// k-means clustering of the embedding (Sec. 5.2: the embeddings are clustered with kmeans).
// Lloyd's algorithm from the caller's initial centres, in FP64:
//   assignment  each point goes to the centre of least squared distance, summed over the
//               coordinates in order with every product and sum rounded separately (no
//               fused multiply-add), equal distances to the lower centre index;
//   update      each centre becomes the mean of its points: the sum of each coordinate,
//               accumulated as a compensated double-double (TwoSum) and rounded once, divided
//               by the count; a centre without points stays where it is;
//   stop        after an assignment step (other than the first) that changed nothing, or
//               after max_iters assignment steps.
// The rounded double-double sum is the exactly rounded sum unless the exact value lies within
// about n 2^-106 sum |x| of a rounding boundary, so assignments are a function of the inputs.
//
// Kernels: one thread per point for the assignment (centres in shared memory); the sums in
// tiles of points staged in shared memory, one thread per (centre, coordinate) pair walking
// the tile in point order, block partials combined in block order by one thread per pair.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "mge_internal.cuh"

namespace mge {
namespace km {
namespace {

constexpr int kBlock = 256;

// a += x as a double-double (hi, lo): TwoSum of hi and x, the error into lo
__device__ __forceinline__ void dd_add(double& hi, double& lo, double x) {
  const double s = __dadd_rn(hi, x);
  const double bp = __dsub_rn(s, hi);
  const double e = __dadd_rn(__dsub_rn(hi, __dsub_rn(s, bp)), __dsub_rn(x, bp));
  hi = s;
  lo = __dadd_rn(lo, e);
}

// X column-major [n x K] (X[k * n + i]); centres row-major [C x K]
__global__ void __launch_bounds__(kBlock) k_assign(int64_t n, int K, int C, const double* __restrict__ X,
                                                   const double* __restrict__ centres,
                                                   int32_t* __restrict__ assign,
                                                   unsigned long long* __restrict__ changes) {
  extern __shared__ double sc[];
  for (int t = threadIdx.x; t < C * K; t += blockDim.x) sc[t] = centres[t];
  __syncthreads();
  unsigned long long changed = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double best = 0.0;
    int bc = 0;
    for (int c = 0; c < C; ++c) {
      double s = 0.0;
      for (int k = 0; k < K; ++k) {
        const double t = __dsub_rn(X[(int64_t)k * n + i], sc[c * K + k]);
        s = __dadd_rn(s, __dmul_rn(t, t));
      }
      if (c == 0 || s < best) { best = s; bc = c; }
    }
    changed += assign[i] != bc;
    assign[i] = bc;
  }
  for (int o = 16; o > 0; o >>= 1) changed += __shfl_xor_sync(0xffffffffu, changed, o);
  if ((threadIdx.x & 31) == 0 && changed) atomicAdd(changes, changed);
}

// Block partial sums over tiles of tp points (tiles b, b + gridDim.x, ...): thread j owns the
// pairs (c, k) = (j / K, j % K), j += blockDim.x, and walks each tile in point order.
__global__ void __launch_bounds__(kBlock) k_partial(int64_t n, int K, int C, int tp, const double* __restrict__ X,
                                                    const int32_t* __restrict__ assign,
                                                    double* __restrict__ part, int64_t* __restrict__ pcnt) {
  extern __shared__ double smem[];
  double* sx = smem;                                                  // [K][tp]
  int32_t* sa = reinterpret_cast<int32_t*>(smem + (size_t)K * tp);    // [tp]
  const int pairs = C * K;
  const int per = (pairs + blockDim.x - 1) / blockDim.x;              // pairs per thread (<= 16)
  double hi[16], lo[16];
  int64_t cnt[16];
  for (int u = 0; u < per; ++u) { hi[u] = 0.0; lo[u] = 0.0; cnt[u] = 0; }
  const int64_t ntiles = (n + tp - 1) / tp;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t i0 = tile * tp;
    const int len = (int)(n - i0 < (int64_t)tp ? n - i0 : (int64_t)tp);
    __syncthreads();
    for (int t = threadIdx.x; t < len; t += blockDim.x) sa[t] = assign[i0 + t];
    for (int t = threadIdx.x; t < K * len; t += blockDim.x) {
      const int k = t / len, p = t % len;
      sx[k * tp + p] = X[(int64_t)k * n + i0 + p];
    }
    __syncthreads();
    for (int u = 0; u < per; ++u) {
      const int j = threadIdx.x + u * blockDim.x;
      if (j >= pairs) break;
      const int c = j / K, k = j % K;
      double h = hi[u], l = lo[u];
      int64_t m = cnt[u];
      for (int p = 0; p < len; ++p)
        if (sa[p] == c) { dd_add(h, l, sx[k * tp + p]); ++m; }
      hi[u] = h; lo[u] = l; cnt[u] = m;
    }
  }
  for (int u = 0; u < per; ++u) {
    const int j = threadIdx.x + u * blockDim.x;
    if (j >= pairs) break;
    part[((size_t)blockIdx.x * pairs + j) * 2] = hi[u];
    part[((size_t)blockIdx.x * pairs + j) * 2 + 1] = lo[u];
    if (j % K == 0) pcnt[(size_t)blockIdx.x * C + j / K] = cnt[u];
  }
}

// new centres: block partials combined in block order, rounded once, divided by the count
__global__ void k_finish(int K, int C, int nb, const double* __restrict__ part, const int64_t* __restrict__ pcnt,
                         double* __restrict__ centres) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= C * K) return;
  const int c = j / K;
  double h = 0.0, l = 0.0;
  int64_t m = 0;
  for (int b = 0; b < nb; ++b) {
    dd_add(h, l, part[((size_t)b * C * K + j) * 2]);
    l = __dadd_rn(l, part[((size_t)b * C * K + j) * 2 + 1]);
    m += pcnt[(size_t)b * C + c];
  }
  if (m > 0) centres[j] = __ddiv_rn(__dadd_rn(h, l), (double)m);
}

}  // namespace
}  // namespace km

mge_status kmeans_run(Ctx* ctx, cudaStream_t st, int64_t n, int K, const double* X, int C, double* centres,
                      int max_iters, int32_t* assign, int* iters_out) {
  using namespace km;
  if (n < 1 || K < 1 || K > 64 || C < 1 || C > 1024 || C * K > 4096 || max_iters < 1) {
    set_error(ctx, "kmeans: need n >= 1, 1 <= K <= 64, 1 <= C, C K <= 4096, max_iters >= 1");
    return MGE_EINVAL;
  }
  const int tp = std::max(32, std::min(256, 8192 / K));
  const int64_t ntiles = (n + tp - 1) / tp;
  const int nb = (int)std::max<int64_t>(1, std::min<int64_t>(ntiles, 2 * ctx->num_sms));
  const int pairs = C * K;
  DevBuf<double> part;
  DevBuf<int64_t> pcnt;
  DevBuf<unsigned long long> changes;
  MGE_TRY(part.scratch(ctx, (size_t)nb * pairs * 2, st));
  MGE_TRY(pcnt.scratch(ctx, (size_t)nb * C, st));
  MGE_TRY(changes.scratch(ctx, 1, st));
  MGE_CUDA(ctx, cudaMemsetAsync(assign, 0xff, n * sizeof(int32_t), st));    // -1: no centre yet
  const size_t smem_a = (size_t)C * K * sizeof(double);
  const size_t smem_p = (size_t)K * tp * sizeof(double) + (size_t)tp * sizeof(int32_t);
  if (smem_a > 48 * 1024) MGE_CUDA(ctx, cudaFuncSetAttribute(k_assign, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_a));
  if (smem_p > 48 * 1024) MGE_CUDA(ctx, cudaFuncSetAttribute(k_partial, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_p));
  const unsigned ga = (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + kBlock - 1) / kBlock, 8 * ctx->num_sms));
  int steps = 0;
  for (int t = 0; t < max_iters; ++t) {
    MGE_CUDA(ctx, cudaMemsetAsync(changes.p, 0, sizeof(unsigned long long), st));
    k_assign<<<ga, kBlock, smem_a, st>>>(n, K, C, X, centres, assign, changes.p);
    MGE_LAUNCHED(ctx, 1);
    unsigned long long ch = 0;
    MGE_CUDA(ctx, cudaMemcpyAsync(&ch, changes.p, sizeof(ch), cudaMemcpyDeviceToHost, st));
    MGE_CUDA(ctx, cudaStreamSynchronize(st));
    steps = t + 1;
    if (t > 0 && ch == 0) break;
    k_partial<<<nb, kBlock, smem_p, st>>>(n, K, C, tp, X, assign, part.p, pcnt.p);
    k_finish<<<(pairs + kBlock - 1) / kBlock, kBlock, 0, st>>>(K, C, nb, part.p, pcnt.p, centres);
    MGE_LAUNCHED(ctx, 2);
  }
  MGE_CUDA(ctx, cudaGetLastError());
  MGE_CUDA(ctx, cudaStreamSynchronize(st));
  *iters_out = steps;
  return MGE_OK;
}

}  // namespace mge
