// Operator build of Sec. 3.1 and Sec. 4: two-hop sets, Q (Eq. 5), eps (Sec. 4.2), mu (Eq. 9),
// A = L - mu Q + eps I (Eq. 6), Gershgorin radii and B (Sec. 4.3).  All on the device.
#include "mge_internal.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>

namespace mge {

namespace {

constexpr int kWarpCap = 1024;          // candidates a warp sorts in shared memory
constexpr int kWarpsPerBlock = 8;

enum : unsigned {
  ERR_RANGE = 1u, ERR_ORDER = 2u, ERR_DIAG = 4u, ERR_WEIGHT = 8u, ERR_PTR = 16u,
  ERR_ASYM = 32u, ERR_ISOLATED = 64u, ERR_LOOP = 128u
};

// ---------------------------------------------------------------------------------------
// input validation: canonical symmetric CSR
// ---------------------------------------------------------------------------------------
__global__ void k_validate(int64_t n, int64_t nnz, const int64_t* __restrict__ rp,
                           const int32_t* __restrict__ col, const double* __restrict__ w, unsigned* err) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  int64_t s = rp[i], e = rp[i + 1];
  unsigned f = 0;
  if (e < s || s < 0 || e > nnz) { atomicOr(err, (unsigned)ERR_PTR); return; }
  int32_t prev = -1;
  for (int64_t p = s; p < e; ++p) {
    int32_t c = col[p];
    double x = w[p];
    if (c < 0 || c >= n) f |= ERR_RANGE;
    if (c <= prev) f |= ERR_ORDER;
    if (c == i) f |= ERR_DIAG;
    if (!(x > 0.0) || !isfinite(x)) f |= ERR_WEIGHT;
    prev = c;
  }
  if (f) atomicOr(err, f);
}

// W_ij must equal W_ji bitwise: binary search i in row j
__global__ void k_symcheck(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                           const double* __restrict__ w, unsigned* err) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
    int32_t j = col[p];
    int64_t lo = rp[j], hi = rp[j + 1];
    while (lo < hi) {
      int64_t mid = (lo + hi) >> 1;
      if (col[mid] < i) lo = mid + 1; else hi = mid;
    }
    if (lo >= rp[j + 1] || col[lo] != i || w[lo] != w[p]) { atomicOr(err, (unsigned)ERR_ASYM); return; }
  }
}

// ---------------------------------------------------------------------------------------
// exclusive scan of int64 counts (three passes; deterministic)
// ---------------------------------------------------------------------------------------
constexpr int kScanBlock = 1024;

__global__ void k_scan_partial(const int64_t* __restrict__ in, int64_t n, int64_t* __restrict__ part) {
  __shared__ int64_t sh[32];
  int64_t base = (int64_t)blockIdx.x * kScanBlock;
  int64_t v = 0;
  int64_t idx = base + threadIdx.x;
  if (idx < n) v = in[idx];
  for (int o = 16; o; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    v = sh[threadIdx.x];
    for (int o = 16; o; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) part[blockIdx.x] = v;
  }
}

__device__ __forceinline__ int64_t block_excl_scan(int64_t v, int64_t* sh, int64_t* total) {
  // blockDim.x == 1024
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int64_t x = v;
  for (int o = 1; o < 32; o <<= 1) {
    int64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sh[wid] = x;
  __syncthreads();
  if (wid == 0) {
    int64_t s = sh[lane];
    for (int o = 1; o < 32; o <<= 1) {
      int64_t y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    sh[lane] = s;
  }
  __syncthreads();
  int64_t incl = x + (wid > 0 ? sh[wid - 1] : 0);
  *total = sh[31];
  __syncthreads();
  return incl - v;
}

__global__ void k_scan_top(int64_t* part, int64_t nb) {
  __shared__ int64_t sh[32];
  int64_t carry = 0;
  for (int64_t base = 0; base < nb; base += kScanBlock) {
    int64_t idx = base + threadIdx.x;
    int64_t v = idx < nb ? part[idx] : 0;
    int64_t tot;
    int64_t ex = block_excl_scan(v, sh, &tot);
    if (idx < nb) part[idx] = ex + carry;
    carry += tot;
  }
}

__global__ void k_scan_final(const int64_t* __restrict__ in, int64_t n, const int64_t* __restrict__ part,
                             int64_t* __restrict__ out) {
  __shared__ int64_t sh[32];
  int64_t base = (int64_t)blockIdx.x * kScanBlock;
  int64_t idx = base + threadIdx.x;
  int64_t v = idx < n ? in[idx] : 0;
  int64_t tot;
  int64_t ex = block_excl_scan(v, sh, &tot);
  if (idx < n) out[idx] = ex + part[blockIdx.x];
  if (idx == n - 1) out[n] = ex + part[blockIdx.x] + v;
}

// out[0..n] = exclusive scan of in[0..n-1], out[n] = total
mge_status exclusive_scan(Ctx* ctx, cudaStream_t st, const int64_t* in, int64_t n, int64_t* out) {
  if (n == 0) {
    MGE_CUDA(ctx, cudaMemsetAsync(out, 0, sizeof(int64_t), st));
    return MGE_OK;
  }
  int64_t nb = (n + kScanBlock - 1) / kScanBlock;
  DevBuf<int64_t> part;
  MGE_TRY(part.scratch(ctx, nb, st));
  k_scan_partial<<<(unsigned)nb, kScanBlock, 0, st>>>(in, n, part.p);
  k_scan_top<<<1, kScanBlock, 0, st>>>(part.p, nb);
  k_scan_final<<<(unsigned)nb, kScanBlock, 0, st>>>(in, n, part.p, out);
  MGE_LAUNCHED(ctx, 3);
  MGE_CUDA(ctx, cudaGetLastError());
  return MGE_OK;
}

// ---------------------------------------------------------------------------------------
// two-hop sets (Sec. 4.1.1): T_i = (union_{m in N(i)} N(m)) \ ({i} u N(i))
// ---------------------------------------------------------------------------------------
__global__ void k_cand_count(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                             int64_t* __restrict__ cnt, int32_t* __restrict__ big_list, int* big_count) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  int64_t c = 0;
  for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
    int32_t m = col[p];
    c += rp[m + 1] - rp[m];
  }
  cnt[i] = c;
  if (c > kWarpCap) {
    int slot = atomicAdd(big_count, 1);
    big_list[slot] = (int32_t)i;
  }
}

__device__ __forceinline__ bool in_sorted(const int32_t* __restrict__ a, int64_t lo, int64_t hi, int32_t x) {
  while (lo < hi) {
    int64_t mid = (lo + hi) >> 1;
    int32_t v = a[mid];
    if (v == x) return true;
    if (v < x) lo = mid + 1; else hi = mid;
  }
  return false;
}

// one warp per row whose candidate count fits kWarpCap: gather, bitonic sort, unique, filter
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
k_twohop_warp(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
              const int64_t* __restrict__ cnt, const int64_t* __restrict__ U,
              int32_t* __restrict__ tlist, int32_t* __restrict__ T) {
  __shared__ int32_t buf[kWarpsPerBlock][kWarpCap];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int32_t* b = buf[wid];
  for (int64_t i = (int64_t)blockIdx.x * kWarpsPerBlock + wid; i < n;
       i += (int64_t)gridDim.x * kWarpsPerBlock) {
    int64_t c = cnt[i];
    if (c > kWarpCap) continue;  // handled by the bitmap kernel
    // gather candidates: walk N(i), each neighbour's list split over lanes
    int pos = 0;
    for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
      int32_t m = col[p];
      int64_t s = rp[m], d = rp[m + 1] - s;
      for (int64_t q = lane; q < d; q += 32) b[pos + q] = col[s + q];
      pos += (int)d;
    }
    int len = 1;
    while (len < pos) len <<= 1;
    for (int q = pos + lane; q < len; q += 32) b[q] = 0x7fffffff;
    __syncwarp();
    // bitonic sort of b[0..len)
    for (int k = 2; k <= len; k <<= 1) {
      for (int j = k >> 1; j > 0; j >>= 1) {
        for (int t = lane; t < len; t += 32) {
          int u = t ^ j;
          if (u > t) {
            int32_t x = b[t], y = b[u];
            bool up = (t & k) == 0;
            if ((x > y) == up) { b[t] = y; b[u] = x; }
          }
        }
        __syncwarp();
      }
    }
    // unique + filter, stream-compacted in ascending order
    int64_t out = U[i];
    int total = 0;
    const int64_t rs = rp[i], re = rp[i + 1];
    for (int base = 0; base < pos; base += 32) {
      int t = base + lane;
      bool keep = false;
      int32_t x = 0;
      if (t < pos) {
        x = b[t];
        keep = (t == 0 || b[t - 1] != x) && x != (int32_t)i && !in_sorted(col, rs, re, x);
      }
      unsigned bal = __ballot_sync(0xffffffffu, keep);
      if (keep) tlist[out + total + __popc(bal & ((1u << lane) - 1))] = x;
      total += __popc(bal);
    }
    if (lane == 0) T[i] = total;
    __syncwarp();
  }
}

// one CTA per large row: a bitmap of n bits in global scratch marks the candidates
__global__ void k_twohop_big(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                             const int32_t* __restrict__ big_list, int nbig, const int64_t* __restrict__ U,
                             unsigned* __restrict__ bitmaps, int32_t* __restrict__ tlist,
                             int32_t* __restrict__ T) {
  __shared__ int32_t warp_tot[32];
  __shared__ int64_t carry;
  const int64_t words = (n + 31) / 32;
  unsigned* bm = bitmaps + (size_t)blockIdx.x * words;
  for (int r = blockIdx.x; r < nbig; r += gridDim.x) {
    const int32_t i = big_list[r];
    for (int64_t q = threadIdx.x; q < words; q += blockDim.x) bm[q] = 0u;
    __syncthreads();
    for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
      int32_t m = col[p];
      for (int64_t q = rp[m] + threadIdx.x; q < rp[m + 1]; q += blockDim.x) {
        int32_t x = col[q];
        atomicOr(&bm[x >> 5], 1u << (x & 31));
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) atomicAnd(&bm[i >> 5], ~(1u << (i & 31)));
    for (int64_t p = rp[i] + threadIdx.x; p < rp[i + 1]; p += blockDim.x) {
      int32_t x = col[p];
      atomicAnd(&bm[x >> 5], ~(1u << (x & 31)));
    }
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    // ordered extraction: chunks of blockDim.x words
    for (int64_t base = 0; base < words; base += blockDim.x) {
      int64_t q = base + threadIdx.x;
      unsigned v = q < words ? bm[q] : 0u;
      int c = __popc(v);
      // block exclusive scan of c
      int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
      int x = c;
      for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
      }
      if (lane == 31) warp_tot[wid] = x;
      __syncthreads();
      if (wid == 0) {
        int s = lane < (int)(blockDim.x >> 5) ? warp_tot[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
          int y = __shfl_up_sync(0xffffffffu, s, o);
          if (lane >= o) s += y;
        }
        warp_tot[lane] = s;
      }
      __syncthreads();
      int64_t off = carry + (x - c) + (wid > 0 ? warp_tot[wid - 1] : 0);
      int64_t dst = U[i] + off;
      while (v) {
        int bpos = __ffs(v) - 1;
        tlist[dst++] = (int32_t)(q * 32 + bpos);
        v &= v - 1;
      }
      __syncthreads();
      if (threadIdx.x == 0) carry += warp_tot[(blockDim.x >> 5) - 1];
      __syncthreads();
    }
    if (threadIdx.x == 0) T[i] = (int32_t)carry;
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------------------
// Q = sum_i Theta_i (Eq. 5, Laplacian reading): Q_ij = -(1/T_i + 1/T_j) for j in T_i,
// Q_ii = -sum_{j != i} Q_ij.  Also the Eq. 9 denominators Q_ii - sum_{j != i} Q_ij.
// ---------------------------------------------------------------------------------------
__global__ void k_counts(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ T,
                         int64_t* __restrict__ qcnt, int64_t* __restrict__ acnt) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  qcnt[i] = 1 + (int64_t)T[i];
  acnt[i] = 1 + (rp[i + 1] - rp[i]) + (int64_t)T[i];
}

__device__ __forceinline__ void atomic_max_nonneg(double* addr, double v) {
  // non-negative doubles order like their bit patterns
  atomicMax(reinterpret_cast<unsigned long long*>(addr), (unsigned long long)__double_as_longlong(v));
}

__global__ void k_fill_q(int64_t n, const int32_t* __restrict__ T, const int64_t* __restrict__ U,
                         const int32_t* __restrict__ tlist, const int64_t* __restrict__ qp,
                         int32_t* __restrict__ qc, double* __restrict__ qv, float* __restrict__ qv32,
                         double* __restrict__ dinv, float* __restrict__ dinv32, double* den_max,
                         double* norm_max, double* beta_max) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int Ti = T[i];
  const double inv_i = Ti > 0 ? 1.0 / (double)Ti : 0.0;
  const int32_t* tl = tlist + U[i];
  int64_t o = qp[i];
  double diag = 0.0, offsum = 0.0;
  int64_t dpos = -1;
  for (int k = 0; k < Ti; ++k) {
    int32_t j = tl[k];
    if (dpos < 0 && j > i) { dpos = o++; }
    double v = -(inv_i + 1.0 / (double)T[j]);
    qc[o] = j; qv[o] = v; qv32[o] = (float)v;
    offsum += v;
    ++o;
  }
  if (dpos < 0) dpos = o;
  diag = 0.0 - offsum;
  qc[dpos] = (int32_t)i; qv[dpos] = diag; qv32[dpos] = (float)diag;
  double den = diag - offsum;             // Eq. 9 denominator, literally
  atomic_max_nonneg(den_max, den > 0 ? den : 0.0);
  atomic_max_nonneg(norm_max, diag - offsum);
  double d = diag > 0 ? 1.0 / diag : 1.0;
  dinv[i] = d; dinv32[i] = (float)d;
  // Gershgorin bound of the spectrum of D^-1 Q (the polynomial preconditioner's interval)
  if (diag > 0) atomic_max_nonneg(beta_max, (diag - offsum) * d);
}

// ---------------------------------------------------------------------------------------
// connected components of (V, T) by lock-free union-find (bounded loops)
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ int32_t uf_find(int32_t* parent, int32_t x) {
  for (int it = 0; it < (1 << 26); ++it) {
    int32_t p = parent[x];
    if (p == x) return x;
    int32_t g = parent[p];
    if (g != p) atomicCAS(&parent[x], p, g);   // path halving
    x = g;
  }
  return x;
}

__global__ void k_cc_init(int64_t n, int32_t* parent) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) parent[i] = (int32_t)i;
}

__global__ void k_cc_union(int64_t n, const int32_t* __restrict__ T, const int64_t* __restrict__ U,
                           const int32_t* __restrict__ tlist, int32_t* parent, unsigned* err) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int32_t* tl = tlist + U[i];
  for (int k = 0; k < T[i]; ++k) {
    int32_t j = tl[k];
    if (j < i) continue;
    bool done = false;
    for (int it = 0; it < (1 << 20) && !done; ++it) {
      int32_t a = uf_find(parent, (int32_t)i), b = uf_find(parent, j);
      if (a == b) { done = true; break; }
      if (a < b) { int32_t t = a; a = b; b = t; }   // hook the larger root under the smaller
      if (atomicCAS(&parent[a], a, b) == a) done = true;
    }
    if (!done) atomicOr(err, (unsigned)ERR_LOOP);
  }
}

__global__ void k_cc_count(int64_t n, int32_t* parent, int* ncomp) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (parent[i] == (int32_t)i) atomicAdd(ncomp, 1);
}

// ---------------------------------------------------------------------------------------
// A = L - mu Q + eps I on the structure diag + E + T (ascending columns); radii r_i
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ int64_t count_less(const int32_t* __restrict__ a, int64_t len, int32_t x) {
  int64_t lo = 0, hi = len;
  while (lo < hi) {
    int64_t mid = (lo + hi) >> 1;
    if (a[mid] < x) lo = mid + 1; else hi = mid;
  }
  return lo;
}

__global__ void k_fill_a(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                         const double* __restrict__ w, const int32_t* __restrict__ T,
                         const int64_t* __restrict__ U, const int32_t* __restrict__ tlist,
                         const int64_t* __restrict__ qp, const double* __restrict__ qv,
                         const int32_t* __restrict__ qc, double mu, double eps,
                         const int64_t* __restrict__ ap, int32_t* __restrict__ ac, double* __restrict__ av,
                         double* __restrict__ r_out, double* __restrict__ logr, unsigned* err) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t s = rp[i], deg = rp[i + 1] - s;
  const int Ti = T[i];
  const double inv_i = Ti > 0 ? 1.0 / (double)Ti : 0.0;
  const int32_t* tl = tlist + U[i];
  // Q_ii from Q's row
  double qii = 0.0;
  for (int64_t p = qp[i]; p < qp[i + 1]; ++p)
    if (qc[p] == (int32_t)i) { qii = qv[p]; break; }
  double dii = 0.0;
  for (int64_t p = 0; p < deg; ++p) dii += w[s + p];
  // merge three ascending lists into A's row
  int64_t o = ap[i];
  int64_t pe = 0, pt = 0;
  bool diag_done = false;
  for (int64_t k = 0; k < deg + Ti + 1; ++k) {
    int32_t ce = pe < deg ? col[s + pe] : 0x7fffffff;
    int32_t ct = pt < Ti ? tl[pt] : 0x7fffffff;
    int32_t cd = diag_done ? 0x7fffffff : (int32_t)i;
    if (cd < ce && cd < ct) {
      ac[o] = (int32_t)i; av[o] = dii - mu * qii + eps; diag_done = true;
    } else if (ce < ct) {
      ac[o] = ce; av[o] = -w[s + pe]; ++pe;
    } else {
      ac[o] = ct; av[o] = mu * (inv_i + 1.0 / (double)T[ct]); ++pt;   // -mu * Q_ij
    }
    ++o;
  }
  double r = 0.0;
  for (int64_t p = ap[i]; p < ap[i + 1]; ++p)
    if (ac[p] != (int32_t)i) r += fabs(av[p]);
  r_out[i] = r;
  if (!(r > 0.0)) { atomicOr(err, (unsigned)ERR_ISOLATED); logr[i] = 0.0; }
  else logr[i] = log(r);
}

// deterministic sum: per-block partials in fixed order, then one block
__global__ void k_sum_partial(const double* __restrict__ x, int64_t n, double* __restrict__ part) {
  __shared__ double sh[32];
  double v = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    v += x[i];
  for (int o = 16; o; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    v = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
    for (int o = 16; o; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) part[blockIdx.x] = v;
  }
}

__global__ void k_sum_final(const double* __restrict__ part, int np, double* out) {
  __shared__ double sh[32];
  double v = 0.0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) v += part[i];
  for (int o = 16; o; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    v = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
    for (int o = 16; o; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) *out = v;
  }
}

// b_i = r_i / exp(mean log r); Jacobi preconditioner 1/A_ii; ||A||_G = max(A_ii + r_i)
__global__ void k_finish_a(int64_t n, const int64_t* __restrict__ ap, const int32_t* __restrict__ ac,
                           const double* __restrict__ av, const double* __restrict__ r,
                           const double* __restrict__ sumlog, double* __restrict__ b,
                           float* __restrict__ b32, double* __restrict__ dinv, float* __restrict__ dinv32,
                           float* __restrict__ av32, double* norm_max, double* bmax, double* beta_max) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  double g = exp(*sumlog / (double)n);
  double bi = r[i] / g;
  b[i] = bi; b32[i] = (float)bi;
  double aii = 0.0;
  for (int64_t p = ap[i]; p < ap[i + 1]; ++p) {
    av32[p] = (float)av[p];
    if (ac[p] == (int32_t)i) aii = av[p];
  }
  double d = aii > 0 ? 1.0 / aii : 1.0;
  dinv[i] = d; dinv32[i] = (float)d;
  atomic_max_nonneg(norm_max, fmax(aii + r[i], 0.0));
  atomic_max_nonneg(bmax, bi);
  // Gershgorin bound of the spectrum of D^-1 A (the polynomial preconditioner's interval)
  if (aii > 0) atomic_max_nonneg(beta_max, (aii + r[i]) * d);
}

// L + eps I for the preconditioner: values -w_ij (difference form, shift eps), its diagonal
// scaling 1 / (d_i + eps) and the Gershgorin bound of the scaled spectrum
__global__ void k_fill_proxy(int64_t n, const int64_t* __restrict__ rp, const double* __restrict__ w,
                             double eps, double* __restrict__ lv, float* __restrict__ lv32,
                             double* __restrict__ ldinv, float* __restrict__ ldinv32, double* beta_max) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  double deg = 0.0;
  for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
    const double v = w[p];
    deg += v;
    lv[p] = -v;
    lv32[p] = (float)(-v);
  }
  const double diag = deg + eps;
  const double d = diag > 0 ? 1.0 / diag : 1.0;
  ldinv[i] = d; ldinv32[i] = (float)d;
  if (diag > 0) atomic_max_nonneg(beta_max, (diag + deg) * d);
}

inline unsigned grid_for(int64_t n, int block) { return (unsigned)((n + block - 1) / block); }

// ---------------------------------------------------------------------------------------
// sliced copy of a CSR operator (layout in mge_internal.cuh)
// ---------------------------------------------------------------------------------------
// One CTA per tile: the sorted position of each row (longest first, ties by row), and the
// padded slot count of each slice
__global__ void __launch_bounds__(kSliceTileRows) k_slice_rank(int64_t n, const int64_t* __restrict__ rp,
                                                               uint8_t* __restrict__ perm, int64_t* __restrict__ cnt,
                                                               unsigned long long* __restrict__ max_tile) {
  __shared__ int64_t len[kSliceTileRows];
  __shared__ int64_t sorted_len[kSliceTileRows];
  __shared__ unsigned long long tile_slots;
  const int64_t t = blockIdx.x;
  const int r = threadIdx.x;
  const int64_t row = t * kSliceTileRows + r;
  const int64_t l = row < n ? rp[row + 1] - rp[row] : -1;
  len[r] = l;
  if (r == 0) tile_slots = 0;
  __syncthreads();
  int rank = 0;
  for (int q = 0; q < kSliceTileRows; ++q) {
    const int64_t lq = len[q];
    rank += (lq > l) || (lq == l && q < r);
  }
  perm[t * kSliceTileRows + rank] = row < n ? (uint8_t)r : (uint8_t)0xFF;
  sorted_len[rank] = l;
  __syncthreads();
  if (r < kSlicesPerTile) {
    const int64_t m = sorted_len[r * kSliceRows] > 0 ? sorted_len[r * kSliceRows] : 0;
    const int64_t c = (int64_t)kSliceRows * ((m + 3) & ~(int64_t)3);
    cnt[t * kSlicesPerTile + r] = c;
    atomicAdd(&tile_slots, (unsigned long long)c);
  }
  __syncthreads();
  if (r == 0) atomicMax(max_tile, tile_slots);
}

// One thread per sorted position: its row's entries and padding, in slot order
__global__ void k_slice_fill(int64_t ntiles, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                             const double* __restrict__ val, const float* __restrict__ val32,
                             const uint8_t* __restrict__ perm, const int64_t* __restrict__ slp,
                             int32_t* __restrict__ scol, double* __restrict__ sval, float* __restrict__ sval32) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= ntiles * kSliceTileRows) return;
  const int64_t t = p / kSliceTileRows, s = p / kSliceRows;
  const int q = (int)(p % kSliceRows);
  const int64_t base = slp[s];
  const int64_t plen = (slp[s + 1] - base) / kSliceRows;
  if (plen == 0) return;
  const int lr = perm[p];
  // the slice's first row is its longest, so it exists whenever the slice has slots
  const int32_t pad = (int32_t)(t * kSliceTileRows + perm[s * kSliceRows]);
  int64_t b = 0, len = 0;
  if (lr != 0xFF) {
    b = rp[t * kSliceTileRows + lr];
    len = rp[t * kSliceTileRows + lr + 1] - b;
  }
  for (int64_t k = 0; k < plen; ++k) {
    const int64_t d = base + (k >> 2) * (4 * kSliceRows) + q * 4 + (k & 3);
    const bool in = k < len;
    scol[d] = in ? col[b + k] : pad;
    sval[d] = in ? val[b + k] : 0.0;
    sval32[d] = in ? val32[b + k] : 0.0f;
  }
}

// Builds the sliced copy of (rp, col, val, val32); leaves `out` unbuilt when the padding
// would more than double the entries (a few very long rows among short ones)
mge_status build_sliced(Ctx* ctx, cudaStream_t st, int64_t n, const int64_t* rp, const int32_t* col,
                        const double* val, const float* val32, int64_t nnz, Sliced* out) {
  const int64_t ntiles = (n + kSliceTileRows - 1) / kSliceTileRows;
  const int64_t ns = ntiles * kSlicesPerTile;
  DevBuf<int64_t> slp, cnt;
  DevBuf<uint8_t> perm;
  DevBuf<unsigned long long> mx;
  MGE_TRY(slp.alloc(ctx, ns + 4));
  MGE_TRY(perm.alloc(ctx, ntiles * kSliceTileRows));
  MGE_TRY(cnt.scratch(ctx, ns, st));
  MGE_TRY(mx.scratch(ctx, 1, st));
  MGE_CUDA(ctx, cudaMemsetAsync(mx.p, 0, sizeof(unsigned long long), st));
  k_slice_rank<<<(unsigned)ntiles, kSliceTileRows, 0, st>>>(n, rp, perm.p, cnt.p, mx.p);
  MGE_LAUNCHED(ctx, 1);
  MGE_CUDA(ctx, cudaGetLastError());
  MGE_TRY(exclusive_scan(ctx, st, cnt.p, ns, slp.p));     // synchronises the stream
  int64_t slots = 0;
  unsigned long long h_mx = 0;
  MGE_CUDA(ctx, cudaMemcpyAsync(&slots, slp.p + ns, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  MGE_CUDA(ctx, cudaMemcpyAsync(&h_mx, mx.p, sizeof(h_mx), cudaMemcpyDeviceToHost, st));
  MGE_CUDA(ctx, cudaStreamSynchronize(st));
  if (slots > 2 * nnz + 4 * (int64_t)kSliceRows * ns) return MGE_OK;
  const int64_t tail[3] = {slots, slots, slots};
  MGE_CUDA(ctx, cudaMemcpyAsync(slp.p + ns + 1, tail, sizeof(tail), cudaMemcpyHostToDevice, st));
  MGE_TRY(out->col.alloc(ctx, slots));
  MGE_TRY(out->val.alloc(ctx, slots));
  MGE_TRY(out->val32.alloc(ctx, slots));
  if (slots > 0) {
    k_slice_fill<<<grid_for(ntiles * kSliceTileRows, 256), 256, 0, st>>>(ntiles, rp, col, val, val32, perm.p, slp.p,
                                                                          out->col.p, out->val.p, out->val32.p);
    MGE_LAUNCHED(ctx, 1);
  }
  MGE_CUDA(ctx, cudaGetLastError());
  MGE_CUDA(ctx, cudaStreamSynchronize(st));   // `tail` is a host array on this frame
  out->ntiles = ntiles;
  out->slots = slots;
  out->max_tile_slots = (int64_t)h_mx;
  out->slp.swap(slp);
  out->perm.swap(perm);
  return MGE_OK;
}

}  // namespace

// ---------------------------------------------------------------------------------------
// host driver
// ---------------------------------------------------------------------------------------
mge_status scan_exclusive(Ctx* ctx, cudaStream_t st, const int64_t* in, int64_t n, int64_t* out) {
  return exclusive_scan(ctx, st, in, n, out);
}

mge_status build_phase1(Ctx* ctx, cudaStream_t st, int64_t n, const int64_t* rp_in, const int32_t* col_in,
                        const double* w_in, int on_device, const mge_ops_opts* opts, Ops* ops, BuildState* bs) {
  NvtxRange range("mge.build.two_hop_and_Q");
  bs->ctx = ctx;
  bs->st = st;
  bs->n = n;
  if (n < 1) { set_error(ctx, "n must be >= 1"); return MGE_EINVAL; }
  // the handle's arrays come from the context's pool, ordered on this stream
  PersistentPoolScope pool_scope(st);
  if (!rp_in || !col_in || !w_in) { set_error(ctx, "null CSR pointer"); return MGE_EINVAL; }
  mge_ops_opts& o = bs->o;
  o = mge_ops_opts{};
  o.precision = MGE_FP32;
  if (opts) o = *opts;
  if (o.precision < MGE_FP64 || o.precision > MGE_BF16) { set_error(ctx, "bad precision"); return MGE_EINVAL; }
  ops->ctx = ctx;
  ops->n = n;
  MGE_CUDA(ctx, cudaEventCreate(&bs->e0));
  MGE_CUDA(ctx, cudaEventCreate(&bs->e1));
  MGE_CUDA(ctx, cudaEventRecord(bs->e0, st));

  // row pointers first (host check of the ends), then the arrays
  int64_t ends[2];
  if (on_device) {
    MGE_CUDA(ctx, cudaMemcpyAsync(&ends[0], rp_in, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    MGE_CUDA(ctx, cudaMemcpyAsync(&ends[1], rp_in + n, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    MGE_CUDA(ctx, cudaStreamSynchronize(st));
  } else {
    ends[0] = rp_in[0];
    ends[1] = rp_in[n];
  }
  if (ends[0] != 0 || ends[1] < 0 || ends[1] > ((int64_t)1 << 40)) {
    set_error(ctx, "row_ptr[0] must be 0 and row_ptr[n] a valid nnz");
    return MGE_EINVAL;
  }
  const int64_t nnz = ends[1];
  ops->nnz_w = nnz;
  if (n > 0x7ffffffe) { set_error(ctx, "n exceeds int32 column range"); return MGE_EINVAL; }
  MGE_TRY(ops->w_ptr.alloc(ctx, n + 2));
  MGE_TRY(ops->w_col.alloc(ctx, nnz + 4));
  MGE_CUDA(ctx, cudaMemsetAsync(ops->w_ptr.p + n + 1, 0, sizeof(int64_t), st));
  MGE_CUDA(ctx, cudaMemsetAsync(ops->w_col.p + nnz, 0, 4 * sizeof(int32_t), st));
  MGE_TRY(ops->w_val.alloc(ctx, nnz));
  cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  MGE_CUDA(ctx, cudaMemcpyAsync(ops->w_ptr.p, rp_in, (n + 1) * sizeof(int64_t), kind, st));
  if (nnz) {
    MGE_CUDA(ctx, cudaMemcpyAsync(ops->w_col.p, col_in, nnz * sizeof(int32_t), kind, st));
    MGE_CUDA(ctx, cudaMemcpyAsync(ops->w_val.p, w_in, nnz * sizeof(double), kind, st));
  }
  const int64_t* rp = ops->w_ptr.p;
  const int32_t* col = ops->w_col.p;
  const double* w = ops->w_val.p;

  // small device scalars: [err, big_count, ncomp] and doubles [den_max, normq, norma, bmax, sumlog]
  DevBuf<unsigned>& d_err = bs->d_err;  MGE_TRY(d_err.scratch(ctx, 4, st));
  DevBuf<double>& d_sc = bs->d_sc;      MGE_TRY(d_sc.scratch(ctx, 8, st));
  MGE_CUDA(ctx, cudaMemsetAsync(d_err.p, 0, 4 * sizeof(unsigned), st));
  MGE_CUDA(ctx, cudaMemsetAsync(d_sc.p, 0, 8 * sizeof(double), st));
  unsigned* err = d_err.p;
  int* big_count = reinterpret_cast<int*>(d_err.p + 1);
  int* ncomp = reinterpret_cast<int*>(d_err.p + 2);
  double* den_max = d_sc.p + 0;
  double* normq = d_sc.p + 1;
  double* norma = d_sc.p + 2;
  double* bmax = d_sc.p + 3;
  double* sumlog = d_sc.p + 4;
  double* beta_q = d_sc.p + 5;
  double* beta_a = d_sc.p + 6;

  const int B = 256;
  // structure first; the symmetry check indexes rows by column values, so it runs only on a
  // CSR that passed
  k_validate<<<grid_for(n, B), B, 0, st>>>(n, nnz, rp, col, w, err);
  MGE_LAUNCHED(ctx, 1);
  MGE_CUDA(ctx, cudaGetLastError());
  unsigned h_err = 0;
  MGE_CUDA(ctx, cudaMemcpyAsync(&h_err, err, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
  MGE_CUDA(ctx, cudaStreamSynchronize(st));
  if (h_err & (ERR_RANGE | ERR_ORDER | ERR_DIAG | ERR_WEIGHT | ERR_PTR)) {
    set_error(ctx, "malformed CSR (flags 0x%x: 1 range, 2 order, 4 diagonal, 8 weight, 16 row_ptr)", h_err);
    return MGE_EINVAL;
  }
  k_symcheck<<<grid_for(n, B), B, 0, st>>>(n, rp, col, w, err);
  MGE_LAUNCHED(ctx, 1);
  MGE_CUDA(ctx, cudaGetLastError());
  MGE_CUDA(ctx, cudaMemcpyAsync(&h_err, err, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
  MGE_CUDA(ctx, cudaStreamSynchronize(st));
  if (h_err & ERR_ASYM) { set_error(ctx, "W is not symmetric"); return MGE_ENOTSYM; }

  // --- node order: everything below runs on W renamed into the locality order ---
  if (!o.keep_order && n > 1) {
    DevBuf<int64_t> rp2;
    DevBuf<int32_t> col2;
    DevBuf<double> w2;
    MGE_TRY(locality_order(ctx, st, n, ops->w_ptr.p, ops->w_col.p, ops->w_val.p, nnz, &ops->order, &ops->rank,
                           &rp2, &col2, &w2));
    ops->w_ptr.swap(rp2);
    ops->w_col.swap(col2);
    ops->w_val.swap(w2);
    rp = ops->w_ptr.p;
    col = ops->w_col.p;
    w = ops->w_val.p;
  }

  // --- two-hop sets ---
  DevBuf<int64_t> cnt;
  DevBuf<int64_t>& U = bs->U;
  DevBuf<int32_t> big_list;
  MGE_TRY(cnt.scratch(ctx, n, st));
  MGE_TRY(U.scratch(ctx, n + 1, st));
  MGE_TRY(big_list.scratch(ctx, n, st));
  k_cand_count<<<grid_for(n, B), B, 0, st>>>(n, rp, col, cnt.p, big_list.p, big_count);
  MGE_LAUNCHED(ctx, 1);
  MGE_TRY(exclusive_scan(ctx, st, cnt.p, n, U.p));
  int64_t total_cand = 0;
  int h_big = 0;
  MGE_CUDA(ctx, cudaMemcpyAsync(&total_cand, U.p + n, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  MGE_CUDA(ctx, cudaMemcpyAsync(&h_big, big_count, sizeof(int), cudaMemcpyDeviceToHost, st));
  MGE_CUDA(ctx, cudaStreamSynchronize(st));
  DevBuf<int32_t>& tlist = bs->tlist;
  MGE_TRY(tlist.scratch(ctx, std::max<int64_t>(total_cand, 1), st));
  MGE_TRY(ops->T.alloc(ctx, n));
  {
    int blocks = std::min<int64_t>(grid_for(n, kWarpsPerBlock), (int64_t)ctx->num_sms * 16);
    k_twohop_warp<<<blocks, kWarpsPerBlock * 32, 0, st>>>(n, rp, col, cnt.p, U.p, tlist.p, ops->T.p);
    MGE_LAUNCHED(ctx, 1);
  }
  if (h_big > 0) {
    int nb = std::min(h_big, 64);
    DevBuf<unsigned> bitmaps;
    MGE_TRY(bitmaps.scratch(ctx, (size_t)nb * ((n + 31) / 32), st));
    k_twohop_big<<<nb, 1024, 0, st>>>(n, rp, col, big_list.p, h_big, U.p, bitmaps.p, tlist.p, ops->T.p);
    MGE_LAUNCHED(ctx, 1);
    MGE_CUDA(ctx, cudaGetLastError());
    MGE_CUDA(ctx, cudaStreamSynchronize(st));
  }
  MGE_CUDA(ctx, cudaGetLastError());

  // --- structures of Q and A ---
  DevBuf<int64_t> qcnt, acnt;
  MGE_TRY(qcnt.scratch(ctx, n, st));
  MGE_TRY(acnt.scratch(ctx, n, st));
  // CSR arrays carry a few zeroed elements past their ends: the LOBPCG SpMM copies row
  // pointers, column indices and values in tiles whose byte counts are rounded up to 16
  MGE_TRY(ops->q_ptr.alloc(ctx, n + 2));
  MGE_TRY(ops->a_ptr.alloc(ctx, n + 2));
  MGE_CUDA(ctx, cudaMemsetAsync(ops->q_ptr.p + n + 1, 0, sizeof(int64_t), st));
  MGE_CUDA(ctx, cudaMemsetAsync(ops->a_ptr.p + n + 1, 0, sizeof(int64_t), st));
  k_counts<<<grid_for(n, B), B, 0, st>>>(n, rp, ops->T.p, qcnt.p, acnt.p);
  MGE_LAUNCHED(ctx, 1);
  MGE_TRY(exclusive_scan(ctx, st, qcnt.p, n, ops->q_ptr.p));
  MGE_TRY(exclusive_scan(ctx, st, acnt.p, n, ops->a_ptr.p));
  MGE_CUDA(ctx, cudaMemcpyAsync(&ops->nnz_q, ops->q_ptr.p + n, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  MGE_CUDA(ctx, cudaMemcpyAsync(&ops->nnz_a, ops->a_ptr.p + n, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  MGE_CUDA(ctx, cudaStreamSynchronize(st));

  // --- Q values, Eq. 9 denominators, preconditioner ---
  MGE_TRY(ops->q_col.alloc(ctx, ops->nnz_q + 4));
  MGE_TRY(ops->q_val.alloc(ctx, ops->nnz_q + 4));
  MGE_TRY(ops->q_val32.alloc(ctx, ops->nnz_q + 4));
  MGE_CUDA(ctx, cudaMemsetAsync(ops->q_col.p + ops->nnz_q, 0, 4 * sizeof(int32_t), st));
  MGE_CUDA(ctx, cudaMemsetAsync(ops->q_val.p + ops->nnz_q, 0, 4 * sizeof(double), st));
  MGE_CUDA(ctx, cudaMemsetAsync(ops->q_val32.p + ops->nnz_q, 0, 4 * sizeof(float), st));
  MGE_TRY(ops->dinv_q.alloc(ctx, n + 4));
  MGE_CUDA(ctx, cudaMemsetAsync(ops->dinv_q.p + n, 0, 4 * sizeof(double), st));
  MGE_TRY(ops->dinv_q32.alloc(ctx, n + 4));
  MGE_CUDA(ctx, cudaMemsetAsync(ops->dinv_q32.p + n, 0, 4 * sizeof(float), st));
  k_fill_q<<<grid_for(n, B), B, 0, st>>>(n, ops->T.p, U.p, tlist.p, ops->q_ptr.p, ops->q_col.p,
                                          ops->q_val.p, ops->q_val32.p, ops->dinv_q.p, ops->dinv_q32.p,
                                          den_max, normq, beta_q);
  MGE_LAUNCHED(ctx, 1);
  MGE_TRY(build_sliced(ctx, st, n, ops->q_ptr.p, ops->q_col.p, ops->q_val.p, ops->q_val32.p, ops->nnz_q,
                       &ops->q_sl));

  // --- components of the two-hop graph (eps = 0 when more than one) ---
  {
    DevBuf<int32_t> parent;
    MGE_TRY(parent.scratch(ctx, n, st));
    k_cc_init<<<grid_for(n, B), B, 0, st>>>(n, parent.p);
    k_cc_union<<<grid_for(n, B), B, 0, st>>>(n, ops->T.p, U.p, tlist.p, parent.p, err);
    k_cc_count<<<grid_for(n, B), B, 0, st>>>(n, parent.p, ncomp);
    MGE_LAUNCHED(ctx, 3);
    MGE_CUDA(ctx, cudaGetLastError());
    int h_ncomp = 0;
    double h_den = 0, h_nq = 0, h_bq = 0;
    MGE_CUDA(ctx, cudaMemcpyAsync(&h_bq, beta_q, sizeof(double), cudaMemcpyDeviceToHost, st));
    MGE_CUDA(ctx, cudaMemcpyAsync(&h_ncomp, ncomp, sizeof(int), cudaMemcpyDeviceToHost, st));
    MGE_CUDA(ctx, cudaMemcpyAsync(&h_den, den_max, sizeof(double), cudaMemcpyDeviceToHost, st));
    MGE_CUDA(ctx, cudaMemcpyAsync(&h_nq, normq, sizeof(double), cudaMemcpyDeviceToHost, st));
    MGE_CUDA(ctx, cudaMemcpyAsync(&h_err, err, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    MGE_CUDA(ctx, cudaStreamSynchronize(st));
    if (h_err & ERR_LOOP) { set_error(ctx, "union-find iteration limit reached"); return MGE_ETIMEOUT; }
    ops->ncomp = h_ncomp;
    ops->norm_q = h_nq > 0 ? h_nq : 1.0;
    ops->beta_q = h_bq > 0 ? h_bq : 2.0;
    bs->h_ncomp = h_ncomp;
    bs->h_den = h_den;
    // --- the eps = lambda_2(Q) solve, prepared for build_eps_single or a batched launch ---
    bs->need_eps = !o.eps_override_set && n >= 2 && h_ncomp == 1;
    if (bs->need_eps) {
      LobOp& qop = bs->qop;
      qop = LobOp{};
      qop.n = n; qop.ptr = ops->q_ptr.p; qop.col = ops->q_col.p;
      qop.val = (o.precision == MGE_FP64) ? (const void*)ops->q_val.p : (const void*)ops->q_val32.p;
      qop.shift = 0.0; qop.b = nullptr;
      qop.dinv = (o.precision == MGE_FP64) ? (const void*)ops->dinv_q.p : (const void*)ops->dinv_q32.p;
      qop.norm = ops->norm_q; qop.bmax = 1.0; qop.deflate = true; qop.beta = ops->beta_q;
      qop.precond_degree = o.eps_precond_degree > 0 ? std::min(o.eps_precond_degree, kMaxPrecondDegree) : default_eps_precond_degree(n);
      qop.nnz = ops->nnz_q;
      qop.rr_fp64 = o.precision == MGE_FP64;
      qop.pc_bf16 = o.precision == MGE_BF16;
      if (qop.pc_bf16) qop.precond_degree = std::min(qop.precond_degree, kBf16MaxPrecondDegree);
      if (ops->q_sl.built()) {
        qop.sl_slp = ops->q_sl.slp.p; qop.sl_perm = ops->q_sl.perm.p; qop.sl_col = ops->q_sl.col.p;
        qop.sl_val = (o.precision == MGE_FP64) ? (const void*)ops->q_sl.val.p : (const void*)ops->q_sl.val32.p;
        qop.sl_max_tile_slots = ops->q_sl.max_tile_slots;
      }
      // default block m = 8 (fewer iterations than m = 4 at about the same SpMM time), m = 4
      // on graphs too small for it
      int guard = o.eps_guard > 0 ? o.eps_guard : (n >= 2 * 8 ? 7 : 3);
      int m = round_block_width(1 + guard);
      if (m > n - 1) m = -1;
      // FP32: eps enters A as a shift, so its relative error passes to the eigenvalues about
      // one to one; at 1e-4 in the relative residual it is below 1e-6 (measured: 7.1e-7 on a
      // 200k-node graph against the exact value; 18 -> 16 and 50 -> 41 iterations at 200k and
      // 2M nodes against 1e-5), inside the 1e-4 accuracy FP32 eigenvalues are held to
      double tol = o.eps_tol > 0 ? o.eps_tol : (o.precision == MGE_FP64 ? 1e-10 : 1e-4);
      int maxit = o.eps_maxiter > 0 ? o.eps_maxiter : 20000;
      if (m < 0) {
        set_error(ctx, "graph too small for the eps solve block (n = %lld)", (long long)n);
        return MGE_EINVAL;
      }
      bs->eps_m = m;
      bs->eps_tol = tol;
      bs->eps_maxiter = maxit;
      bs->eps_precision = (o.precision == MGE_FP64) ? MGE_FP64 : MGE_FP32;
      bs->eps_seed = o.seed ^ 0x9e3779b97f4a7c15ull;
    }
  }
  return MGE_OK;
}

// The single eps solve of a build (phase 2 when the build runs alone).
mge_status build_eps_single(BuildState* bs, Ops* ops, double* eps) {
  NvtxRange range("mge.build.eps_solve");
  LobResult lr;
  mge_status s = lobpcg_solve(bs->ctx, bs->st, bs->qop, bs->eps_precision, 1, bs->eps_m, bs->eps_tol,
                              bs->eps_maxiter, bs->eps_seed, 16, true, nullptr, 0, nullptr, &lr);
  if (s != MGE_OK && s != MGE_ENOTCONVERGED) return s;
  *eps = lr.lambda[0];
  ops->eps_iters = lr.iters;
  ops->eps_resid = lr.eta.empty() ? 0.0 : lr.eta[0];
  return MGE_OK;
}

// Phase 3: mu (Eq. 9), A, the radii and B (Sec. 4.3), the preconditioner's operator.
mge_status build_phase3(BuildState* bs, Ops* ops, double eps) {
  NvtxRange range("mge.build.mu_A_B");
  Ctx* ctx = bs->ctx;
  cudaStream_t st = bs->st;
  const int64_t n = bs->n;
  const mge_ops_opts& o = bs->o;
  PersistentPoolScope pool_scope(st);
  const int64_t* rp = ops->w_ptr.p;
  const int32_t* col = ops->w_col.p;
  const double* w = ops->w_val.p;
  DevBuf<int64_t>& U = bs->U;
  DevBuf<int32_t>& tlist = bs->tlist;
  DevBuf<double>& d_sc = bs->d_sc;
  unsigned* err = bs->d_err.p;
  double* norma = d_sc.p + 2;
  double* bmax = d_sc.p + 3;
  double* sumlog = d_sc.p + 4;
  double* beta_a = d_sc.p + 6;
  cudaEvent_t e0 = bs->e0, e1 = bs->e1;
  unsigned h_err = 0;
  const int B = 256;
  {
    if (o.eps_override_set) eps = o.eps_override;
    ops->degenerate = (!o.eps_override_set && bs->h_ncomp > 1) ? 1 : 0;
    ops->eps = eps;
    // --- mu (Eq. 9) ---
    double mu = 0.0;
    if (o.mu_override_set) mu = o.mu_override;
    else if (eps != 0.0 && bs->h_den > 0) mu = eps / bs->h_den;
    ops->mu = mu;
  }

  // --- A values, radii, B ---
  MGE_TRY(ops->a_col.alloc(ctx, ops->nnz_a + 4));
  MGE_TRY(ops->a_val.alloc(ctx, ops->nnz_a + 4));
  MGE_TRY(ops->a_val32.alloc(ctx, ops->nnz_a + 4));
  MGE_CUDA(ctx, cudaMemsetAsync(ops->a_col.p + ops->nnz_a, 0, 4 * sizeof(int32_t), st));
  MGE_CUDA(ctx, cudaMemsetAsync(ops->a_val.p + ops->nnz_a, 0, 4 * sizeof(double), st));
  MGE_CUDA(ctx, cudaMemsetAsync(ops->a_val32.p + ops->nnz_a, 0, 4 * sizeof(float), st));
  // b carries 4 zeroed elements past n: the LOBPCG Gram copies b in tiles whose byte
  // count is rounded up to a multiple of 16
  MGE_TRY(ops->b.alloc(ctx, n + 4));
  MGE_TRY(ops->b32.alloc(ctx, n + 4));
  MGE_CUDA(ctx, cudaMemsetAsync(ops->b.p + n, 0, 4 * sizeof(double), st));
  MGE_CUDA(ctx, cudaMemsetAsync(ops->b32.p + n, 0, 4 * sizeof(float), st));
  MGE_TRY(ops->dinv_a.alloc(ctx, n + 4));
  MGE_CUDA(ctx, cudaMemsetAsync(ops->dinv_a.p + n, 0, 4 * sizeof(double), st));
  MGE_TRY(ops->dinv_a32.alloc(ctx, n + 4));
  MGE_CUDA(ctx, cudaMemsetAsync(ops->dinv_a32.p + n, 0, 4 * sizeof(float), st));
  DevBuf<double> r, logr;
  MGE_TRY(r.scratch(ctx, n, st));
  MGE_TRY(logr.scratch(ctx, n, st));
  k_fill_a<<<grid_for(n, B), B, 0, st>>>(n, rp, col, w, ops->T.p, U.p, tlist.p, ops->q_ptr.p,
                                          ops->q_val.p, ops->q_col.p, ops->mu, ops->eps, ops->a_ptr.p,
                                          ops->a_col.p, ops->a_val.p, r.p, logr.p, err);
  MGE_LAUNCHED(ctx, 1);
  {
    const int np = 256;
    DevBuf<double> part;
    MGE_TRY(part.scratch(ctx, np, st));
    k_sum_partial<<<np, 256, 0, st>>>(logr.p, n, part.p);
    k_sum_final<<<1, 256, 0, st>>>(part.p, np, sumlog);
    MGE_LAUNCHED(ctx, 2);
    k_finish_a<<<grid_for(n, B), B, 0, st>>>(n, ops->a_ptr.p, ops->a_col.p, ops->a_val.p, r.p, sumlog,
                                              ops->b.p, ops->b32.p, ops->dinv_a.p, ops->dinv_a32.p,
                                              ops->a_val32.p, norma, bmax, beta_a);
    MGE_LAUNCHED(ctx, 1);
    MGE_CUDA(ctx, cudaGetLastError());
    double h_na = 0, h_bm = 0, h_ba = 0;
    MGE_CUDA(ctx, cudaMemcpyAsync(&h_ba, beta_a, sizeof(double), cudaMemcpyDeviceToHost, st));
    MGE_CUDA(ctx, cudaMemcpyAsync(&h_err, err, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    MGE_CUDA(ctx, cudaMemcpyAsync(&h_na, norma, sizeof(double), cudaMemcpyDeviceToHost, st));
    MGE_CUDA(ctx, cudaMemcpyAsync(&h_bm, bmax, sizeof(double), cudaMemcpyDeviceToHost, st));
    MGE_CUDA(ctx, cudaEventRecord(e1, st));
    MGE_CUDA(ctx, cudaStreamSynchronize(st));
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    bs->e0 = bs->e1 = nullptr;
    ops->build_ms = ms;
    ops->norm_a = h_na > 0 ? h_na : 1.0;
    ops->bmax = h_bm > 0 ? h_bm : 1.0;
    ops->beta_a = h_ba > 0 ? h_ba : 2.0;
  }
  {
    const int64_t nnz_w = ops->nnz_w;
    MGE_TRY(ops->l_val.alloc(ctx, nnz_w + 4));
    MGE_TRY(ops->l_val32.alloc(ctx, nnz_w + 4));
    MGE_TRY(ops->l_dinv.alloc(ctx, n + 4));
    MGE_TRY(ops->l_dinv32.alloc(ctx, n + 4));
    MGE_CUDA(ctx, cudaMemsetAsync(ops->l_val.p + nnz_w, 0, 4 * sizeof(double), st));
    MGE_CUDA(ctx, cudaMemsetAsync(ops->l_val32.p + nnz_w, 0, 4 * sizeof(float), st));
    MGE_CUDA(ctx, cudaMemsetAsync(ops->l_dinv.p + n, 0, 4 * sizeof(double), st));
    MGE_CUDA(ctx, cudaMemsetAsync(ops->l_dinv32.p + n, 0, 4 * sizeof(float), st));
    double* beta_l = d_sc.p + 7;
    MGE_CUDA(ctx, cudaMemsetAsync(beta_l, 0, sizeof(double), st));
    k_fill_proxy<<<grid_for(n, B), B, 0, st>>>(n, ops->w_ptr.p, ops->w_val.p, ops->eps, ops->l_val.p,
                                                ops->l_val32.p, ops->l_dinv.p, ops->l_dinv32.p, beta_l);
    MGE_LAUNCHED(ctx, 1);
    double h_bl = 0;
    MGE_CUDA(ctx, cudaMemcpyAsync(&h_bl, beta_l, sizeof(double), cudaMemcpyDeviceToHost, st));
    MGE_CUDA(ctx, cudaStreamSynchronize(st));
    ops->beta_l = h_bl > 0 ? h_bl : 2.0;
    MGE_TRY(build_sliced(ctx, st, n, ops->w_ptr.p, ops->w_col.p, ops->l_val.p, ops->l_val32.p, nnz_w, &ops->l_sl));
  }
  if (h_err & ERR_ISOLATED) {
    set_error(ctx, "isolated node: a Gershgorin radius r_i is zero, so B is singular");
    return MGE_EISOLATED;
  }
  return ops->degenerate ? MGE_EDEGENERATE : MGE_OK;
}

mge_status build_graph_ops_impl(Ctx* ctx, cudaStream_t st, int64_t n, const int64_t* rp_in,
                                const int32_t* col_in, const double* w_in, int on_device,
                                const mge_ops_opts* opts, Ops* ops) {
  BuildState bs;
  MGE_TRY(build_phase1(ctx, st, n, rp_in, col_in, w_in, on_device, opts, ops, &bs));
  double eps = 0.0;
  if (bs.need_eps) MGE_TRY(build_eps_single(&bs, ops, &eps));
  return build_phase3(&bs, ops, eps);
}

}  // namespace mge
