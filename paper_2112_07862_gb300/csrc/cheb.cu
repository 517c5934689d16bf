// Chebyshev steps of the LOBPCG polynomial preconditioner on the sliced copy of an operator
// (Saad, Iterative Methods for Sparse Linear Systems, Alg. 12.1; the preconditioner itself is
// described in lobpcg.cu).  One launch per step:
//
//   y = A x,   z = R - D^-1 (sy y),   d_out = c1 (sd d) + c2 z,   x_out = sy x + d_out
//
// with A in the difference form (A x)_i = shift x_i + sum_j a_ij (x_j - x_i).
//
// The operator's rows are sorted by length inside each 128-row tile and padded per 16-row
// slice (layout in mge_internal.cuh), so that every lane of a slice walks the same number of
// 4-slot chunks, a chunk's indices and values are one 16-byte load each, and no per-entry
// bounds test is left in the inner loop.  Each CTA is a producer warp that streams tiles
// into a ring of shared-memory stages with 1-D bulk copies (TMA: the slice offsets, the row
// order and the chunk indices and values) and eight consumer warps that gather the x rows of
// the column indices from global memory (L2), then read the row's own R, d and D^-1.  The
// stages are kept small: the L1 part of the
// SM's 256 KB holds the gathers in flight, and with most of it given to shared memory the
// gathers queue (measured: 2 x 111 KB of stages per SM made the step 1.7x slower).
#include "lobpcg_common.cuh"

#include <type_traits>

namespace mge {
namespace lob {
namespace {

constexpr int kChebConsumers = kThreads;           // 8 consumer warps
constexpr int kChebThreads = kThreads + 32;        // plus one producer warp

// Row teams: a row's M columns are split over G lanes of 4 columns (padded to a power of
// two); at M = 4 two lanes share a row, taking its chunks alternately.
template <int M>
struct ChebShape {
  static constexpr int G = M / 4;
  static constexpr int GP = (G <= 1) ? 1 : (G <= 2) ? 2 : (G <= 4) ? 4 : 8;
  static constexpr int S = (G == 1) ? 2 : 1;
  static constexpr int TEAM = GP * S;
  static constexpr int RPW = 32 / TEAM;                           // rows per warp and pass
  static constexpr int PASSES = kSliceTileRows / (8 * RPW);
  static_assert(M % 4 == 0 && PASSES * 8 * RPW == kSliceTileRows, "row teams must tile the slice rows");
};

// One stage: slice offsets (80 bytes used), row order (128 bytes), then chunk indices and
// values (cap slots).  Byte offsets.
template <typename T>
struct ChebLayout {
  uint32_t col, val, bytes;
  __host__ __device__ explicit ChebLayout(int cap) {
    col = 256;
    val = col + (uint32_t)cap * 4u;
    bytes = val + (uint32_t)cap * (uint32_t)sizeof(T);
  }
};

struct ChebMeta {
  int64_t pb;      // first slot of the tile
  int staged;      // indices and values are in the stage (else read from global memory)
  int pad;
};

__device__ __forceinline__ void ld4i(const int32_t* p, int32_t v[4]) {
  int4 t = *reinterpret_cast<const int4*>(p);
  v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}

// PF: load the row's own R, d and D^-1 before its gathers rather than after them, so that
// their latency (DRAM when the blocks exceed L2) overlaps the gathers' at the cost of nine
// registers through the chunk loop (measured on one GB300: 5% faster per step on a 2M-node
// graph, 4% slower on a 200k-node one; the autotuner chooses per operator).
template <typename T, typename SB, typename SO, int M, bool PF>
__global__ void __launch_bounds__(kChebThreads, sizeof(T) == 4 ? 2 : 1) k_cheb(ChebArgs<T> a, int cap, int nst) {
  const SB* __restrict__ X = static_cast<const SB*>(a.X);
  const SB* __restrict__ Rb = static_cast<const SB*>(a.R);
  const SB* Db = static_cast<const SB*>(a.D);        // may alias Dout: no __restrict__
  SB* Dout = static_cast<SB*>(a.Dout);
  SO* __restrict__ Xout = static_cast<SO*>(a.Xout);
  using Sh = ChebShape<M>;
  constexpr int G = Sh::G, GP = Sh::GP, S = Sh::S, TEAM = Sh::TEAM, RPW = Sh::RPW;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw);                       // [3]
  uint64_t* empty = full + 4;                                                   // [3]
  ChebMeta* meta = reinterpret_cast<ChebMeta*>(smem_raw + 64);                  // [3]
  unsigned char* stages = smem_raw + 256;
  const ChebLayout<T> L(cap);
  const int wid = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int64_t ntiles = (a.n + kSliceTileRows - 1) / kSliceTileRows;
  // a solve that has stopped (converged, or failed) leaves its remaining captured steps idle;
  // thread 0 reads the state once for the whole CTA
  __shared__ int s_done;
  if (threadIdx.x == 0) {
    s_done = (a.st && a.st->done) ? 1 : 0;
    for (int s = 0; s < nst; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], kChebConsumers);
    }
    mbar_fence_init();
  }
  __syncthreads();
  if (s_done) return;

  // ---------------- producer ----------------
  if (wid == kChebConsumers / 32) {
    if (lane == 0) {
      int64_t t = blockIdx.x;
      int64_t pb = t < ntiles ? a.slp[t * kSlicesPerTile] : 0;
      int64_t pe = t < ntiles ? a.slp[(t + 1) * kSlicesPerTile] : 0;
      int i = 0;
      for (; t < ntiles; t += gridDim.x, ++i) {
        const int s = i % nst;
        // the next tile's slot range is loaded now, so that its latency overlaps the wait
        const int64_t tn = t + gridDim.x;
        const int64_t nb = tn < ntiles ? a.slp[tn * kSlicesPerTile] : 0;
        const int64_t ne = tn < ntiles ? a.slp[(tn + 1) * kSlicesPerTile] : 0;
        if (i >= nst && !mbar_wait(&empty[s], (uint32_t)((i / nst) - 1) & 1u)) {
          if (a.st) { a.st->err = MGE_ETIMEOUT; a.st->bad_stage = 7; a.st->done = DONE_ERROR; }
          break;
        }
        const bool staged = pe - pb <= cap;
        const uint32_t ns = staged ? (uint32_t)(pe - pb) : 0u;
        const uint32_t total = 80u + 128u + ns * (4u + (uint32_t)sizeof(T));
        meta[s].pb = pb;
        meta[s].staged = staged;
        unsigned char* sb = stages + (size_t)s * L.bytes;
        fence_proxy_async();
        mbar_arrive_expect_tx(&full[s], total);
        bulk_g2s(sb, a.slp + t * kSlicesPerTile, 80u, &full[s]);
        bulk_g2s(sb + 128, a.perm + t * kSliceTileRows, 128u, &full[s]);
        if (ns > 0) {
          bulk_g2s(sb + L.col, a.col + pb, ns * 4u, &full[s]);
          bulk_g2s(sb + L.val, a.val + pb, ns * (uint32_t)sizeof(T), &full[s]);
        }
        pb = nb;
        pe = ne;
      }
      // no copy may still be landing when the block's shared memory is released
      for (int u = max(0, i - nst); u < i; ++u) mbar_wait(&full[u % nst], (uint32_t)(u / nst) & 1u);
    }
    return;
  }

  // ---------------- consumer warps ----------------
  const int team = lane / TEAM, tl = lane % TEAM;
  const int sub = tl / GP, g = tl % GP, c0 = g * 4;
  const bool lane_ok = g < G;
  int i = 0;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x, ++i) {
    const int s = i % nst;
    if (!mbar_wait(&full[s], (uint32_t)(i / nst) & 1u)) {
      if (a.st) { a.st->err = MGE_ETIMEOUT; a.st->bad_stage = 7; a.st->done = DONE_ERROR; }
      break;
    }
    const unsigned char* sb = stages + (size_t)s * L.bytes;
    const int64_t* sslp = reinterpret_cast<const int64_t*>(sb);
    const uint8_t* sperm = sb + 128;
    const int32_t* scol = reinterpret_cast<const int32_t*>(sb + L.col);
    const T* sval = reinterpret_cast<const T*>(sb + L.val);
    const int64_t tb = meta[s].pb;
    const bool staged = meta[s].staged != 0;
    const int64_t r0 = t * kSliceTileRows;
#pragma unroll
    for (int pass = 0; pass < Sh::PASSES; ++pass) {
      const int p = (pass * 8 + wid) * RPW + team;        // sorted position in the tile
      const int sl = p / kSliceRows, q = p % kSliceRows;
      const int lr = sperm[p];
      const bool valid = lane_ok && lr != 0xFF;
      // The rows of a warp lie in one slice, so every lane runs the same chunk loop; lanes
      // without a row (past the last row, or beyond the block's columns) read row 0 and
      // column 0 instead and drop the result.  No lane-dependent branch before the store.
      const int64_t row = r0 + (valid ? lr : 0);
      const int cc = lane_ok ? c0 : 0;
      const int nch = (int)((sslp[sl + 1] - sslp[sl]) / (4 * kSliceRows));   // 4-slot chunks
      const int nit = (nch + S - 1) / S;                                       // per lane
      const int off = (int)(sslp[sl] - tb) + q * 4;
      T acc[4] = {0, 0, 0, 0}, wi[4];
      ldg4(X + row * M + cc, wi);
      T rr[4], dd[4], dv;
      if constexpr (PF) {
        ldg4(Rb + row * M + cc, rr);
        ld4(Db + row * M + cc, dd);           // D may be the output array: plain load
        dv = __ldg(a.dinv + row);
      }
      // chunk c of the row: indices and values at off + 64 c, then the four gathers; two
      // register sets in turn keep the next chunk's gathers in flight while one is summed.
      // With two lanes per row, lane `sub` takes chunks sub, sub + 2, ...; the second lane of
      // an odd count repeats the last chunk with zero values.
      auto run = [&](const int32_t* cp, const T* vp) {
        int32_t jA[4], jB[4];
        T vA[4], vB[4], wA[4][4], wB[4][4];
        auto load = [&](int k, int32_t* j, T* v, T (*w)[4]) {
          int c = sub + k * S;
          const bool in = c < nch;
          c = in ? c : nch - 1;
          ld4i(cp + c * (4 * kSliceRows), j);
          ld4(vp + c * (4 * kSliceRows), v);
          if constexpr (S > 1) {
#pragma unroll
            for (int b = 0; b < 4; ++b) v[b] = in ? v[b] : T(0);
          }
#pragma unroll
          for (int b = 0; b < 4; ++b) ldg4(X + (size_t)j[b] * M + cc, w[b]);
        };
        auto consume = [&](const T* v, const T (*w)[4]) {
#pragma unroll
          for (int b = 0; b < 4; ++b)
#pragma unroll
            for (int u = 0; u < 4; ++u) acc[u] += v[b] * (w[b][u] - wi[u]);
        };
        if (nit == 0) return;
        load(0, jA, vA, wA);
        for (int k = 0;;) {
          if (k + 1 < nit) load(k + 1, jB, vB, wB);
          consume(vA, wA);
          if (++k >= nit) break;
          if (k + 1 < nit) load(k + 1, jA, vA, wA);
          consume(vB, wB);
          if (++k >= nit) break;
        }
      };
      if (staged) run(scol + off, sval + off);
      else run(a.col + tb + off, a.val + tb + off);
      if constexpr (S == 2) {
        // the two lanes of a row (adjacent) took alternate chunks
#pragma unroll
        for (int u = 0; u < 4; ++u) acc[u] += __shfl_xor_sync(0xffffffffu, acc[u], 1);
      }
      if (valid && sub == 0) {
        T dn[4], xn[4];
        if constexpr (!PF) {
          ldg4(Rb + row * M + c0, rr);
          ld4(Db + row * M + c0, dd);         // D may be the output array: plain load
          dv = __ldg(a.dinv + row);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const T y = a.shift * wi[u] + acc[u];
          const T z = rr[u] - dv * (a.sy * y);
          dn[u] = a.c1 * (a.sd * dd[u]) + a.c2 * z;
          xn[u] = a.sy * wi[u] + dn[u];
        }
        st4(Dout + row * M + c0, dn);
        st4(Xout + row * M + c0, xn);
      }
    }
    mbar_arrive(&empty[s]);      // this thread is done with stage s (no lane-dependent branch)
  }
}

// Stage capacity and count: the densest tile's slots, in three stages if they fit the
// per-CTA budget, else two, else the capacity two stages of the budget hold (denser tiles
// read their indices and values from global memory).  The budget is the tuned one (default
// 64 KB: the L1 part of the SM keeps room for the gathers in flight).
constexpr int kChebBudgets[] = {32 * 1024, 48 * 1024, 64 * 1024, 96 * 1024};
constexpr int kChebMaxBudget = 96 * 1024;
template <typename T>
void cheb_config(int64_t max_tile_slots, int64_t budget, int* cap, int* nst) {
  const int64_t fixed = ChebLayout<T>(0).bytes;
  const int64_t per = 4 + sizeof(T);
  const int64_t want = std::max<int64_t>(64, (max_tile_slots + 63) / 64 * 64);
  for (int k : {3, 2}) {
    if (256 + k * (fixed + want * per) <= budget) {
      *cap = (int)want;
      *nst = k;
      return;
    }
  }
  *nst = 2;
  *cap = (int)std::max<int64_t>(64, ((budget - 256) / 2 - fixed) / per / 64 * 64);
}

// the early-load variant exists for FP32 throughout
template <typename T, typename S, typename SO>
constexpr bool cheb_has_pf() { return std::is_same<T, float>::value && std::is_same<S, float>::value && std::is_same<SO, float>::value; }

template <typename T, typename S, typename SO, int M, bool PF>
cudaError_t cheb_launch_v(const Ctx* ctx, cudaStream_t st, const ChebArgs<T>& a, int64_t max_tile_slots, int budget) {
  int cap = 0, nst = 0;
  cheb_config<T>(max_tile_slots, budget, &cap, &nst);
  const size_t smem = 256 + (size_t)nst * ChebLayout<T>(cap).bytes;
  // resident CTAs per SM for this stage size (cached per host thread: the serving slots
  // launch from several threads; the size is fixed per operator)
  thread_local size_t last_smem = 0;
  thread_local int per_sm = 1;
  if (smem != last_smem) {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_cheb<T, S, SO, M, PF>, kChebThreads, smem) != cudaSuccess || b < 1)
      b = 1;
    per_sm = b;
    last_smem = smem;
  }
  const int64_t ntiles = (a.n + kSliceTileRows - 1) / kSliceTileRows;
  const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(ntiles, (int64_t)ctx->num_sms * per_sm));
  k_cheb<T, S, SO, M, PF><<<(unsigned)grid, kChebThreads, smem, st>>>(a, cap, nst);
  return cudaGetLastError();
}

}  // namespace

template <typename T, typename S, typename SO, int M>
cudaError_t cheb_configure() {
  cudaError_t e = cudaFuncSetAttribute(k_cheb<T, S, SO, M, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 256 + kChebMaxBudget);
  if constexpr (cheb_has_pf<T, S, SO>()) {
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_cheb<T, S, SO, M, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 256 + kChebMaxBudget);
  }
  return e;
}

template <typename T, typename S, typename SO, int M>
cudaError_t cheb_launch(const Ctx* ctx, cudaStream_t st, const ChebArgs<T>& a, int64_t max_tile_slots, ChebTune tune) {
  if (a.n <= 0) return cudaSuccess;
  const int budget = tune.budget > 0 ? std::min(tune.budget, kChebMaxBudget) : 64 * 1024;
  if constexpr (cheb_has_pf<T, S, SO>()) {
    if (tune.prefetch) return cheb_launch_v<T, S, SO, M, true>(ctx, st, a, max_tile_slots, budget);
  }
  return cheb_launch_v<T, S, SO, M, false>(ctx, st, a, max_tile_slots, budget);
}

template <typename T, int M>
cudaError_t cheb_tune(const Ctx* ctx, cudaStream_t st, const ChebArgs<T>& a, int64_t max_tile_slots,
                      ChebTune* best, double* best_us, int* launches) {
  *best = ChebTune{};
  *best_us = 0;
  *launches = 0;
  if (a.n <= 0) return cudaSuccess;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t err = cudaEventCreate(&e0);
  if (err == cudaSuccess) err = cudaEventCreate(&e1);
  double bu = 1e30;
  constexpr int kReps = 3;
  for (int pf = 0; pf < (cheb_has_pf<T, T, T>() ? 2 : 1) && err == cudaSuccess; ++pf) {
    for (int budget : kChebBudgets) {
      const ChebTune c{budget, pf};
      err = cheb_launch<T, T, T, M>(ctx, st, a, max_tile_slots, c);         // warm-up
      *launches += 1 + kReps;
      if (err == cudaSuccess) err = cudaEventRecord(e0, st);
      for (int r = 0; r < kReps && err == cudaSuccess; ++r) err = cheb_launch<T, T, T, M>(ctx, st, a, max_tile_slots, c);
      if (err == cudaSuccess) err = cudaEventRecord(e1, st);
      if (err == cudaSuccess) err = cudaEventSynchronize(e1);
      float ms = 0;
      if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
      if (err != cudaSuccess) break;
      const double us = 1e3 * ms / kReps;
      if (us < bu) { bu = us; *best = c; }
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (err == cudaSuccess) *best_us = bu;
  return err;
}

#define MGE_CHEB_INST(T, S, SO, M)                                                           \
  template cudaError_t cheb_configure<T, S, SO, M>();                                        \
  template cudaError_t cheb_launch<T, S, SO, M>(const Ctx*, cudaStream_t, const ChebArgs<T>&, int64_t, ChebTune);
#define MGE_CHEB_INST_M(M)                                                                   \
  MGE_CHEB_INST(float, float, float, M)                                                      \
  MGE_CHEB_INST(double, double, double, M)                                                   \
  MGE_CHEB_INST(float, __nv_bfloat16, __nv_bfloat16, M)                                      \
  MGE_CHEB_INST(float, __nv_bfloat16, float, M)
MGE_CHEB_INST_M(4)
MGE_CHEB_INST_M(8)
MGE_CHEB_INST_M(12)
MGE_CHEB_INST_M(16)
MGE_CHEB_INST_M(24)
#define MGE_CHEB_TUNE_INST(M)                                                                \
  template cudaError_t cheb_tune<float, M>(const Ctx*, cudaStream_t, const ChebArgs<float>&, int64_t, ChebTune*, double*, int*); \
  template cudaError_t cheb_tune<double, M>(const Ctx*, cudaStream_t, const ChebArgs<double>&, int64_t, ChebTune*, double*, int*);
MGE_CHEB_TUNE_INST(4)
MGE_CHEB_TUNE_INST(8)
MGE_CHEB_TUNE_INST(12)
MGE_CHEB_TUNE_INST(16)
MGE_CHEB_TUNE_INST(24)
#undef MGE_CHEB_TUNE_INST
#undef MGE_CHEB_INST_M
#undef MGE_CHEB_INST

}  // namespace lob
}  // namespace mge
