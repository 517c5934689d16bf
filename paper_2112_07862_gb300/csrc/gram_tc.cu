// Rayleigh-Ritz Grams on the tensor cores (tcgen05): for S = [X W P] (3m columns) and
// AS = [AX AW AP],
//   G = S^T [AS | BS],   G_A = S^T A S (first 3m columns), G_B = S^T B S (last 3m),
// as one MMA chain per CTA, D[128 x N] += A[128 x 32] B[N x 32]^T per tile of 32 rows,
// with A = S^T (rows 3m..127 unused) and B = [AS | BS]^T (N = 6m rounded up to 16).
//
// FP32 accuracy from TF32 tensor cores: every FP32 value x is split into hi = x rounded to
// TF32 (to nearest) and lo = x - hi (exact in FP32) rounded to TF32; each tile issues
// hi*hi + hi*lo + lo*hi, so a product carries about 2^-22 relative error, unbiased, instead
// of TF32's 2^-11.  Sums: the tensor-memory accumulator (FP32) runs over a few tiles only
// (TcShape::GROUP); the consumer warps then drain it into FP32 sums held in registers
// (Kahan-compensated where they fit) while the next run accumulates in a second
// tensor-memory region.  A single FP32 accumulator over all of a CTA's rows (13,000 at
// n = 2M) put an error of ~8e-6 relative into the Ritz values, which floored the relative
// residual just under a 1e-5 tolerance.  The CTAs' sums are reduced in FP64.
//
// Per CTA: a producer warp streams each tile's six 32 x m block slices and the 32 b_i into a
// ring of shared-memory stages (7, or 4 at m = 24) with 1-D bulk copies (TMA); eight consumer warps split
// the values and write both operands in the K-major, non-swizzled layout of the tensor cores
// (8-row x 16-byte core matrices: element (row r, k) at (r/8)*1024 + (k/4)*128 + (r%8)*16 +
// (k%4)*4), into one of two operand buffers; one thread issues the twelve MMAs of the tile and
// commits them to the buffer's mbarrier, which the consumers wait on before refilling it.
// A drain reads the accumulator back (tcgen05.ld.32x32b: warp w reads tensor-memory lanes
// 32 (w % 4) .. + 31, i.e. Gram rows, and column half w / 4).  The epilogue writes the
// compensated sums to shared memory in FP64; the eight CTAs of a cluster add their copies
// through distributed shared memory (each rank a slice of the entries) and add the cluster's
// sums into the Gram accumulators with FP64 atomics.
#include "lobpcg_common.cuh"

namespace mge {
namespace lob {
namespace {

constexpr int kTcConsumers = 256;                 // 8 warps
constexpr int kTcThreads = kTcConsumers + 32;     // plus the producer warp
constexpr int kTcT = 32;                          // rows per tile (the MMAs' K)
constexpr int kLBO = 128;                         // bytes between K-adjacent core matrices
constexpr int kSBO = (kTcT / 4) * 128;            // bytes between 8-row groups
constexpr int kTcCluster = 8;                     // CTAs per cluster (DSMEM reduction)

template <int M>
struct TcShape {
  static constexpr int NS = 3 * M;
  static constexpr int NB = 6 * M;
  static constexpr int NMMA = ((NB + 15) / 16) * 16;
  static constexpr int RAW = ((6 * kTcT * M * 4 + kTcT * 4) + 127) / 128 * 128;
  static constexpr int A_BYTES = 128 * kTcT * 4;
  static constexpr int B_BYTES = NMMA * kTcT * 4;
  static constexpr int BUF = 2 * A_BYTES + 2 * B_BYTES;
  static constexpr int HDR = 1024;
  // raw stages in flight: as many as shared memory allows, up to 7 (the tile loads are the
  // kernel's critical path: ~40 KB in flight per SM with 3 stages left it waiting on them)
  static constexpr int NRAW = M == 24 ? 4 : 7;
  static constexpr int SMEM = HDR + NRAW * RAW + 2 * BUF;
  static_assert(SMEM <= 227 * 1024, "shared memory");
  static constexpr int TMEM_COLS = NMMA <= 32 ? 32 : NMMA <= 64 ? 64 : NMMA <= 128 ? 128 : 256;
  static constexpr int TMEM_ALLOC = 2 * TMEM_COLS;                // two accumulator regions
  static constexpr int H0 = (NB / 2 + 7) / 8 * 8;                 // columns of half 0 (x8 loads)
  static constexpr int H1 = NB - H0;
  static constexpr int QUARTERS = (NS + 31) / 32;                 // lane quarters holding rows
  // Register sums: compensated (Kahan) where two floats per column fit the 168 registers a
  // thread gets at 288 threads per CTA (m <= 16), plain FP32 at m = 24.  Runs of 8 tiles: the
  // error of a run grows with its length, that of plain register sums as sqrt(runs).
  static constexpr bool KAHAN = M <= 16;
  static constexpr int GROUP = 8;                                // tiles per accumulation run
  static constexpr int NC = KAHAN ? H0 : 1;                      // compensation terms
  static_assert(GROUP >= 2, "a region is drained two tiles after its run ends");
  static_assert(NS <= 128 && NMMA <= 256, "Gram shape exceeds one MMA");
  static_assert(H1 > 0 && H1 % 8 == 0 && H0 >= H1, "column halves");
  static_assert(NS * NB * 8 <= 2 * BUF, "epilogue does not fit the operand buffers");
};

__device__ __forceinline__ int kmaj(int r, int k) {
  return (r >> 3) * kSBO + (k >> 2) * kLBO + (r & 7) * 16 + (k & 3) * 4;
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  uint64_t d = (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)((kLBO >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((kSBO >> 4) & 0x3FFF) << 32;
  d |= 1ull << 46;                                // descriptor version; no swizzle, base offset 0
  return d;
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
               " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}"
               ::"r"(tmem), "l"(a), "l"(b), "r"(idesc), "r"(acc) : "memory");
}

// x rounded to the 10-bit TF32 mantissa, to nearest with ties away from zero: add half a unit
// of the 13th bit to the magnitude's bit pattern (a carry moves into the exponent as it
// should) and clear the 13 low bits.  Integer operations: the conversion instruction runs
// at a fraction of the FP32 rate, and every Gram tile converts ~9,000 values.
__device__ __forceinline__ float tf32_rna(float x) {
  return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}

__device__ __forceinline__ void tf32_split(float x, float& hi, float& lo) {
  hi = tf32_rna(x);
  lo = tf32_rna(__fsub_rn(x, hi));     // x - hi is exact: it holds x's low 13 bits
}

// Kahan summation: s + (-c) carries the sum with the rounding errors of its additions
__device__ __forceinline__ void kahan_add(float& s, float& c, float v) {
  const float y = __fsub_rn(v, c);
  const float t = __fadd_rn(s, y);
  c = __fsub_rn(__fsub_rn(t, s), y);
  s = t;
}

// Adds one accumulator region into this thread's register sums: its lane (a Gram row) and W
// columns from taddr on.  Warp-collective (tcgen05.ld .sync.aligned).
template <int W, bool KAHAN, int NA, int NCA>
__device__ __forceinline__ void tc_drain(uint32_t taddr, float (&s)[NA], float (&c)[NCA]) {
  static_assert(W <= NA && W % 8 == 0 && (!KAHAN || W <= NCA), "drain width");
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
  for (int c0 = 0; c0 < W; c0 += 8) {
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr + (uint32_t)c0));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      if constexpr (KAHAN) kahan_add(s[c0 + j], c[c0 + j], __uint_as_float(r[j]));
      else s[c0 + j] = __fadd_rn(s[c0 + j], __uint_as_float(r[j]));
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

template <int M>
__global__ void __cluster_dims__(kTcCluster, 1, 1) __launch_bounds__(kTcThreads, 1) k_gram_tc(GramTcArgs a) {
  using Sh = TcShape<M>;
  extern __shared__ __align__(1024) unsigned char smem[];
  static_assert(Sh::NRAW <= 8, "header layout");
  uint64_t* full = reinterpret_cast<uint64_t*>(smem);            // [NRAW]
  uint64_t* empty = full + 8;                                    // [NRAW]
  uint64_t* mmab = full + 16;                                    // [2]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + 160);
  int* s_fail = reinterpret_cast<int*>(smem + 192);      // a consumer wait gave up
  int* s_done = reinterpret_cast<int*>(smem + 196);
  int* p_fail = reinterpret_cast<int*>(smem + 200);      // the producer's wait gave up
  unsigned char* raw = smem + Sh::HDR;
  unsigned char* bufs = raw + Sh::NRAW * Sh::RAW;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  cg::cluster_group cl = cg::this_cluster();

  if (tid == 0) {
    for (int s = 0; s < Sh::NRAW; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], kTcConsumers); }
    mbar_init(&mmab[0], 1);
    mbar_init(&mmab[1], 1);
    *s_fail = 0;
    *p_fail = 0;
    *s_done = (a.st && a.st->done) ? 1 : 0;
    mbar_fence_init();
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 ::"r"(smem_u32(tmem_slot)), "r"(Sh::TMEM_ALLOC) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  const bool active = *s_done == 0;

  const int64_t ntiles = (a.n + kTcT - 1) / kTcT;
  const int64_t my_tiles = active && blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  // compensated sums of this thread's Gram row (lane) over its warp's column half
  const int quarter = warp & 3, half = warp >> 2;
  const bool drainer = warp < kTcConsumers / 32 && quarter < Sh::QUARTERS;
  float ks_s[Sh::H0], ks_c[Sh::NC];
#pragma unroll
  for (int j = 0; j < Sh::H0; ++j) ks_s[j] = 0.f;
#pragma unroll
  for (int j = 0; j < Sh::NC; ++j) ks_c[j] = 0.f;
  // region (g & 1) holds run g; warp-uniform
  auto drain = [&](int64_t g) {
    if (!drainer) return;
    const uint32_t addr = tmem + (uint32_t)((g & 1) * Sh::TMEM_COLS) + ((uint32_t)(32 * quarter) << 16) +
                          (uint32_t)(half ? Sh::H0 : 0);
    if (half == 0) tc_drain<Sh::H0, Sh::KAHAN>(addr, ks_s, ks_c);
    else tc_drain<Sh::H1, Sh::KAHAN>(addr, ks_s, ks_c);
  };

  if (warp == kTcConsumers / 32) {
    // ---------------- producer ----------------
    if (lane == 0) {
      for (int64_t i = 0; i < my_tiles; ++i) {
        const int s = (int)(i % Sh::NRAW);
        if (i >= Sh::NRAW && !mbar_wait(&empty[s], (uint32_t)((i / Sh::NRAW) - 1) & 1u)) { *p_fail = 1; break; }
        const int64_t r0 = (blockIdx.x + i * gridDim.x) * kTcT;
        const int nr = (int)(a.n - r0 < (int64_t)kTcT ? a.n - r0 : (int64_t)kTcT);
        const uint32_t blk = (uint32_t)nr * M * 4u;
        const uint32_t bb = a.b ? (uint32_t)((nr + 3) / 4 * 4) * 4u : 0u;
        unsigned char* st = raw + (size_t)s * Sh::RAW;
        fence_proxy_async();
        mbar_arrive_expect_tx(&full[s], 6u * blk + bb);
        for (int q = 0; q < 3; ++q) {
          bulk_g2s(st + (size_t)q * kTcT * M * 4, a.S[q] + r0 * M, blk, &full[s]);
          bulk_g2s(st + (size_t)(3 + q) * kTcT * M * 4, a.AS[q] + r0 * M, blk, &full[s]);
        }
        if (a.b) bulk_g2s(st + (size_t)6 * kTcT * M * 4, a.b + r0, bb, &full[s]);
      }
    }
  } else {
    // ---------------- consumers ----------------
    const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(Sh::NMMA >> 3) << 17) |
                           ((uint32_t)(128 >> 4) << 24);
    int64_t issued = 0;                 // tiles whose MMAs were issued (the same in every consumer)
    int64_t drained = 0;                // runs drained (the same in every consumer)
    for (int64_t i = 0; i < my_tiles; ++i) {
      const int s = (int)(i % Sh::NRAW), buf = (int)(i & 1);
      const int64_t r0 = (blockIdx.x + i * gridDim.x) * kTcT;
      const int nr = (int)(a.n - r0 < (int64_t)kTcT ? a.n - r0 : (int64_t)kTcT);
      bool ok = mbar_wait(&full[s], (uint32_t)(i / Sh::NRAW) & 1u);
      if (ok && i >= 2) ok = mbar_wait(&mmab[buf], (uint32_t)((i - 2) >> 1) & 1u);
      if (!ok) *s_fail = 1;               // written before the barrier below, read after it
      const unsigned char* st = raw + (size_t)s * Sh::RAW;
      const float* rb = reinterpret_cast<const float*>(st + (size_t)6 * kTcT * M * 4);
      unsigned char* bp = bufs + (size_t)buf * Sh::BUF;
      unsigned char* Ahi = bp;
      unsigned char* Alo = bp + Sh::A_BYTES;
      unsigned char* Bhi = bp + 2 * Sh::A_BYTES;
      unsigned char* Blo = Bhi + Sh::B_BYTES;
      // operand rows: A rows c < 3m (S columns); B rows j < 6m ([AS | BS] columns); tile rows
      // k >= nr are zero in both.  A thread takes one operand row j and four consecutive k:
      // four reads of the raw tile (consecutive threads, consecutive j: conflict-free) and one
      // 16-byte store per operand copy (the four k of a core-matrix row are contiguous).
      for (int it = tid; it < Sh::NB * (kTcT / 4); it += kTcConsumers) {
        const int j = it % Sh::NB, k0 = (it / Sh::NB) * 4;
        const int jj = j < Sh::NS ? j : j - Sh::NS;
        const int q = jj / M, c = jj - q * M;
        const float* sraw = reinterpret_cast<const float*>(st + (size_t)q * kTcT * M * 4) + c;
        const float* araw = reinterpret_cast<const float*>(st + (size_t)(3 + q) * kTcT * M * 4) + c;
        float sv[4], v[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const int k = k0 + t;
          const bool in = k < nr;
          sv[t] = in ? sraw[k * M] : 0.f;
          v[t] = !in ? 0.f : (j < Sh::NS) ? araw[k * M] : (a.b ? rb[k] * sv[t] : sv[t]);
        }
        float4 h, l;
        tf32_split(v[0], h.x, l.x); tf32_split(v[1], h.y, l.y);
        tf32_split(v[2], h.z, l.z); tf32_split(v[3], h.w, l.w);
        const int o = kmaj(j, k0);
        *reinterpret_cast<float4*>(Bhi + o) = h;
        *reinterpret_cast<float4*>(Blo + o) = l;
        if (j < Sh::NS) {
          tf32_split(sv[0], h.x, l.x); tf32_split(sv[1], h.y, l.y);
          tf32_split(sv[2], h.z, l.z); tf32_split(sv[3], h.w, l.w);
          *reinterpret_cast<float4*>(Ahi + o) = h;
          *reinterpret_cast<float4*>(Alo + o) = l;
        }
      }
      fence_proxy_async();
      mbar_arrive(&empty[s]);
      asm volatile("bar.sync 1, %0;" ::"r"(kTcConsumers) : "memory");
      if (*reinterpret_cast<volatile int*>(s_fail)) break;      // uniform: set before the barrier
      ++issued;
      // a run that ended with tile i - 2 is complete (every consumer waited for that tile's
      // commit above); its region is next written by run g + 2, after later barriers
      if (i >= 2 && (i - 2) % Sh::GROUP == Sh::GROUP - 1) {
        drain((i - 2) / Sh::GROUP);
        drained = (i - 2) / Sh::GROUP + 1;
      }
      if (tid == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t ah = smem_u32(Ahi), al = smem_u32(Alo), bh = smem_u32(Bhi), bl = smem_u32(Blo);
        const uint32_t dt = tmem + (uint32_t)(((i / Sh::GROUP) & 1) * Sh::TMEM_COLS);
        const bool first = i % Sh::GROUP == 0;
#pragma unroll
        for (int ks = 0; ks < kTcT / 8; ++ks) {
          const uint32_t o = (uint32_t)ks * 2u * kLBO;
          const uint32_t acc = (first && ks == 0) ? 0u : 1u;
          mma_tf32(dt, smem_desc(ah + o), smem_desc(bh + o), idesc, acc);
          mma_tf32(dt, smem_desc(ah + o), smem_desc(bl + o), idesc, 1u);
          mma_tf32(dt, smem_desc(al + o), smem_desc(bh + o), idesc, 1u);
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                     ::"r"(smem_u32(&mmab[buf])) : "memory");
      }
    }
    // the last commit covers every MMA this CTA issued
    if (issued > 0) {
      const int64_t last = issued - 1;
      if (!mbar_wait(&mmab[last & 1], (uint32_t)(last >> 1) & 1u)) *s_fail = 1;
    }
    asm volatile("bar.sync 1, %0;" ::"r"(kTcConsumers) : "memory");
    // the last one or two runs (consecutive: distinct regions)
    if (!*reinterpret_cast<volatile int*>(s_fail))
      for (int64_t g = drained; g < (issued + Sh::GROUP - 1) / Sh::GROUP; ++g) drain(g);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  // ---------------- epilogue: compensated sums -> FP64 [3m][6m] in shared memory ----------------
  double* E = reinterpret_cast<double*>(bufs);
  auto sum_of = [](const float (&sv)[Sh::H0], const float (&cv)[Sh::NC], int j) -> double {
    if constexpr (Sh::KAHAN) return (double)sv[j] - (double)cv[j];
    else return (double)sv[j];
  };
  if (drainer) {
    const int row = quarter * 32 + lane;
    const bool ok = my_tiles > 0 && !*s_fail && !*p_fail;
    if (row < Sh::NS) {
      if (half == 0) {
#pragma unroll
        for (int j = 0; j < Sh::H0; ++j) E[row * Sh::NB + j] = ok ? sum_of(ks_s, ks_c, j) : 0.0;
      } else {
#pragma unroll
        for (int j = 0; j < Sh::H1; ++j) E[row * Sh::NB + Sh::H0 + j] = ok ? sum_of(ks_s, ks_c, j) : 0.0;
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(Sh::TMEM_ALLOC) : "memory");
  if ((*s_fail || *p_fail) && a.st && threadIdx.x == 0) {
    a.st->err = MGE_ETIMEOUT; a.st->bad_stage = 8; a.st->done = DONE_ERROR;
  }
  // ---------------- the cluster's copies summed through DSMEM, added into slot 0 ----------------
  cl.sync();
  if (active) {
    const int r = (int)cl.block_rank();
    const int len = Sh::NS * Sh::NB, per = (len + kTcCluster - 1) / kTcCluster;
    const int lo = r * per, hi = min(len, lo + per);
    for (int e = lo + tid; e < hi; e += kTcThreads) {
      double v = 0.0;
#pragma unroll
      for (int q = 0; q < kTcCluster; ++q) v += cl.map_shared_rank(E, q)[e];
      const int i = e / Sh::NB, j = e % Sh::NB;
      if (j < Sh::NS) atomicAdd(a.outA + (size_t)i * MAXS + j, v);
      else atomicAdd(a.outB + (size_t)i * MAXS + (j - Sh::NS), v);
    }
  }
  cl.sync();
}

}  // namespace

template <int M>
cudaError_t gram_tc_configure() {
  return cudaFuncSetAttribute(k_gram_tc<M>, cudaFuncAttributeMaxDynamicSharedMemorySize, TcShape<M>::SMEM);
}

template <int M>
int gram_tc_clusters(const Ctx* ctx, int64_t n) {
  const int64_t ntiles = (n + kTcT - 1) / kTcT;
  const int64_t cls = std::min<int64_t>((ntiles + kTcCluster - 1) / kTcCluster,
                                        (int64_t)std::max(1, ctx->num_sms / kTcCluster));
  return (int)std::max<int64_t>(1, cls);
}

template <int M>
cudaError_t gram_tc_launch(const Ctx* ctx, cudaStream_t st, const GramTcArgs& a, int clusters) {
  k_gram_tc<M><<<kTcCluster * clusters, kTcThreads, TcShape<M>::SMEM, st>>>(a);
  return cudaGetLastError();
}

#define MGE_GRAM_TC_INST(M)                                                                  \
  template cudaError_t gram_tc_configure<M>();                                               \
  template int gram_tc_clusters<M>(const Ctx*, int64_t);                                      \
  template cudaError_t gram_tc_launch<M>(const Ctx*, cudaStream_t, const GramTcArgs&, int);
MGE_GRAM_TC_INST(12)
MGE_GRAM_TC_INST(16)
MGE_GRAM_TC_INST(24)
#undef MGE_GRAM_TC_INST

}  // namespace lob
}  // namespace mge
