// Device-side state, scratch layout and helpers shared by the LOBPCG kernels (lobpcg.cu)
// and the small dense kernels (rr.cu).
#pragma once

#include <cooperative_groups.h>

#include "mge_internal.cuh"

namespace mge {
namespace lob {

namespace cg = cooperative_groups;

constexpr int MAXM = 24;             // widest block
constexpr int MAXS = 3 * MAXM;       // widest Rayleigh-Ritz basis [X W P]
constexpr int CL = 8;                // CTAs per cluster in the reducing kernels
constexpr int MAXCL = 64;            // clusters per reducing launch (grid <= 512 CTAs)
constexpr int kThreads = 256;

enum : int { DONE_RUNNING = 0, DONE_CONVERGED = 1, DONE_ERROR = 2, DONE_MAXITER = 3, DONE_STALLED = 4 };

struct State {
  int done;
  int iter;
  int err;
  int drops;
  int kept;
  int bad_stage;     // 1: Rayleigh-Ritz input, 2: residual / Ritz values, 3: W Gram, 4: RR output
  int loops;         // passes of the device-side iteration loop (graph mode)
  int rr64;          // FP32 blocks: Rayleigh-Ritz and W's Cholesky now run in FP64
  int rr64_iter;     // iteration after which they switched (0: from the start)
  int best_iter;     // last iteration that halved the largest relative residual (near tol)
  float best_rho;    // that residual
  int pbest_iter;    // the same at any level of the residual
  float pbest_rho;
  int refine;        // the FP32 Rayleigh-Ritz applies its FP64 correction step: the largest
                     // residual is within kRRStallGate of the tolerance and has halved in the
                     // last kRRStallIters iterations
  int pad1;
  long long rr_clk[16];     // clock64 deltas at the phase boundaries of the last Rayleigh-Ritz
  long long wp_clk[8];      // and of the last wprep (diagnostics)
  double lambda[MAXM];
  double eta[MAXM];
};

// FP64 results of the small kernels and the per-cluster partial sums they consume.
struct Small {
  double partA[MAXCL][MAXS * MAXS];   // G_A = S^T A S, per cluster
  double partB[MAXCL][MAXS * MAXS];   // G_B = S^T B S (block-upper part), per cluster
  double partW[MAXCL][MAXS * MAXM];   // [X' P' W_raw]^T B W_raw, per cluster
  double partC[MAXCL][MAXM];          // column sums of W_raw (deflation), per cluster
  double partN[MAXCL][2 * MAXM];      // ||r_k||^2 and ||x_k||^2, per cluster
  double Cx[MAXS * MAXM], Cp[MAXS * MAXM];
  double lam[MAXM];
  unsigned long long vmax[MAXM];
  unsigned long long vidx[MAXM];
};

// Block-precision copies the streaming kernels read.
template <typename T>
struct SmallT {
  T Cx[MAXS * MAXM], Cp[MAXS * MAXM];
  T lam[MAXM];
  // W normalisation L (upper triangular, right factor) and the products the SpMM epilogue
  // applies: W = W_raw L - X (M_x L) - P (M_p L) - 1 (c L)
  T Linv[MAXM * MAXM], MxL[MAXM * MAXM], MpL[MAXM * MAXM], cL[MAXM];
};

// ---- 4-wide vector access -------------------------------------------------------------
__device__ __forceinline__ void ld4(const float* p, float v[4]) {
  float4 t = *reinterpret_cast<const float4*>(p);
  v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
__device__ __forceinline__ void ld4(const double* p, double v[4]) {
  double2 a = reinterpret_cast<const double2*>(p)[0];
  double2 b = reinterpret_cast<const double2*>(p)[1];
  v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}
__device__ __forceinline__ void st4(float* p, const float v[4]) {
  *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void st4(double* p, const double v[4]) {
  reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
  reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
}
__device__ __forceinline__ void ldg4(const float* p, float v[4]) {
  float4 t = __ldg(reinterpret_cast<const float4*>(p));
  v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
__device__ __forceinline__ void ldg4(const double* p, double v[4]) {
  double2 a = __ldg(reinterpret_cast<const double2*>(p));
  double2 b = __ldg(reinterpret_cast<const double2*>(p) + 1);
  v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}

// BF16 blocks (4 columns = 8 bytes): widening is exact (a bfloat16 is the top half of a
// float); narrowing rounds to nearest even
__device__ __forceinline__ void bf16x4_to_f32(uint2 t, float v[4]) {
  v[0] = __uint_as_float(t.x << 16); v[1] = __uint_as_float(t.x & 0xffff0000u);
  v[2] = __uint_as_float(t.y << 16); v[3] = __uint_as_float(t.y & 0xffff0000u);
}
__device__ __forceinline__ void ld4(const __nv_bfloat16* p, float v[4]) {
  bf16x4_to_f32(*reinterpret_cast<const uint2*>(p), v);
}
__device__ __forceinline__ void ldg4(const __nv_bfloat16* p, float v[4]) {
  bf16x4_to_f32(__ldg(reinterpret_cast<const uint2*>(p)), v);
}
__device__ __forceinline__ void st4(__nv_bfloat16* p, const float v[4]) {
  __nv_bfloat162 a = __floats2bfloat162_rn(v[0], v[1]);
  __nv_bfloat162 b = __floats2bfloat162_rn(v[2], v[3]);
  uint2 t;
  t.x = *reinterpret_cast<const uint32_t*>(&a);
  t.y = *reinterpret_cast<const uint32_t*>(&b);
  *reinterpret_cast<uint2*>(p) = t;
}

// Sums `len` doubles that every CTA of the cluster holds at `buf` (shared memory) and stores
// the cluster total through store(index, value).  Rank r reduces the slice r of the vector,
// reading all peers' copies through distributed shared memory.
template <typename F>
__device__ __forceinline__ void cluster_sum(const double* buf, int len, F store) {
  cg::cluster_group cl = cg::this_cluster();
  cl.sync();
  const int r = (int)cl.block_rank();
  const int nr = (int)cl.num_blocks();
  const int per = (len + nr - 1) / nr;
  const int lo = r * per, hi = min(len, lo + per);
  for (int t = lo + (int)threadIdx.x; t < hi; t += blockDim.x) {
    double s = 0.0;
    for (int q = 0; q < nr; ++q) s += cl.map_shared_rank(buf, q)[t];
    store(t, s);
  }
  cl.sync();   // peers keep their shared memory until every slice is read
}

__device__ __forceinline__ int cluster_id() { return blockIdx.x / CL; }

// ---- bulk asynchronous copies (TMA, 1-D) and mbarriers -----------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
// make initialised barriers visible to the asynchronous (copy) proxy
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
// global -> this CTA's shared memory; dst, src 16-byte aligned, bytes a multiple of 16
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t done;
  asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
               : "=r"(done) : "r"(smem_u32(bar)), "r"(parity) : "memory");
  return done != 0;
}
// The same, suspending the thread until the phase completes or about ns nanoseconds pass:
// a waiting thread issues no instructions meanwhile.
__device__ __forceinline__ bool mbar_try_wait_suspend(uint64_t* bar, uint32_t parity, uint32_t ns) {
  uint32_t done;
  asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}"
               : "=r"(done) : "r"(smem_u32(bar)), "r"(parity), "r"(ns) : "memory");
  return done != 0;
}
// Waits for the phase with the given parity to complete; gives up (false) after about
// max_cycles SM cycles so that a lost copy cannot hang the GPU.
constexpr long long kWaitCycles = 1ll << 31;
// Waiting threads are suspended by the hardware between polls (a spinning wait took most of
// the issue slots of the SM from the CTAs that had their data).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long long max_cycles = kWaitCycles) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait_suspend(bar, parity, 1000000u))
    if (clock64() - t0 > max_cycles) return false;
  return true;
}

// Sum of p[c * stride] for c < n with eight loads in flight (the partial sums sit in L2; a
// plain dependent loop pays the full load latency per term).
__device__ __forceinline__ double sum_strided(const double* p, int n, size_t stride) {
  double s0 = 0, s1 = 0, s2 = 0, s3 = 0, s4 = 0, s5 = 0, s6 = 0, s7 = 0;
  int c = 0;
  for (; c + 8 <= n; c += 8) {
    double v0 = p[(size_t)(c + 0) * stride], v1 = p[(size_t)(c + 1) * stride];
    double v2 = p[(size_t)(c + 2) * stride], v3 = p[(size_t)(c + 3) * stride];
    double v4 = p[(size_t)(c + 4) * stride], v5 = p[(size_t)(c + 5) * stride];
    double v6 = p[(size_t)(c + 6) * stride], v7 = p[(size_t)(c + 7) * stride];
    s0 += v0; s1 += v1; s2 += v2; s3 += v3; s4 += v4; s5 += v5; s6 += v6; s7 += v7;
  }
  for (; c < n; ++c) s0 += p[(size_t)c * stride];
  return ((s0 + s1) + (s2 + s3)) + ((s4 + s5) + (s6 + s7));
}

// FP64 reciprocal square root from an FP32 seed and two Newton steps
// (y <- y (3 - x y^2) / 2); avoids the long-latency FP64 division/sqrt sequences.
__device__ __forceinline__ double drsqrt(double x) {
  double y = (double)rsqrtf((float)x);
  y = y * (1.5 - 0.5 * x * y * y);
  y = y * (1.5 - 0.5 * x * y * y);
  return y;
}
// FP64 reciprocal from an FP32 seed and two Newton steps (y <- y (2 - x y)).
__device__ __forceinline__ double drcp(double x) {
  double y = (double)(1.0f / (float)x);
  y = y * (2.0 - x * y);
  y = y * (2.0 - x * y);
  return y;
}


// Arguments of the single-CTA kernels in rr.cu (launched from lobpcg.cu).
struct RRArgs {
  Small* sm;
  void* smt;            // SmallT<float> or SmallT<double>
  int is_double;
  int ncl;              // clusters that wrote Gram partials
  int M, nb, nx;        // basis: nb blocks of M columns, the first nx of which are X
  double tau;           // dependence threshold (pivot^2 of a unit-diagonal Gram)
  double tau_p;         // threshold for dropping an empty P direction
  int sel;              // RR_ALWAYS, or RR_FP32 / RR_FP64: run only in that phase of a solve
  State* st;
};

// Rayleigh-Ritz precision of an FP32 solve that may switch (State::rr64): both forms are
// launched each iteration and the one not selected returns at once.
enum : int { RR_ALWAYS = 0, RR_FP32 = 1, RR_FP64 = 2 };
// An FP32 solve moves to the FP64 Rayleigh-Ritz once the largest relative residual of the
// wanted pairs, below kRRStallGate times the tolerance, has not halved for kRRStallIters
// iterations.  (The first iterations of a preconditioned solve can go that long without
// halving it; measured on a 2M-node sphere: 9.4 after 10 iterations, 0.36 after 20.)
constexpr int kRRStallIters = 10;
constexpr float kRRStallGate = 1000.f;
__device__ __forceinline__ bool rr_selected(int sel, const State* st) {
  return sel == RR_ALWAYS || (sel == RR_FP64) == (st->rr64 != 0);
}

struct WprepArgs {
  Small* sm;
  void* smt;
  int is_double;
  int ncl_w;            // clusters that wrote W-side Gram partials
  int ncl_n;            // clusters that wrote norm partials
  int M, K;
  int has_x, has_p;
  int check;
  int deflate;
  int64_t n;
  double tol, norm, bmax, tau_w;
  int maxiter;
  int sel;              // as RRArgs::sel
  int rr_switch;        // this launch may move the solve to the FP64 Rayleigh-Ritz
  State* st;
};

cudaError_t rr_configure();
void launch_rr(cudaStream_t st, const RRArgs& a, bool inverse_form);
void launch_wprep(cudaStream_t st, const WprepArgs& a, bool fp64);

// One Chebyshev step of the LOBPCG preconditioner on the sliced copy of an operator (cheb.cu):
//   y = A x (difference form),  z = R - dinv (sy y),  d_out = c1 (sd D) + c2 z,
//   x_out = sy x + d_out.
// X, R, D, Dout, Xout: [n x M] row-major; D and Dout may be the same array (each row of D is
// read before the same row of Dout is written); dinv carries zeroed elements up to n rounded
// up to 16 bytes.
template <typename T>
struct ChebArgs {
  int64_t n;
  const int64_t* slp;
  const uint8_t* perm;
  const int32_t* col;
  const T* val;
  T shift;
  // blocks: T, or bfloat16 storage (S, and SO for x_out) with T = float arithmetic
  const void* X;
  const void* R;
  const void* D;
  const T* dinv;
  void* Dout;
  void* Xout;
  T sy, sd, c1, c2;
  State* st;
};

// Tensor-core Grams of S = [X W P] (gram_tc.cu): G_A = S^T [AX AW AP] into outA and
// G_B = S^T B S into outB, added with FP64 atomics (the accumulators start at zero).
struct GramTcArgs {
  int64_t n;
  const float* S[3];
  const float* AS[3];
  const float* b;            // NULL: B = I (else padded with 4 zeros)
  double* outA;
  double* outB;
  State* st;
};
template <int M>
cudaError_t gram_tc_configure();
template <int M>
int gram_tc_clusters(const Ctx* ctx, int64_t n);
template <int M>
cudaError_t gram_tc_launch(const Ctx* ctx, cudaStream_t st, const GramTcArgs& a, int clusters);

// Launches the step on stream st; max_tile_slots (the densest tile of the sliced copy) sizes
// the shared-memory stages.  S is the storage type of x, R, d and d_out, SO that of x_out
// (T, or __nv_bfloat16 with T = float).  cheb_configure raises the dynamic shared-memory limit.
// A tuned configuration of the step (stage budget in bytes, early loads; cheb.cu, tune.cu).
struct ChebTune {
  int budget = 64 * 1024;
  int prefetch = 0;
};
template <typename T, typename S, typename SO, int M>
cudaError_t cheb_launch(const Ctx* ctx, cudaStream_t st, const ChebArgs<T>& a, int64_t max_tile_slots,
                        ChebTune tune = ChebTune{});
template <typename T, typename S, typename SO, int M>
cudaError_t cheb_configure();
// Times every configuration on the step `a` (its buffers are overwritten: scratch only) and
// returns the fastest with its time per launch.  Synchronises the stream; not during capture.
template <typename T, int M>
cudaError_t cheb_tune(const Ctx* ctx, cudaStream_t st, const ChebArgs<T>& a, int64_t max_tile_slots,
                      ChebTune* best, double* best_us, int* launches);

}  // namespace lob
}  // namespace mge
