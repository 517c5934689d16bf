// LOBPCG for the first K generalized eigenpairs of (A, B) (Sec. 4.3), in the library's own
// kernels.  One iteration is six launches:
//
//   spmm_w   W = (W_raw - 1 c^T - X Mx - P Mp) L^-T and AW = A W: the projections and the
//            normalisation of the preconditioned residual are fused into the SpMM
//   gram     G_A = S^T A S, G_B = S^T B S for S = [X W P]   (FP32 accumulation, cluster sums)
//   rr       Rayleigh-Ritz on one CTA (rr.cu): coefficients C_x, C_p and Ritz values
//   update   X' = S C_x, AX' = AS C_x, P' = S C_p, AP' = AS C_p, R = AX' - B X' Lambda,
//            W_raw = diag(A)^-1 R, residual and vector norms          (cluster sums)
//   gram     [X' P' W_raw]^T B W_raw (+ column sums of W_raw when deflating)
//   wprep    backward errors, convergence flag, Mx, Mp and L^-T for the next SpMM (rr.cu)
//
// A is a graph Laplacian plus a multiple of I in every use (A = L - mu Q + eps I, or Q), so
// (A x)_i = shift x_i + sum_j A_ij (x_j - x_i): the SpMM sums differences, which keeps FP32
// accuracy where A x is small next to ||A|| ||x|| (smooth vectors); the diagonal entry
// contributes A_ii (x_i - x_i) = 0.
//
// Cross-CTA reductions: each CTA reduces in registers/shared memory, the 8 CTAs of a cluster
// sum through distributed shared memory, and each cluster stores one partial; the single-CTA
// consumer adds the (at most MAXCL) cluster partials in FP64.  No contended atomics.
#include "lobpcg_common.cuh"

#include <memory>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>

namespace mge {
namespace lob {

namespace {

// =======================================================================================
// SpMM with fused projection and normalisation of W
// =======================================================================================
template <typename T>
struct SpmmArgs {
  int64_t n;
  const int64_t* ptr;        // n + 2 entries (one padding entry)
  const int32_t* col;        // nnz + 4 entries (padding)
  const T* val;              // nnz + 4 entries (padding)
  T shift;
  const T* Wr;
  const T* X; const T* AX; const T* P; const T* AP;   // NULL when absent
  const SmallT<T>* sm;                                 // L, M_x L, M_p L, c L (NULL: plain A*Wr)
  T* W; T* AW;
  const int32_t* out_row;    // plain product only: row r of the result goes to row out_row[r]
                             // of AW (NULL: row r)
  State* st;
  int tiles_per_cta;
  // one step of the Chebyshev preconditioner (cheb != 0; Wr is then the iterate x_k):
  //   z = R - D^-1 A (sy x_k),  d' = c1 (sd d) + c2 z,  x_{k+1} = sy x_k + d'
  // with R the Jacobi-scaled residual block (cr), d the previous correction (cd), D^-1 (cdinv)
  int cheb;
  const T* cr; const T* cd; const T* cdinv;
  T* cd_out; T* cx_out;
  T sy, sd, c1, c2;
};

// Lanes per row: G = M/4 column groups (4-wide vectors) times S, the split of the row's
// nonzeros; every row is a team of 12 or 16 lanes, two rows per warp.
// SHORT is for operators whose rows hold at most about half a batch of nonzeros (the
// preconditioner's L + eps I, and Q, on k-NN graphs): two lanes per row at m <= 8, each lane
// walking the row's nonzeros itself (no split, no reduction), 16 rows per warp.
template <int M, bool SHORT = false> struct SpmmShape {
  static constexpr int G = M / 4;
  static constexpr int SL = (G == 1) ? 16 : (G == 2) ? 8 : (G <= 4) ? 4 : 2;
  static constexpr int S = !SHORT ? SL : (G == 1) ? 4 : (G == 2) ? 1 : (SL > 1 ? SL / 2 : 1);
  static constexpr int TEAM = G * S;
  static constexpr int RPW = 32 / TEAM;
  static constexpr int BATCH = 4;     // nonzeros per lane whose gathers are issued together
};

// One pipeline stage of the SpMM: a tile of R rows with its row pointers, column indices and
// values (when they fit in CAP), and the rows of W_raw, X, AX, P, AP the rows need.  Byte
// offsets; every segment starts on a 128-byte boundary.
template <typename T, int M, bool SHORT = false>
struct SpmmTile {
  // one pass of the 8 consumer warps covers R rows (32, or the number of row teams)
  static constexpr int TEAMS = SpmmShape<M, SHORT>::RPW * 8;
  static constexpr int R = TEAMS <= 32 ? 32 : TEAMS;
  static constexpr int CAP = (R > 32 || !SHORT) ? 2048 : 1024;
  static constexpr int ST = (R >= 128) ? 2 : 3;      // pipeline stages
  static constexpr int up(int x) { return (x + 127) / 128 * 128; }
  static constexpr int PTR = 0;
  static constexpr int COL = up((R + 2) * 8);
  static constexpr int VAL = COL + up((CAP + 8) * 4);
  static constexpr int ROWB = up(R * M * (int)sizeof(T));
  static constexpr int WR = VAL + up((CAP + 8) * (int)sizeof(T));
  // the short variant never runs the fused epilogue (no X, AX, P, AP rows): its stage holds
  // W_raw (the iterate), R and d (XR, AXR) and D^-1 (PR) only
  static constexpr int XR = WR + ROWB, AXR = XR + ROWB, PR = AXR + ROWB;
  static constexpr int APR = PR + (SHORT ? up(R * (int)sizeof(T)) : ROWB);
  static constexpr int BYTES = APR + (SHORT ? 0 : ROWB);
};
constexpr int kSpmmConsumers = kThreads;           // 8 consumer warps
constexpr int kSpmmThreads = kThreads + 32;        // plus one producer warp

struct SpmmMeta {
  int64_t pb;      // first nonzero of the tile
  int64_t c0;      // first column index copied (pb rounded down to 16 bytes)
  int64_t v0;      // first value copied
  int rows;
  int staged;      // column indices and values are in the stage
};

// Y = A X with A = shift I + the difference-form Laplacian part (a_ij (x_j - x_i)), fused with
// the projection and normalisation of W when a.sm is set.  Each CTA owns a contiguous range
// of tiles; its producer warp streams them through a ring of shared-memory stages with 1-D
// bulk copies (TMA) so that the row pointers, column indices, values and row blocks never sit
// on a dependent load chain; the consumer warps wait only for the gathers of X rows.
template <typename T, int M, bool SHORT>
__global__ void __launch_bounds__(kSpmmThreads) k_spmm_w(SpmmArgs<T> a) {
  if (a.st && a.st->done) return;
  using Sh = SpmmShape<M, SHORT>;
  using Tl = SpmmTile<T, M, SHORT>;
  constexpr int G = Sh::G, S = Sh::S, TEAM = Sh::TEAM, RPW = Sh::RPW, BT = Sh::BATCH;
  constexpr int NW = kSpmmConsumers / 32;
  constexpr int TEAMS = NW * RPW;
  constexpr int ST = Tl::ST;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw);
  uint64_t* empty = full + ST;
  SpmmMeta* meta = reinterpret_cast<SpmmMeta*>(smem_raw + 64);
  unsigned char* stages = smem_raw + 256;
  // blocks of at most 8 columns keep the epilogue's row vectors in registers (assembled by
  // shuffles); wider blocks stage them in shared memory
  constexpr bool REG = (G <= 2) && (TEAM >= 2 * M);
  // epilogue matrices stored transposed (column c contiguous) with a padded column stride,
  // so that the 16-byte loads of different columns fall in different banks
  constexpr int CS = M + 4;
  __shared__ __align__(16) T sMxLt[M * CS], sMpLt[M * CS], sLt[M * CS];
  __shared__ T scL[M];
  // row vectors of the shared-memory epilogue (fused mode, long variant only)
  __shared__ __align__(16) T sW[(REG || SHORT) ? 1 : NW][(REG || SHORT) ? 1 : RPW][M];
  __shared__ __align__(16) T sAW[(REG || SHORT) ? 1 : NW][(REG || SHORT) ? 1 : RPW][M];
  const bool fused = a.sm != nullptr;
  const bool hx = fused && a.X, hp = fused && a.P;
  const bool cheb = !fused && a.cheb != 0;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t ntiles = (a.n + Tl::R - 1) / Tl::R;
  const int64_t t0 = (int64_t)blockIdx.x * a.tiles_per_cta;
  const int my = (int)max((int64_t)0, min((int64_t)a.tiles_per_cta, ntiles - t0));
  if (threadIdx.x == 0) {
    for (int s = 0; s < ST; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], kSpmmConsumers); }
    mbar_fence_init();
  }
  if (fused) {
    for (int t = threadIdx.x; t < M * M; t += kSpmmThreads) {
      const int r = t / M, c = t % M;
      sMxLt[c * CS + r] = a.sm->MxL[r * MAXM + c];
      sMpLt[c * CS + r] = a.sm->MpL[r * MAXM + c];
      sLt[c * CS + r] = a.sm->Linv[r * MAXM + c];
    }
    for (int t = threadIdx.x; t < M; t += kSpmmThreads) scL[t] = a.sm->cL[t];
  }
  __syncthreads();

  if (wid == NW) {
    // ---------------- producer warp (one thread) ----------------
    if (lane == 0) {
      // the end of the next tile is loaded one iteration early, so that its latency overlaps
      // the wait for a free stage instead of delaying the copies
      int64_t pb = my > 0 ? a.ptr[t0 * Tl::R] : 0;
      int64_t pe_next = my > 0 ? a.ptr[min(a.n, (t0 + 1) * Tl::R)] : 0;
      int i = 0;
      for (; i < my; ++i) {
        const int s = i % ST;
        const int64_t pe = pe_next;
        if (i + 1 < my) pe_next = a.ptr[min(a.n, (t0 + i + 2) * Tl::R)];
        if (i >= ST && !mbar_wait(&empty[s], (uint32_t)((i / ST) - 1) & 1u)) {
          if (a.st) { a.st->err = MGE_ETIMEOUT; a.st->bad_stage = 6; a.st->done = DONE_ERROR; }
          break;
        }
        const int64_t r0 = (t0 + i) * Tl::R;
        const int rows = (int)min((int64_t)Tl::R, a.n - r0);
        const bool staged = pe - pb <= Tl::CAP;
        constexpr int VE = 16 / (int)sizeof(T);              // values per 16 bytes
        const int64_t c0 = pb & ~(int64_t)3, c1 = (pe + 3) & ~(int64_t)3;
        const int64_t v0 = pb & ~(int64_t)(VE - 1), v1 = (pe + VE - 1) & ~(int64_t)(VE - 1);
        const uint32_t bp = (uint32_t)(((rows + 2) / 2) * 2 * 8);
        const uint32_t bc = staged ? (uint32_t)((c1 - c0) * 4) : 0u;
        const uint32_t bv = staged ? (uint32_t)((v1 - v0) * (int64_t)sizeof(T)) : 0u;
        const uint32_t br = (uint32_t)rows * M * (uint32_t)sizeof(T);
        const uint32_t bd = cheb ? (((uint32_t)rows * (uint32_t)sizeof(T) + 15u) & ~15u) : 0u;
        const uint32_t total = bp + bc + bv + br * (1u + (hx ? 2u : 0u) + (hp ? 2u : 0u) + (cheb ? 2u : 0u)) + bd;
        meta[s].pb = pb; meta[s].c0 = c0; meta[s].v0 = v0; meta[s].rows = rows; meta[s].staged = staged;
        unsigned char* sb = stages + (size_t)s * Tl::BYTES;
        fence_proxy_async();
        mbar_arrive_expect_tx(&full[s], total);
        bulk_g2s(sb + Tl::PTR, a.ptr + r0, bp, &full[s]);
        if (staged) {
          bulk_g2s(sb + Tl::COL, a.col + c0, bc, &full[s]);
          bulk_g2s(sb + Tl::VAL, a.val + v0, bv, &full[s]);
        }
        bulk_g2s(sb + Tl::WR, a.Wr + r0 * M, br, &full[s]);
        if (hx) {
          bulk_g2s(sb + Tl::XR, a.X + r0 * M, br, &full[s]);
          bulk_g2s(sb + Tl::AXR, a.AX + r0 * M, br, &full[s]);
        }
        if (hp) {
          bulk_g2s(sb + Tl::PR, a.P + r0 * M, br, &full[s]);
          bulk_g2s(sb + Tl::APR, a.AP + r0 * M, br, &full[s]);
        }
        if (cheb) {
          bulk_g2s(sb + Tl::XR, a.cr + r0 * M, br, &full[s]);
          bulk_g2s(sb + Tl::AXR, a.cd + r0 * M, br, &full[s]);
          bulk_g2s(sb + Tl::PR, a.cdinv + r0, bd, &full[s]);
        }
        pb = pe;
      }
      // no copy may still be landing when the block's shared memory is released
      for (int u = max(0, i - ST); u < i; ++u) mbar_wait(&full[u % ST], (uint32_t)(u / ST) & 1u);
    }
    return;
  }

  // ---------------- consumer warps ----------------
  const int team = lane / TEAM, tl = lane % TEAM;
  const int sub = tl / G, g = tl % G, c0 = g * 4;     // nonzero slice and column group
  const bool lane_ok = team < RPW;
  for (int i = 0; i < my; ++i) {
    const int s = i % ST;
    if (!mbar_wait(&full[s], (uint32_t)(i / ST) & 1u)) {
      if (a.st) { a.st->err = MGE_ETIMEOUT; a.st->bad_stage = 6; a.st->done = DONE_ERROR; }
      break;
    }
    const unsigned char* sb = stages + (size_t)s * Tl::BYTES;
    const int64_t* sptr = reinterpret_cast<const int64_t*>(sb + Tl::PTR);
    const int32_t* scol = reinterpret_cast<const int32_t*>(sb + Tl::COL);
    const T* sval = reinterpret_cast<const T*>(sb + Tl::VAL);
    const T* sWr = reinterpret_cast<const T*>(sb + Tl::WR);
    const int64_t mpb = meta[s].pb, mc0 = meta[s].c0, mv0 = meta[s].v0;
    const int rows = meta[s].rows;
    const bool staged = meta[s].staged != 0;
    const int64_t r0 = (t0 + i) * Tl::R;
    for (int pass = 0; pass < (Tl::R + TEAMS - 1) / TEAMS; ++pass) {
      const int r = pass * TEAMS + wid * RPW + team;
      const bool valid = lane_ok && r < rows;
      const int64_t row = r0 + r;
      T acc[4] = {0, 0, 0, 0}, wi[4] = {0, 0, 0, 0};
      if (valid) {
        ld4(sWr + r * M + c0, wi);
        const int64_t pb = sptr[r];
        const int len = (int)(sptr[r + 1] - pb);
        // BATCH nonzeros per lane at a time: their indices and values, then their gathers;
        // indices and values come from the stage (shared-memory loads) or, for tiles too
        // dense to stage, from global memory
        auto gather = [&](const int32_t* cp, const T* vp) {
          // short rows are software-pipelined: the indices and gathers of batch b + 1 are
          // issued before batch b is consumed, so a row's batches overlap instead of queueing
          int32_t j[BT];
          T v[BT], w[BT][4];
          auto issue = [&](int k0, int32_t* jj, T* vv, T (*ww)[4]) {
#pragma unroll
            for (int b = 0; b < BT; ++b) {
              const int k = k0 + b * S;
              jj[b] = k < len ? cp[k] : -1;
              vv[b] = k < len ? vp[k] : T(0);
            }
#pragma unroll
            for (int b = 0; b < BT; ++b) {
              if (jj[b] >= 0) {
                ldg4(a.Wr + (size_t)jj[b] * M + c0, ww[b]);
              } else {
#pragma unroll
                for (int q = 0; q < 4; ++q) ww[b][q] = wi[q];
              }
            }
          };
          auto consume = [&](const T* vv, const T (*ww)[4]) {
#pragma unroll
            for (int b = 0; b < BT; ++b)
#pragma unroll
              for (int q = 0; q < 4; ++q) acc[q] += vv[b] * (ww[b][q] - wi[q]);
          };
          if constexpr (SHORT) {
            // two register sets in turn, so that no batch is copied from one set to the other
            int32_t jn[BT];
            T vn[BT], wn[BT][4];
            issue(sub, j, v, w);
            for (int k0 = sub; k0 < len; k0 += 2 * BT * S) {
              const int k1 = k0 + BT * S, k2 = k1 + BT * S;
              if (k1 < len) issue(k1, jn, vn, wn);
              consume(v, w);
              if (k1 >= len) break;
              if (k2 < len) issue(k2, j, v, w);
              consume(vn, wn);
            }
          } else {
            // long rows: each lane's share of a row is about one batch
            for (int k0 = sub; k0 < len; k0 += BT * S) {
              issue(k0, j, v, w);
              consume(v, w);
            }
          }
        };
        if (staged) gather(scol + (pb - mc0), sval + (pb - mv0));
        else gather(a.col + pb, a.val + pb);
      }
      const bool lead = valid && sub == 0;
      if (!fused || !REG) {
        // combine the S nonzero slices: lanes of slice 0 end up with the row sums
#pragma unroll
        for (int off = (S / 2) * G; off >= G && off > 0; off >>= 1) {
#pragma unroll
          for (int q = 0; q < 4; ++q) acc[q] += __shfl_down_sync(0xffffffffu, acc[q], off);
        }
      }
      if (!fused) {
        if (lead) {
          T y[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) y[q] = a.shift * wi[q] + acc[q];
          if (cheb) {
            T rr[4], dd[4], dn[4], xn[4];
            ld4(reinterpret_cast<const T*>(sb + Tl::XR) + r * M + c0, rr);
            ld4(reinterpret_cast<const T*>(sb + Tl::AXR) + r * M + c0, dd);
            const T dv = reinterpret_cast<const T*>(sb + Tl::PR)[r];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              const T z = rr[q] - dv * (a.sy * y[q]);
              dn[q] = a.c1 * (a.sd * dd[q]) + a.c2 * z;
              xn[q] = a.sy * wi[q] + dn[q];
            }
            st4(a.cd_out + row * M + c0, dn);
            st4(a.cx_out + row * M + c0, xn);
          } else {
            st4(a.AW + (a.out_row ? (int64_t)a.out_row[row] : row) * M + c0, y);
          }
        }
        continue;
      }
      // projection against X, P and the constant vector, then the normalisation, folded
      // into one product per output (L, M_x L, M_p L, c L prepared by the small kernel):
      //   W  = W_raw L - X (M_x L) - P (M_p L) - 1 (c L)
      //   AW = (A W_raw) L - shift 1 (c L) - AX (M_x L) - AP (M_p L)
      // lane tl of the team computes outputs tl, tl + TEAM, ... (W column o for o < M, AW
      // column o - M otherwise); the X, AX, P, AP rows come from the stage
      const T* sX = reinterpret_cast<const T*>(sb + Tl::XR) + r * M;
      const T* sAX = reinterpret_cast<const T*>(sb + Tl::AXR) + r * M;
      const T* sP = reinterpret_cast<const T*>(sb + Tl::PR) + r * M;
      const T* sAP = reinterpret_cast<const T*>(sb + Tl::APR) + r * M;
      if constexpr (REG) {
        // every lane gets its column group's row sums (butterfly over the slices), then the
        // whole row of W_raw and of A W_raw from the lanes of the other group
#pragma unroll
        for (int off = (S / 2) * G; off >= G && off > 0; off >>= 1) {
#pragma unroll
          for (int q = 0; q < 4; ++q) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], off);
        }
        T wf[M], yf[M];
#pragma unroll
        for (int gg = 0; gg < G; ++gg) {
          const int src = lane - g + gg;
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const T wq = __shfl_sync(0xffffffffu, wi[q], src);
            const T aq = __shfl_sync(0xffffffffu, acc[q], src);
            wf[gg * 4 + q] = wq;
            yf[gg * 4 + q] = a.shift * wq + aq;
          }
        }
        if (valid && tl < 2 * M) {
          const bool isw = tl < M;
          const int c = isw ? tl : tl - M;
          T r0v = (isw ? T(-1) : -a.shift) * scL[c], r1v = T(0);
#pragma unroll
          for (int l = 0; l < M; l += 4) {
            T lc[4];
            ld4(sLt + c * CS + l, lc);
#pragma unroll
            for (int t = 0; t < 4; ++t) r0v += (isw ? wf[l + t] : yf[l + t]) * lc[t];
          }
          if (hx) {
            const T* xr = isw ? sX : sAX;
#pragma unroll
            for (int l = 0; l < M; l += 4) {
              T xv[4], mc[4];
              ld4(xr + l, xv);
              ld4(sMxLt + c * CS + l, mc);
#pragma unroll
              for (int t = 0; t < 4; ++t) r1v -= xv[t] * mc[t];
            }
          }
          if (hp) {
            const T* pr = isw ? sP : sAP;
#pragma unroll
            for (int l = 0; l < M; l += 4) {
              T pv[4], mc[4];
              ld4(pr + l, pv);
              ld4(sMpLt + c * CS + l, mc);
#pragma unroll
              for (int t = 0; t < 4; ++t) r1v -= pv[t] * mc[t];
            }
          }
          (isw ? a.W : a.AW)[row * M + c] = r0v + r1v;
        }
      } else {
        // the row's W_raw and A W_raw go to shared memory for the whole team
        if (lead) {
          T y[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) y[q] = a.shift * wi[q] + acc[q];
          st4(&sW[wid][team][c0], wi);
          st4(&sAW[wid][team][c0], y);
        }
        __syncwarp();
        if (valid) {
          for (int o = tl; o < 2 * M; o += TEAM) {
            const bool isw = o < M;
            const int c = isw ? o : o - M;
            T r0v = (isw ? T(-1) : -a.shift) * scL[c], r1v = T(0);
#pragma unroll
            for (int l = 0; l < M; l += 4) {
              T vv[4], lc[4];
              if (isw) ld4(&sW[wid][team][l], vv);
              else ld4(&sAW[wid][team][l], vv);
              ld4(sLt + c * CS + l, lc);
#pragma unroll
              for (int t = 0; t < 4; ++t) r0v += vv[t] * lc[t];
            }
            if (hx) {
              const T* xr = isw ? sX : sAX;
#pragma unroll
              for (int l = 0; l < M; l += 4) {
                T xv[4], mc[4];
                ld4(xr + l, xv);
                ld4(sMxLt + c * CS + l, mc);
#pragma unroll
                for (int t = 0; t < 4; ++t) r1v -= xv[t] * mc[t];
              }
            }
            if (hp) {
              const T* pr = isw ? sP : sAP;
#pragma unroll
              for (int l = 0; l < M; l += 4) {
                T pv[4], mc[4];
                ld4(pr + l, pv);
                ld4(sMpLt + c * CS + l, mc);
#pragma unroll
                for (int t = 0; t < 4; ++t) r1v -= pv[t] * mc[t];
              }
            }
            (isw ? a.W : a.AW)[row * M + c] = r0v + r1v;
          }
        }
        __syncwarp();
      }
    }
    mbar_arrive(&empty[s]);      // this thread is done with stage s (no lane-dependent branch)
  }
}

template <typename T, int M, bool SHORT>
size_t spmm_smem() { return 256 + (size_t)SpmmTile<T, M, SHORT>::ST * SpmmTile<T, M, SHORT>::BYTES; }

// rows short enough for the halved split: at most half a batch of nonzeros on average
template <int M>
bool spmm_short(int64_t nnz, int64_t n) {
  return n > 0 && 2 * nnz <= (int64_t)SpmmShape<M>::SL * SpmmShape<M>::BATCH * n;
}

// grid: as many CTAs as fit on the GPU at once (by shared memory), each owning a
// contiguous range of tiles
template <typename T, int M, bool SHORT>
int spmm_grid(const Ctx* ctx, int64_t n, int* tiles_per_cta) {
  static int per_sm = 0;                 // resident CTAs per SM (registers, shared memory)
  if (per_sm == 0) {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_spmm_w<T, M, SHORT>, kSpmmThreads,
                                                      spmm_smem<T, M, SHORT>()) != cudaSuccess || b < 1)
      b = 1;
    per_sm = b;
  }
  const int64_t ntiles = (n + SpmmTile<T, M, SHORT>::R - 1) / SpmmTile<T, M, SHORT>::R;
  const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(ntiles, (int64_t)ctx->num_sms * per_sm));
  *tiles_per_cta = (int)((ntiles + grid - 1) / grid);
  return (int)((ntiles + *tiles_per_cta - 1) / *tiles_per_cta);
}

template <typename T, int M>
void spmm_launch(const Ctx* ctx, cudaStream_t st, SpmmArgs<T> s, bool short_rows) {
  if (short_rows) {
    const int grid = spmm_grid<T, M, true>(ctx, s.n, &s.tiles_per_cta);
    k_spmm_w<T, M, true><<<grid, kSpmmThreads, spmm_smem<T, M, true>(), st>>>(s);
  } else {
    const int grid = spmm_grid<T, M, false>(ctx, s.n, &s.tiles_per_cta);
    k_spmm_w<T, M, false><<<grid, kSpmmThreads, spmm_smem<T, M, false>(), st>>>(s);
  }
}

template <typename T, int M>
cudaError_t spmm_configure() {
  cudaError_t e = cudaFuncSetAttribute(k_spmm_w<T, M, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)spmm_smem<T, M, false>());
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_spmm_w<T, M, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)spmm_smem<T, M, true>());
}


// =======================================================================================
// Gram products over row tiles: out1 = L^T R1, out2 = L^T diag(b) R2 (block-upper part of
// L^T B L when R2 is L).  Each CTA streams its contiguous rows through a ring of shared-
// memory stages filled by 1-D bulk copies (TMA), one per source block and tile; threads own
// 4x4 output blocks and accumulate them from shared memory, with a compensated fold of the
// per-chunk sums.
// =======================================================================================
template <typename T>
struct GramArgs {
  int64_t n;
  int nl, n1, n2;
  bool sym2;
  const T* b;                // NULL = unit weights; else at least n rounded up to 4 elements
  double* out1;              // accumulator of out1, [MAXS * MAXS], ld MAXS
  double* out2;              // accumulator of out2, leading dimension ld2
  int ld2;
  int stride2;
  double* csum;              // column sums of R2 (deflation), [MAXM] (NULL: skip)
  State* st;
  const T* src[9];           // distinct source blocks, each [n x M] row-major
  int nsrc;
  int lmap[3], r1map[3], r2map[3];   // source index of each block of L, R1, R2
  int tr;                    // rows per tile, a multiple of 4
  int64_t per;               // rows per CTA, a multiple of tr
  uint32_t stage_bytes;      // bytes per stage, a multiple of 128
};

constexpr int kGramStages = 4;
constexpr int kTileRows = 32;

// Neumaier's compensated step acc += x, the lost low part collected in cmp; all in the
// accumulator's own precision (FP64 arithmetic would run at GB300's low FP64 rate)
template <typename A>
__device__ __forceinline__ void neumaier(A& acc, A& cmp, A x) {
  const A s = acc + x;
  const A aa = acc < A(0) ? -acc : acc, ax = x < A(0) ? -x : x;
  cmp += (aa >= ax) ? (acc - s) + x : (x - s) + acc;
  acc = s;
}

__device__ __forceinline__ void decode_item(int item, int nb1, int b1, int bl, bool sym2, int b2, int& prod,
                                            int& bi, int& bj) {
  if (item < nb1) {
    prod = 1; bi = item / b1; bj = item % b1;
    return;
  }
  int r = item - nb1;
  prod = 2;
  if (sym2) {
    int i = 0;
    while (r >= bl - i) { r -= bl - i; ++i; }
    bi = i; bj = i + r;
  } else {
    bi = r / b2; bj = r % b2;
  }
}

template <typename T, int M>
__global__ void __cluster_dims__(CL, 1, 1) __launch_bounds__(kThreads) k_gram(GramArgs<T> a) {
  if (a.st && a.st->done) return;
  using A = T;   // accumulate in the block precision (FP32 for FP32 blocks), compensated
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw);       // one mbarrier per stage
  unsigned char* data = smem_raw + 128;
  const int wl = a.nl * M, w1 = a.n1 * M, ws = a.sym2 ? 0 : a.n2 * M;
  const int bl = wl / 4, b1 = w1 / 4, b2 = (a.sym2 ? wl : a.n2 * M) / 4;
  const int nb1 = bl * b1;
  const int nb2 = a.sym2 ? bl * (bl + 1) / 2 : bl * b2;
  const int nblk = nb1 + nb2;
  constexpr int IPT = (M <= 16) ? 1 : 2;
  int rs = kThreads / nblk;
  if (rs < 1) rs = 1;
  const int tpi = (nblk * rs <= kThreads) ? nblk : kThreads;
  const int rg = threadIdx.x / tpi;
  const int ti = threadIdx.x % tpi;
  const bool has_group = rg < rs;
  const int tr = a.tr;
  // each item: a 4x4 block of one product; offsets of its two 4-column slices in a stage
  int lo[IPT], ro[IPT];
  bool it_ok[IPT], it_w[IPT];
#pragma unroll
  for (int u = 0; u < IPT; ++u) {
    const int item = ti + u * tpi;
    it_ok[u] = has_group && item < nblk;
    lo[u] = ro[u] = 0;
    it_w[u] = false;
    if (it_ok[u]) {
      int prod, bi, bj;
      decode_item(item, nb1, b1, bl, a.sym2, b2, prod, bi, bj);
      const int ci = bi * 4, cj = bj * 4;
      lo[u] = a.lmap[ci / M] * tr * M + ci % M;
      if (prod == 1) ro[u] = a.r1map[cj / M] * tr * M + cj % M;
      else if (a.sym2) { ro[u] = a.lmap[cj / M] * tr * M + cj % M; it_w[u] = true; }
      else { ro[u] = a.r2map[cj / M] * tr * M + cj % M; it_w[u] = true; }
    }
  }
  const bool weighted = a.b != nullptr;
  const int boff = a.nsrc * tr * M;
  const int64_t r0 = (int64_t)blockIdx.x * a.per;
  const int64_t r1 = min(a.n, r0 + a.per);
  const int ntiles = r0 < r1 ? (int)((r1 - r0 + tr - 1) / tr) : 0;
  // column sums of R2 (deflation): thread c + ws*g sums rows g, g + ng, ... of column c
  const int ng = ws > 0 ? kThreads / ws : 0;
  const int csg = ws > 0 ? threadIdx.x / ws : 0, csc = ws > 0 ? threadIdx.x % ws : 0;
  const bool do_cs = a.csum && csg < ng;
  const int cso = do_cs ? a.r2map[csc / M] * tr * M + csc % M : 0;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kGramStages; ++s) mbar_init(&full[s], 1);
    mbar_fence_init();
  }
  __syncthreads();
  // thread 0: copy tile t of every source block (and of b) into stage t mod kGramStages
  auto issue = [&](int t) {
    const int s = t % kGramStages;
    const int64_t row = r0 + (int64_t)t * tr;
    const int rows = (int)min((int64_t)tr, r1 - row);
    const uint32_t bb = (uint32_t)rows * M * (uint32_t)sizeof(T);
    const uint32_t wb = weighted ? (((uint32_t)rows * (uint32_t)sizeof(T) + 15u) & ~15u) : 0u;
    T* dst = reinterpret_cast<T*>(data + (size_t)s * a.stage_bytes);
    fence_proxy_async();
    mbar_arrive_expect_tx(&full[s], bb * (uint32_t)a.nsrc + wb);
    for (int i = 0; i < a.nsrc; ++i) bulk_g2s(dst + (size_t)i * tr * M, a.src[i] + row * M, bb, &full[s]);
    if (weighted) bulk_g2s(dst + boff, a.b + row, wb, &full[s]);
  };
  if (threadIdx.x == 0)
    for (int t = 0; t < ntiles && t < kGramStages; ++t) issue(t);

  A acc[IPT][16], cmp[IPT][16], at[IPT][16];
#pragma unroll
  for (int u = 0; u < IPT; ++u)
#pragma unroll
    for (int e = 0; e < 16; ++e) { acc[u][e] = A(0); cmp[u][e] = A(0); at[u][e] = A(0); }
  constexpr int CHUNK = 16;             // rows summed before the compensated fold
  int steps = 0;
  A cs = A(0);
  int t = 0;
  bool ok = true;
  for (; t < ntiles; ++t) {
    const int s = t % kGramStages;
    const bool got = mbar_wait(&full[s], (uint32_t)(t / kGramStages) & 1u);
    if (got) {
      const T* stg = reinterpret_cast<const T*>(data + (size_t)s * a.stage_bytes);
      const int rows = (int)min((int64_t)tr, r1 - (r0 + (int64_t)t * tr));
      if (has_group) {
#pragma unroll 2
        for (int r = rg; r < rows; r += rs) {
          const T bw = weighted ? stg[boff + r] : T(1);
#pragma unroll
          for (int u = 0; u < IPT; ++u) {
            if (!it_ok[u]) continue;
            T lv[4], rv[4];
            ld4(stg + lo[u] + r * M, lv);
            ld4(stg + ro[u] + r * M, rv);
            const A w = it_w[u] ? (A)bw : A(1);
#pragma unroll
            for (int p = 0; p < 4; ++p) {
              const A lb = (A)lv[p] * w;
#pragma unroll
              for (int q = 0; q < 4; ++q) at[u][p * 4 + q] += lb * (A)rv[q];
            }
          }
          if (++steps == CHUNK) {
            steps = 0;
#pragma unroll
            for (int u = 0; u < IPT; ++u)
#pragma unroll
              for (int e = 0; e < 16; ++e) {
                neumaier(acc[u][e], cmp[u][e], at[u][e]);
                at[u][e] = A(0);
              }
          }
        }
      }
      if (do_cs)
        for (int r = csg; r < rows; r += ng) cs += (A)stg[cso + r * M];
    }
    ok = __syncthreads_and(got) != 0;   // also: every thread is done with stage s
    if (!ok) break;
    if (threadIdx.x == 0 && t + kGramStages < ntiles) issue(t + kGramStages);
  }
  if (!ok && threadIdx.x == 0) {
    // a copy did not arrive in time: report it, then wait (bounded) for the copies still
    // in flight before the stages are reused below; the cluster reduction still runs so
    // that no peer CTA waits for this one
    for (int u = t; u < ntiles && u < t + kGramStages; ++u)
      mbar_wait(&full[u % kGramStages], (uint32_t)(u / kGramStages) & 1u);
    if (a.st) { a.st->err = MGE_ETIMEOUT; a.st->bad_stage = 5; a.st->done = DONE_ERROR; }
  }
  __syncthreads();
#pragma unroll
  for (int u = 0; u < IPT; ++u)
#pragma unroll
    for (int e = 0; e < 16; ++e) neumaier(acc[u][e], cmp[u][e], at[u][e]);
  // CTA reduction: stage [rs][nblk][16], sum over row groups into FP64, then the cluster
  const int len = nblk * 16;
  A* stage = reinterpret_cast<A*>(data);
  A* cstage = stage + (size_t)rs * len;
  double* part = reinterpret_cast<double*>(data + ((((size_t)rs * len + kThreads) * sizeof(A) + 15) / 16) * 16);
#pragma unroll
  for (int u = 0; u < IPT; ++u)
    if (it_ok[u]) {
      const int item = ti + u * tpi;
#pragma unroll
      for (int e = 0; e < 16; ++e) stage[(size_t)rg * len + item * 16 + e] = acc[u][e] + cmp[u][e];
    }
  if (a.csum) cstage[threadIdx.x] = do_cs ? cs : A(0);
  __syncthreads();
  // row groups summed in the accumulator precision (compensated), one conversion per entry
  for (int i = threadIdx.x; i < len; i += kThreads) {
    A sum = A(0), c = A(0);
    for (int g = 0; g < rs; ++g) neumaier(sum, c, stage[(size_t)g * len + i]);
    part[i] = (double)sum + (double)c;
  }
  if (a.csum && threadIdx.x < ws) {
    A sum = A(0), c = A(0);
    for (int g = 0; g < ng; ++g) neumaier(sum, c, cstage[g * ws + threadIdx.x]);
    part[len + threadIdx.x] = (double)sum + (double)c;
  }
  const int tot = len + (a.csum ? ws : 0);
  // each cluster adds its total into the single accumulator the consumer reads (and zeroes)
  cluster_sum(part, tot, [&](int i, double v) {
    if (i >= len) { atomicAdd(a.csum + (i - len), v); return; }
    int item = i / 16, e = i % 16, p = e / 4, q = e % 4;
    int prod, bi, bj;
    decode_item(item, nb1, b1, bl, a.sym2, b2, prod, bi, bj);
    if (prod == 1) atomicAdd(a.out1 + (bi * 4 + p) * MAXS + bj * 4 + q, v);
    else atomicAdd(a.out2 + (bi * 4 + p) * a.ld2 + bj * 4 + q, v);
  });
}

// =======================================================================================
// update: X' = S Cx, AX' = AS Cx, P' = S Cp, AP' = AS Cp, R, W_raw, residual norms
// =======================================================================================
template <typename T>
struct UpdArgs {
  int64_t n;
  int nb;
  T* S[3];
  T* AS[3];
  T* Xo; T* AXo; T* Po; T* APo;
  bool produce_p;
  const SmallT<T>* smt;
  const T* b;
  const T* dinv;
  T* Wr;
  __nv_bfloat16* WrB;        // not NULL: W_raw is stored here in BF16 instead of Wr
  double* partN;             // [ncl][2*MAXM]
  const State* st;
};

template <typename T, int M, int NB>
__global__ void __cluster_dims__(CL, 1, 1) __launch_bounds__(kThreads) k_update(UpdArgs<T> a) {
  if (a.st->done) return;
  using A = T;
  constexpr int G = M / 4, RPW = 32 / G, NW = kThreads / 32;
  constexpr int NS = NB * M;
  __shared__ T sCx[NS * M], sCp[NS * M], sLam[M];
  __shared__ A red[NW][2 * M];
  __shared__ double part[2 * M];
  for (int t = threadIdx.x; t < NS * M; t += kThreads) {
    int r = t / M, c = t % M;
    sCx[t] = a.smt->Cx[r * MAXM + c];
    sCp[t] = a.smt->Cp[r * MAXM + c];
  }
  for (int t = threadIdx.x; t < M; t += kThreads) sLam[t] = a.smt->lam[t];
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int team = lane / G, tl = lane % G, c0 = tl * 4;
  const bool lane_ok = team < RPW;
  A pr[4] = {0, 0, 0, 0}, px[4] = {0, 0, 0, 0};
  for (int64_t base = ((int64_t)blockIdx.x * NW + wid) * RPW; base < a.n;
       base += (int64_t)gridDim.x * NW * RPW) {
    const int64_t row = base + team;
    const bool valid = lane_ok && row < a.n;
    T x[4] = {0, 0, 0, 0}, ax[4] = {0, 0, 0, 0}, p[4] = {0, 0, 0, 0}, ap[4] = {0, 0, 0, 0};
    T bi = T(1), di = T(0);
    if (valid) {
      bi = a.b ? a.b[row] : T(1);
      di = a.dinv[row];
      // PB blocks of the row are loaded before their first use (all of them when they fit)
      constexpr int PB = (NB * M <= 48) ? NB : 1;
#pragma unroll
      for (int b0 = 0; b0 < NB; b0 += PB) {
        T sv[PB][M], av[PB][M];
#pragma unroll
        for (int k = 0; k < PB; ++k)
#pragma unroll
          for (int l = 0; l < M; l += 4) {
            ld4(a.S[b0 + k] + row * M + l, &sv[k][l]);
            ld4(a.AS[b0 + k] + row * M + l, &av[k][l]);
          }
#pragma unroll
        for (int k = 0; k < PB; ++k)
#pragma unroll
          for (int l = 0; l < M; ++l) {
            const int rr = (b0 + k) * M + l;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              const T cx = sCx[rr * M + c0 + q], cp = sCp[rr * M + c0 + q];
              x[q] += sv[k][l] * cx;
              ax[q] += av[k][l] * cx;
              p[q] += sv[k][l] * cp;
              ap[q] += av[k][l] * cp;
            }
          }
      }
    }
    __syncwarp();   // every lane of the team has read the row before any lane overwrites it
    if (valid) {
      st4(a.Xo + row * M + c0, x);
      st4(a.AXo + row * M + c0, ax);
      if (a.produce_p) {
        st4(a.Po + row * M + c0, p);
        st4(a.APo + row * M + c0, ap);
      }
      T r[4], w[4];
      // norms for the convergence test: ||r||_{B^-1}^2 = sum r^2 / b and ||x||_B^2 = sum b x^2
      // (1/b in FP32: the norms only meet a tolerance)
      const T ib = (T)(1.0f / (float)bi);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        r[q] = ax[q] - bi * x[q] * sLam[c0 + q];
        w[q] = r[q] * di;
        pr[q] += r[q] * r[q] * ib;
        px[q] += bi * x[q] * x[q];
      }
      if constexpr (sizeof(T) == 4) {
        if (a.WrB) st4(a.WrB + row * M + c0, w);
        else st4(a.Wr + row * M + c0, w);
      } else {
        st4(a.Wr + row * M + c0, w);
      }
    }
    __syncwarp();
  }
  // per-column sums: across the teams of a warp (lanes with equal tl), then across warps
  if ((G & (G - 1)) == 0) {
#pragma unroll
    for (int off = 16; off >= G; off >>= 1)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        pr[q] += __shfl_xor_sync(0xffffffffu, pr[q], off);
        px[q] += __shfl_xor_sync(0xffffffffu, px[q], off);
      }
    if (lane < G)
#pragma unroll
      for (int q = 0; q < 4; ++q) { red[wid][c0 + q] = pr[q]; red[wid][M + c0 + q] = px[q]; }
  } else {
    // team sizes of 3 or 6 lanes: lanes of the same column group sum through shared memory
    __shared__ A lanes[NW][32][8];
#pragma unroll
    for (int q = 0; q < 4; ++q) { lanes[wid][lane][q] = lane_ok ? pr[q] : A(0); lanes[wid][lane][4 + q] = lane_ok ? px[q] : A(0); }
    __syncwarp();
    if (lane < G) {
      A sr[4] = {0, 0, 0, 0}, sx[4] = {0, 0, 0, 0};
      for (int l = lane; l < RPW * G; l += G)
#pragma unroll
        for (int q = 0; q < 4; ++q) { sr[q] += lanes[wid][l][q]; sx[q] += lanes[wid][l][4 + q]; }
#pragma unroll
      for (int q = 0; q < 4; ++q) { red[wid][c0 + q] = sr[q]; red[wid][M + c0 + q] = sx[q]; }
    }
  }
  __syncthreads();
  if (threadIdx.x < 2 * M) {
    A s = A(0);
#pragma unroll
    for (int w = 0; w < NW; ++w) s += red[w][threadIdx.x];
    part[threadIdx.x] = (double)s;
  }
  const int cl = cluster_id();
  (void)cl;
  cluster_sum(part, 2 * M, [&](int t, double v) {
    const int which = t / M, c = t % M;
    atomicAdd(a.partN + which * MAXM + c, v);
  });
}

// =======================================================================================
// initial block and output
// =======================================================================================
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  // SplitMix64 (Steele, Lea, Flood 2014): golden-ratio increment, then the finaliser
  x += 0x9e3779b97f4a7c15ull;
  x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ull;
  x = (x ^ (x >> 27)) * 0x94d049bb133111ebull;
  return x ^ (x >> 31);
}

template <typename T>
__global__ void k_init_block(int64_t n, int M, uint64_t seed, const double* x0, int x0_cols,
                             const int32_t* row_order, T* Wr) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n * M) return;
  int64_t i = t / M;
  int c = (int)(t % M);
  double v;
  if (x0 && c < x0_cols) {
    v = x0[(int64_t)c * n + (row_order ? (int64_t)row_order[i] : i)];   // x0 is in the caller's order
  } else {
    // Box-Muller on two uniforms from the counter (i, c)
    uint64_t h1 = splitmix64(seed ^ splitmix64((uint64_t)t * 2));
    uint64_t h2 = splitmix64(seed ^ splitmix64((uint64_t)t * 2 + 1));
    double u1 = ((h1 >> 11) + 1) * (1.0 / 9007199254740993.0);   // (0, 1]
    double u2 = (h2 >> 11) * (1.0 / 9007199254740992.0);
    v = sqrt(-2.0 * log(u1)) * cospi(2.0 * u2);
  }
  Wr[t] = (T)v;
}

template <typename T>
__global__ void k_vmax(int64_t n, int M, int K, const T* X, unsigned long long* vmax) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n * K) return;
  int64_t i = t / K;
  int c = (int)(t % K);
  double v = fabs((double)X[i * M + c]);
  atomicMax(vmax + c, (unsigned long long)__double_as_longlong(v));
}

template <typename T>
__global__ void k_vidx(int64_t n, int M, int K, const T* X, const unsigned long long* vmax,
                       const int32_t* row_order, unsigned long long* vidx) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n * K) return;
  int64_t i = t / K;
  int c = (int)(t % K);
  double v = fabs((double)X[i * M + c]);
  // ties go to the smallest node index in the caller's order
  const int64_t e = row_order ? (int64_t)row_order[i] : i;
  if ((unsigned long long)__double_as_longlong(v) == vmax[c]) atomicMin(vidx + c, (unsigned long long)e);
}

template <typename T>
__global__ void k_write_v(int64_t n, int M, int K, const T* X, const unsigned long long* vidx,
                          const int32_t* row_order, const int32_t* row_rank, double* V) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n * K) return;
  int c = (int)(t / n);
  int64_t i = t % n;
  unsigned long long r = vidx[c];                       // in the caller's order
  const int64_t ri = (r < (unsigned long long)n) ? (row_rank ? (int64_t)row_rank[r] : (int64_t)r) : -1;
  double s = (ri >= 0 && (double)X[ri * M + c] < 0.0) ? -1.0 : 1.0;
  V[(int64_t)c * n + (row_order ? (int64_t)row_order[i] : i)] = s * (double)X[i * M + c];
}

inline unsigned gridn(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

// Last node of the device-side iteration loop: run another pass while the solve is running
// (and below the iteration limit, a bound that does not rely on the solver's own check).
__global__ void k_loop_cond(cudaGraphConditionalHandle h, State* st, int maxiter) {
  if (threadIdx.x == 0) {
    st->loops += 1;
    const bool more = st->done == DONE_RUNNING && st->iter < maxiter;
    cudaGraphSetConditional(h, more ? 1u : 0u);
  }
}

// =======================================================================================
// host driver
// =======================================================================================
template <typename T, int M>
struct Solver {
  Ctx* ctx;
  cudaStream_t st;
  const LobOp& op;
  int K;
  int64_t n;
  DevBuf<T> X, AX, P, AP, W, AW, Wr;
  // Chebyshev preconditioner: iterates x_k (two buffers), corrections d_k, and the block the
  // W-side kernels read (W_raw itself at the start, the preconditioned block afterwards)
  int cheb_deg = 1;
  double ch_theta = 1, ch_delta = 1, ch_sigma = 1;
  DevBuf<T> Yc0, Yc1, Dc;
  // BF16 form: the preconditioner's right-hand side D^-1 R, iterates and corrections in BF16
  // (its last step writes the preconditioned block to Wr in T)
  bool pc_bf16 = false;
  DevBuf<__nv_bfloat16> WrB, Yb0, Yb1, Db;
  const T* wsrc = nullptr;
  std::vector<uint64_t> cap_bytes;     // bytes of the SpMM launches timed inside the graph
  DevBuf<unsigned char> small;
  Small* sm = nullptr;
  SmallT<T>* smt = nullptr;
  State* state = nullptr;
  int grid_upd = 0, grid_gram = 0;
  double tol;
  int maxiter;
  bool inverse_rr = true;
  bool rr_auto = false;             // inverse form first, FP64 Jacobi once the residuals stall
  ChebTune ctune;                   // the Chebyshev step's configuration (tuned per shape)
  double tau = 1e-12, tau_p = 1e-16, tau_w = 1e-10;
  int64_t nnz_a = 0, nnz_pc = 0;

  Solver(Ctx* c, cudaStream_t s, const LobOp& o, int k) : ctx(c), st(s), op(o), K(k), n(o.n) {}

  static int clusters_for(int64_t units, int per_cta, int max_ctas) {
    int64_t ctas = (units + per_cta - 1) / per_cta;
    int64_t cls = (ctas + CL - 1) / CL;
    cls = std::max<int64_t>(1, std::min<int64_t>(cls, std::min(max_ctas / CL, MAXCL)));
    return (int)cls;
  }

  mge_status setup() {
    size_t blk = (size_t)n * M;
    MGE_TRY(X.scratch(ctx, blk, st)); MGE_TRY(AX.scratch(ctx, blk, st));
    MGE_TRY(P.scratch(ctx, blk, st)); MGE_TRY(AP.scratch(ctx, blk, st));
    MGE_TRY(W.scratch(ctx, blk, st)); MGE_TRY(AW.scratch(ctx, blk, st));
    MGE_TRY(Wr.scratch(ctx, blk, st));
    wsrc = Wr.p;
    cheb_deg = std::max(1, std::min(op.precond_degree, kMaxPrecondDegree));
    pc_bf16 = sizeof(T) == 4 && op.pc_bf16 && cheb_deg > 1 && op.sl_slp != nullptr;
    if (pc_bf16) {
      MGE_TRY(WrB.scratch(ctx, blk, st)); MGE_TRY(Yb0.scratch(ctx, blk, st));
      MGE_TRY(Yb1.scratch(ctx, blk, st)); MGE_TRY(Db.scratch(ctx, blk, st));
    }
    if (cheb_deg > 1) {
      if (!pc_bf16) {
        MGE_TRY(Yc0.scratch(ctx, blk, st)); MGE_TRY(Yc1.scratch(ctx, blk, st)); MGE_TRY(Dc.scratch(ctx, blk, st));
      }
      // Chebyshev iteration for A y = r on [alpha, beta] of the spectrum of D^-1 A: beta is the
      // Gershgorin bound, alpha = beta / (2 d^2) so that the polynomial reduces the condition
      // number of the preconditioned block by about d^2
      const double beta_in = op.pc_ptr ? op.pc_beta : op.beta;
      const double beta = beta_in > 0 ? beta_in : 2.0;
      const double alpha = beta * 0.5 / ((double)cheb_deg * cheb_deg);
      ch_theta = 0.5 * (beta + alpha);
      ch_delta = 0.5 * (beta - alpha);
      ch_sigma = ch_theta / ch_delta;
    }
    size_t off_t = ((sizeof(Small) + 255) / 256) * 256;
    size_t off_s = off_t + ((sizeof(SmallT<T>) + 255) / 256) * 256;
    size_t bytes = off_s + sizeof(State);
    MGE_TRY(small.scratch(ctx, bytes, st));
    MGE_CUDA(ctx, cudaMemsetAsync(small.p, 0, bytes, st));
    sm = reinterpret_cast<Small*>(small.p);
    smt = reinterpret_cast<SmallT<T>*>(small.p + off_t);
    state = reinterpret_cast<State*>(small.p + off_s);
    constexpr int RPW = 32 / (M / 4);
    const int rows_per_cta = RPW * (kThreads / 32);
    const int max_red = std::min(2 * ctx->num_sms, MAXCL * CL);
    grid_upd = CL * clusters_for(n, rows_per_cta, max_red);
    grid_gram = CL * clusters_for(n, kTileRows * 4, max_red);
    if (sizeof(T) == 4) { tau = 1e-6; tau_p = 1e-8; tau_w = 1e-4; }
    // the inverse-pencil Rayleigh-Ritz needs G_A positive definite: A = L - mu Q + eps I with
    // eps > 0, or Q with the constant vector deflated
    inverse_rr = (sizeof(T) == 4) && !op.rr_fp64 && (op.shift > 0.0 || op.deflate);
    rr_auto = inverse_rr && op.rr_switch;
    return MGE_OK;
  }

  // The Chebyshev step's configuration for this shape (width, precision, size class and slot
  // density of the sliced operator): the context's tuned entry, measured here -- before the
  // solve's first launch and outside any stream capture -- when the context tunes and the
  // shape is new.  The trial steps run on the solve's scratch blocks.
  mge_status tune_cheb() {
    if (cheb_deg <= 1 || !op.sl_slp || pc_bf16 || ctx->tune_mode == 0) return MGE_OK;
    char key[128];
    const int lg = (int)std::floor(std::log2((double)std::max<int64_t>(n, 1)));
    const int spr = (int)std::lround((double)op.sl_max_tile_slots / kSliceTileRows);
    snprintf(key, sizeof key, "cheb/m%d/%s/n2^%d/slots%d", M, sizeof(T) == 8 ? "f64" : "f32", lg, spr);
    TuneEntry e;
    if (tune_lookup(ctx, key, &e)) {
      ctune.budget = e.budget;
      ctune.prefetch = e.prefetch;
      return MGE_OK;
    }
    if (ctx->tune_mode != 1) return MGE_OK;
    cudaStreamCaptureStatus cs;
    MGE_CUDA(ctx, cudaStreamIsCapturing(st, &cs));
    if (cs != cudaStreamCaptureStatusNone) return MGE_OK;
    const size_t blk = (size_t)n * M * sizeof(T);
    MGE_CUDA(ctx, cudaMemsetAsync(Wr.p, 0, blk, st));
    MGE_CUDA(ctx, cudaMemsetAsync(Yc0.p, 0, blk, st));
    MGE_CUDA(ctx, cudaMemsetAsync(Dc.p, 0, blk, st));
    ChebArgs<T> c{};
    c.n = n;
    c.slp = op.sl_slp; c.perm = op.sl_perm; c.col = op.sl_col;
    c.val = static_cast<const T*>(op.sl_val);
    c.shift = (T)(op.pc_ptr ? op.pc_shift : op.shift);
    c.X = Yc0.p; c.R = Wr.p; c.D = Dc.p;
    c.dinv = static_cast<const T*>(op.pc_ptr ? op.pc_dinv : op.dinv);
    c.Dout = Dc.p; c.Xout = Yc1.p;
    c.sy = T(1); c.sd = T(1); c.c1 = T(0.5); c.c2 = T(0.5);
    c.st = state;
    ChebTune best;
    double us = 0;
    int launched = 0;
    MGE_CUDA(ctx, (cheb_tune<T, M>(ctx, st, c, op.sl_max_tile_slots, &best, &us, &launched)));
    MGE_LAUNCHED(ctx, launched);
    ctune = best;
    tune_store(ctx, key, TuneEntry{best.budget, best.prefetch, us});
    return MGE_OK;
  }

  // shared memory of the Gram epilogue (row-group stage, column-sum stage, FP64 partials)
  size_t gram_epi_bytes(int nl, int n1, int n2, bool sym2, bool csum) const {
    int bl = nl * M / 4;
    int nblk = bl * (n1 * M / 4) + (sym2 ? bl * (bl + 1) / 2 : bl * (n2 * M / 4));
    int rs = std::max(1, kThreads / nblk);
    size_t len = (size_t)nblk * 16;
    return (((rs * len + kThreads) * sizeof(T) + 15) / 16) * 16 + (len + (csum ? (size_t)n2 * M : 0)) * sizeof(double);
  }

  void launch_gram(int nl, const T* const* L, int n1, const T* const* R1, int n2, const T* const* R2,
                   bool sym2, bool weighted, double* out1, double* out2, int ld2, int stride2, bool csum) {
    GramArgs<T> g{};
    g.n = n; g.nl = nl; g.n1 = n1; g.n2 = n2;
    g.sym2 = sym2;
    g.b = weighted ? static_cast<const T*>(op.b) : nullptr;
    g.out1 = out1; g.out2 = out2; g.ld2 = ld2; g.stride2 = stride2;
    g.csum = csum ? &sm->partC[0][0] : nullptr;
    g.st = state;
    auto source = [&g](const T* p) {
      for (int i = 0; i < g.nsrc; ++i)
        if (g.src[i] == p) return i;
      g.src[g.nsrc] = p;
      return g.nsrc++;
    };
    for (int i = 0; i < nl; ++i) g.lmap[i] = source(L[i]);
    for (int i = 0; i < n1; ++i) g.r1map[i] = source(R1[i]);
    if (!sym2)
      for (int i = 0; i < n2; ++i) g.r2map[i] = source(R2[i]);
    auto stage_bytes = [&](int tr) {
      size_t b = (size_t)g.nsrc * tr * M * sizeof(T) + (weighted ? ((tr * sizeof(T) + 15) / 16) * 16 : 0);
      return ((b + 127) / 128) * 128;
    };
    int tr = 64;
    while (tr > 16 && stage_bytes(tr) > 24576) tr /= 2;
    g.tr = tr;
    g.stage_bytes = (uint32_t)stage_bytes(tr);
    int64_t per = (n + grid_gram - 1) / grid_gram;
    g.per = ((per + tr - 1) / tr) * tr;
    size_t smem = 128 + std::max((size_t)kGramStages * g.stage_bytes, gram_epi_bytes(nl, n1, n2, sym2, csum));
    k_gram<T, M><<<grid_gram, kThreads, smem, st>>>(g);
    MGE_LAUNCHED(ctx, 1);
  }

  // algorithmic bytes of one SpMM launch: A's column indices and values, the row pointers,
  // the gathered block once, the projection blocks read, W and AW written
  uint64_t spmm_bytes(bool hx, bool hp) const {
    uint64_t blk = (uint64_t)n * M * sizeof(T);
    uint64_t b = (uint64_t)nnz_a * (4 + sizeof(T)) + (uint64_t)(n + 1) * 8 + blk + 2 * blk;
    if (hx) b += 2 * blk;
    if (hp) b += 2 * blk;
    return b;
  }

  // algorithmic bytes of one Chebyshev step: the operator's indices, values and row
  // pointers, the gathered iterate once, R, d and D^-1 read, d and the next iterate written
  // (BF16 form: x, R, d and d_out in 2-byte storage; x_out in T on the last step)
  uint64_t cheb_bytes(bool last = false) const {
    const uint64_t s = pc_bf16 ? 2 : sizeof(T), so = (pc_bf16 && !last) ? 2 : sizeof(T);
    const uint64_t nm = (uint64_t)n * M;
    return (uint64_t)nnz_pc * (4 + sizeof(T)) + (uint64_t)(n + 1) * 8 + nm * (4 * s + so) +
           (uint64_t)n * sizeof(T);
  }

  // CUDA-event timing of the SpMM launches (ctx->timing): inside a stream capture the
  // records become external event nodes of the graph
  cudaEvent_t tev1 = nullptr;
  bool tcap = false;
  mge_status time_begin(uint64_t bytes) {
    if (ctx->ev_used >= ctx->ev_pool.size()) {
      cudaEvent_t x, y;
      MGE_CUDA(ctx, cudaEventCreate(&x));
      MGE_CUDA(ctx, cudaEventCreate(&y));
      ctx->ev_pool.push_back({x, y});
    }
    cudaEvent_t e0 = ctx->ev_pool[ctx->ev_used].first;
    tev1 = ctx->ev_pool[ctx->ev_used].second;
    ctx->ev_used++;
    ctx->ev_bytes.push_back(bytes);
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    MGE_CUDA(ctx, cudaStreamIsCapturing(st, &cap));
    tcap = cap == cudaStreamCaptureStatusActive;
    if (tcap) MGE_CUDA(ctx, cudaEventRecordWithFlags(e0, st, cudaEventRecordExternal));
    else MGE_CUDA(ctx, cudaEventRecord(e0, st));
    return MGE_OK;
  }
  mge_status time_end() {
    if (tcap) MGE_CUDA(ctx, cudaEventRecordWithFlags(tev1, st, cudaEventRecordExternal));
    else MGE_CUDA(ctx, cudaEventRecord(tev1, st));
    return MGE_OK;
  }

  mge_status launch_spmm(bool hx, bool hp, bool timed) {
    SpmmArgs<T> s{};
    s.n = n; s.ptr = op.ptr; s.col = op.col; s.val = static_cast<const T*>(op.val);
    s.shift = (T)op.shift;
    s.Wr = wsrc;
    s.X = hx ? X.p : nullptr; s.AX = hx ? AX.p : nullptr;
    s.P = hp ? P.p : nullptr; s.AP = hp ? AP.p : nullptr;
    s.sm = smt;
    s.W = W.p; s.AW = AW.p;
    s.st = state;
    if (timed) MGE_TRY(time_begin(spmm_bytes(hx, hp)));
    spmm_launch<T, M>(ctx, st, s, false);      // the fused epilogue runs in the long variant
    MGE_LAUNCHED(ctx, 1);
    if (timed) MGE_TRY(time_end());
    return MGE_OK;
  }

  void launch_rr_(int nb, int nx) {
    RRArgs r{};
    r.sm = sm; r.smt = smt; r.is_double = sizeof(T) == 8; r.ncl = gram_ncl;
    r.M = M; r.nb = nb; r.nx = nx; r.tau = tau; r.tau_p = tau_p; r.st = state;
    r.sel = rr_auto ? RR_FP32 : RR_ALWAYS;
    launch_rr(st, r, inverse_rr);
    MGE_LAUNCHED(ctx, 1);
    if (rr_auto) {
      r.sel = RR_FP64;
      launch_rr(st, r, false);
      MGE_LAUNCHED(ctx, 1);
    }
  }

  void launch_update(int nb, bool init, bool produce_p) {
    UpdArgs<T> u{};
    u.n = n; u.nb = nb;
    if (init) { u.S[0] = W.p; u.AS[0] = AW.p; }
    else {
      u.S[0] = X.p; u.AS[0] = AX.p;
      u.S[1] = W.p; u.AS[1] = AW.p;
      u.S[2] = P.p; u.AS[2] = AP.p;
    }
    u.Xo = X.p; u.AXo = AX.p; u.Po = P.p; u.APo = AP.p;
    u.produce_p = produce_p;
    u.smt = smt;
    u.b = static_cast<const T*>(op.b);
    // the residual is scaled by the diagonal of the operator the preconditioner applies
    u.dinv = static_cast<const T*>(op.pc_ptr ? op.pc_dinv : op.dinv);
    u.Wr = Wr.p;
    u.WrB = pc_bf16 ? WrB.p : nullptr;
    u.partN = &sm->partN[0][0];
    u.st = state;
    if (nb == 1) k_update<T, M, 1><<<grid_upd, kThreads, 0, st>>>(u);
    else if (nb == 2) k_update<T, M, 2><<<grid_upd, kThreads, 0, st>>>(u);
    else k_update<T, M, 3><<<grid_upd, kThreads, 0, st>>>(u);
    MGE_LAUNCHED(ctx, 1);
  }

  // W_raw <- p(D^-1 A) D^-1 R: cheb_deg - 1 steps of the Chebyshev iteration for A y = R with
  // y_0 = 0 (Saad, Iterative Methods for Sparse Linear Systems, Alg. 12.1), each one SpMM
  mge_status launch_cheb(bool timed) {
    wsrc = Wr.p;
    if (cheb_deg <= 1) return MGE_OK;
    if constexpr (sizeof(T) == 4) {
      if (pc_bf16) return launch_cheb_bf16(timed);
    }
    T* ys[2] = {Yc0.p, Yc1.p};
    double rho_prev = 1.0 / ch_sigma;
    for (int k = 1; k < cheb_deg; ++k) {
      const double rho = 1.0 / (2.0 * ch_sigma - rho_prev);
      if (op.sl_slp) {
        // the sliced copy of the operator (rows sorted and padded per slice)
        ChebArgs<T> c{};
        c.n = n;
        c.slp = op.sl_slp; c.perm = op.sl_perm; c.col = op.sl_col;
        c.val = static_cast<const T*>(op.sl_val);
        c.shift = (T)(op.pc_ptr ? op.pc_shift : op.shift);
        c.X = (k == 1) ? Wr.p : ys[k % 2];
        c.R = Wr.p;
        c.D = (k == 1) ? Wr.p : Dc.p;
        c.dinv = static_cast<const T*>(op.pc_ptr ? op.pc_dinv : op.dinv);
        c.Dout = Dc.p;
        c.Xout = ys[(k + 1) % 2];
        c.sy = (k == 1) ? (T)(1.0 / ch_theta) : T(1);
        c.sd = (k == 1) ? (T)(1.0 / ch_theta) : T(1);
        c.c1 = (T)(rho * rho_prev);
        c.c2 = (T)(2.0 * rho / ch_delta);
        c.st = state;
        if (timed) MGE_TRY(time_begin(cheb_bytes()));
        MGE_CUDA(ctx, (cheb_launch<T, T, T, M>(ctx, st, c, op.sl_max_tile_slots, ctune)));
        MGE_LAUNCHED(ctx, 1);
        if (timed) MGE_TRY(time_end());
        rho_prev = rho;
        continue;
      }
      SpmmArgs<T> s{};
      s.n = n;
      if (op.pc_ptr) {
        s.ptr = op.pc_ptr; s.col = op.pc_col; s.val = static_cast<const T*>(op.pc_val);
        s.shift = (T)op.pc_shift;
      } else {
        s.ptr = op.ptr; s.col = op.col; s.val = static_cast<const T*>(op.val);
        s.shift = (T)op.shift;
      }
      s.Wr = (k == 1) ? Wr.p : ys[k % 2];                 // x_k (x_1 = R / theta)
      s.sm = nullptr; s.W = nullptr; s.AW = nullptr;
      s.st = state;
        s.cheb = 1;
      s.cr = Wr.p;
      s.cd = (k == 1) ? Wr.p : Dc.p;                      // d_0 = R / theta
      s.cdinv = static_cast<const T*>(op.pc_ptr ? op.pc_dinv : op.dinv);
      s.cd_out = Dc.p;
      s.cx_out = ys[(k + 1) % 2];
      s.sy = (k == 1) ? (T)(1.0 / ch_theta) : T(1);
      s.sd = (k == 1) ? (T)(1.0 / ch_theta) : T(1);
      s.c1 = (T)(rho * rho_prev);
      s.c2 = (T)(2.0 * rho / ch_delta);
      if (timed) MGE_TRY(time_begin(cheb_bytes()));
      spmm_launch<T, M>(ctx, st, s, spmm_short<M>(nnz_pc, n));
      MGE_LAUNCHED(ctx, 1);
      if (timed) MGE_TRY(time_end());
      rho_prev = rho;
    }
    wsrc = ys[cheb_deg % 2];
    return MGE_OK;
  }

  // The same steps with the right-hand side, iterates and corrections in BF16 (written by
  // k_update and the steps themselves); the last step writes the preconditioned block to Wr.
  mge_status launch_cheb_bf16(bool timed) {
    __nv_bfloat16* yb[2] = {Yb0.p, Yb1.p};
    double rho_prev = 1.0 / ch_sigma;
    for (int k = 1; k < cheb_deg; ++k) {
      const double rho = 1.0 / (2.0 * ch_sigma - rho_prev);
      const bool last = k == cheb_deg - 1;
      ChebArgs<T> c{};
      c.n = n;
      c.slp = op.sl_slp; c.perm = op.sl_perm; c.col = op.sl_col;
      c.val = static_cast<const T*>(op.sl_val);
      c.shift = (T)(op.pc_ptr ? op.pc_shift : op.shift);
      c.X = (k == 1) ? (const void*)WrB.p : (const void*)yb[k % 2];
      c.R = WrB.p;
      c.D = (k == 1) ? (const void*)WrB.p : (const void*)Db.p;
      c.dinv = static_cast<const T*>(op.pc_ptr ? op.pc_dinv : op.dinv);
      c.Dout = Db.p;
      c.Xout = last ? (void*)Wr.p : (void*)yb[(k + 1) % 2];
      c.sy = (k == 1) ? (T)(1.0 / ch_theta) : T(1);
      c.sd = (k == 1) ? (T)(1.0 / ch_theta) : T(1);
      c.c1 = (T)(rho * rho_prev);
      c.c2 = (T)(2.0 * rho / ch_delta);
      c.st = state;
      if (timed) MGE_TRY(time_begin(cheb_bytes(last)));
      if (last) MGE_CUDA(ctx, (cheb_launch<float, __nv_bfloat16, float, M>(ctx, st, c, op.sl_max_tile_slots)));
      else MGE_CUDA(ctx, (cheb_launch<float, __nv_bfloat16, __nv_bfloat16, M>(ctx, st, c, op.sl_max_tile_slots)));
      MGE_LAUNCHED(ctx, 1);
      if (timed) MGE_TRY(time_end());
      rho_prev = rho;
    }
    wsrc = Wr.p;
    return MGE_OK;
  }

  void launch_wprep_(bool hx, bool hp, bool check) {
    WprepArgs w{};
    w.sm = sm; w.smt = smt; w.is_double = sizeof(T) == 8;
    w.ncl_w = 1; w.ncl_n = 1;
    w.M = M; w.K = K; w.has_x = hx; w.has_p = hp; w.check = check;
    w.deflate = op.deflate; w.n = n; w.tol = tol; w.norm = op.norm; w.bmax = op.bmax;
    w.tau_w = tau_w; w.maxiter = maxiter; w.st = state;
    if (rr_auto) {
      // the FP64 launch first: a switch made by the FP32 launch takes effect next iteration
      w.sel = RR_FP64; w.rr_switch = 0;
      launch_wprep(st, w, true);
      w.sel = RR_FP32; w.rr_switch = 1;
      launch_wprep(st, w, false);
      MGE_LAUNCHED(ctx, 2);
    } else {
      w.sel = RR_ALWAYS; w.rr_switch = 0;
      launch_wprep(st, w, sizeof(T) == 8 || op.rr_fp64);
      MGE_LAUNCHED(ctx, 1);
    }
  }

  void launch_gram_w(bool hx, bool hp) {
    const T* L[3];
    int nl = 0;
    if (hx) L[nl++] = X.p;
    if (hp) L[nl++] = P.p;
    L[nl++] = wsrc;
    const T* R2[1] = {wsrc};
    launch_gram(nl, L, 0, nullptr, 1, R2, false, op.b != nullptr, nullptr, &sm->partW[0][0], MAXM,
                MAXS * MAXM, op.deflate);
  }

  // S-side Grams on the tensor cores (gram_tc.cu) for FP32 blocks of width 12, 16, 24 with the
  // full basis [X W P], on graphs of at least kTcMinRows rows: the kernel holds one CTA per SM
  // with ~150-190 KB of shared memory, which on small graphs costs more than it saves and, in
  // a batch of small solves, keeps the other solves' kernels off the SMs (measured on 512
  // graphs of 2k-50k nodes: 5.4M node-embeddings/s with it against 6.8M without)
  static constexpr bool kTcWidth = sizeof(T) == 4 && (M == 12 || M == 16 || M == 24);
  static constexpr int64_t kTcMinRows = 65536;
  int gram_ncl = 1;
  bool use_tc_gram() const { return kTcWidth && !op.gram_cuda_cores && n >= kTcMinRows; }

  mge_status launch_gram_s_tc() {
    if constexpr (kTcWidth) {
      GramTcArgs g{};
      g.n = n;
      g.S[0] = X.p; g.S[1] = W.p; g.S[2] = P.p;
      g.AS[0] = AX.p; g.AS[1] = AW.p; g.AS[2] = AP.p;
      g.b = static_cast<const float*>(op.b);
      g.outA = &sm->partA[0][0];
      g.outB = &sm->partB[0][0];
      g.st = state;
      MGE_CUDA(ctx, gram_tc_launch<M>(ctx, st, g, gram_tc_clusters<M>(ctx, n)));
      MGE_LAUNCHED(ctx, 1);
    }
    return MGE_OK;
  }

  mge_status launch_gram_s(int nb) {
    gram_ncl = 1;
    if (nb == 3 && use_tc_gram()) return launch_gram_s_tc();
    const T* L[3] = {X.p, W.p, P.p};
    const T* R[3] = {AX.p, AW.p, AP.p};
    if (nb == 1) { L[0] = W.p; R[0] = AW.p; }
    launch_gram(nb, L, nb, R, nb, L, true, op.b != nullptr, &sm->partA[0][0], &sm->partB[0][0], MAXS,
                MAXS * MAXS, false);
    return MGE_OK;
  }

  mge_status iteration(int nb, bool timed) {
    bool hp = nb == 3;
    MGE_TRY(launch_spmm(true, hp, timed));
    MGE_TRY(launch_gram_s(nb));
    launch_rr_(nb, M);
    launch_update(nb, false, true);
    MGE_TRY(launch_cheb(timed));
    launch_gram_w(true, true);
    launch_wprep_(true, true, true);
    return MGE_OK;
  }

  // the initial block (W_raw = X0, normalised, Rayleigh-Ritz on span(W)) and the first
  // iteration, S = [X W]
  mge_status prologue(uint64_t seed, const double* x0, int x0_cols, bool timed) {
    k_init_block<T><<<gridn(n * M, 256), 256, 0, st>>>(n, M, seed, x0, x0_cols, op.row_order, Wr.p);
    MGE_LAUNCHED(ctx, 1);
    wsrc = Wr.p;
    launch_gram_w(false, false);
    launch_wprep_(false, false, false);
    MGE_TRY(launch_spmm(false, false, timed));
    MGE_TRY(launch_gram_s(1));
    launch_rr_(1, 0);
    launch_update(1, true, false);
    MGE_TRY(launch_cheb(timed));
    launch_gram_w(true, false);
    launch_wprep_(true, false, true);
    MGE_TRY(launch_spmm(true, false, timed));
    MGE_TRY(launch_gram_s(2));
    launch_rr_(2, M);
    launch_update(2, false, true);
    MGE_TRY(launch_cheb(timed));
    launch_gram_w(true, true);
    launch_wprep_(true, true, true);
    return MGE_OK;
  }

  // Appends this solve to `graph`: the prologue (initial block and first iteration) as a
  // child graph, then a conditional while node whose body is one iteration ending in a
  // one-thread kernel that sets the loop condition from the device status word.  The new
  // nodes depend on nothing else in `graph`.  per_pass receives the body's kernel launches.
  mge_status add_loop(cudaGraph_t graph, uint64_t seed, const double* x0, int x0_cols, uint64_t* per_pass) {
    cudaGraph_t pro = nullptr;
    MGE_CUDA(ctx, cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    mge_status cap = prologue(seed, x0, x0_cols, false);
    cudaError_t ce = cudaStreamEndCapture(st, &pro);
    if (cap != MGE_OK) { if (pro) cudaGraphDestroy(pro); return cap; }
    if (ce != cudaSuccess) { set_error(ctx, "graph capture failed: %s", cudaGetErrorString(ce)); return MGE_EDEVICE; }
    cudaGraphNode_t npro = nullptr, nloop = nullptr;
    cudaError_t e1c = cudaGraphAddChildGraphNode(&npro, graph, nullptr, 0, pro);
    cudaGraphDestroy(pro);                      // the node holds its own copy
    MGE_CUDA(ctx, e1c);
    cudaGraphConditionalHandle h;
    MGE_CUDA(ctx, cudaGraphConditionalHandleCreate(&h, graph, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    MGE_CUDA(ctx, cudaGraphAddNode(&nloop, graph, &npro, nullptr, 1, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    MGE_CUDA(ctx, cudaStreamBeginCaptureToGraph(st, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    const uint64_t before = ctx->kernel_launches;
    cap = iteration(3, false);
    if (cap == MGE_OK) {
      k_loop_cond<<<1, 32, 0, st>>>(h, state, maxiter);
      MGE_LAUNCHED(ctx, 1);
    }
    cudaGraph_t body_out = nullptr;
    ce = cudaStreamEndCapture(st, &body_out);
    *per_pass = ctx->kernel_launches - before;
    ctx->kernel_launches = before;
    if (cap != MGE_OK) return cap;
    if (ce != cudaSuccess) {
      set_error(ctx, "graph capture failed: %s", cudaGetErrorString(ce));
      return MGE_EDEVICE;
    }
    return MGE_OK;
  }

  // After the solve has run: the status from the host copy of the device status word, the
  // eigenvalues and backward errors, and (V_out not NULL) the sign-fixed vectors written in
  // the caller's node order, launched on the solver's stream.
  mge_status finish_result(const State* hst, mge_status* status, double* V_out, LobResult* res) {
    if (hst->done == DONE_ERROR) {
      *status = (mge_status)hst->err;
      set_error(ctx, "LOBPCG stopped at iteration %d: %s (stage %d, kept %d)", hst->iter,
                mge_strerror(*status), hst->bad_stage, hst->kept);
    } else if (hst->done == DONE_MAXITER || hst->done == DONE_RUNNING) {
      *status = MGE_ENOTCONVERGED;
    } else if (hst->done == DONE_STALLED) {
      *status = MGE_ENOTCONVERGED;
      set_error(ctx, "LOBPCG stagnated at iteration %d (basis of %d directions, fewer than m): the "
                "tolerance is below what the block precision reaches; current pairs returned",
                hst->iter, hst->kept);
    }
    if (getenv("MGE_PHASES")) {
      fprintf(stderr, "[mge] n=%lld M=%d iters=%d rr_clk:", (long long)n, M, hst->iter);
      for (int i = 0; i < 12; ++i) fprintf(stderr, " %lld", hst->rr_clk[i]);
      fprintf(stderr, " | wprep_clk:");
      for (int i = 0; i < 4; ++i) fprintf(stderr, " %lld", hst->wp_clk[i]);
      fprintf(stderr, "\n");
    }
    res->iters = hst->iter;
    res->drops = hst->drops;
    res->rr64_from = op.rr_fp64 || sizeof(T) == 8 || !inverse_rr ? 0 : hst->rr64 ? hst->rr64_iter : -1;
    res->lambda.assign(hst->lambda, hst->lambda + K);
    res->eta.assign(hst->eta, hst->eta + K);
    if (V_out && (*status == MGE_OK || *status == MGE_ENOTCONVERGED)) {
      MGE_CUDA(ctx, cudaMemsetAsync(sm->vmax, 0, sizeof(sm->vmax), st));
      MGE_CUDA(ctx, cudaMemsetAsync(sm->vidx, 0xff, sizeof(sm->vidx), st));
      k_vmax<T><<<gridn(n * K, 256), 256, 0, st>>>(n, M, K, X.p, sm->vmax);
      k_vidx<T><<<gridn(n * K, 256), 256, 0, st>>>(n, M, K, X.p, sm->vmax, op.row_order, sm->vidx);
      k_write_v<T><<<gridn(n * K, 256), 256, 0, st>>>(n, M, K, X.p, sm->vidx, op.row_order, op.row_rank, V_out);
      MGE_LAUNCHED(ctx, 3);
      MGE_CUDA(ctx, cudaGetLastError());
    }
    return MGE_OK;
  }

  mge_status run(int check_every, bool use_graph, uint64_t seed, const double* x0, int x0_cols,
                 double* V_out, LobResult* res) {
    cudaEvent_t e0, e1;
    MGE_CUDA(ctx, cudaEventCreate(&e0));
    MGE_CUDA(ctx, cudaEventCreate(&e1));
    MGE_CUDA(ctx, cudaEventRecord(e0, st));
    const bool timed = ctx->timing;
    bool graph_ok = use_graph;
    if (graph_ok) {
      cudaStreamCaptureStatus cs;
      MGE_CUDA(ctx, cudaStreamIsCapturing(st, &cs));
      if (cs != cudaStreamCaptureStatusNone) graph_ok = false;
    }
    // Without per-launch events (which a graph loop cannot hold) the whole solve is one graph:
    // the prologue, then a conditional (while) node whose body is one iteration and ends with
    // a kernel that decides on the device whether to run another pass.
    const bool loop_graph = graph_ok && !timed;
    cudaGraphExec_t gexec = nullptr;
    cudaGraph_t graph = nullptr;
    uint64_t per_pass = 0;
    if (loop_graph) {
      MGE_CUDA(ctx, cudaGraphCreate(&graph, 0));
      const mge_status ag = add_loop(graph, seed, x0, x0_cols, &per_pass);
      if (ag != MGE_OK) { cudaGraphDestroy(graph); return ag; }
      MGE_CUDA(ctx, cudaGraphInstantiate(&gexec, graph, 0));
      MGE_CUDA(ctx, cudaGraphLaunch(gexec, st));
    } else {
      MGE_TRY(prologue(seed, x0, x0_cols, timed));
    }
    MGE_CUDA(ctx, cudaGetLastError());
    State* hst = nullptr;
    {
      // a pinned status buffer from the context's free list (pinned allocation is slow)
      std::lock_guard<std::mutex> lock(ctx->state_mu);
      if (!ctx->state_host.empty()) {
        hst = static_cast<State*>(ctx->state_host.back());
        ctx->state_host.pop_back();
      }
    }
    if (!hst) MGE_CUDA(ctx, cudaMallocHost(&hst, sizeof(State)));
    mge_status status = MGE_OK;
    if (check_every < 1) check_every = 1;
    auto finish_timing = [&]() -> mge_status {
      if (!timed) return MGE_OK;
      MGE_CUDA(ctx, cudaStreamSynchronize(st));
      for (size_t i = 0; i < ctx->ev_used; ++i) {
        float ms = 0;
        if (cudaEventElapsedTime(&ms, ctx->ev_pool[i].first, ctx->ev_pool[i].second) == cudaSuccess) {
          ctx->spmm_ms += ms;
          ctx->spmm_launches += 1;
          ctx->spmm_bytes += ctx->ev_bytes[i];
        }
      }
      ctx->ev_used = 0;
      ctx->ev_bytes.clear();
      return MGE_OK;
    };
    MGE_TRY(finish_timing());
    if (graph_ok && !loop_graph) {
      MGE_CUDA(ctx, cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
      uint64_t before = ctx->kernel_launches;
      mge_status cap = MGE_OK;
      for (int i = 0; i < check_every && cap == MGE_OK; ++i) cap = iteration(3, timed && i == 0);
      cudaError_t ce = cudaStreamEndCapture(st, &graph);
      if (cap != MGE_OK) return cap;
      if (ce != cudaSuccess) { set_error(ctx, "graph capture failed: %s", cudaGetErrorString(ce)); return MGE_EDEVICE; }
      ctx->kernel_launches = before;
      MGE_CUDA(ctx, cudaGraphInstantiate(&gexec, graph, 0));
      if (timed) { cap_bytes = ctx->ev_bytes; ctx->ev_used = 0; ctx->ev_bytes.clear(); }
    }
    const uint64_t per_chunk = (uint64_t)check_every * (6 + (cheb_deg - 1) + (rr_auto ? 2 : 0));
    for (;;) {
      MGE_CUDA(ctx, cudaMemcpyAsync(hst, state, sizeof(State), cudaMemcpyDeviceToHost, st));
      MGE_CUDA(ctx, cudaStreamSynchronize(st));
      if (loop_graph) {
        ctx->kernel_launches += per_pass * (uint64_t)hst->loops;
        break;
      }
      if (hst->done != DONE_RUNNING) break;
      if (graph_ok) {
        if (timed) {
          // the events recorded in the first captured iteration fire on every launch
          ctx->ev_used = cap_bytes.size();
          ctx->ev_bytes = cap_bytes;
        }
        MGE_CUDA(ctx, cudaGraphLaunch(gexec, st));
        ctx->kernel_launches += per_chunk;
        MGE_TRY(finish_timing());
      } else {
        for (int i = 0; i < check_every; ++i) MGE_TRY(iteration(3, timed));
        MGE_CUDA(ctx, cudaGetLastError());
        MGE_TRY(finish_timing());
      }
    }
    if (gexec) cudaGraphExecDestroy(gexec);
    if (graph) cudaGraphDestroy(graph);
    MGE_CUDA(ctx, cudaEventRecord(e1, st));
    MGE_TRY(finish_result(hst, &status, V_out, res));
    MGE_CUDA(ctx, cudaStreamSynchronize(st));
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    res->ms = ms;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    {
      std::lock_guard<std::mutex> lock(ctx->state_mu);
      ctx->state_host.push_back(hst);
    }
    res->status = status;
    return status;
  }
};

// Buffers, the operators' entry counts and the kernels' shared-memory limits of one solve
template <typename T, int M>
mge_status prepare_solver(Solver<T, M>& s) {
  Ctx* ctx = s.ctx;
  cudaStream_t st = s.st;
  const LobOp& op = s.op;
  MGE_TRY(s.setup());
  // entry counts from the host copy when the caller has them (no device round trip, so that a
  // batch can prepare its next solves while earlier ones run)
  int64_t nnz = op.nnz;
  if (nnz < 0) {
    MGE_CUDA(ctx, cudaMemcpyAsync(&nnz, op.ptr + op.n, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    MGE_CUDA(ctx, cudaStreamSynchronize(st));
  }
  s.nnz_a = nnz;
  s.nnz_pc = nnz;
  if (op.pc_ptr) {
    s.nnz_pc = op.pc_nnz;
    if (s.nnz_pc < 0) {
      MGE_CUDA(ctx, cudaMemcpyAsync(&s.nnz_pc, op.pc_ptr + op.n, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
      MGE_CUDA(ctx, cudaStreamSynchronize(st));
    }
  }
  MGE_CUDA(ctx, cudaFuncSetAttribute(k_gram<T, M>, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024));
  MGE_CUDA(ctx, (spmm_configure<T, M>()));
  MGE_CUDA(ctx, (cheb_configure<T, T, T, M>()));
  if constexpr (Solver<T, M>::kTcWidth) {
    if (s.use_tc_gram()) MGE_CUDA(ctx, gram_tc_configure<M>());
  }
  if constexpr (sizeof(T) == 4) {
    if (s.pc_bf16) {
      MGE_CUDA(ctx, (cheb_configure<float, __nv_bfloat16, __nv_bfloat16, M>()));
      MGE_CUDA(ctx, (cheb_configure<float, __nv_bfloat16, float, M>()));
    }
  }
  MGE_CUDA(ctx, rr_configure());
  MGE_TRY(s.tune_cheb());
  return MGE_OK;
}

template <typename T, int M>
mge_status solve_m(Ctx* ctx, cudaStream_t st, const LobOp& op, int K, double tol, int maxiter, uint64_t seed,
                   int check_every, bool use_graph, const double* x0, int x0_cols, double* V_out,
                   LobResult* res) {
  Solver<T, M> s(ctx, st, op, K);
  s.tol = tol;
  s.maxiter = maxiter;
  MGE_TRY(prepare_solver(s));
  return s.run(check_every, use_graph, seed, x0, x0_cols, V_out, res);
}

// One solve of a batch (solves of several widths and precisions share one graph)
struct BatchItem {
  virtual ~BatchItem() {}
  virtual mge_status prepare() = 0;
  virtual mge_status add(cudaGraph_t g, uint64_t seed) = 0;
  virtual const State* device_state() const = 0;
  virtual mge_status finish(const State* hst, mge_status* status, double* V_out, LobResult* res) = 0;
  uint64_t per_pass = 0;
};

template <typename T, int M>
struct BatchItemT : BatchItem {
  Solver<T, M> s;
  BatchItemT(Ctx* c, cudaStream_t st, const LobOp& op, int K, double tol, int maxiter) : s(c, st, op, K) {
    s.tol = tol;
    s.maxiter = maxiter;
  }
  mge_status prepare() override { return prepare_solver(s); }
  mge_status add(cudaGraph_t g, uint64_t seed) override { return s.add_loop(g, seed, nullptr, 0, &per_pass); }
  const State* device_state() const override { return s.state; }
  mge_status finish(const State* hst, mge_status* status, double* V_out, LobResult* res) override {
    return s.finish_result(hst, status, V_out, res);
  }
};

template <typename T>
BatchItem* make_batch_item_t(Ctx* ctx, cudaStream_t st, const LobOp& op, int K, int m, double tol, int maxiter) {
  switch (m) {
    case 4: return new BatchItemT<T, 4>(ctx, st, op, K, tol, maxiter);
    case 8: return new BatchItemT<T, 8>(ctx, st, op, K, tol, maxiter);
    case 12: return new BatchItemT<T, 12>(ctx, st, op, K, tol, maxiter);
    case 16: return new BatchItemT<T, 16>(ctx, st, op, K, tol, maxiter);
    case 24: return new BatchItemT<T, 24>(ctx, st, op, K, tol, maxiter);
    default: return nullptr;
  }
}

template <typename T>
mge_status solve_t(Ctx* ctx, cudaStream_t st, const LobOp& op, int K, int m, double tol, int maxiter,
                   uint64_t seed, int check_every, bool use_graph, const double* x0, int x0_cols,
                   double* V_out, LobResult* res) {
  switch (m) {
    case 4: return solve_m<T, 4>(ctx, st, op, K, tol, maxiter, seed, check_every, use_graph, x0, x0_cols, V_out, res);
    case 8: return solve_m<T, 8>(ctx, st, op, K, tol, maxiter, seed, check_every, use_graph, x0, x0_cols, V_out, res);
    case 12: return solve_m<T, 12>(ctx, st, op, K, tol, maxiter, seed, check_every, use_graph, x0, x0_cols, V_out, res);
    case 16: return solve_m<T, 16>(ctx, st, op, K, tol, maxiter, seed, check_every, use_graph, x0, x0_cols, V_out, res);
    case 24: return solve_m<T, 24>(ctx, st, op, K, tol, maxiter, seed, check_every, use_graph, x0, x0_cols, V_out, res);
    default:
      set_error(ctx, "unsupported block width %d", m);
      return MGE_EINVAL;
  }
}

template <typename T, int M>
mge_status apply_m(Ctx* ctx, cudaStream_t st, const LobOp& op, const void* X, void* Y, const int32_t* out_row) {
  SpmmArgs<T> s{};
  s.n = op.n; s.ptr = op.ptr; s.col = op.col; s.val = static_cast<const T*>(op.val);
  s.shift = (T)op.shift; s.Wr = static_cast<const T*>(X); s.AW = static_cast<T*>(Y);
  s.out_row = out_row;
  s.W = nullptr; s.sm = nullptr; s.st = nullptr;
  MGE_CUDA(ctx, (spmm_configure<T, M>()));
  int64_t nnz = 0;
  MGE_CUDA(ctx, cudaMemcpyAsync(&nnz, op.ptr + op.n, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  MGE_CUDA(ctx, cudaStreamSynchronize(st));
  spmm_launch<T, M>(ctx, st, s, spmm_short<M>(nnz, op.n));
  MGE_LAUNCHED(ctx, 1);
  MGE_CUDA(ctx, cudaGetLastError());
  return MGE_OK;
}

}  // namespace
}  // namespace lob

mge_status lobpcg_solve(Ctx* ctx, cudaStream_t st, const LobOp& op, int precision, int K, int m, double tol,
                        int maxiter, uint64_t seed, int check_every, bool use_graph, const double* x0_dev,
                        int x0_cols, double* V_out, LobResult* res) {
  using namespace lob;
  if (m > MAXM || m < 4) { set_error(ctx, "block width %d out of range", m); return MGE_EINVAL; }
  if (K < 1 || K > m) { set_error(ctx, "K = %d out of range for block width %d", K, m); return MGE_EINVAL; }
  if (op.n < 2 * m) { set_error(ctx, "n = %lld too small for block width %d", (long long)op.n, m); return MGE_EINVAL; }
  if (precision == MGE_FP64)
    return solve_t<double>(ctx, st, op, K, m, tol, maxiter, seed, check_every, use_graph, x0_dev, x0_cols, V_out, res);
  if (precision == MGE_FP32)
    return solve_t<float>(ctx, st, op, K, m, tol, maxiter, seed, check_every, use_graph, x0_dev, x0_cols, V_out, res);
  set_error(ctx, "precision %d not supported by the solver", precision);
  return MGE_EINVAL;
}

// Several solves in one CUDA graph: each solve is a branch of its own (prologue, then its
// conditional while loop) with no edge to the others, so one launch runs them side by side
// and each branch stops when its own solve has converged.
mge_status lobpcg_solve_batch(Ctx* ctx, cudaStream_t st, int count, const LobOp* ops, int precision, const int* K,
                              const int* m, double tol, int maxiter, uint64_t seed, double* const* V_out,
                              LobResult* res, mge_status* status, double* batch_ms) {
  using namespace lob;
  if (precision != MGE_FP64 && precision != MGE_FP32) {
    set_error(ctx, "precision %d not supported by the solver", precision);
    return MGE_EINVAL;
  }
  std::vector<std::unique_ptr<BatchItem>> items;
  items.reserve(count);
  for (int i = 0; i < count; ++i) {
    if (m[i] > MAXM || m[i] < 4) { set_error(ctx, "batch item %d: block width %d out of range", i, m[i]); return MGE_EINVAL; }
    if (K[i] < 1 || K[i] > m[i]) { set_error(ctx, "batch item %d: K = %d out of range", i, K[i]); return MGE_EINVAL; }
    if (ops[i].n < 2 * m[i]) {
      set_error(ctx, "batch item %d: n = %lld too small for block width %d", i, (long long)ops[i].n, m[i]);
      return MGE_EINVAL;
    }
    BatchItem* it = precision == MGE_FP64 ? make_batch_item_t<double>(ctx, st, ops[i], K[i], m[i], tol, maxiter)
                                          : make_batch_item_t<float>(ctx, st, ops[i], K[i], m[i], tol, maxiter);
    if (!it) { set_error(ctx, "batch item %d: unsupported block width %d", i, m[i]); return MGE_EINVAL; }
    items.emplace_back(it);
  }
  // The solves go out in chunks of kChunk: each chunk is prepared (allocations and set-up on
  // st, which nothing else uses meanwhile), captured as one graph with a branch per solve,
  // instantiated and launched on one of kLanes streams, so that the host work of the next chunk
  // overlaps the device work of the launched ones (instantiating one graph of hundreds of
  // solves took longer than much of their device time).
  constexpr int kChunk = 64, kLanes = 4;
  State* hst = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  mge_status out = MGE_OK;
  auto fail = [&](cudaError_t e, const char* what) {
    set_error(ctx, "%s: %s", what, cudaGetErrorString(e));
    out = MGE_EDEVICE;
  };
  cudaError_t e;
  std::vector<cudaStream_t> lanes;
  std::vector<cudaGraphExec_t> execs;
  std::vector<cudaEvent_t> evs;
  auto new_event = [&]() -> cudaEvent_t {
    cudaEvent_t ev = nullptr;
    if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess) { fail(e, "cudaEventCreate"); return nullptr; }
    evs.push_back(ev);
    return ev;
  };
  if ((e = cudaMallocHost(&hst, sizeof(State) * (size_t)count)) != cudaSuccess) fail(e, "cudaMallocHost");
  if (out == MGE_OK && (e = cudaEventCreate(&e0)) != cudaSuccess) fail(e, "cudaEventCreate");
  if (out == MGE_OK && (e = cudaEventCreate(&e1)) != cudaSuccess) fail(e, "cudaEventCreate");
  for (int l = 0; l < kLanes && out == MGE_OK; ++l) {
    cudaStream_t s = nullptr;
    if ((e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking)) != cudaSuccess) fail(e, "cudaStreamCreate");
    else lanes.push_back(s);
  }
  for (int c0 = 0, lane = 0; c0 < count && out == MGE_OK; c0 += kChunk, lane = (lane + 1) % kLanes) {
    const int c1 = std::min(count, c0 + kChunk);
    for (int i = c0; i < c1 && out == MGE_OK; ++i) {
      const mge_status p = items[i]->prepare();
      if (p != MGE_OK) out = p;
    }
    if (out != MGE_OK) break;
    cudaGraph_t graph = nullptr;
    if ((e = cudaGraphCreate(&graph, 0)) != cudaSuccess) { fail(e, "cudaGraphCreate"); break; }
    for (int i = c0; i < c1 && out == MGE_OK; ++i) {
      const mge_status a = items[i]->add(graph, seed);
      if (a != MGE_OK) out = a;
    }
    cudaGraphExec_t gexec = nullptr;
    if (out == MGE_OK && (e = cudaGraphInstantiate(&gexec, graph, 0)) != cudaSuccess) fail(e, "batch graph instantiation");
    cudaGraphDestroy(graph);
    if (out != MGE_OK) break;
    execs.push_back(gexec);
    // the chunk's buffers were allocated and set up on st
    if (c0 == 0 && (e = cudaEventRecord(e0, st)) != cudaSuccess) { fail(e, "cudaEventRecord"); break; }
    cudaEvent_t ready = new_event();
    if (!ready) break;
    if ((e = cudaEventRecord(ready, st)) != cudaSuccess) { fail(e, "cudaEventRecord"); break; }
    if ((e = cudaStreamWaitEvent(lanes[lane], ready, 0)) != cudaSuccess) { fail(e, "cudaStreamWaitEvent"); break; }
    if ((e = cudaGraphLaunch(gexec, lanes[lane])) != cudaSuccess) { fail(e, "cudaGraphLaunch"); break; }
  }
  // join the lanes back into st
  for (cudaStream_t s : lanes) {
    cudaEvent_t done = new_event();
    if (!done) break;
    if ((e = cudaEventRecord(done, s)) != cudaSuccess) { fail(e, "cudaEventRecord"); break; }
    if ((e = cudaStreamWaitEvent(st, done, 0)) != cudaSuccess) { fail(e, "cudaStreamWaitEvent"); break; }
  }
  if (out == MGE_OK && (e = cudaEventRecord(e1, st)) != cudaSuccess) fail(e, "cudaEventRecord");
  for (int i = 0; i < count && out == MGE_OK; ++i)
    if ((e = cudaMemcpyAsync(&hst[i], items[i]->device_state(), sizeof(State), cudaMemcpyDeviceToHost, st)) !=
        cudaSuccess)
      fail(e, "cudaMemcpyAsync");
  if (out == MGE_OK && (e = cudaStreamSynchronize(st)) != cudaSuccess) fail(e, "batch solve");
  if (out == MGE_OK) {
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    *batch_ms = ms;
    for (int i = 0; i < count; ++i) {
      ctx->kernel_launches += items[i]->per_pass * (uint64_t)hst[i].loops;
      status[i] = MGE_OK;
      const mge_status f = items[i]->finish(&hst[i], &status[i], V_out ? V_out[i] : nullptr, &res[i]);
      if (f != MGE_OK) status[i] = f;
      res[i].status = status[i];
      res[i].ms = ms;
    }
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) fail(e, "batch results");
  }
  for (cudaStream_t s : lanes) cudaStreamSynchronize(s);
  for (cudaGraphExec_t x : execs) cudaGraphExecDestroy(x);
  for (cudaStream_t s : lanes) cudaStreamDestroy(s);
  for (cudaEvent_t ev : evs) cudaEventDestroy(ev);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (hst) cudaFreeHost(hst);
  return out;
}

// Y = A X with X already in the library's node order; row r of the product goes to row
// out_row[r] of Y (NULL: row r)
mge_status apply_internal(Ctx* ctx, cudaStream_t st, const LobOp& op, int precision, int m, const void* X, void* Y,
                          const int32_t* out_row) {
  using namespace lob;
  if (precision == MGE_FP64) {
    switch (m) {
      case 4: return apply_m<double, 4>(ctx, st, op, X, Y, out_row);
      case 8: return apply_m<double, 8>(ctx, st, op, X, Y, out_row);
      case 12: return apply_m<double, 12>(ctx, st, op, X, Y, out_row);
      case 16: return apply_m<double, 16>(ctx, st, op, X, Y, out_row);
      case 24: return apply_m<double, 24>(ctx, st, op, X, Y, out_row);
    }
  } else if (precision == MGE_FP32) {
    switch (m) {
      case 4: return apply_m<float, 4>(ctx, st, op, X, Y, out_row);
      case 8: return apply_m<float, 8>(ctx, st, op, X, Y, out_row);
      case 12: return apply_m<float, 12>(ctx, st, op, X, Y, out_row);
      case 16: return apply_m<float, 16>(ctx, st, op, X, Y, out_row);
      case 24: return apply_m<float, 24>(ctx, st, op, X, Y, out_row);
    }
  }
  set_error(ctx, "unsupported precision %d / width %d for apply", precision, m);
  return MGE_EINVAL;
}

// rows of `vec` 16-byte vectors: dst row r = src row order[r]
__global__ void k_gather_rows(int64_t n, int vec, const int32_t* __restrict__ order, const uint4* __restrict__ src,
                              uint4* __restrict__ dst) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n * vec) return;
  const int64_t r = t / vec;
  dst[t] = src[(int64_t)order[r] * vec + (t % vec)];
}

mge_status spmm_apply(Ctx* ctx, cudaStream_t st, const LobOp& op, int precision, int m, const void* X, void* Y) {
  if (!op.row_order) return apply_internal(ctx, st, op, precision, m, X, Y, nullptr);
  // X into the library's node order, the product back into the caller's
  const size_t elem = precision == MGE_FP64 ? sizeof(double) : sizeof(float);
  const int vec = (int)((size_t)m * elem / 16);
  DevBuf<uint4> xi;
  MGE_TRY(xi.scratch(ctx, (size_t)op.n * vec, st));
  k_gather_rows<<<lob::gridn(op.n * vec, 256), 256, 0, st>>>(op.n, vec, op.row_order, static_cast<const uint4*>(X), xi.p);
  MGE_LAUNCHED(ctx, 1);
  MGE_CUDA(ctx, cudaGetLastError());
  MGE_TRY(apply_internal(ctx, st, op, precision, m, xi.p, Y, op.row_order));
  MGE_CUDA(ctx, cudaStreamSynchronize(st));     // xi is freed on return
  return MGE_OK;
}

// ---------------------------------------------------------------------------------------
// In-place apply that allocates nothing.  The SpMM reads the rows of X at a row's
// neighbours while it writes that row of Y, so Y = A Y needs a copy of the block; the copy
// goes into one fixed device array that every call on the device shares.  Nothing in the
// array has to start at zero: each call overwrites the bytes it reads before reading them.
// Two calls whose copies or kernels overlap in time (several host threads, or streams the
// caller does not order) race on the array.
// ---------------------------------------------------------------------------------------
constexpr size_t kInplaceScratchBytes = size_t(32) << 20;      // 32 MiB per device
static __device__ __align__(256) unsigned char g_inplace_scratch[kInplaceScratchBytes];

namespace {
constexpr int kInplaceMaxDevices = 64;
std::mutex g_inplace_mu;
void* g_inplace_addr[kInplaceMaxDevices] = {};
}  // namespace

size_t inplace_scratch_bytes() { return kInplaceScratchBytes; }

mge_status spmm_apply_inplace(Ctx* ctx, cudaStream_t st, const LobOp& op, int precision, int m, void* XY) {
  const size_t elem = precision == MGE_FP64 ? sizeof(double) : sizeof(float);
  const size_t bytes = (size_t)op.n * (size_t)m * elem;
  if (bytes > kInplaceScratchBytes) {
    set_error(ctx, "apply_inplace: the block (%lld x %d, %zu bytes) exceeds the fixed %zu-byte scratch",
              (long long)op.n, m, bytes, kInplaceScratchBytes);
    return MGE_EINVAL;
  }
  if (ctx->device < 0 || ctx->device >= kInplaceMaxDevices) {
    set_error(ctx, "apply_inplace: device ordinal %d out of range", ctx->device);
    return MGE_EINVAL;
  }
  void* scratch = nullptr;
  {
    // set-up, once per device, with that device current (the caller made it current)
    std::lock_guard<std::mutex> lock(g_inplace_mu);
    if (!g_inplace_addr[ctx->device]) {
      void* p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, g_inplace_scratch);
      if (e != cudaSuccess || !p) {
        set_error(ctx, "apply_inplace: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
        return MGE_EDEVICE;
      }
      g_inplace_addr[ctx->device] = p;
    }
    scratch = g_inplace_addr[ctx->device];
  }
  if (op.row_order) {
    // the copy is made in the library's node order; the product lands in the caller's
    const int vec = (int)((size_t)m * elem / 16);
    k_gather_rows<<<lob::gridn(op.n * vec, 256), 256, 0, st>>>(op.n, vec, op.row_order, static_cast<const uint4*>(XY),
                                                          static_cast<uint4*>(scratch));
    MGE_LAUNCHED(ctx, 1);
    MGE_CUDA(ctx, cudaGetLastError());
  } else {
    MGE_CUDA(ctx, cudaMemcpyAsync(scratch, XY, bytes, cudaMemcpyDeviceToDevice, st));
  }
  return apply_internal(ctx, st, op, precision, m, scratch, XY, op.row_order);
}

}  // namespace mge
