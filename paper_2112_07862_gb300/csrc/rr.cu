// Small dense kernels of the LOBPCG iteration (Sec. 4.3): Rayleigh-Ritz on the basis
// S = [X W P] and the preparation of the next W block.  One CTA each.
//
// Rayleigh-Ritz solves G_A c = theta G_B c (G_A = S^T A S, G_B = S^T B S) for the m smallest
// theta.  Two forms:
//
//  * k_rr_inv (FP32 and BF16 blocks).  FP64 sums of the per-cluster Gram partials, FP64
//    scaling to unit G_A diagonal, then the inverse pencil in FP32: with G^_A = L L^T,
//    M = L^-1 G^_B L^-T has eigenvalues mu = 1/theta, so the wanted (smallest) theta are the
//    largest mu, which a backward-stable FP32 eigensolver gets to relative accuracy ~u times
//    the ratio mu_max / mu (the spread of the wanted eigenvalues only).  A plain FP32
//    eigensolve of (G_A, G_B) would give the small theta only to absolute accuracy
//    u ||G_A||.  Eigenpairs of M: Householder tridiagonalisation, multisection bisection for
//    the m largest eigenvalues, inverse iteration and CGS2 for their vectors.
//  * k_rr_jacobi (FP64 blocks, and operators with a zero shift, for which G_A may be
//    singular).  FP64 Cholesky of G^_B with dropping, reduction to standard form, cyclic
//    two-sided Jacobi.
//
// Both drop basis directions that are numerically dependent (pivots below a threshold) and
// return C_x (Ritz vectors, G_B-orthonormal), Lambda, and C_p (the next P: the W/P part of
// the Ritz coefficients made G_B-orthogonal to C_x and G_B-orthonormal).
#include "lobpcg_common.cuh"

#include <cmath>

namespace mge {
namespace lob {

// ---------------------------------------------------------------------------------------
// shared: sum the cluster partials into gA, gB (FP64, row-major, leading dimension ld)
// ---------------------------------------------------------------------------------------
// G_A[i][j] holds s_i^T (A s_j).  Its rounding error is about u times sum_r |s_i[r]| |(A s_j)[r]|,
// small when A acts on the smoother of the two columns (the smaller Rayleigh quotient,
// G_A[j][j]): for a Ritz vector x against a rough search direction w, (A x)^T w has terms of
// size lambda while x^T (A w) has terms of size w's Rayleigh quotient and cancels to the
// small true value.  So the symmetrised entry takes the product whose A-side column has the
// smaller diagonal, and averages the two when the diagonals are within a factor of two.
template <typename R>
__device__ __forceinline__ R sym_a_entry(R gij, R gji, R gii, R gjj) {
  if (gjj <= R(0.5) * gii) return gij;
  if (gii <= R(0.5) * gjj) return gji;
  return R(0.5) * (gij + gji);
}

// Largest relative size of the FP64 correction of the FP32 Ritz coefficients (the corrections
// the FP32 eigensolve needs are of order u theta_K / theta_1, about 1e-6).
constexpr float kRefineMax = 1e-5f;

// A basis that collapses (fewer than m independent directions) after the solve has made
// progress means the iteration has stagnated at its precision's floor: the current pairs
// stand and the solve ends as not converged.  At the start it is a rank-deficient block.
__device__ __forceinline__ int stall_or_error(const State* st) {
  return st->iter >= 2 ? DONE_STALLED : DONE_ERROR;
}

__device__ bool load_grams(const RRArgs& a, double* gA, double* gB, int n, int ld) {
  __shared__ int nonfinite;
  if (threadIdx.x == 0) nonfinite = 0;
  const Small* sm = a.sm;
  for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
    int i = t / n, j = t % n;
    int bi = i / 4, bj = j / 4;
    int si = (bi <= bj) ? i : j, sj = (bi <= bj) ? j : i;
    gA[i * ld + j] = sum_strided(&sm->partA[0][i * MAXS + j], a.ncl, MAXS * MAXS);
    gB[i * ld + j] = sum_strided(&sm->partB[0][si * MAXS + sj], a.ncl, MAXS * MAXS);
  }
  __syncthreads();
  // the accumulators start the next Gram from zero
  for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
    int i = t / n, j = t % n;
    for (int c = 0; c < a.ncl; ++c) { a.sm->partA[c][i * MAXS + j] = 0.0; a.sm->partB[c][i * MAXS + j] = 0.0; }
  }
  for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
    int i = t / n, j = t % n;
    if (i < j) {
      double va = sym_a_entry(gA[i * ld + j], gA[j * ld + i], gA[i * ld + i], gA[j * ld + j]);
      gA[i * ld + j] = va; gA[j * ld + i] = va;
      if (i / 4 == j / 4) {
        double vb = 0.5 * (gB[i * ld + j] + gB[j * ld + i]);
        gB[i * ld + j] = vb; gB[j * ld + i] = vb;
      }
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
    int i = t / n, j = t % n;
    if (!isfinite(gA[i * ld + j]) || !isfinite(gB[i * ld + j])) nonfinite = 1;
  }
  __syncthreads();
  return nonfinite == 0;
}

// In-place Cholesky (lower) of the leading n x n block, dropping column j when its pivot^2
// <= tau[j] or keep[j] == 0 (dropped columns and rows are zeroed); rd[j] = 1 / L_jj.
template <typename R>
__device__ void chol_drop(R* S, int ld, int n, const R* tau, int* keep, R* rd) {
  __shared__ R piv;
  for (int j = 0; j < n; ++j) {
    if (threadIdx.x == 0) {
      R v = S[j * ld + j];
      if (keep[j] && v > tau[j] && isfinite((double)v)) {
        piv = sqrt(v);
        S[j * ld + j] = piv;
        rd[j] = R(1) / piv;
      } else {
        keep[j] = 0;
        piv = R(0);
        S[j * ld + j] = R(0);
        rd[j] = R(0);
      }
    }
    __syncthreads();
    const R p = piv;
    const R rp = rd[j];
    for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) S[i * ld + j] = (p > R(0)) ? S[i * ld + j] * rp : R(0);
    __syncthreads();
    if (p > R(0)) {
      const int m = n - j - 1;
      for (int t = threadIdx.x; t < m * m; t += blockDim.x) {
        int i = j + 1 + t / m, k = j + 1 + t % m;
        if (k <= i) S[i * ld + k] -= S[i * ld + j] * S[k * ld + j];
      }
    }
    __syncthreads();
  }
  for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
    int i = t / n, k = t % n;
    if (k > i) S[i * ld + k] = R(0);
  }
  __syncthreads();
}

template <typename T, typename R>
__device__ void store_coeffs(const RRArgs& a) {
  SmallT<T>* o = static_cast<SmallT<T>*>(a.smt);
  const Small* sm = a.sm;
  for (int t = threadIdx.x; t < MAXS * MAXM; t += blockDim.x) { o->Cx[t] = (T)sm->Cx[t]; o->Cp[t] = (T)sm->Cp[t]; }
  for (int t = threadIdx.x; t < MAXM; t += blockDim.x) o->lam[t] = (T)sm->lam[t];
}

// ---------------------------------------------------------------------------------------
// Sturm count: eigenvalues of the symmetric tridiagonal (d, e) below x
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ int sturm_count(const float* d, const float* e2, int k, float x, float pivmin) {
  int c = 0;
  float q = d[0] - x;
  if (fabsf(q) < pivmin) q = -pivmin;
  c += q < 0.f;
  for (int i = 1; i < k; ++i) {
    q = (d[i] - x) - __fdividef(e2[i - 1], q);
    if (fabsf(q) < pivmin) q = -pivmin;
    c += q < 0.f;
  }
  return c;
}

// ---------------------------------------------------------------------------------------
// fast form: FP32 inverse pencil (see the file comment)
// ---------------------------------------------------------------------------------------
constexpr int kRRThreads = 512;

__global__ void __launch_bounds__(kRRThreads) k_rr_inv(RRArgs a) {
  if (a.st->done || !rr_selected(a.sel, a.st)) return;
  long long clk0 = clock64();
#define RR_MARK(k) do { __syncthreads(); if (threadIdx.x == 0) a.st->rr_clk[k] = clock64() - clk0; } while (0)
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int M = a.M, n = a.nb * a.M, nx = a.nx;
  const int ldd = n + 1;         // FP64 leading dimension
  const int ldf = n + 1;         // FP32 leading dimension
  double* gA = reinterpret_cast<double*>(smem_raw);
  double* gB = gA + n * ldd;
  float* Lf = reinterpret_cast<float*>(gB + n * ldd);   // Cholesky factor of G^_A (compacted)
  float* Mf = Lf + n * ldf;                              // M = L^-1 G^_B L^-T (kept for C_p)
  float* Hf = Mf + n * ldf;                              // tridiagonalisation workspace
  float* Yf = Hf + n * ldf;                              // eigenvectors of M, k x MAXM
  float* scr = Yf + n * MAXM;                            // inverse-iteration scratch, 6 x k per vector
  __shared__ double dsc[MAXS];
  __shared__ float tauv[MAXS], rd[MAXS], td[MAXS], te[MAXS], te2[MAXS], ht[MAXS], wv[MAXS], pv[MAXS];
  __shared__ float mu[MAXM], dots[MAXM], gp[MAXM * MAXM], rdp[MAXM], taup[MAXM];
  __shared__ int keep[MAXS], idx[MAXS], pkeep[MAXM];
  __shared__ int kcount, bad;
  __shared__ float sh_f[4];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;

  RR_MARK(1);
  if (!load_grams(a, gA, gB, n, ldd)) {
    if (threadIdx.x == 0) { a.st->done = DONE_ERROR; a.st->err = MGE_ENOTFINITE; a.st->bad_stage = 1; }
    return;
  }
  // 1. scale to unit G_A diagonal; columns with empty A or B norm are dead
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double ga = gA[i * ldd + i], gb = gB[i * ldd + i];
    bool live = ga > 1e-30 && gb > 1e-30 && ga < 1e30 && gb < 1e30;
    dsc[i] = live ? drsqrt(ga) : 0.0;
    keep[i] = live ? 1 : 0;
    tauv[i] = (float)a.tau;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
    int i = t / n, j = t % n;
    double s = dsc[i] * dsc[j];
    Hf[i * ldf + j] = (float)(gA[i * ldd + j] * s);   // G^_A
    Mf[i * ldf + j] = (float)(gB[i * ldd + j] * s);   // G^_B
  }
  __syncthreads();
  RR_MARK(2);
  // 2. Cholesky of G^_A with dropping
  chol_drop<float>(Hf, ldf, n, tauv, keep, rd);
  if (threadIdx.x == 0) {
    int c = 0;
    for (int i = 0; i < n; ++i) if (keep[i]) idx[c++] = i;
    kcount = c;
  }
  __syncthreads();
  const int k = kcount;
  if (k < M) {
    if (threadIdx.x == 0) { a.st->done = stall_or_error(a.st); a.st->err = MGE_ECHOLESKY; a.st->kept = k; }
    return;
  }
  if (threadIdx.x == 0 && k < n) atomicAdd(&a.st->drops, 1);
  // compact: L -> Lf, G^_B -> Yf temporarily (k x k, ld ldf), rd -> rd compacted
  for (int t = threadIdx.x; t < k * k; t += blockDim.x) {
    int r = t / k, c = t % k;
    Lf[r * ldf + c] = Hf[idx[r] * ldf + idx[c]];
  }
  __syncthreads();
  for (int t = threadIdx.x; t < k * k; t += blockDim.x) {
    int r = t / k, c = t % k;
    Hf[r * ldf + c] = Mf[idx[r] * ldf + idx[c]];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    float tmp[MAXS];
    for (int r = 0; r < k; ++r) tmp[r] = rd[idx[r]];
    for (int r = 0; r < k; ++r) rd[r] = tmp[r];
  }
  __syncthreads();
  RR_MARK(3);
  // 3. M = L^-1 G^_B L^-T: Y = L^-1 G^_B in Hf (column-parallel), then M = L^-1 Y^T into Mf
  for (int c = threadIdx.x; c < k; c += blockDim.x) {
    for (int r = 0; r < k; ++r) {
      float v = Hf[r * ldf + c];
      for (int s = 0; s < r; ++s) v -= Lf[r * ldf + s] * Hf[s * ldf + c];
      Hf[r * ldf + c] = v * rd[r];
    }
  }
  __syncthreads();
  for (int c = threadIdx.x; c < k; c += blockDim.x) {
    for (int r = 0; r < k; ++r) {
      float v = Hf[c * ldf + r];
      for (int s = 0; s < r; ++s) v -= Lf[r * ldf + s] * Mf[s * ldf + c];
      Mf[r * ldf + c] = v * rd[r];
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < k * k; t += blockDim.x) {
    int r = t / k, c = t % k;
    float v = (r == c) ? Mf[r * ldf + c] : 0.5f * (Mf[r * ldf + c] + Mf[c * ldf + r]);
    Hf[r * ldf + c] = v;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < k * k; t += blockDim.x) Mf[(t / k) * ldf + t % k] = Hf[(t / k) * ldf + t % k];
  __syncthreads();
  RR_MARK(4);
  // 4. Householder tridiagonalisation of Hf (k x k): T = Q^T M Q
  for (int j = 0; j + 2 < k; ++j) {
    const int len = k - j - 1;
    if (wid == 0) {
      float s2 = 0.f;
      for (int i = lane; i < len; i += 32) { float x = Hf[(j + 1 + i) * ldf + j]; s2 += x * x; }
      for (int o = 16; o; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
      if (lane == 0) {
        float x0 = Hf[(j + 1) * ldf + j];
        float tail = s2 - x0 * x0;
        if (!(tail > 1e-30f * s2) || s2 == 0.f) {
          ht[j] = 0.f;
          te[j] = x0;
        } else {
          float alpha = -copysignf(sqrtf(s2), x0);
          float v0 = x0 - alpha;
          Hf[(j + 1) * ldf + j] = v0;
          ht[j] = 2.f / (tail + v0 * v0);
          te[j] = alpha;
        }
        td[j] = Hf[j * ldf + j];
      }
    }
    __syncthreads();
    const float tj = ht[j];
    if (tj != 0.f) {
      // p = tau * A22 v
      for (int r = threadIdx.x; r < len; r += blockDim.x) {
        const float* row = Hf + (j + 1 + r) * ldf + (j + 1);
        float s0 = 0.f, s1 = 0.f;
        int c = 0;
        for (; c + 1 < len; c += 2) {
          s0 += row[c] * Hf[(j + 1 + c) * ldf + j];
          s1 += row[c + 1] * Hf[(j + 2 + c) * ldf + j];
        }
        if (c < len) s0 += row[c] * Hf[(j + 1 + c) * ldf + j];
        pv[r] = tj * (s0 + s1);
      }
      __syncthreads();
      if (wid == 0) {
        float s = 0.f;
        for (int i = lane; i < len; i += 32) s += pv[i] * Hf[(j + 1 + i) * ldf + j];
        for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) sh_f[0] = 0.5f * tj * s;
      }
      __syncthreads();
      const float K = sh_f[0];
      for (int r = threadIdx.x; r < len; r += blockDim.x) wv[r] = pv[r] - K * Hf[(j + 1 + r) * ldf + j];
      __syncthreads();
      for (int t = threadIdx.x; t < len * len; t += blockDim.x) {
        int r = t / len, c = t % len;
        float vr = Hf[(j + 1 + r) * ldf + j], vc = Hf[(j + 1 + c) * ldf + j];
        Hf[(j + 1 + r) * ldf + (j + 1 + c)] -= vr * wv[c] + wv[r] * vc;
      }
      __syncthreads();
    }
  }
  if (threadIdx.x == 0) {
    if (k >= 2) {
      td[k - 2] = Hf[(k - 2) * ldf + (k - 2)];
      te[k - 2] = Hf[(k - 1) * ldf + (k - 2)];
      if (k >= 3) {}  // ht[k-2] unused
    }
    td[k - 1] = Hf[(k - 1) * ldf + (k - 1)];
    for (int i = 0; i + 1 < k; ++i) te2[i] = te[i] * te[i];
  }
  __syncthreads();
  RR_MARK(5);
  // 5. the M largest eigenvalues of T by multisection bisection (one warp per eigenvalue)
  {
    float glo = 3.4e38f, ghi = -3.4e38f, emax = 0.f;
    for (int i = 0; i < k; ++i) {
      float r = (i > 0 ? fabsf(te[i - 1]) : 0.f) + (i + 1 < k ? fabsf(te[i]) : 0.f);
      glo = fminf(glo, td[i] - r);
      ghi = fmaxf(ghi, td[i] + r);
      emax = fmaxf(emax, fabsf(td[i]) + r);
    }
    const float pivmin = fmaxf(1e-30f, 1e-37f * emax * emax);
    const float width = fmaxf(ghi - glo, 1e-30f);
    glo -= 2e-6f * width + pivmin;
    ghi += 2e-6f * width + pivmin;
    for (int q = wid; q < M; q += nw) {
      const int target = k - 1 - q;           // ascending index of the q-th largest
      float lo = glo, hi = ghi;
      for (int round = 0; round < 10; ++round) {
        float step = (hi - lo) / 33.f;
        float x = lo + step * (float)(lane + 1);
        int c = sturm_count(td, te2, k, x, pivmin);
        unsigned above = __ballot_sync(0xffffffffu, c > target);
        float nlo = lo, nhi = hi;
        if (above) {
          int f = __ffs(above) - 1;
          nhi = __shfl_sync(0xffffffffu, x, f);
          if (f > 0) nlo = __shfl_sync(0xffffffffu, x, f - 1);
        } else {
          nlo = __shfl_sync(0xffffffffu, x, 31);
        }
        lo = nlo; hi = nhi;
        if (hi - lo <= 1.2e-7f * fmaxf(fabsf(lo), fabsf(hi))) break;
      }
      if (lane == 0) mu[q] = 0.5f * (lo + hi);
    }
  }
  __syncthreads();
  RR_MARK(6);
  // 6. inverse iteration on T - mu I (tridiagonal LU with partial pivoting), one thread per vector
  for (int q = threadIdx.x; q < M; q += blockDim.x) {
    float* u0 = scr + (size_t)q * 6 * k;
    float* u1 = u0 + k;
    float* u2 = u1 + k;
    float* lm = u2 + k;
    float* y = lm + k;
    int* pv_ = reinterpret_cast<int*>(y + k);
    float nrmT = 0.f;
    for (int i = 0; i < k; ++i) nrmT = fmaxf(nrmT, fabsf(td[i]) + (i > 0 ? fabsf(te[i - 1]) : 0.f) + (i + 1 < k ? fabsf(te[i]) : 0.f));
    const float tiny = fmaxf(nrmT * 1.2e-7f, 1e-30f);
    const float lam = mu[q];
    float p = td[0] - lam, qq = (k > 1) ? te[0] : 0.f;
    for (int i = 0; i + 1 < k; ++i) {
      float c = te[i], an = td[i + 1] - lam, bn = (i + 2 < k) ? te[i + 1] : 0.f;
      if (fabsf(c) > fabsf(p)) {
        float l = p / c;
        u0[i] = c; u1[i] = an; u2[i] = bn; lm[i] = l; pv_[i] = 1;
        p = qq - l * an; qq = -l * bn;
      } else {
        if (fabsf(p) < tiny) p = copysignf(tiny, p == 0.f ? 1.f : p);
        float l = c / p;
        u0[i] = p; u1[i] = qq; u2[i] = 0.f; lm[i] = l; pv_[i] = 0;
        p = an - l * qq; qq = bn;
      }
    }
    if (fabsf(p) < tiny) p = copysignf(tiny, p == 0.f ? 1.f : p);
    u0[k - 1] = p;
    // starting vector: deterministic, not orthogonal to any eigenvector in practice
    for (int i = 0; i < k; ++i) y[i] = 1.f + 0.37f * __sinf(1.3f * i + 0.7f * q);
    for (int itn = 0; itn < 3; ++itn) {
      for (int i = 0; i + 1 < k; ++i) {
        if (pv_[i]) { float t = y[i]; y[i] = y[i + 1]; y[i + 1] = t; }
        y[i + 1] -= lm[i] * y[i];
      }
      for (int i = k - 1; i >= 0; --i) {
        float v = y[i];
        if (i + 1 < k) v -= u1[i] * y[i + 1];
        if (i + 2 < k) v -= u2[i] * y[i + 2];
        y[i] = v / u0[i];
      }
      float s = 0.f;
      for (int i = 0; i < k; ++i) s = fmaxf(s, fabsf(y[i]));
      float inv = s > 0.f ? 1.f / s : 1.f;
      for (int i = 0; i < k; ++i) y[i] *= inv;
    }
    for (int i = 0; i < k; ++i) Yf[i * MAXM + q] = y[i];
  }
  __syncthreads();
  RR_MARK(7);
  // 7. CGS2 over the M vectors (in order of decreasing mu), then unit norm
  for (int j = 0; j < M; ++j) {
    for (int pass = 0; pass < 2; ++pass) {
      for (int i = wid; i < j; i += nw) {
        float s = 0.f;
        for (int r = lane; r < k; r += 32) s += Yf[r * MAXM + i] * Yf[r * MAXM + j];
        for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) dots[i] = s;
      }
      __syncthreads();
      for (int r = threadIdx.x; r < k; r += blockDim.x) {
        float v = Yf[r * MAXM + j];
        for (int i = 0; i < j; ++i) v -= dots[i] * Yf[r * MAXM + i];
        Yf[r * MAXM + j] = v;
      }
      __syncthreads();
    }
    if (wid == 0) {
      float s = 0.f;
      for (int r = lane; r < k; r += 32) { float v = Yf[r * MAXM + j]; s += v * v; }
      for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) sh_f[1] = s > 0.f ? rsqrtf(s) : 0.f;
    }
    __syncthreads();
    for (int r = threadIdx.x; r < k; r += blockDim.x) Yf[r * MAXM + j] *= sh_f[1];
    __syncthreads();
  }
  RR_MARK(8);
  // 8. back-transform y <- Q y (Householder reflectors in reverse), one warp per vector
  for (int q = wid; q < M; q += nw) {
    for (int j = k - 3; j >= 0; --j) {
      const float tj = ht[j];
      if (tj == 0.f) continue;
      float s = 0.f;
      for (int r = j + 1 + lane; r < k; r += 32) s += Hf[r * ldf + j] * Yf[r * MAXM + q];
      for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      s *= tj;
      for (int r = j + 1 + lane; r < k; r += 32) Yf[r * MAXM + q] -= s * Hf[r * ldf + j];
      __syncwarp();
    }
  }
  __syncthreads();
  RR_MARK(9);
  // 9. Ritz values and coefficients: theta = 1/mu, c = D L^-T y / sqrt(mu) (then c^T G_B c = 1)
  if (threadIdx.x == 0) {
    int b = 0;
    for (int q = 0; q < M; ++q) if (!(mu[q] > 0.f) || !isfinite(mu[q])) b = 1;
    bad = b;
  }
  __syncthreads();
  if (bad) {
    if (threadIdx.x == 0) { a.st->done = DONE_ERROR; a.st->err = MGE_ENOTFINITE; a.st->bad_stage = 4; }
    return;
  }
  Small* sm = a.sm;
  for (int t = threadIdx.x; t < n * M; t += blockDim.x) { sm->Cx[(t / M) * MAXM + t % M] = 0.0; sm->Cp[(t / M) * MAXM + t % M] = 0.0; }
  // z = L^-T y (k x M, leading dimension M) in Hf; the reflectors are no longer needed
  float* Z = Hf;
  float* U = scr;   // k x M, leading dimension M; the inverse-iteration scratch is free
  __syncthreads();
  for (int q = threadIdx.x; q < M; q += blockDim.x) {
    for (int r = k - 1; r >= 0; --r) {
      float v = Yf[r * MAXM + q];
      for (int s = r + 1; s < k; ++s) v -= Lf[s * ldf + r] * Z[s * M + q];
      Z[r * M + q] = v * rd[r];
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < k * M; t += blockDim.x) {
    int r = t / M, q = t % M;
    double s = (double)rsqrtf(mu[q]);
    sm->Cx[idx[r] * MAXM + q] = dsc[idx[r]] * (double)Z[r * M + q] * s;
  }
  for (int q = threadIdx.x; q < M; q += blockDim.x) sm->lam[q] = 1.0 / (double)mu[q];
  RR_MARK(10);
  // 10. C_p.  In u = L^T z coordinates the G_B inner product is u^T M u', and a Ritz vector
  //     is u = y / sqrt(mu) with M y = mu y, so M-orthogonality to it is Euclidean
  //     orthogonality to y.
  if (nx > 0) {
    __syncthreads();
    // z_p: the W/P rows of z (X rows zeroed), in place
    for (int t = threadIdx.x; t < k * M; t += blockDim.x) {
      int r = t / M;
      if (idx[r] < nx) Z[t] = 0.f;
    }
    __syncthreads();
    // u = L^T z_p
    for (int t = threadIdx.x; t < k * M; t += blockDim.x) {
      int r = t / M, q = t % M;
      float v = 0.f;
      for (int s_ = r; s_ < k; ++s_) v += Lf[s_ * ldf + r] * Z[s_ * M + q];
      U[r * M + q] = v;
    }
    __syncthreads();
    // u <- u - Y (Y^T u)
    for (int t = threadIdx.x; t < M * M; t += blockDim.x) {
      int i = t / M, q = t % M;
      float v = 0.f;
      for (int r = 0; r < k; ++r) v += Yf[r * MAXM + i] * U[r * M + q];
      gp[i * MAXM + q] = v;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < k * M; t += blockDim.x) {
      int r = t / M, q = t % M;
      float v = U[r * M + q];
      for (int i = 0; i < M; ++i) v -= Yf[r * MAXM + i] * gp[i * MAXM + q];
      U[r * M + q] = v;
    }
    __syncthreads();
    // Gram u^T M u -> Cholesky with dropping -> u <- u L_p^-T
    for (int t = threadIdx.x; t < k * M; t += blockDim.x) {
      int r = t / M, q = t % M;
      float v = 0.f;
      for (int c = 0; c < k; ++c) v += Mf[r * ldf + c] * U[c * M + q];
      Z[r * M + q] = v;       // M u
    }
    __syncthreads();
    for (int t = threadIdx.x; t < M * M; t += blockDim.x) {
      int i = t / M, q = t % M;
      float v = 0.f;
      for (int r = 0; r < k; ++r) v += U[r * M + i] * Z[r * M + q];
      gp[i * MAXM + q] = v;
    }
    for (int i = threadIdx.x; i < M; i += blockDim.x) { pkeep[i] = 1; taup[i] = (float)a.tau_p; }
    __syncthreads();
    for (int t = threadIdx.x; t < M * M; t += blockDim.x) {
      int i = t / M, q = t % M;
      if (i < q) { float v = 0.5f * (gp[i * MAXM + q] + gp[q * MAXM + i]); gp[i * MAXM + q] = v; gp[q * MAXM + i] = v; }
    }
    __syncthreads();
    chol_drop<float>(gp, MAXM, M, taup, pkeep, rdp);
    for (int r = threadIdx.x; r < k; r += blockDim.x) {
      for (int c = 0; c < M; ++c) {
        float v = U[r * M + c];
        if (rdp[c] > 0.f) {
          for (int s_ = 0; s_ < c; ++s_) v -= U[r * M + s_] * gp[c * MAXM + s_];
          U[r * M + c] = v * rdp[c];
        } else {
          U[r * M + c] = 0.f;
        }
      }
    }
    __syncthreads();
    // z_p = L^-T u into Z, C_p = D z_p
    for (int q = threadIdx.x; q < M; q += blockDim.x) {
      for (int r = k - 1; r >= 0; --r) {
        float v = U[r * M + q];
        for (int s_ = r + 1; s_ < k; ++s_) v -= Lf[s_ * ldf + r] * Z[s_ * M + q];
        Z[r * M + q] = v * rd[r];
      }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < k * M; t += blockDim.x) {
      int r = t / M, q = t % M;
      sm->Cp[idx[r] * MAXM + q] = dsc[idx[r]] * (double)Z[r * M + q];
    }
  }
  __syncthreads();
  RR_MARK(11);
  // 11. One correction step for the Ritz coefficients against the FP64 pencil.  The FP32
  //     eigenvectors of M carry absolute errors of about u mu_max, i.e. components of
  //     relative size u theta_k / theta_1 along basis directions of large Rayleigh quotient
  //     theta_j, which put u theta_j / theta_1 into the relative residual (measured floors:
  //     ~3e-6 at 20k nodes, ~1e-5 at 200k, 1-2e-5 at 2M).  With the FP64 residual
  //     r = (G_A - theta G_B) c and the correction d = -G_A^-1 r (the FP32 Cholesky factor of
  //     G^_A), a component along an eigenvector j of the pencil shrinks by the factor
  //     theta_k / theta_j: the large-theta errors go, the ones along nearby eigenvectors
  //     change little, and those along smaller theta (of size u) grow by at most
  //     theta_K / theta_1.  Applied only near the tolerance (the floor matters there) and
  //     not once the residuals have stopped falling: at a floor set by the FP32 blocks the
  //     correction only feeds rounding back into the basis, and over thousands of such
  //     iterations that diverged (measured on a 2000-node graph).
  if (a.st->refine) {
    float* Rf = scr;                        // k x M: D r, then d in the u coordinates
    for (int t = threadIdx.x; t < k * M; t += blockDim.x) {
      const int r = t / M, q = t % M;
      const int i = idx[r];
      const double th = sm->lam[q];
      double s = 0.0;
      for (int c_ = 0; c_ < k; ++c_) {
        const int j = idx[c_];
        s += (gA[i * ldd + j] - th * gB[i * ldd + j]) * sm->Cx[j * MAXM + q];
      }
      Rf[r * M + q] = (float)(dsc[i] * s);
    }
    __syncthreads();
    // G_A^-1 = D L^-T L^-1 D on the kept directions: w = L^-1 (D r), then z = L^-T w
    for (int q = threadIdx.x; q < M; q += blockDim.x) {
      for (int r = 0; r < k; ++r) {
        float v = Rf[r * M + q];
        for (int s_ = 0; s_ < r; ++s_) v -= Lf[r * ldf + s_] * Rf[s_ * M + q];
        Rf[r * M + q] = v * rd[r];
      }
      for (int r = k - 1; r >= 0; --r) {
        float v = Rf[r * M + q];
        for (int s_ = r + 1; s_ < k; ++s_) v -= Lf[s_ * ldf + r] * Rf[s_ * M + q];
        Rf[r * M + q] = v * rd[r];
      }
    }
    __syncthreads();
    // a correction is kept only while it is small against the coefficients (both in the
    // unit-diagonal scaling): near-dependent bases, where G_A^-1 amplifies the residual's
    // rounding, leave the FP32 coefficients as they are
    for (int q = threadIdx.x; q < M; q += blockDim.x) {
      float nz = 0.f, nc = 0.f;
      for (int r = 0; r < k; ++r) {
        const float z = Rf[r * M + q];
        const float c = (float)(sm->Cx[idx[r] * MAXM + q] / dsc[idx[r]]);
        nz += z * z;
        nc += c * c;
      }
      dots[q] = (nz <= kRefineMax * kRefineMax * nc) ? 1.f : 0.f;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < k * M; t += blockDim.x) {
      const int r = t / M, q = t % M;
      if (dots[q] != 0.f) sm->Cx[idx[r] * MAXM + q] -= dsc[idx[r]] * (double)Rf[r * M + q];
    }
  }
  __syncthreads();
  if (a.is_double) store_coeffs<double, float>(a);
  else store_coeffs<float, float>(a);
  if (threadIdx.x == 0) a.st->kept = k;
  RR_MARK(12);
#undef RR_MARK
}

// ---------------------------------------------------------------------------------------
// fast form for bases of at most 32 directions: the inverse-pencil algorithm above on
// 32 x 32 shared-memory matrices, one CTA of 8 warps.  Warp w owns rows 4w .. 4w+3 of every
// matrix update; the per-step reductions (pivot columns, Householder vectors) are
// recomputed by every warp so that one barrier per elimination step suffices.
//
// Lane-dependent branches are avoided in the warp-synchronous parts: a warp left diverged
// by such a branch executes later shuffles and barriers one thread group at a time, which
// multiplied the cost of this kernel several times over.
// ---------------------------------------------------------------------------------------
constexpr int WN = 32;
constexpr int kRWThreads = 256;
constexpr int kRWRows = WN / (kRWThreads / 32);     // rows per warp: 4

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Four warp sums at once (transposed butterfly, six shuffles): lane l returns the total of
// value (l >> 3) & 3.
__device__ __forceinline__ float warp_sum4(float s0, float s1, float s2, float s3, int lane) {
  const bool h16 = lane & 16, h8 = lane & 8;
  float a0 = h16 ? s2 : s0, a1 = h16 ? s3 : s1;
  const float b0 = h16 ? s0 : s2, b1 = h16 ? s1 : s3;
  a0 += __shfl_xor_sync(0xffffffffu, b0, 16);
  a1 += __shfl_xor_sync(0xffffffffu, b1, 16);
  float c = h8 ? a1 : a0;
  const float d = h8 ? a0 : a1;
  c += __shfl_xor_sync(0xffffffffu, d, 8);
  c += __shfl_xor_sync(0xffffffffu, c, 4);
  c += __shfl_xor_sync(0xffffffffu, c, 2);
  c += __shfl_xor_sync(0xffffffffu, c, 1);
  return c;
}

__global__ void __launch_bounds__(kRWThreads) k_rr_warp(RRArgs a) {
  if (a.st->done || !rr_selected(a.sel, a.st)) return;
  const long long clk0 = clock64();
  __shared__ long long sclk[12];
  // phase clocks: written by every thread (a branch around clock64 leaves warps diverged)
#define RW_MARK(k) (sclk[k] = clock64() - clk0)
  const int M = a.M, n = a.nb * a.M, nx = a.nx;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int row0 = wid * kRWRows;
  __shared__ float sA[WN][WN + 1];       // G^_A and its Schur complements, then L (compact)
  __shared__ float sB[WN][WN + 1];       // G^_B (full index), then Y = L^-1 G^_B, then T
  __shared__ float sL[WN][WN + 1];       // L (full index), then L^-1 (compact)
  __shared__ float sM[WN][WN + 1];       // G^_B (compact), then M = L^-1 G^_B L^-T
  __shared__ float sH[WN][WN + 1];       // Householder vectors: sH[j][i] = v_i of reflector j
  __shared__ float sZ[WN][MAXM + 1];     // eigenvectors (compact coordinate r, vector q)
  __shared__ float sU[WN][MAXM + 1];
  __shared__ float sV[WN][MAXM + 1];
  __shared__ float sgp[MAXM][MAXM + 1];
  __shared__ float sdf[WN];             // scaling D (unit G_A diagonal)
  __shared__ float srd[WN], sd[WN], se[WN], se2[WN], sht[WN], sp[WN], smu[MAXM], srdp[MAXM];
  __shared__ int sidx[WN], sinv[WN];    // compact -> full index, full -> compact (-1: dropped)
  __shared__ unsigned slive;
  Small* sm = a.sm;
  if (threadIdx.x < 12) sclk[threadIdx.x] = 0;

  // ---- 1. FP64 Grams scaled to unit G_A diagonal, rounded to FP32 ----
  if (wid == 0) {
    const int li = lane < n ? lane : 0;
    const double gaii = sm->partA[0][li * MAXS + li], gbii = sm->partB[0][li * MAXS + li];
    const bool live = lane < n && gaii > 1e-30 && gbii > 1e-30 && gaii < 1e30 && gbii < 1e30;
    // any positive scaling is exact enough: it is undone in C_x and C_p with the same factors
    sdf[lane] = live ? rsqrtf((float)gaii) : 0.f;
    const unsigned lm = __ballot_sync(0xffffffffu, live);
    slive = lm;
  }
  __syncthreads();
  // each FP64 partial is rounded to FP32 once (GB300's FP64 rate is a small fraction of its
  // FP32 rate); G_B holds only its block-upper part
  int bad = 0;
  for (int t = threadIdx.x; t < WN * WN; t += kRWThreads) {
    const int i = t >> 5, j = t & 31;
    double ga = 0.0, gb = 0.0;
    if (i < n && j < n) {
      const int bi = i / 4, bj = j / 4;
      ga = sym_a_entry(sm->partA[0][i * MAXS + j], sm->partA[0][j * MAXS + i],
                       sm->partA[0][i * MAXS + i], sm->partA[0][j * MAXS + j]);
      const double b1 = (bi <= bj) ? sm->partB[0][i * MAXS + j] : 0.0;
      const double b2 = (bi >= bj) ? sm->partB[0][j * MAXS + i] : 0.0;
      gb = (bi < bj) ? b1 : (bi > bj) ? b2 : 0.5 * (b1 + b2);
      bad |= !(isfinite((float)ga) && isfinite((float)gb));
    }
    const float sc = sdf[i] * sdf[j];
    sA[i][j] = (float)ga * sc;
    sB[i][j] = (float)gb * sc;
  }
  bad = __syncthreads_or(bad);
  if (bad) {
    if (threadIdx.x == 0) { a.st->done = DONE_ERROR; a.st->err = MGE_ENOTFINITE; a.st->bad_stage = 1; }
    return;
  }
  RW_MARK(1);

  // ---- 2. Cholesky of G^_A with dropping: step j scales column j, every warp updates its
  //      rows of the Schur complement (lane = column); dropped directions are skipped ----
  unsigned keep = slive;
  {
    const float tau = (float)a.tau;
#pragma unroll 1
    for (int j = 0; j < n; ++j) {
      const float ajj = sA[j][j];
      const bool ok = ((keep >> j) & 1u) && ajj > tau && isfinite(ajj);
      const float rinv = ok ? rsqrtf(ajj) : 0.f;
      const float lj = (lane > j && lane < n) ? sA[lane][j] * rinv : 0.f;      // l_{lane j}
      keep = ok ? keep : (keep & ~(1u << j));
      if (wid == (j & 7)) sL[lane][j] = (lane == j) ? ajj * rinv : lj;
      // l_kj = 0 for k <= j, so column j and the rows above j are left unchanged
#pragma unroll
      for (int r = 0; r < kRWRows; ++r) {
        const float li = __shfl_sync(0xffffffffu, lj, row0 + r);
        sA[row0 + r][lane] -= li * lj;
      }
      __syncthreads();
    }
  }
  const int k = __popc(keep);
  if (threadIdx.x < WN) {                    // compaction map: kept index of rank r at sidx[r]
    const int i = threadIdx.x;
    const bool kept = (keep >> i) & 1u;
    const int pos = __popc(keep & ((1u << i) - 1u));
    sidx[kept ? pos : k + (i - pos)] = kept ? i : 0;
    sinv[i] = kept ? pos : -1;
  }
  RW_MARK(9);
  if (k < M) {
    if (threadIdx.x == 0) { a.st->done = stall_or_error(a.st); a.st->err = MGE_ECHOLESKY; a.st->kept = k; }
    return;
  }
  if (threadIdx.x == 0 && k < n) atomicAdd(&a.st->drops, 1);
  __syncthreads();
  for (int t = threadIdx.x; t < WN * WN; t += kRWThreads) {
    const int r = t >> 5, c = t & 31;
    const bool in = r < k && c < k;
    const int sr = sidx[r], sc = sidx[c];
    sA[r][c] = (in && c <= r) ? sL[sr][sc] : 0.f;
    sM[r][c] = in ? sB[sr][sc] : 0.f;
  }
  if (threadIdx.x < WN) {
    const int r = threadIdx.x;
    srd[r] = r < k ? 1.f / sL[sidx[r]][sidx[r]] : 0.f;
  }
  __syncthreads();
  RW_MARK(2);

  // ---- 3. L^-1 by forward substitution (row r final after step r, lane = column), then
  //      M = L^-1 G^_B L^-T as two products ----
  for (int t = threadIdx.x; t < WN * WN; t += kRWThreads) {
    const int r = t >> 5, c = t & 31;
    sL[r][c] = (r == c && r < k) ? 1.f : 0.f;
  }
  __syncthreads();
#pragma unroll 1
  for (int r = 0; r < k; ++r) {
    const float xr = sL[r][lane] * srd[r];
#pragma unroll
    for (int q = 0; q < kRWRows; ++q) {
      const int s_ = row0 + q;
      if (s_ > r && s_ < k) sL[s_][lane] -= sA[s_][r] * xr;
    }
    __syncthreads();
  }
  for (int t = threadIdx.x; t < WN * WN; t += kRWThreads) sL[t >> 5][t & 31] *= srd[t >> 5];
  __syncthreads();
  {
    const int i = threadIdx.x >> 3, c0 = (threadIdx.x & 7) * 4;
    float y0 = 0.f, y1 = 0.f, y2 = 0.f, y3 = 0.f;
#pragma unroll 8
    for (int s_ = 0; s_ < k; ++s_) {
      const float l = sL[i][s_];
      y0 += l * sM[s_][c0]; y1 += l * sM[s_][c0 + 1]; y2 += l * sM[s_][c0 + 2]; y3 += l * sM[s_][c0 + 3];
    }
    sB[i][c0] = y0; sB[i][c0 + 1] = y1; sB[i][c0 + 2] = y2; sB[i][c0 + 3] = y3;
    __syncthreads();
    float m0 = 0.f, m1 = 0.f, m2 = 0.f, m3 = 0.f;
#pragma unroll 8
    for (int s_ = 0; s_ < k; ++s_) {
      const float y = sB[i][s_];
      m0 += y * sL[c0][s_]; m1 += y * sL[c0 + 1][s_]; m2 += y * sL[c0 + 2][s_]; m3 += y * sL[c0 + 3][s_];
    }
    sM[i][c0] = m0; sM[i][c0 + 1] = m1; sM[i][c0 + 2] = m2; sM[i][c0 + 3] = m3;
    __syncthreads();
  }
  for (int t = threadIdx.x; t < WN * WN; t += kRWThreads) {     // T = symmetric part of M
    const int r = t >> 5, c = t & 31;
    sB[r][c] = 0.5f * (sM[r][c] + sM[c][r]);
  }
  __syncthreads();
  RW_MARK(3);

  // ---- 4. Householder tridiagonalisation of T (in sB) ----
#pragma unroll 1
  for (int j = 0; j + 2 < k; ++j) {
    const float x = (lane > j && lane < k) ? sB[lane][j] : 0.f;
    const float s2 = warp_sum(x * x);
    const float x0 = __shfl_sync(0xffffffffu, x, j + 1);
    const float tail = s2 - x0 * x0;
    const bool refl = tail > 1e-30f * s2 && s2 > 0.f;
    const float alpha = refl ? -copysignf(sqrtf(s2), x0) : x0;
    const float v0 = x0 - alpha;
    const float tau = refl ? 2.f / (tail + v0 * v0) : 0.f;
    const float v = refl ? ((lane == j + 1) ? v0 : x) : 0.f;
    if (wid == 0) {
      sd[j] = sB[j][j]; se[j] = alpha; sht[j] = tau;
      sH[j][lane] = v;
    }
    if (refl) {
      // p_i = tau sum_c T_ic v_c for this warp's rows (lane = c)
      const float pr = warp_sum4(sB[row0][lane] * v, sB[row0 + 1][lane] * v, sB[row0 + 2][lane] * v,
                                 sB[row0 + 3][lane] * v, lane);
      const int ir = row0 + ((lane >> 3) & 3);
      sp[ir] = (ir > j && ir < k) ? tau * pr : 0.f;
      __syncthreads();
      const float p = sp[lane];
      const float K = 0.5f * tau * warp_sum(p * v);
      const float w = p - K * v;
#pragma unroll
      for (int r = 0; r < kRWRows; ++r) {
        const int i = row0 + r;
        const float vi = __shfl_sync(0xffffffffu, v, i), wi = __shfl_sync(0xffffffffu, w, i);
        if (i > j && i < k) sB[i][lane] -= vi * w + wi * v;
      }
    }
    __syncthreads();
  }
  if (wid == 0) {
    sd[k - 2] = sB[k - 2][k - 2];
    se[k - 2] = sB[k - 1][k - 2];
    sd[k - 1] = sB[k - 1][k - 1];
    sht[k - 2] = 0.f;
    __syncwarp();
    se2[lane] = (lane + 1 < k) ? se[lane] * se[lane] : 0.f;
  }
  __syncthreads();
  RW_MARK(4);

  // ---- 5. the M largest eigenvalues of T: multisection bisection, one warp per eigenvalue ----
  {
    float glo = 3.4e38f, ghi = -3.4e38f, emax = 0.f;
    for (int r = 0; r < k; ++r) {
      const float rad = (r > 0 ? fabsf(se[r - 1]) : 0.f) + (r + 1 < k ? fabsf(se[r]) : 0.f);
      glo = fminf(glo, sd[r] - rad);
      ghi = fmaxf(ghi, sd[r] + rad);
      emax = fmaxf(emax, fabsf(sd[r]) + rad);
    }
    const float pivmin = fmaxf(1e-30f, 1e-37f * emax * emax);
    const float width = fmaxf(ghi - glo, 1e-30f);
    glo -= 2e-6f * width + pivmin;
    ghi += 2e-6f * width + pivmin;
    for (int q = wid; q < M; q += kRWThreads / 32) {
      const int target = k - 1 - q;
      float lo = glo, hi = ghi;
      for (int round = 0; round < 10; ++round) {
        const float step = (hi - lo) / 33.f;
        const float xs = lo + step * (float)(lane + 1);
        const int cnt = sturm_count(sd, se2, k, xs, pivmin);
        const unsigned above = __ballot_sync(0xffffffffu, cnt > target);
        float nlo = lo, nhi = hi;
        if (above) {
          const int f = __ffs(above) - 1;
          nhi = __shfl_sync(0xffffffffu, xs, f);
          const float pl = __shfl_sync(0xffffffffu, xs, f > 0 ? f - 1 : 0);
          nlo = f > 0 ? pl : lo;
        } else {
          nlo = __shfl_sync(0xffffffffu, xs, 31);
        }
        lo = nlo; hi = nhi;
        if (hi - lo <= 1.2e-7f * fmaxf(fabsf(lo), fabsf(hi))) break;
      }
      smu[q] = 0.5f * (lo + hi);
    }
  }
  __syncthreads();
  RW_MARK(5);

  // ---- 6. inverse iteration on T - mu I (tridiagonal LU with partial pivoting), one thread
  //      per eigenvalue; loops unrolled over the 32 possible rows so that the factors stay in
  //      registers, pivoting by selects (no divergence between the eigenvalues) ----
  for (int q = threadIdx.x; q < M; q += kRWThreads) {
    float nrmT = 0.f;
    for (int r = 0; r < k; ++r)
      nrmT = fmaxf(nrmT, fabsf(sd[r]) + (r > 0 ? fabsf(se[r - 1]) : 0.f) + (r + 1 < k ? fabsf(se[r]) : 0.f));
    const float tiny = fmaxf(nrmT * 1.2e-7f, 1e-30f);
    const float lam = smu[q];
    float u0[WN], u1[WN], lm[WN], y[WN];     // reciprocal pivots, first superdiagonal, multipliers
    unsigned pvm = 0u;                       // bit r: rows r and r + 1 exchanged
    float p = sd[0] - lam, qq = se[0];
#pragma unroll
    for (int r = 0; r < WN; ++r) {
      if (r + 1 < k) {
        const float c = se[r], an = sd[r + 1] - lam, bn = (r + 2 < k) ? se[r + 1] : 0.f;
        const bool piv = fabsf(c) > fabsf(p);
        const float pc = (fabsf(p) < tiny) ? copysignf(tiny, p == 0.f ? 1.f : p) : p;
        const float id = __fdividef(1.f, piv ? c : pc);
        const float l = (piv ? p : c) * id;
        u0[r] = id;
        u1[r] = piv ? an : qq;
        lm[r] = l;
        pvm |= piv ? (1u << r) : 0u;
        const float np = piv ? qq - l * an : an - l * qq;
        qq = piv ? -l * bn : bn;
        p = np;
      } else if (r + 1 == k) {
        const float pc = (fabsf(p) < tiny) ? copysignf(tiny, p == 0.f ? 1.f : p) : p;
        u0[r] = __fdividef(1.f, pc);
        u1[r] = 0.f;
        lm[r] = 0.f;
      } else {
        u0[r] = 0.f; u1[r] = 0.f; lm[r] = 0.f;
      }
      y[r] = (r < k) ? 1.f + 0.37f * __sinf(1.3f * r + 0.7f * q) : 0.f;
    }
#pragma unroll 1
    for (int itn = 0; itn < 2; ++itn) {
#pragma unroll
      for (int r = 0; r + 1 < WN; ++r) {
        if (r + 1 < k) {
          const bool piv = (pvm >> r) & 1u;
          const float a0 = piv ? y[r + 1] : y[r], a1 = piv ? y[r] : y[r + 1];
          y[r] = a0;
          y[r + 1] = a1 - lm[r] * a0;
        }
      }
      float mx = 0.f;
#pragma unroll
      for (int r = WN - 1; r >= 0; --r) {
        if (r < k) {
          float v = y[r];
          if (r + 1 < WN && r + 1 < k) v -= u1[r] * y[r + 1];
          // the second superdiagonal is nonzero only where rows were exchanged
          if (r + 2 < WN && r + 2 < k && ((pvm >> r) & 1u)) v -= se[r + 1] * y[r + 2];
          v *= u0[r];
          y[r] = v;
          mx = fmaxf(mx, fabsf(v));
        }
      }
      const float inv = (mx > 0.f && isfinite(mx)) ? 1.f / mx : 1.f;
#pragma unroll
      for (int r = 0; r < WN; ++r) y[r] *= inv;
    }
#pragma unroll
    for (int r = 0; r < WN; ++r) sZ[r][q] = y[r];
  }
  __syncthreads();
  RW_MARK(6);

  // ---- 7. CGS2 (warp 0, lane = coordinate), then the back-transform y <- H_0 ... H_{k-3} y
  //      (vector q by warp q mod 8) ----
  if (wid == 0) {
#pragma unroll 1
    for (int j = 0; j < M; ++j) {
      float zj = sZ[lane][j];
#pragma unroll 1
      for (int pass = 0; pass < 2; ++pass) {
        int i2 = 0;
#pragma unroll 1
        for (; i2 + 4 <= j; i2 += 4) {
          const float z0 = sZ[lane][i2], z1 = sZ[lane][i2 + 1], z2 = sZ[lane][i2 + 2], z3 = sZ[lane][i2 + 3];
          float d0 = z0 * zj, d1 = z1 * zj, d2 = z2 * zj, d3 = z3 * zj;
#pragma unroll
          for (int o = 16; o; o >>= 1) {
            d0 += __shfl_xor_sync(0xffffffffu, d0, o);
            d1 += __shfl_xor_sync(0xffffffffu, d1, o);
            d2 += __shfl_xor_sync(0xffffffffu, d2, o);
            d3 += __shfl_xor_sync(0xffffffffu, d3, o);
          }
          zj -= d0 * z0 + d1 * z1 + d2 * z2 + d3 * z3;
        }
#pragma unroll 1
        for (; i2 < j; ++i2) {
          const float zi = sZ[lane][i2];
          zj -= warp_sum(zi * zj) * zi;
        }
      }
      const float nn = warp_sum(zj * zj);
      sZ[lane][j] = (nn > 0.f) ? zj * rsqrtf(nn) : 0.f;
      __syncwarp();
    }
  }
  __syncthreads();
  for (int q = wid; q < M; q += kRWThreads / 32) {
    float z = sZ[lane][q];
#pragma unroll 1
    for (int j = k - 3; j >= 0; --j) {
      const float tj = sht[j], hv = sH[j][lane];
      z -= tj * warp_sum(hv * z) * hv;
    }
    sZ[lane][q] = (lane < k) ? z : 0.f;
  }
  __syncthreads();
  RW_MARK(7);

  // ---- 8. Ritz coefficients: z = L^-T y, C_x = D z / sqrt(mu), Lambda = 1 / mu ----
  for (int t = threadIdx.x; t < WN * M; t += kRWThreads) {
    const int r = t / M, q = t % M;
    float v = 0.f;
#pragma unroll 8
    for (int s_ = 0; s_ < k; ++s_) v += sL[s_][r] * sZ[s_][q];
    sU[r][q] = v;
  }
  const int badmu = __syncthreads_or(threadIdx.x < M && !(smu[threadIdx.x] > 0.f && isfinite(smu[threadIdx.x])));
  if (badmu) {
    if (threadIdx.x == 0) { a.st->done = DONE_ERROR; a.st->err = MGE_ENOTFINITE; a.st->bad_stage = 4; }
    return;
  }
  // the coefficients go straight into the block-precision copies the update kernel reads
  // (this form runs for FP32 blocks only); rows of dropped directions are zero
  SmallT<float>* cf = static_cast<SmallT<float>*>(a.smt);
  for (int t = threadIdx.x; t < n * M; t += kRWThreads) {
    const int i = t / M, q = t % M, r = sinv[i];
    cf->Cx[i * MAXM + q] = r >= 0 ? sdf[i] * (sU[r][q] * rsqrtf(smu[q])) : 0.f;
    if (nx == 0) cf->Cp[i * MAXM + q] = 0.f;
  }
  if (threadIdx.x < M) {
    const double lam = 1.0 / (double)smu[threadIdx.x];
    sm->lam[threadIdx.x] = lam;
    cf->lam[threadIdx.x] = (float)lam;
  }
  RW_MARK(8);

  // ---- 9. C_p: in u = L^T z coordinates the G_B inner product is u^T M u'; the Ritz vectors
  //      are y / sqrt(mu) with M y = mu y, so M-orthogonality to them is orthogonality to y.
  //      All matrices are zero outside k x k, so the sums run over all 32 indices. ----
  if (nx > 0) {
    if (threadIdx.x < WN) sp[threadIdx.x] = (threadIdx.x < k && sidx[threadIdx.x] >= nx) ? 1.f : 0.f;
    __syncthreads();
    for (int t = threadIdx.x; t < WN * M; t += kRWThreads) {    // u = L^T z_p (X rows of z zeroed)
      const int r = t / M, q = t % M;
      float v0 = 0.f, v1 = 0.f;
#pragma unroll
      for (int s_ = 0; s_ < WN; s_ += 2) {
        v0 += sA[s_][r] * (sU[s_][q] * sp[s_]);
        v1 += sA[s_ + 1][r] * (sU[s_ + 1][q] * sp[s_ + 1]);
      }
      sV[r][q] = v0 + v1;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < M * M; t += kRWThreads) {     // Y^T u
      const int i2 = t / M, q = t % M;
      float v0 = 0.f, v1 = 0.f;
#pragma unroll
      for (int r = 0; r < WN; r += 2) {
        v0 += sZ[r][i2] * sV[r][q];
        v1 += sZ[r + 1][i2] * sV[r + 1][q];
      }
      sgp[i2][q] = v0 + v1;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < WN * M; t += kRWThreads) {    // u <- u - Y (Y^T u)
      const int r = t / M, q = t % M;
      float v = sV[r][q];
#pragma unroll
      for (int i2 = 0; i2 < MAXM; ++i2)
        if (i2 < M) v -= sZ[r][i2] * sgp[i2][q];
      sU[r][q] = v;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < WN * M; t += kRWThreads) {    // M u
      const int r = t / M, q = t % M;
      float v0 = 0.f, v1 = 0.f;
#pragma unroll
      for (int c = 0; c < WN; c += 2) {
        v0 += sM[r][c] * sU[c][q];
        v1 += sM[r][c + 1] * sU[c + 1][q];
      }
      sV[r][q] = v0 + v1;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < MAXM * MAXM; t += kRWThreads) {   // G_p = u^T M u (zero padded)
      const int i2 = t / MAXM, q = t % MAXM;
      float v0 = 0.f, v1 = 0.f;
      if (i2 < M && q < M) {
#pragma unroll
        for (int r = 0; r < WN; r += 2) {
          v0 += sU[r][i2] * sV[r][q];
          v1 += sU[r + 1][i2] * sV[r + 1][q];
        }
      }
      sgp[i2][q] = v0 + v1;
    }
    __syncthreads();
    if (wid == 0) {                 // Cholesky of G_p with dropping (lower triangle), lane = row
      const float tp = (float)a.tau_p;
#pragma unroll 1
      for (int j = 0; j < M; ++j) {
        const float gjj = sgp[j][j];
        const bool ok = gjj > tp && isfinite(gjj);
        const float rinv = ok ? rsqrtf(gjj) : 0.f;
        const int rl = lane < MAXM ? lane : 0;
        const float lj = (lane > j && lane < M) ? sgp[rl][j] * rinv : 0.f;
        __syncwarp();
        const float dj = (lane == j) ? gjj * rinv : lj;
        if (lane < MAXM) sgp[lane][j] = dj;
        // l_cj = 0 for c <= j: entries above the diagonal pick up values that are never read
#pragma unroll
        for (int c = 0; c < MAXM; ++c) {
          const float lc = __shfl_sync(0xffffffffu, lj, c);
          if (c > j && lane < MAXM) sgp[lane][c] -= lj * lc;
        }
        __syncwarp();
      }
      if (lane < M) srdp[lane] = sgp[lane][lane] > 0.f ? 1.f / sgp[lane][lane] : 0.f;
    }
    __syncthreads();
    for (int r = threadIdx.x; r < k; r += kRWThreads) {         // u <- u L_p^-T, row by row
      float ur[MAXM];
#pragma unroll
      for (int c = 0; c < MAXM; ++c) {
        if (c < M) {
          float v = sU[r][c];
#pragma unroll
          for (int s_ = 0; s_ < c; ++s_) v -= ur[s_] * sgp[c][s_];
          ur[c] = v * srdp[c];
          sU[r][c] = ur[c];
        } else {
          ur[c] = 0.f;
        }
      }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < n * M; t += kRWThreads) {     // z_p = L^-T u, C_p = D z_p
      const int i = t / M, q = t % M, r = sinv[i];
      float v0 = 0.f, v1 = 0.f;
      if (r >= 0) {
#pragma unroll
        for (int s_ = 0; s_ < WN; s_ += 2) {
          v0 += sL[s_][r] * sU[s_][q];
          v1 += sL[s_ + 1][r] * sU[s_ + 1][q];
        }
      }
      cf->Cp[i * MAXM + q] = sdf[i] * (v0 + v1);
    }
  }
  __syncthreads();
  // ---- correction of the Ritz coefficients against the FP64 pencil (see k_rr_inv, step 11):
  //      c -= G_A^-1 (G_A - theta G_B) c, with G_A^-1 = D L^-T L^-1 D and L^-1 in sL (compact).
  //      runs after C_p, whose sU and sV it reuses: sV holds D r (compact rows), sU
  //      w = L^-1 D r.  The FP64 Gram partials are read again here and cleared after. ----
  const bool refine = a.st->refine != 0;
  for (int t = threadIdx.x; t < WN * M && refine; t += kRWThreads) {
    const int r = t / M, q = t % M;
    float v = 0.f;
    if (r < k) {
      const int i = sidx[r];
      const double th = sm->lam[q];
      double acc = 0.0;
      for (int j = 0; j < n; ++j) {
        const int bi = i / 4, bj = j / 4;      // the Grams as step 1 symmetrised them, in FP64
        const double ga = sym_a_entry(sm->partA[0][i * MAXS + j], sm->partA[0][j * MAXS + i],
                                      sm->partA[0][i * MAXS + i], sm->partA[0][j * MAXS + j]);
        const double gb = bi < bj ? sm->partB[0][i * MAXS + j] : bi > bj ? sm->partB[0][j * MAXS + i]
                                  : 0.5 * (sm->partB[0][i * MAXS + j] + sm->partB[0][j * MAXS + i]);
        acc += (ga - th * gb) * (double)cf->Cx[j * MAXM + q];
      }
      v = (float)((double)sdf[i] * acc);
    }
    sV[r][q] = v;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < WN * M; t += kRWThreads) {      // w = L^-1 (D r), lower triangular
    const int r = t / M, q = t % M;
    float v = 0.f;
    for (int s_ = 0; s_ <= r && s_ < k; ++s_) v += sL[r][s_] * sV[s_][q];
    sU[r][q] = v;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < WN * M; t += kRWThreads) {      // z = L^-T w (compact rows)
    const int r = t / M, q = t % M;
    float v = 0.f;
    for (int s_ = r; s_ < k; ++s_) v += sL[s_][r] * sU[s_][q];
    sV[r][q] = v;
  }
  __syncthreads();
  if (threadIdx.x < M) {                 // kept only while small (see kRefineMax)
    const int q = threadIdx.x;
    float nz = 0.f, nc = 0.f;
    for (int r = 0; r < k; ++r) {
      const float z = sV[r][q], c = cf->Cx[sidx[r] * MAXM + q] / sdf[sidx[r]];
      nz += z * z;
      nc += c * c;
    }
    smu[q] = (refine && nz <= kRefineMax * kRefineMax * nc) ? 1.f : 0.f;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < n * M; t += kRWThreads) {       // C_x -= D z
    const int i = t / M, q = t % M, r = sinv[i];
    if (r >= 0 && smu[q] != 0.f) cf->Cx[i * MAXM + q] -= sdf[i] * sV[r][q];
  }
  __syncthreads();
  for (int t = threadIdx.x; t < n * n; t += kRWThreads) {      // the next Gram starts from zero
    const int i = t / n, j = t % n;
    sm->partA[0][i * MAXS + j] = 0.0;
    sm->partB[0][i * MAXS + j] = 0.0;
  }
  RW_MARK(11);
  __syncthreads();
  if (threadIdx.x < 12) a.st->rr_clk[threadIdx.x] = sclk[threadIdx.x];
  if (threadIdx.x == 0) a.st->kept = k;
#undef RW_MARK
}

// ---------------------------------------------------------------------------------------
// FP64 form: Cholesky of G^_B with dropping, standard form, cyclic two-sided Jacobi
// ---------------------------------------------------------------------------------------
__device__ int jacobi_eig(double* A, double* V, int ld, int k) {
  __shared__ int rotated;
  __shared__ double cs_c[MAXS / 2 + 1], cs_s[MAXS / 2 + 1];
  __shared__ int pr_p[MAXS / 2 + 1], pr_q[MAXS / 2 + 1];
  for (int t = threadIdx.x; t < k * k; t += blockDim.x) V[(t / k) * ld + t % k] = (t / k == t % k) ? 1.0 : 0.0;
  const int kk = k + (k & 1);
  const int np = kk / 2;
  int sweeps = 0;
  __syncthreads();
  if (k < 2) return 0;
  for (; sweeps < 60; ++sweeps) {
    if (threadIdx.x == 0) rotated = 0;
    __syncthreads();
    for (int s = 0; s < kk - 1; ++s) {
      if (threadIdx.x < np) {
        int i = threadIdx.x;
        int p, q;
        if (i == 0) { p = kk - 1; q = s; }
        else { p = (s + i) % (kk - 1); q = (s - i + kk - 1) % (kk - 1); }
        if (p > q) { int t = p; p = q; q = t; }
        double c = 1.0, sn = 0.0;
        if (q < k) {
          double app = A[p * ld + p], aqq = A[q * ld + q], apq = A[p * ld + q];
          if (apq != 0.0 && fabs(apq) > 1e-17 * sqrt(fabs(app * aqq))) {
            double theta = (aqq - app) / (2.0 * apq);
            double t;
            if (fabs(theta) > 1e150) t = 0.5 / theta;
            else t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
            c = 1.0 / sqrt(t * t + 1.0);
            sn = t * c;
            rotated = 1;
          }
        }
        pr_p[i] = p; pr_q[i] = q; cs_c[i] = c; cs_s[i] = sn;
      }
      __syncthreads();
      for (int t = threadIdx.x; t < np * k; t += blockDim.x) {
        int i = t / k, j = t % k;
        double s_ = cs_s[i];
        if (s_ == 0.0) continue;
        double c = cs_c[i];
        int p = pr_p[i], q = pr_q[i];
        double ap = A[p * ld + j], aq = A[q * ld + j];
        A[p * ld + j] = c * ap - s_ * aq;
        A[q * ld + j] = s_ * ap + c * aq;
      }
      __syncthreads();
      for (int t = threadIdx.x; t < np * k; t += blockDim.x) {
        int i = t / k, j = t % k;
        double s_ = cs_s[i];
        if (s_ == 0.0) continue;
        double c = cs_c[i];
        int p = pr_p[i], q = pr_q[i];
        double ap = A[j * ld + p], aq = A[j * ld + q];
        A[j * ld + p] = c * ap - s_ * aq;
        A[j * ld + q] = s_ * ap + c * aq;
        double vp = V[j * ld + p], vq = V[j * ld + q];
        V[j * ld + p] = c * vp - s_ * vq;
        V[j * ld + q] = s_ * vp + c * vq;
      }
      __syncthreads();
    }
    int r = rotated;
    __syncthreads();
    if (!r) break;
  }
  return sweeps;
}

__global__ void __launch_bounds__(kThreads) k_rr_jacobi(RRArgs a) {
  if (a.st->done || !rr_selected(a.sel, a.st)) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int M = a.M, n = a.nb * a.M, nx = a.nx;
  const int ld = n + 1;
  double* bufA = reinterpret_cast<double*>(smem_raw);
  double* bufB = bufA + n * ld;
  double* bufC = bufB + n * ld;
  double* bufV = bufC + n * ld;
  __shared__ double dsc[MAXS], tau[MAXS], theta[MAXS], rdb[MAXS];
  __shared__ int keep[MAXS], idx[MAXS], order[MAXS], pkeep[MAXM];
  __shared__ int kcount;
  Small* sm = a.sm;
  if (!load_grams(a, bufA, bufB, n, ld)) {
    if (threadIdx.x == 0) { a.st->done = DONE_ERROR; a.st->err = MGE_ENOTFINITE; a.st->bad_stage = 1; }
    return;
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double d = bufB[i * ld + i];
    bool live = d > 0.0 && isfinite(d);
    dsc[i] = live ? 1.0 / sqrt(d) : 0.0;
    keep[i] = live ? 1 : 0;
    tau[i] = a.tau;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
    int i = t / n, j = t % n;
    double s = dsc[i] * dsc[j];
    bufA[i * ld + j] *= s;
    bufB[i * ld + j] *= s;
  }
  __syncthreads();
  chol_drop<double>(bufB, ld, n, tau, keep, rdb);
  if (threadIdx.x == 0) {
    int c = 0;
    for (int i = 0; i < n; ++i) if (keep[i]) idx[c++] = i;
    kcount = c;
  }
  __syncthreads();
  const int k = kcount;
  if (k < M) {
    if (threadIdx.x == 0) { a.st->done = stall_or_error(a.st); a.st->err = MGE_ECHOLESKY; a.st->kept = k; }
    return;
  }
  if (threadIdx.x == 0 && k < n) atomicAdd(&a.st->drops, 1);
  for (int t = threadIdx.x; t < k * k; t += blockDim.x) {
    int r = t / k, c = t % k;
    bufC[r * ld + c] = bufA[idx[r] * ld + idx[c]];
  }
  __syncthreads();
  for (int t = threadIdx.x; t < k * k; t += blockDim.x) {
    int r = t / k, c = t % k;
    bufA[r * ld + c] = bufB[idx[r] * ld + idx[c]];
  }
  __syncthreads();
  double* Lk = bufA;
  for (int c = threadIdx.x; c < k; c += blockDim.x) {
    for (int r = 0; r < k; ++r) {
      double v = bufC[r * ld + c];
      for (int s = 0; s < r; ++s) v -= Lk[r * ld + s] * bufC[s * ld + c];
      bufC[r * ld + c] = v / Lk[r * ld + r];
    }
  }
  __syncthreads();
  for (int c = threadIdx.x; c < k; c += blockDim.x) {
    for (int r = 0; r < k; ++r) {
      double v = bufC[c * ld + r];
      for (int s = 0; s < r; ++s) v -= Lk[r * ld + s] * bufB[s * ld + c];
      bufB[r * ld + c] = v / Lk[r * ld + r];
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < k * k; t += blockDim.x) {
    int r = t / k, c = t % k;
    if (c > r) {
      double v = 0.5 * (bufB[r * ld + c] + bufB[c * ld + r]);
      bufB[r * ld + c] = v;
      bufB[c * ld + r] = v;
    }
  }
  __syncthreads();
  jacobi_eig(bufB, bufV, ld, k);
  for (int i = threadIdx.x; i < k; i += blockDim.x) theta[i] = bufB[i * ld + i];
  __syncthreads();
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    int rank = 0;
    double ti = theta[i];
    for (int j = 0; j < k; ++j) {
      double tj = theta[j];
      if (tj < ti || (tj == ti && j < i)) ++rank;
    }
    order[rank] = i;
  }
  __syncthreads();
  for (int c = threadIdx.x; c < M; c += blockDim.x) {
    int e = order[c];
    for (int r = k - 1; r >= 0; --r) {
      double v = bufV[r * ld + e];
      for (int s = r + 1; s < k; ++s) v -= Lk[s * ld + r] * bufC[s * ld + c];
      bufC[r * ld + c] = v / Lk[r * ld + r];
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < n * M; t += blockDim.x) { sm->Cx[(t / M) * MAXM + t % M] = 0.0; sm->Cp[(t / M) * MAXM + t % M] = 0.0; }
  __syncthreads();
  for (int t = threadIdx.x; t < k * M; t += blockDim.x) {
    int r = t / M, c = t % M;
    sm->Cx[idx[r] * MAXM + c] = dsc[idx[r]] * bufC[r * ld + c];
  }
  for (int c = threadIdx.x; c < M; c += blockDim.x) sm->lam[c] = theta[order[c]];
  if (nx > 0) {
    double* U = bufB;
    double* Z = bufC;
    __syncthreads();
    for (int t = threadIdx.x; t < k * M; t += blockDim.x) {
      int r = t / M, c = t % M;
      double v = 0.0;
      for (int s = r; s < k; ++s)
        if (idx[s] >= nx) v += Lk[s * ld + r] * Z[s * ld + c];
      U[r * ld + c] = v;
    }
    double* Gc = bufC + M;
    __syncthreads();
    for (int t = threadIdx.x; t < M * M; t += blockDim.x) {
      int i = t / M, c = t % M;
      double v = 0.0;
      int e = order[i];
      for (int r = 0; r < k; ++r) v += bufV[r * ld + e] * U[r * ld + c];
      Gc[i * ld + c] = v;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < k * M; t += blockDim.x) {
      int r = t / M, c = t % M;
      double v = U[r * ld + c];
      for (int i = 0; i < M; ++i) v -= bufV[r * ld + order[i]] * Gc[i * ld + c];
      U[r * ld + c] = v;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < M * M; t += blockDim.x) {
      int i = t / M, c = t % M;
      double v = 0.0;
      for (int r = 0; r < k; ++r) v += U[r * ld + i] * U[r * ld + c];
      Gc[i * ld + c] = v;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < M; i += blockDim.x) { pkeep[i] = 1; tau[i] = a.tau_p; }
    __syncthreads();
    chol_drop<double>(Gc, ld, M, tau, pkeep, rdb);
    for (int r = threadIdx.x; r < k; r += blockDim.x) {
      for (int c = 0; c < M; ++c) {
        double v = U[r * ld + c];
        double lcc = Gc[c * ld + c];
        if (lcc > 0.0) {
          for (int s = 0; s < c; ++s) v -= U[r * ld + s] * Gc[c * ld + s];
          U[r * ld + c] = v / lcc;
        } else {
          U[r * ld + c] = 0.0;
        }
      }
    }
    __syncthreads();
    for (int c = threadIdx.x; c < M; c += blockDim.x) {
      for (int r = k - 1; r >= 0; --r) {
        double v = U[r * ld + c];
        for (int s = r + 1; s < k; ++s) v -= Lk[s * ld + r] * Z[s * ld + c];
        Z[r * ld + c] = v / Lk[r * ld + r];
      }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < k * M; t += blockDim.x) {
      int r = t / M, c = t % M;
      sm->Cp[idx[r] * MAXM + c] = dsc[idx[r]] * Z[r * ld + c];
    }
  }
  __syncthreads();
  if (a.is_double) store_coeffs<double, double>(a);
  else store_coeffs<float, double>(a);
  if (threadIdx.x == 0) a.st->kept = k;
}

// Same factorisation for n <= 32 by one warp (lane = row, columns broadcast by shuffles);
// called by the whole warp, no block barrier.
template <typename R>
__device__ void chol_drop_warp(R* S, int ld, int n, const R* tau, int* keep, R* rd) {
  const int i = threadIdx.x & 31;
  const int ri = i < n ? i : 0;
  for (int j = 0; j < n; ++j) {
    const R v = S[j * ld + j];
    const bool ok = keep[j] && v > tau[j] && isfinite((double)v);
    const R piv = ok ? (R)sqrt(v) : R(0);
    const R rp = ok ? R(1) / piv : R(0);
    const R lij = (i > j && i < n) ? S[ri * ld + j] * rp : R(0);
    __syncwarp();
    for (int k = j + 1; k < n; ++k) {
      const R lkj = __shfl_sync(0xffffffffu, lij, k);
      if (k <= i && i < n) S[ri * ld + k] -= lij * lkj;
    }
    if (i == j) { S[j * ld + j] = piv; rd[j] = rp; keep[j] = ok ? 1 : 0; }
    if (i > j && i < n) S[ri * ld + j] = lij;
    __syncwarp();
  }
  for (int k = i + 1; k < n; ++k) S[ri * ld + k] = R(0);
  __syncwarp();
}

// ---------------------------------------------------------------------------------------
// wprep: backward errors and convergence; projections Mx, Mp and the normalisation of the
// projected W_raw (Cholesky with dropping, in R precision)
// ---------------------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(kThreads) k_wprep(WprepArgs a) {
  if (a.st->done || !rr_selected(a.sel, a.st)) return;
  const int M = a.M;
  Small* sm = a.sm;
  // The FP64 Gram partials are rounded to R once; everything after runs in R (FP32 for FP32
  // blocks: GB300's FP64 rate is a small fraction of its FP32 rate, conversions included).
  __shared__ R G2[MAXS * MAXM];
  __shared__ R cs[MAXM];
  __shared__ R G[MAXM * (MAXM + 1)];
  __shared__ R tau[MAXM], rdw[MAXM];
  __shared__ R sLinv[MAXM][MAXM + 1];
  __shared__ int keep[MAXM];
  __shared__ long long sclk[4];
  // phase clocks written by every thread (a branch around clock64 leaves warps diverged)
  const long long clk0 = clock64();
#define WP_MARK(k) (sclk[k] = clock64() - clk0)
  const int ld = M + 1;
  const int rows = (a.has_x ? M : 0) + (a.has_p ? M : 0) + M;
  for (int t = threadIdx.x; t < rows * M; t += blockDim.x) {
    int i = t / M, j = t % M;
    const double v = a.ncl_w == 1 ? sm->partW[0][i * MAXM + j] : sum_strided(&sm->partW[0][i * MAXM + j], a.ncl_w, MAXS * MAXM);
    G2[i * MAXM + j] = (R)v;
  }
  for (int t = threadIdx.x; t < M; t += blockDim.x) {
    const double v = !a.deflate ? 0.0 : a.ncl_w == 1 ? sm->partC[0][t] : sum_strided(&sm->partC[0][t], a.ncl_w, MAXM);
    cs[t] = (R)v;
  }
  int bad = 0, unconv = 0;
  __shared__ int rmax_bits;     // largest relative residual of the wanted pairs (float bits)
  if (threadIdx.x == 0) rmax_bits = 0;
  __syncthreads();
  if (a.check) {
    for (int k = threadIdx.x; k < M; k += blockDim.x) {
      const double rn2 = a.ncl_n == 1 ? sm->partN[0][k] : sum_strided(&sm->partN[0][k], a.ncl_n, 2 * MAXM);
      const double xn2 = a.ncl_n == 1 ? sm->partN[0][MAXM + k] : sum_strided(&sm->partN[0][MAXM + k], a.ncl_n, 2 * MAXM);
      const double lam = sm->lam[k];
      // relative residual rho = ||A x - lam B x||_{B^-1} / ((|lam| + u ||A||_G) ||x||_B): the
      // residual of the symmetric form B^-1/2 A B^-1/2 relative to the eigenvalue, with the
      // block precision's unit roundoff u times ||A||_G as a floor for lam = 0.  FP32
      // arithmetic is ample for a number compared with a tolerance.
      const float ufloor = a.is_double ? 1.1102230e-16f : 5.9604645e-8f;
      const float den = fabsf((float)lam) + ufloor * (float)a.norm;
      const float eta = sqrtf((float)rn2) / (den * sqrtf((float)xn2));
      bad |= !isfinite(eta) || !isfinite(lam);
      a.st->eta[k] = (double)eta;
      a.st->lambda[k] = lam;
      unconv |= k < a.K && !(eta <= (float)a.tol);
      if (k < a.K && isfinite(eta)) atomicMax(&rmax_bits, __float_as_int(eta));   // eta >= 0
    }
  }
  bad = __syncthreads_or(bad);
  unconv = __syncthreads_or(unconv);
  WP_MARK(0);
  if (a.check && threadIdx.x == 0) {
    a.st->iter += 1;
    if (bad) { a.st->done = DONE_ERROR; a.st->err = MGE_ENOTFINITE; a.st->bad_stage = 2; }
    else if (!unconv) a.st->done = DONE_CONVERGED;
    else if (a.st->iter >= a.maxiter) a.st->done = DONE_MAXITER;
    // stagnation of an FP32 Rayleigh-Ritz: its eigenvectors carry errors of about u times the
    // spread of the pencil, which floor the relative residual (measured: ~1e-5 on a 2M-node
    // sphere, whose eigenvalues come in near-degenerate groups); the FP64 form continues
    if (!a.st->done) {
      const float r = __int_as_float(rmax_bits);
      if (a.st->pbest_iter == 0 || r <= 0.5f * a.st->pbest_rho) { a.st->pbest_rho = r; a.st->pbest_iter = a.st->iter; }
      a.st->refine = r <= kRRStallGate * (float)a.tol && a.st->iter - a.st->pbest_iter < kRRStallIters;
    }
    if (a.rr_switch && !a.st->done && !a.st->rr64) {
      const float r = __int_as_float(rmax_bits);
      if (!(r <= kRRStallGate * (float)a.tol)) a.st->best_iter = 0;     // not near the target yet
      else if (a.st->best_iter == 0 || r <= 0.5f * a.st->best_rho) { a.st->best_rho = r; a.st->best_iter = a.st->iter; }
      else if (a.st->iter - a.st->best_iter >= kRRStallIters) { a.st->rr64 = 1; a.st->rr64_iter = a.st->iter; }
    }
  }
  const int ox = 0, op = a.has_x ? M : 0, ow = (a.has_x ? M : 0) + (a.has_p ? M : 0);
  const R inv_n = (R)(1.0 / (double)a.n);
  // the accumulators start the next reduction from zero (everything was read above)
  for (int t = threadIdx.x; t < rows * M; t += blockDim.x) {
    int i = t / M, j = t % M;
    for (int c = 0; c < a.ncl_w; ++c) sm->partW[c][i * MAXM + j] = 0.0;
  }
  for (int t = threadIdx.x; t < MAXM; t += blockDim.x) {
    for (int c = 0; c < a.ncl_w; ++c) sm->partC[c][t] = 0.0;
    for (int c = 0; c < a.ncl_n; ++c) { sm->partN[c][t] = 0.0; sm->partN[c][MAXM + t] = 0.0; }
  }
  int bad_g = 0;
  for (int t = threadIdx.x; t < M * M; t += blockDim.x) {
    int i = t / M, j = t % M;
    // G_W - M_x^T M_x - M_p^T M_p - n c c^T: entries below tau_w * G_jj are dropped anyway
    R g = R(0.5) * (G2[(ow + i) * MAXM + j] + G2[(ow + j) * MAXM + i]);
    for (int l = 0; l < M; ++l) {
      if (a.has_x) g -= G2[(ox + l) * MAXM + i] * G2[(ox + l) * MAXM + j];
      if (a.has_p) g -= G2[(op + l) * MAXM + i] * G2[(op + l) * MAXM + j];
    }
    if (a.deflate) g -= cs[i] * cs[j] * inv_n;
    G[i * ld + j] = g;
    bad_g |= !isfinite(g);
  }
  for (int t = threadIdx.x; t < M; t += blockDim.x) {
    const R g0 = G2[(ow + t) * MAXM + t];
    tau[t] = (R)a.tau_w * g0;
    keep[t] = (g0 > R(0) && isfinite(g0)) ? 1 : 0;
  }
  bad_g = __syncthreads_or(bad_g);
  if (bad_g) {
    if (threadIdx.x == 0) { a.st->done = DONE_ERROR; a.st->err = MGE_ENOTFINITE; a.st->bad_stage = 3; }
    return;
  }
  WP_MARK(1);
  if (threadIdx.x < 32) chol_drop_warp<R>(G, ld, M, tau, keep, rdw);
  __syncthreads();
  WP_MARK(2);
  // L = L_G^-T (upper triangular): column c solves L_G^T y = e_c, y in registers
  for (int c = threadIdx.x; c < M; c += blockDim.x) {
    R y[MAXM];
#pragma unroll
    for (int r = MAXM - 1; r >= 0; --r) {
      R v = (r == c) ? R(1) : R(0);
#pragma unroll
      for (int s_ = r + 1; s_ < MAXM; ++s_)
        if (s_ < M) v -= G[s_ * ld + r] * y[s_];
      y[r] = (r < M && rdw[r] > R(0)) ? v * rdw[r] : R(0);
    }
#pragma unroll
    for (int r = 0; r < MAXM; ++r)
      if (r < M) sLinv[r][c] = y[r];
  }
  __syncthreads();
  // publish L and the products the SpMM epilogue applies: M_x L, M_p L with
  // M_x = X^T B W_raw, M_p = P^T B W_raw, and c L with c the column means of W_raw
  for (int t = threadIdx.x; t < M * M; t += blockDim.x) {
    const int i = t / M, c = t % M;
    R mxl = R(0), mpl = R(0);
    for (int l = 0; l < M; ++l) {
      if (a.has_x) mxl += G2[(ox + i) * MAXM + l] * sLinv[l][c];
      if (a.has_p) mpl += G2[(op + i) * MAXM + l] * sLinv[l][c];
    }
    const int o = i * MAXM + c;
    if (a.is_double) {
      SmallT<double>* d = static_cast<SmallT<double>*>(a.smt);
      d->Linv[o] = (double)sLinv[i][c]; d->MxL[o] = (double)mxl; d->MpL[o] = (double)mpl;
    } else {
      SmallT<float>* f = static_cast<SmallT<float>*>(a.smt);
      f->Linv[o] = (float)sLinv[i][c]; f->MxL[o] = (float)mxl; f->MpL[o] = (float)mpl;
    }
  }
  for (int c = threadIdx.x; c < M; c += blockDim.x) {
    R cl = R(0);
    if (a.deflate)
      for (int l = 0; l < M; ++l) cl += cs[l] * inv_n * sLinv[l][c];
    if (a.is_double) static_cast<SmallT<double>*>(a.smt)->cL[c] = (double)cl;
    else static_cast<SmallT<float>*>(a.smt)->cL[c] = (float)cl;
  }
  WP_MARK(3);
  __syncthreads();
  if (threadIdx.x < 4) a.st->wp_clk[threadIdx.x] = sclk[threadIdx.x];
#undef WP_MARK
}

// ---------------------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------------------
size_t rr_inv_smem(int n) {
  size_t d = 2 * (size_t)n * (n + 1) * sizeof(double);
  size_t f = 3 * (size_t)n * (n + 1) * sizeof(float) + (size_t)n * MAXM * sizeof(float) +
             (size_t)MAXM * 6 * n * sizeof(float);
  return d + f;
}
size_t rr_jacobi_smem(int n) { return 4 * (size_t)n * (n + 1) * sizeof(double); }

cudaError_t rr_configure() {
  cudaError_t e = cudaFuncSetAttribute(k_rr_inv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rr_inv_smem(MAXS));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_rr_jacobi, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rr_jacobi_smem(MAXS));
}

void launch_rr(cudaStream_t st, const RRArgs& a, bool inverse_form) {
  int n = a.nb * a.M;
  if (inverse_form && n <= WN) k_rr_warp<<<1, kRWThreads, 0, st>>>(a);
  else if (inverse_form) k_rr_inv<<<1, kRRThreads, rr_inv_smem(n), st>>>(a);
  else k_rr_jacobi<<<1, kThreads, rr_jacobi_smem(n), st>>>(a);
}

void launch_wprep(cudaStream_t st, const WprepArgs& a, bool fp64) {
  if (fp64) k_wprep<double><<<1, kThreads, 0, st>>>(a);
  else k_wprep<float><<<1, kThreads, 0, st>>>(a);
}

}  // namespace lob
}  // namespace mge
