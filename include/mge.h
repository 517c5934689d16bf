/*
 * mge.h -- C ABI of libmge: generalized-eigenvector manifold graph embedding on one GPU.
 *
 * The library computes the graph embedding of "Fast computation of Generalized
 * Eigenvectors for Manifold Graph Embedding" (Chen, Cheung, Zhang): for an input graph
 * G(V, E, W) it builds the sparse pair
 *     A = L - mu Q + eps I,   B = diag(b_i)                         (Eq. 6, Sec. 4.3)
 * and returns the first K generalized eigenpairs A q = lambda B q, q_i^T B q_j = delta_ij
 * (Eq. 10-11), found by LOBPCG (Sec. 4.3; Knyazev's locally optimal block
 * preconditioned conjugate gradient method).  All arithmetic runs in the library's own
 * CUDA kernels for sm_103a; there is no CPU fallback.
 *
 * Conventions shared by every entry point
 *   - Errors are returned as mge_status codes; nothing aborts and no C++ exception
 *     crosses this boundary.  mge_ctx_last_error() gives a one-line message for the last
 *     failing call on a context.
 *   - Pointers flagged "host or device" are device pointers when the matching on_device
 *     flag is nonzero, host pointers otherwise.  Device pointers must belong to the
 *     context's device.  Caller buffers stay caller-owned; the library never frees them.
 *   - Handles (mge_ctx, mge_ops) are library-owned and freed by their destroy call.  An ops
 *     handle may outlive its context: after mge_destroy it can still be exported and must
 *     still be passed to mge_ops_destroy, which releases its device memory.
 *   - A context is used by one host thread at a time, except mge_submit/mge_poll/
 *     mge_release, which are thread-safe.
 *   - Streams are passed as void* (a cudaStream_t); NULL selects the context's stream.
 *     Calls return after the results they write are complete on the host side.
 *   - Graph inputs are canonical CSR: row_ptr int64[n+1] with row_ptr[0] = 0, col int32
 *     strictly ascending within each row, no diagonal entries, weights finite and > 0,
 *     and the matrix symmetric (W_ij == W_ji bitwise).
 *   - Block vectors returned to callers (V) are FP64, column-major [n x K].
 *   - Eigenpairs come out in ascending lambda; each vector's sign is fixed so that its
 *     entry of largest magnitude is positive (lowest index on ties).
 */
#ifndef MGE_H
#define MGE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  MGE_OK = 0,
  MGE_EINVAL = 1,         /* invalid argument or malformed CSR                              */
  MGE_ENOTSYM = 2,        /* W is not symmetric                                             */
  MGE_EISOLATED = 3,      /* some r_i = 0 (isolated node): B is singular (Sec. 4.3)          */
  MGE_EDEGENERATE = 4,    /* eps = lambda_2(Q) = 0: the two-hop graph is disconnected
                             (Sec. 4.2); mu = 0 and A = L.  Outputs are still produced.      */
  MGE_ENOTCONVERGED = 5,  /* maxiter reached, or the iteration stagnated below what its
                             precision reaches (its basis collapsed after the first
                             iterations); the current Ritz pairs and residuals returned     */
  MGE_ENOMEM = 6,         /* device allocation failed or the HBM budget is exceeded          */
  MGE_EAGAIN = 7,         /* serving queue or HBM budget full; retry later                   */
  MGE_ETIMEOUT = 8,       /* mge_poll timed out, or a bounded device loop hit its limit      */
  MGE_EDEVICE = 9,        /* a CUDA runtime error                                           */
  MGE_ECHOLESKY = 10,     /* the Rayleigh-Ritz basis collapsed (fewer than m independent
                             directions): the block is rank deficient                       */
  MGE_ENOTFOUND = 11,     /* unknown ticket                                                  */
  MGE_ENOTFINITE = 12     /* a NaN or Inf appeared in the iteration                          */
} mge_status;

/* Arithmetic of the iterated blocks X, W, P and of the stored matrix values.
 *   MGE_FP64  everything in FP64, including the Rayleigh-Ritz eigensolve (cyclic Jacobi).
 *   MGE_FP32  FP32 blocks and SpMM; Gram sums in FP32 with compensation (on graphs of at
 *             least 65,536 nodes: TF32 tensor cores on split operands, see
 *             mge_embed_opts.gram_cuda_cores), reduced across the GPU in FP64; residual
 *             norms in FP64; the Rayleigh-Ritz scaling in FP64 and its eigensolve in FP32 on
 *             the inverse pencil (the wanted smallest eigenvalues become the largest, which
 *             FP32 resolves to relative accuracy), followed by one correction of the Ritz
 *             coefficients against the FP64 residual of the pencil (see
 *             mge_embed_opts.rr_fp64).
 *   MGE_BF16  as MGE_FP32, with the LOBPCG preconditioner's blocks -- its right-hand side
 *             D^-1 R, the Chebyshev iterates and corrections -- stored in BF16 (FP32
 *             arithmetic in registers; the matrix values stay FP32 so that the Chebyshev
 *             interval's Gershgorin bound holds).  These blocks are all but a few of the
 *             bytes a LOBPCG iteration streams.  X, W, P and their products stay FP32: a
 *             Ritz vector rounded to BF16 carries a residual of about u_bf16 ||A|| |x|, which
 *             on manifold graphs (||A|| / lambda_1 ~ 1e5-1e6) is far above any useful
 *             tolerance.  Falls back to FP32 preconditioner blocks when the sliced copy of
 *             the preconditioner's operator was not built.  The preconditioner degree is
 *             capped at 8: the Chebyshev polynomial scales the bottom of the spectrum by
 *             about 2 d^2 against the top, and BF16 rounding of its iterates (u = 2^-8)
 *             spoils the directions LOBPCG needs once u 2 d^2 > 1.  Measured on a 200k-node
 *             swiss roll (K = 8, tol 1e-5): no faster per Chebyshev step than FP32 (the step
 *             is bound by gather latency, not bytes) and more iterations, so MGE_FP32 is the
 *             faster form on this path; MGE_BF16 is kept for callers that must halve the
 *             preconditioner's memory. */
typedef enum { MGE_FP64 = 0, MGE_FP32 = 1, MGE_BF16 = 2 } mge_precision;

typedef struct mge_ctx mge_ctx;
typedef struct mge_ops mge_ops;

/* ---- context ----------------------------------------------------------------------- */

/* Creates a context on CUDA device `device`.  hbm_budget_bytes bounds the device memory the
 * context may hold (0 = no limit beyond the device's).  Errors: MGE_EINVAL, MGE_EDEVICE. */
mge_status mge_create(int device, size_t hbm_budget_bytes, mge_ctx** out);
mge_status mge_destroy(mge_ctx* ctx);
const char* mge_strerror(mge_status s);
const char* mge_ctx_last_error(const mge_ctx* ctx);

typedef struct {
  uint64_t kernel_launches;   /* kernels this context has launched (graph nodes included)   */
  uint64_t spmm_launches;     /* SpMM launches recorded while kernel timing was on           */
  double   spmm_ms;           /* their summed CUDA-event duration                           */
  uint64_t spmm_bytes;        /* their summed algorithmic bytes                             */
  size_t   hbm_in_use;        /* bytes of device memory the context holds                   */
  uint64_t tune_entries;      /* kernel configurations the context's autotuner holds        */
} mge_stats;

/* Copies the context's counters.  mge_ctx_set_timing(ctx, 1) brackets every SpMM launch
 * with CUDA events (for roofline measurement); 0 turns it off; mge_ctx_reset_stats zeroes. */
mge_status mge_ctx_stats(const mge_ctx* ctx, mge_stats* out);
mge_status mge_ctx_set_timing(mge_ctx* ctx, int on);
mge_status mge_ctx_reset_stats(mge_ctx* ctx);

/* Kernel autotuning.  The LOBPCG preconditioner's Chebyshev step (the solve's dominant kernel)
 * has several launch configurations -- its shared-memory stage budget (32, 48, 64 or 96 KB per
 * CTA: staged indices against L1 room for the gathers in flight) and, in FP32, whether each
 * row's own blocks are loaded before its gathers -- which all compute the same values in the
 * same order.  A solve looks up the configuration for its shape, the key
 *   cheb/m<block width>/<f32|f64>/n2^<floor(log2 n)>/slots<densest tile's slots / 128>,
 * and, when the key is new and mode is 1, times every configuration on its own operator
 * before its first launch (outside any stream capture; a few dozen launches of the step) and
 * keeps the fastest.
 *   mode 0: fixed rules (64 KB, no early loads);  1 (default): tune new keys;  2: use known
 *           keys only, fixed rules otherwise.
 *   cache_path: a JSON file (object of key -> {"budget": bytes, "prefetch": 0|1, "us": time
 *           per launch}) read now, if it exists, and rewritten whenever a key is added; NULL
 *           keeps the entries in the context only.
 * Errors: MGE_EINVAL (mode out of range, or a cache file that does not parse). */
mge_status mge_ctx_set_autotune(mge_ctx* ctx, int mode, const char* cache_path);

/* ---- kNN graph from points (Sec. 5.1) ---------------------------------------------- */

/* The paper's input graphs are kNN graphs built from Euclidean distances between samples
 * (Sec. 5.1).  mge_knn_graph builds one on the device:
 *   - the exact k nearest neighbours of every point (itself excluded); the squared distance
 *     is the sum over coordinates, in order, of (p_c - q_c)^2 with every product and sum
 *     rounded to FP64 separately (no fused multiply-add); equal distances go to the lower
 *     index;
 *   - the union of the directed relations (i ~ j when either is among the other's k nearest);
 *   - Gaussian weights w_ij = exp(-d_ij^2 / sigma^2), sigma the mean of the n k directed
 *     nearest-neighbour distances.
 * The result is canonical CSR (ascending columns, no diagonal, symmetric), ready for
 * mge_build_graph_ops with on_device = 1 (see mge_graph_csr).
 * points: row-major [n x dim] FP64, host or device per on_device (a device pointer of the
 * context's device, 16-byte aligned), read only.
 * dim in {2, 3}; 1 <= k <= 32; k < n < 2^31.  stream: cudaStream_t or NULL.
 * Errors: MGE_EINVAL (sizes; non-finite coordinates; all points coincident; a row with more
 * than 1024 candidate neighbours, which only many coincident points produce), MGE_ENOMEM,
 * MGE_EDEVICE. */
typedef struct mge_graph mge_graph;
mge_status mge_knn_graph(mge_ctx* ctx, int64_t n, int dim, const double* points, int on_device, int k,
                         void* stream, mge_graph** out);
/* n, nnz (directed entries of the CSR) and sigma of a graph; any pointer may be NULL. */
mge_status mge_graph_info(const mge_graph* g, int64_t* n, int64_t* nnz, double* sigma);
/* The device arrays of the graph (row_ptr [n+1], col [nnz], w [nnz]), borrowed: valid until
 * mge_graph_destroy.  Pass them to mge_build_graph_ops with on_device = 1. */
mge_status mge_graph_csr(const mge_graph* g, const int64_t** row_ptr, const int32_t** col,
                         const double** w);
/* Copies the CSR out; any pointer may be NULL; on_device selects device or host destinations. */
mge_status mge_graph_export(const mge_graph* g, int64_t* row_ptr, int32_t* col, double* w,
                            int on_device);
mge_status mge_graph_destroy(mge_graph* g);

/* ---- graph operators (Sec. 3.1, Sec. 4.1-4.3) --------------------------------------- */

typedef struct {
  int      precision;         /* mge_precision of the eps solve and of the stored A values  */
  int      eps_override_set;  /* nonzero: use eps_override instead of solving lambda_2(Q)   */
  double   eps_override;
  int      mu_override_set;   /* nonzero: use mu_override instead of Eq. 9                  */
  double   mu_override;
  double   eps_tol;           /* relative-residual tolerance of the eps solve (the measure
                                 of mge_embed; 0 = default: 1e-10 in FP64, 1e-4 otherwise:
                                 eps then carries a relative error below 1e-6, measured)     */
  int      eps_guard;         /* extra LOBPCG columns for the eps solve (default 7)         */
  int      eps_maxiter;       /* default 20000                                              */
  uint64_t seed;              /* seed of the eps solve's initial block                      */
  void*    stream;            /* cudaStream_t or NULL                                       */
  int      eps_precond_degree; /* Chebyshev preconditioner degree of the eps solve (see
                                 mge_embed_opts.precond_degree; 0 = default
                                 round(sqrt(n) / 12) within [8, 32]; at most 256)            */
  int      keep_order;        /* 0 (default): the library renumbers the nodes internally into
                                 a locality order (compact patches of the graph in
                                 consecutive rows, so that the SpMMs' gathers share cache
                                 lines); every API call still takes and returns arrays in
                                 the caller's node order.  1: keep the caller's numbering.   */
} mge_ops_opts;

/* Builds the operators of Sec. 4 for the graph W (n nodes, CSR as described above; host
 * or device pointers per on_device; read only):
 *   T_i    two-hop sets: j reachable in two hops with (i, j) not an edge (Sec. 4.1.1)
 *   Q      sum_i Theta_i (Eq. 5), Theta_i = (1/T_i) * Laplacian of the star (i, T_i)
 *   eps    lambda_2(Q), the Fiedler value, by LOBPCG on (Q, I) with the constant vector
 *          deflated; 0 when the two-hop graph is disconnected (Sec. 4.2)
 *   mu     min_i eps / (Q_ii - sum_{j != i} Q_ij) over rows with a positive denominator
 *          (Eq. 9)
 *   A      L - mu Q + eps I (Eq. 6) on the structure diag + E + T, ascending columns
 *   b_i    r_i / (prod_j r_j)^(1/n), r_i the Gershgorin radius of row i of A (Sec. 4.3)
 * The result is a library-owned handle holding everything on the device.
 * Errors: MGE_EINVAL (malformed CSR), MGE_ENOTSYM, MGE_EISOLATED, MGE_ENOMEM, MGE_EDEVICE.
 * MGE_EDEGENERATE is returned together with a valid handle when eps = 0. */
mge_status mge_build_graph_ops(mge_ctx* ctx, int64_t n, const int64_t* row_ptr,
                               const int32_t* col, const double* w, int on_device,
                               const mge_ops_opts* opts, mge_ops** out);

/* Builds the operators of many graphs (each exactly as mge_build_graph_ops, Sec. 4) with
 * `workers` host threads (0 = 8), each issuing its builds on a CUDA stream of its own: the
 * steps before the eps = lambda_2(Q) solve on the workers, then every eps solve as a branch
 * of ONE CUDA graph launch (as mge_embed_batch), then the steps after it on the workers.
 * n, row_ptr, col, w: count entries each (host or device pointers per on_device; device
 *   inputs written on opts->stream are waited for first).  opts: shared; its stream is not
 *   used by the builds.
 * out[count]: handles (NULL where a build failed); status[count] (may be NULL): each build's
 *   own status (MGE_EDEGENERATE with a valid handle as in mge_build_graph_ops).
 * Returns MGE_OK when every build produced a handle, else the first failing status.
 * Every build's result equals the one mge_build_graph_ops gives alone (up to the order of
 * floating-point atomics in its eps solve). */
mge_status mge_build_graph_ops_batch(mge_ctx* ctx, int count, const int64_t* n,
                                     const int64_t* const* row_ptr, const int32_t* const* col,
                                     const double* const* w, int on_device,
                                     const mge_ops_opts* opts, int workers, mge_ops** out,
                                     mge_status* status);
/* Releases the handle's device arrays.  Call it once no call that uses the handle is in
 * progress on any thread; every call has finished its device work on the handle when it
 * returns.  Performs no device-wide synchronisation. */
mge_status mge_ops_destroy(mge_ops* ops);

typedef struct {
  int64_t n;
  int64_t nnz_w;              /* entries of W                                               */
  int64_t nnz_a;              /* entries of A (diagonal + 1-hop + two-hop)                  */
  int64_t nnz_q;              /* entries of Q (diagonal + two-hop)                          */
  double  eps, mu;
  double  norm_a;             /* max_i (A_ii + r_i), a Gershgorin bound on ||A||_2          */
  double  bmax;               /* max_i b_i                                                  */
  int     degenerate;         /* eps forced to 0                                            */
  int     two_hop_components; /* connected components of (V, T)                             */
  int     eps_iters;          /* LOBPCG iterations of the eps solve                         */
  double  eps_resid;          /* its final relative residual (see mge_embed)               */
  double  build_ms;           /* device time of the whole build                             */
} mge_ops_info_t;

mge_status mge_ops_info(const mge_ops* ops, mge_ops_info_t* out);

/* Copies the operators out (for parity checks).  Any pointer may be NULL to skip it.
 * Sizes: a_ptr/q_ptr [n+1], a_col/a_val [nnz_a], q_col/q_val [nnz_q], b/T [n].  Values are
 * FP64 whatever the precision the iteration uses.  on_device selects device or host
 * destinations. */
mge_status mge_ops_export(const mge_ops* ops, int64_t* a_ptr, int32_t* a_col, double* a_val,
                          int64_t* q_ptr, int32_t* q_col, double* q_val, double* b,
                          int32_t* T, int on_device);

/* The library's node order (see mge_ops_opts.keep_order): order[r] = the caller's node
 * held in row r of the device-resident operators, r < n (the identity when the caller's
 * order was kept).  order: int32 [n], host or device per on_device.  Errors: MGE_EINVAL. */
mge_status mge_ops_node_order(const mge_ops* ops, int32_t* order, int on_device);

/* Y = A X (which = 0) or Y = Q X (which = 1) with the library's SpMM kernel in the given
 * precision (MGE_FP64 or MGE_FP32); X and Y are row-major [n x m] blocks of that precision
 * (double or float), m in {4, 8, 12, 16, 24}, device pointers of the context's device,
 * 16-byte aligned, rows in the caller's node order.  Test and measurement entry point for
 * the SpMM of the iteration (Sec. 4.3: the products A q of the LOBPCG solve).
 * Errors: MGE_EINVAL (bad which, precision or width; a pointer that is misaligned, host
 * memory or on another device -- checked on the host before anything runs), MGE_EDEVICE. */
mge_status mge_ops_apply(mge_ctx* ctx, const mge_ops* ops, int which, int precision, int m,
                         const void* X, void* Y, void* stream);

/* Y = A Y (which = 0) or Y = Q Y (which = 1) in place, for callers that cannot allocate
 * device memory: a process that reserves its whole device-memory budget up front (a
 * serving process, or one sharing the GPU under a fixed quota), or code that must not
 * call cudaMalloc/cudaFree because cudaFree waits for the whole device and would stall
 * the work on its other streams.  The paper has no counterpart; it is a service entry
 * point around the SpMM of the iteration (same kernel, same results as mge_ops_apply).
 *
 * XY: device pointer of the context's device, row-major [n x m] block of the given
 * precision (MGE_FP64 or MGE_FP32), 16-byte aligned, m in {4, 8, 12, 16, 24}; overwritten
 * with the product.  A misaligned, host or foreign pointer is rejected with MGE_EINVAL
 * before anything runs.
 * The copy of the block the product needs goes into one fixed 32 MiB device array inside
 * the library (not counted in the context's HBM budget); a block whose size
 * n * m * sizeof(element) exceeds 32 MiB is rejected with MGE_EINVAL.  Nothing in the array
 * needs to start at zero.  Every call on a device shares the array: calls must not
 * overlap in time (from several host threads, or on streams the caller does not order).
 * The call returns after the product is complete (the stream is synchronised).  The first
 * call on each device performs a set-up step (it looks up the array's device address);
 * make that first call before any stream capture begins.  Allocates no memory. */
mge_status mge_ops_apply_inplace(mge_ctx* ctx, const mge_ops* ops, int which, int precision, int m,
                                 void* XY, void* stream);

/* ---- embedding: LOBPCG for the first K generalized eigenpairs (Sec. 4.3) ------------- */

typedef struct {
  int         precision;      /* mge_precision of the blocks (default MGE_FP32)             */
  int         guard;          /* extra columns beyond K; m = K + guard is rounded up to a
                                 supported block width (4, 8, 12, 16, 24).  0 = default:
                                 K more (m = 2K, at most 24), which the relative-residual
                                 test needs to converge in tens rather than hundreds of
                                 iterations when eigenvalues are ~1% apart; negative: none */
  int         maxiter;        /* default 20000                                             */
  uint64_t    seed;           /* seed of the initial block when x0 is NULL                  */
  int         check_every;    /* iterations between host checks of convergence (default 16)*/
  int         use_graph;      /* capture the iteration in a CUDA graph (default 1)          */
  const double* x0;           /* optional initial block, host or device per x0_on_device,
                                 column-major [n x m_in] FP64, m_in = x0_cols              */
  int         x0_cols;
  int         x0_on_device;
  int         v_on_device;    /* V is a device pointer                                      */
  void*       stream;         /* cudaStream_t or NULL                                       */
  int         precond_degree; /* LOBPCG preconditioner: the residual block R becomes
                                 p(D^-1 L') D^-1 R, p the degree-d Chebyshev iteration for
                                 L' y = R on [beta / (2 d^2), beta], with L' = L + eps I (the
                                 Laplacian of W shifted by eps, a sparser stand-in for A),
                                 D = diag(L') and beta the Gershgorin bound of D^-1 L'.
                                 d = 1 is the Jacobi preconditioner; each degree above 1
                                 costs one SpMM of L' per iteration and cuts the iteration
                                 count about in proportion.  The paper leaves the
                                 preconditioner open.  0 = default round(sqrt(n) / 5)
                                 within [16, 64] (measured best on 2k-50k-node graphs
                                 and at 200k nodes); at most 256.  MGE_BF16 caps it at 8.  */
  int         rr_fp64;        /* arithmetic of the Rayleigh-Ritz eigensolve and of the
                                 Cholesky that B-normalises W, for FP32 blocks:
                                  0 (default) the inverse-pencil FP32 solve described under
                                    MGE_FP32 until the largest relative residual of the K
                                    wanted pairs, once within 1000x of tol, has not halved
                                    for 10 iterations, then cyclic Jacobi in FP64 for the
                                    rest of the solve;
                                  1 cyclic Jacobi on the 3m x 3m pencil in FP64 throughout;
                                 -1 the FP32 form throughout.
                                 The FP32 form's eigenvectors carry errors of about u
                                 theta_k / theta_1 along directions of large Rayleigh
                                 quotient theta_j, which floor the relative residual at
                                 about u theta_j / theta_1 (measured before the correction:
                                 1e-5 at 200k nodes, 1-2e-5 on a 2M-node sphere); one step
                                 c -= G_A^-1 (G_A - theta G_B) c with the residual in FP64
                                 removes them.  Measured on one GB300 (tol 1e-5): 200k-node
                                 swiss roll, K = 8, m = 16: FP32 21 iterations at 2.15 ms,
                                 FP64 23 at 4.0 ms; 2M-node sphere, K = 16, m = 24: FP32 48
                                 iterations, FP64 90.  info.rr_fp64_from reports which ran.
                                 FP64 blocks always use FP64.                               */
  int         gram_cuda_cores; /* FP32 blocks of width 12, 16 or 24 on graphs of at least
                                 65,536 nodes: 0 (default) computes the Rayleigh-Ritz Grams
                                 [X W P]^T A [X W P] and [X W P]^T B [X W P] on the tensor
                                 cores (tcgen05, TF32 with each value split in two so that
                                 products keep about 2^-21 relative accuracy); 1 computes them
                                 on the CUDA cores (compensated FP32), as smaller graphs do. */
} mge_embed_opts;

typedef struct {
  int    status;              /* mge_status of the solve                                   */
  int    iters;               /* LOBPCG iterations                                         */
  int    m;                   /* block width used                                          */
  int    drops;               /* iterations whose Rayleigh-Ritz basis dropped a direction   */
  double resid[64];           /* relative residual rho_k of each returned pair (k < K)      */
  double solve_ms;            /* device time of the solve                                  */
  int    rr_fp64_from;        /* Rayleigh-Ritz in FP64: -1 never, 0 from the start, k > 0
                                 after iteration k (mge_embed_opts.rr_fp64)                 */
} mge_embed_info;

/* Fills lambda[K] (host, ascending) and V (column-major [n x K] FP64, host or device per
 * opts->v_on_device) with the first K generalized eigenpairs of (A, B) of `ops`.
 * Convergence: every returned column has relative residual
 *   rho = ||A x - lambda B x||_{B^-1} / ((|lambda| + u ||A||_G) ||x||_B) <= tol,
 * the residual of the symmetric form B^-1/2 A B^-1/2 relative to the eigenvalue (ARPACK's
 * criterion), with ||v||_{B^-1}^2 = sum v_i^2 / b_i, ||x||_B^2 = sum b_i x_i^2,
 * ||A||_G = max_i (A_ii + r_i) and u the unit roundoff of the block precision (2^-53 or
 * 2^-24) as a floor for lambda = 0.  rho <= tol bounds each eigenvalue's relative error by
 * about tol^2 |lambda| / gap and each vector's angle by about tol |lambda| / gap (gap: the
 * distance to the nearest other eigenvalue).  The residual is the one the iteration
 * carries (A x from its recurrences); a residual recomputed from the returned FP32 vectors
 * also holds their rounding noise, about u ||A|| / |lambda|.
 * Errors: MGE_EINVAL (K < 1, K + guard > 24, n < m), MGE_ENOTCONVERGED (partial results
 * written), MGE_ECHOLESKY, MGE_ENOTFINITE, MGE_ENOMEM, MGE_EDEVICE.  `info` may be NULL. */
mge_status mge_embed(mge_ctx* ctx, const mge_ops* ops, int K, double tol,
                     const mge_embed_opts* opts, double* lambda, void* V,
                     mge_embed_info* info);

/* Batched form of mge_embed: the first K[i] generalized eigenpairs of (A, B) of each of
 * `count` operator handles (Sec. 4.3, Eq. 10-11, as mge_embed), computed in ONE launch of one
 * CUDA graph in which every solve is an independent branch (its initial block and first
 * iteration, then a device-side while loop over its iterations), so graphs of uneven size
 * and iteration count share the GPU and each branch stops at its own convergence.
 * ops[count], K[count]: the handles (all built on this context's device) and their K.
 * opts: as mge_embed, shared by all solves (precision, guard, maxiter, seed, stream,
 *   v_on_device, precond_degree); x0 must be unset; use_graph and check_every are ignored.
 * lambda[count]: host arrays of K[i] doubles each (written, ascending).
 * V: NULL, or count pointers (each NULL or a column-major [n_i x K[i]] FP64 buffer, host or
 *   device per opts->v_on_device).  info: NULL or count entries; solve_ms is the device time
 *   of the whole batch launch.  Every solve's result is the one mge_embed gives alone with
 *   the same options (up to the order of floating-point atomics).
 * Returns MGE_OK when every solve converged; otherwise the first failing solve's status
 * (MGE_ENOTCONVERGED: partial results written; per-solve status in info[i].status).
 * Errors: MGE_EINVAL (count < 1, a NULL handle or lambda, x0 set, K or width out of range),
 * MGE_ENOMEM, MGE_EDEVICE. */
mge_status mge_embed_batch(mge_ctx* ctx, int count, const mge_ops* const* ops, const int* K,
                           double tol, const mge_embed_opts* opts, double* const* lambda,
                           void* const* V, mge_embed_info* info);

/* ---- betweenness centrality and VBC (Sec. 3.3) ------------------------------------- */

/* The paper qualifies an input graph as a manifold graph by the variance of its nodes'
 * betweenness centralities (VBC, Sec. 3.3, Table 1):
 *   C_B(i) = sum over ordered pairs (s, t), s != t, both != i, of sigma_st(i) / sigma_st,
 * sigma_st the number of shortest paths from s to t (counted in hops; the graph's weights are
 * similarities, not lengths) and sigma_st(i) those through i; pairs without a path add
 * nothing.  VBC = (1/n) sum_i (C_B(i) - mean C_B)^2.
 * row_ptr [n+1], col: CSR of an undirected graph (both directions stored), host or device per
 * on_device; cb [n] FP64 written (host or device per on_device); vbc (host, may be NULL).
 * Cost O(n nnz): meant for the graph sizes the paper qualifies (hundreds to tens of
 * thousands of nodes).  Errors: MGE_EINVAL (malformed CSR), MGE_ENOMEM, MGE_EDEVICE. */
mge_status mge_betweenness(mge_ctx* ctx, int64_t n, const int64_t* row_ptr, const int32_t* col,
                           int on_device, double* cb, double* vbc, void* stream);

/* ---- k-means of the embedding (Sec. 5.2) ------------------------------------------- */

/* The paper clusters its embeddings with kmeans (Sec. 5.2, Table 3).  Lloyd's algorithm in
 * FP64 from the caller's initial centres (random choices are the caller's):
 *   assignment  each point to the centre of least squared distance, the squared distance
 *               summed over coordinates in order with each product and sum rounded
 *               separately (no fused multiply-add); equal distances go to the lower index;
 *   update      each centre becomes the mean of its points (each coordinate's sum rounded
 *               once from a compensated double-double, divided by the count); a centre
 *               without points stays;
 *   stop        after an assignment step other than the first that changed nothing, or
 *               after max_iters assignment steps.
 * X: column-major [n x K] FP64 (the layout mge_embed returns V in).  centres0: row-major
 * [C x K].  assign [n] int32 and centres [C x K] (row-major) are written; *iters receives
 * the assignment steps taken.  All pointers host or device per on_device (device pointers
 * 16-byte aligned).  1 <= K <= 64, C >= 1, C K <= 4096.  Errors: MGE_EINVAL, MGE_ENOMEM,
 * MGE_EDEVICE. */
mge_status mge_kmeans(mge_ctx* ctx, int64_t n, int K, const double* X, int C, const double* centres0,
                      int max_iters, int on_device, int32_t* assign, double* centres, int* iters,
                      void* stream);

/* ---- serving: continuous batching of embedding requests ---------------------------- */

typedef struct {
  int64_t        n;
  const int64_t* row_ptr;     /* host CSR of W; copied at submit                            */
  const int32_t* col;
  const double*  w;
  int            K;
  double         tol;
  int            precision;
  int            guard;
  int            maxiter;
  uint64_t       seed;
  /* Alternatively the request is given as points (row_ptr, col, w unused): host row-major
   * [n x dim] FP64, copied at submit; the serving slot builds their kNN graph with knn
   * neighbours on the device (mge_knn_graph, Sec. 5.1) before the operators.            */
  const double*  points;
  int            dim;
  int            knn;
} mge_request;

typedef struct {
  int      status;            /* mge_status of the request                                  */
  int64_t  n;
  int      K;
  double   eps, mu;
  int      iters;
  double   latency_ms;        /* submit to completion, host clock                           */
  double   queue_ms;          /* submit to admission                                        */
  double*  lambda;            /* library-owned, valid until mge_release                     */
  double*  V;                 /* library-owned host buffer, column-major [n x K]            */
} mge_result;

/* Enqueues a request; the serving thread admits it when its HBM footprint fits the
 * context budget and runs it concurrently with the requests already on the device.
 * Errors: MGE_EINVAL, MGE_EAGAIN (queue full). */
mge_status mge_submit(mge_ctx* ctx, const mge_request* req, uint64_t* ticket);
/* Waits up to timeout_ms (negative = forever) for the ticket; MGE_ETIMEOUT if not done. */
mge_status mge_poll(mge_ctx* ctx, uint64_t ticket, int timeout_ms, mge_result* out);
/* Frees the result buffers of a completed ticket. */
mge_status mge_release(mge_ctx* ctx, uint64_t ticket);

#ifdef __cplusplus
}
#endif
#endif /* MGE_H */
