/*
 * cakf.h -- C ABI of the GB300 computation-aware Kalman filter / smoother library (libcakf.so).
 *
 * Method: Pfoertner, Wenger, Cockayne, Hennig, "Computation-Aware Kalman Filtering and
 * Smoothing" (arXiv 2405.08971).  The library runs, on one GPU:
 *   - the CAKF forward pass (Alg. 1 with the iterative update of the appendix, CG actions of
 *     Sec. 3.3, and Truncate of Sec. 3.2),
 *   - the CAKS backward pass (Alg. 3),
 *   - the negative log likelihood of the projected data and its gradient w.r.t. the four
 *     hyperparameters (the paper names these as future work; the definition is given at
 *     cakf_nll below).
 *
 * Model (problem statement, Sec. 2; space-time separable Gauss-Markov lemma in the appendix):
 *   state x_k = values of a spatio-temporal GP on a fixed grid X (n points, dim 1..3),
 *   spatial kernel  K = sf2 * Matern_nu(|x - x'| / lx),
 *   OU time factor  A = a I, Q = (1 - a^2) K, a = exp(-dt / lt), x_0 ~ N(mu_0, K),
 *   observations    y_k = x_k[obs_k] + eps, eps ~ N(0, sn2 I), steps k = 1..T.
 *
 * Conventions shared by every entry point
 *   Pointers   "host or device": the library inspects each pointer (cudaPointerGetAttributes)
 *              and copies host data itself.  Input arrays are caller-owned and only read during
 *              the call.  Output arrays are caller-allocated.
 *   Layout     all 2-D arrays are row-major in the step index: element (k, j) of a (T+1) x n
 *              array is at [k * n + j].
 *   Streams    `cuda_stream` is a cudaStream_t owned by the caller (NULL = legacy default
 *              stream).  Calls return once their results are in the output arrays.
 *   Errors     every call returns a cakf_status; nothing aborts or throws across the ABI.
 *              cakf_last_error() gives a message for the calling thread's last failure.
 *              Device pointers must belong to the current device (CAKF_ERR_ARG otherwise).
 *              cakf_smooth, cakf_nll, cakf_nll_backward and cakf_get_actions on a NULL context
 *              (none created yet) or on one without a successful cakf_filter: CAKF_ERR_STATE.
 *              A cakf_filter rejected by argument validation leaves its context untouched.
 *   Threads    a cakf_ctx may be used by one thread at a time.
 */
#ifndef CAKF_H
#define CAKF_H

#include <stdint.h>
#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CAKF_ABI_VERSION 3

typedef enum {
  CAKF_OK = 0,
  CAKF_ERR_ARG = 1,      /* invalid argument (sizes, indices, enum values, NULL)            */
  CAKF_ERR_CUDA = 2,     /* a CUDA runtime call failed                                      */
  CAKF_ERR_OOM = 3,      /* device memory exhausted                                         */
  CAKF_ERR_NUMERIC = 4,  /* non-finite value, or a non-positive-definite projected Gram      */
  CAKF_ERR_TIMEOUT = 5,  /* a device-side wait exceeded its iteration limit                 */
  CAKF_ERR_STATE = 6     /* call order violated (e.g. smooth before filter)                 */
} cakf_status;

enum { CAKF_MATERN12 = 0, CAKF_MATERN32 = 1, CAKF_MATERN52 = 2 };

/* Temporal factor of the space-time separable prior (the appendix lemma on space-time separable
   Gauss-Markov processes: A = A^t (x) I_n, Q = Q^t (x) K, stationary covariance P^t_inf (x) K). */
enum {
  CAKF_TEMPORAL_OU = 0,        /* Ornstein-Uhlenbeck, D' = 1: A^t = exp(-dt / l_t), P^t_inf = 1;
                                  the state is the n grid values                               */
  CAKF_TEMPORAL_MATERN32 = 1   /* Matern-3/2, D' = 2 (the remark after that lemma: Matern(p + 1/2)
                                  kernels have an exact state-space form): the state holds the
                                  grid values f and their time derivatives (D = 2n);
                                  lam = sqrt(3) / l_t, A^t = expm(F dt) with
                                  F = [[0, 1], [-lam^2, -2 lam]], P^t_inf = diag(1, lam^2).  The
                                  outputs (means, variances) are those of f; a prior mean mu_k
                                  applies to f (zero for the derivatives).  Supported by
                                  cakf_filter / cakf_smooth / cakf_nll with CAKF_STORE_FP32;
                                  cakf_nll_backward, cakf_sample, cakf_interpolate and
                                  freeze_truncation return CAKF_ERR_ARG                        */
};

/* Arithmetic of the kernel-Gram x block products (everything else follows in parentheses). */
enum {
  CAKF_FP64 = 0,   /* all in FP64 (reference mode)                                          */
  CAKF_FP32 = 1,   /* plain FP32 SIMT kernels (factors, CG and tall-skinny GEMMs in FP32)    */
  CAKF_TF32 = 2,   /* Gram tiles x blocks on tcgen05 kind::tf32 (operands rounded to TF32,
                      11 significant bits), FP32 accumulation                                 */
  CAKF_BF16 = 3,   /* Gram tiles x blocks on tcgen05 kind::f16 (bf16), FP32 accumulation    */
  CAKF_FP16X3 = 4, /* Gram tiles x blocks on tcgen05 kind::f16 with split FP16 operands:
                      x = hi + lo (both fp16, B scaled per column by a power of two), three
                      MMAs hi*hi + hi*lo + lo*hi, FP32 accumulation: FP32-class products      */
  CAKF_TF32X3 = 5  /* Gram tiles x blocks on tcgen05 kind::tf32 with split TF32 operands
                      (x = hi + lo, both tf32, no scaling), three MMAs: FP32-class products   */
};

/* How the actions S_k of a step are chosen (Sec. 3.3 and the policy appendix). */
enum {
  CAKF_POLICY_CG = 0,          /* iterative update, the action of iteration j is the current residual
                                  (or replay_actions[j] when given)                               */
  CAKF_POLICY_COORDINATE = 1,  /* batch update (Alg. 2) with unit-vector actions at min(i, m_k)
                                  observations evenly spaced through the step's observation list
                                  (positions floor((q + 1/2) m_k / i)); i <= 160                 */
  CAKF_POLICY_BATCH = 2        /* batch update (Alg. 2) with the actions given in replay_actions
                                  (e.g. Gaussian sketches drawn by the caller); i_k <= 160       */
};

/* Where the per-step factors the smoother and the gradient pass read (M+_k, [P^-W_k P^-w_k],
   K(X, X_o)[V_k v_k], [V_k v_k]) are kept between cakf_filter and cakf_smooth (memory O(n r) per
   step, Sec. 3.2). */
enum {
  CAKF_STORE_FP32 = 0,   /* all steps resident in the working precision (FP64 in CAKF_FP64 mode)   */
  CAKF_STORE_BF16 = 1,   /* all steps kept as BF16 copies (half the bytes; the smoother reads them
                            back rounded to 8 significant bits); FP32-based precisions only        */
  CAKF_RECOMPUTE = 2     /* only M+_k and its eigenvalues every checkpoint_every steps (and the
                            actions of every step) are kept; the smoother and the gradient pass
                            re-run the filter over each segment with the stored actions, which
                            reproduces the first pass's factors exactly                           */
};

typedef struct {
  int32_t abi_version;        /* must equal CAKF_ABI_VERSION                                  */
  int32_t n;                  /* grid points; the state dimension is D = n D' (temporal)       */
  int32_t dim;                /* coordinate dimension, 1..3                                   */
  const double* coords;       /* n*dim, row-major, host or device; sphere grids pass xyz       */
  int32_t kernel;             /* CAKF_MATERN12 | CAKF_MATERN32 | CAKF_MATERN52                */
  double log_lx;              /* log spatial lengthscale                                      */
  double log_lt;              /* log temporal lengthscale (OU or Matern-3/2, see temporal)     */
  double log_sf2;             /* log output variance sigma_f^2                                */
  double log_sn2;             /* log observation-noise variance sigma_n^2                     */
  int32_t T;                  /* number of steps with data; states are k = 0..T              */
  double dt;                  /* time between steps                                           */
  const int32_t* obs_ptr;     /* T+1 offsets, HOST: step k (1-based) owns [obs_ptr[k-1],
                                 obs_ptr[k]); obs_ptr[0] = 0; an empty range = no data       */
  const int32_t* obs_idx;     /* obs_ptr[T] grid indices in [0, n), distinct within a step;
                                 host or device                                               */
  const double* y;            /* obs_ptr[T] observations, host or device                      */
  const double* prior_mean;   /* NULL (zero mean) or (T+1)*n known prior mean mu_k, host/dev  */
  int32_t budget_i;           /* action budget per step (CG iterations), >= 1                 */
  int32_t rank_r;             /* truncation rank of the downdate factors; <= 0: no truncation */
  double cg_rtol;             /* stop a step's CG early when ||r|| <= cg_rtol ||r0||; 0 = never */
  int32_t precision;          /* CAKF_FP64 | CAKF_FP32 | CAKF_TF32 | CAKF_BF16 | CAKF_FP16X3 |
                                 CAKF_TF32X3                                                  */
  const double* replay_actions; /* NULL, or frozen actions: for each step k the m_k x i_k
                                 column-major block S_k, concatenated over k = 1..T (host)    */
  const int32_t* replay_counts; /* with replay_actions: T+1 entries, i_k for k = 0..T (host)  */
  int32_t factor_storage;     /* CAKF_STORE_FP32 | CAKF_STORE_BF16 | CAKF_RECOMPUTE              */
  int32_t checkpoint_every;   /* segment length of CAKF_STORE_BF16 / CAKF_RECOMPUTE (the steps
                                 restored at a time; 0 = 20); ignored for CAKF_STORE_FP32     */
  int32_t policy;             /* CAKF_POLICY_CG | CAKF_POLICY_COORDINATE | CAKF_POLICY_BATCH     */
  int32_t freeze_truncation;  /* 1: instead of eigendecomposing, the filter truncates with the
                                 rotations U_k of the previous cakf_filter on the same context
                                 (same sizes; with replay_actions this evaluates the frozen
                                 modified model of cakf_nll_backward at other hyperparameters, for
                                 finite-difference checks); 0: normal                          */
  int32_t temporal;           /* CAKF_TEMPORAL_OU | CAKF_TEMPORAL_MATERN32                      */
} cakf_problem;

typedef struct cakf_ctx cakf_ctx;   /* library-owned state; holds the stored factors */

typedef struct {
  double filter_ms;           /* device time of the last cakf_filter (CUDA events)            */
  double smooth_ms;           /* device time of the last cakf_smooth                          */
  double gram_block_ms;       /* summed device time of the Gram x block launches (profiling on)*/
  int64_t gram_block_launches;
  double gram_block_flops;    /* algorithmic flops of those launches: 2*rows*cols*(width-1) on
                                 the tensor-core path, 2*rows*cols*width on the SIMT path     */
  double gram_block_evals;    /* kernel-matrix entries evaluated by those launches            */
  double cg_matvec_ms;        /* summed device time of the CG Gram matvec launches            */
  int64_t cg_matvec_launches;
  double cg_matvec_evals;
  double eig_ms;              /* summed device time of the FP64 eigensolver calls             */
  int64_t eig_calls;
  int64_t kernel_launches;    /* kernels this library launched in the last filter + smooth    */
  int64_t device_bytes;       /* device memory held by the context                            */
  /* device time per phase, summed over the steps (profiling on):
     [0] filter CG loop (actions, G s products, G-orthogonalisation)
     [1] filter Gram x block finalize incl. its low-rank correction and outputs
     [2] filter truncation (Gram, FP64 eig, rotation)
     [3] smoother P^- X (K X propagated from the filter's stored K(X, X_o)[V v] blocks, no kernel
         evaluations; low-rank correction)
     [4] smoother combine and outputs (Z, P X, ws)
     [5] smoother truncation (Gram identities, FP64 eig, rotation)
     [6] NLL term per step (side stream: overlaps [2])
     [7] restoring stored factors for the smoother / gradient pass (recomputation of filter
         segments, or BF16 unpacking); zero with CAKF_STORE_FP32                              */
  double phase_ms[8];
  /* summed device time of the eigensolver's parts (profiling on): [0] tridiagonalisation,
     [1] divide & conquer, [2] back-transformation and conversion of the kept vectors      */
  double eig_phase_ms[3];
  double eig_flops[2];        /* algorithmic FP64 flops of those eigensolver calls, per part:
                                 [0] (4/3) N^3 (tridiagonalisation), [1] 2 N^2 keep (back-
                                 transformation); divide & conquer depends on deflation: not counted */
} cakf_stats;

/*
 * cakf_filter -- run the CAKF over k = 1..T (Alg. 1; update: appendix algorithm "CAKF Update
 * Step (Iterative Version)"; Truncate: Sec. 3.2).
 *   p         problem description (read during the call only).
 *   ctx_inout *ctx_inout == NULL: a new context is created and returned there.  Otherwise the
 *             given context is reused (its buffers are kept when the sizes fit).
 *   mean_out  (T+1)*n filter means m_k (host or device), or NULL.
 *   var_out   (T+1)*n filter marginal variances diag(P_k) = sf2 - rowsumsq(M_k) taken before
 *             truncation (host or device), or NULL.
 * The context keeps per-step factors for cakf_smooth / cakf_nll / cakf_nll_backward.
 * Errors: CAKF_ERR_ARG (sizes, indices out of range, abi_version), CAKF_ERR_OOM,
 *         CAKF_ERR_NUMERIC (non-finite result or non-positive-definite action Gram),
 *         CAKF_ERR_CUDA, CAKF_ERR_TIMEOUT, CAKF_ERR_STATE (freeze_truncation without a previous
 *         successful run of the same sizes on the context).
 */
int cakf_filter(const cakf_problem* p, cakf_ctx** ctx_inout, double* mean_out, double* var_out,
                void* cuda_stream);

/*
 * cakf_smooth -- run the CAKS backward pass k = T-1 .. 0 (Alg. 3) on the filter state held by
 * ctx.  Outputs (T+1)*n smoother means and marginal variances (host or device, or NULL).
 * Errors: CAKF_ERR_STATE when no successful cakf_filter preceded it on this context.
 */
int cakf_smooth(cakf_ctx* ctx, double* mean_out, double* var_out, void* cuda_stream);

/*
 * cakf_nll -- negative log likelihood of the projected data of the last cakf_filter:
 *   NLL = sum_k [ 1/2 logdet(2 pi S_k^T G_k S_k) + 1/2 r_k^T S_k (S_k^T G_k S_k)^-1 S_k^T r_k
 *                 - 1/2 logdet(S_k^T S_k) ],
 *   G_k = H_k P^-_k H_k^T + sn2 I, r_k = y_k - H_k m^-_k, S_k the actions (eq. proj-observation,
 *   Sec. 3.1).  Each step's term is formed during the filter from its definition: S^T G S (with
 *   the stored G s_j), S^T S and S^T r in FP64, both Cholesky-factored in FP64 (on a side stream
 *   that overlaps the truncation; cakf_filter returns after it has finished).
 *   nll_out: one double (host).
 */
int cakf_nll(cakf_ctx* ctx, double* nll_out);

/*
 * cakf_nll_backward -- gradient of cakf_nll w.r.t. (log_lx, log_lt, log_sf2, log_sn2) with the
 * actions S_k and truncation rotations of the last filter run held fixed (exact inference in
 * the fixed modified observation model, Sec. 3.1).  grad_out: 4 doubles (host).
 */
int cakf_nll_backward(cakf_ctx* ctx, double* grad_out);

/*
 * cakf_get_actions -- copy the actions used by the last filter run (host outputs):
 *   counts_out  T+1 entries i_k (0 for k = 0 and for steps without data);
 *   actions_out the m_k x i_k column-major blocks for k = 1..T, concatenated (size
 *               sum_k m_k * i_k), suitable for cakf_problem.replay_actions.  May be NULL to
 *               query the counts only.
 */
int cakf_get_actions(cakf_ctx* ctx, double* actions_out, int32_t* counts_out);

/*
 * cakf_gram_matmul -- the matrix-free kernel-Gram product on its own (the Gram x matrix primitive
 * that every CAKF / CAKS covariance product reduces to; Sec. 6, "Implementation"):
 *     Out[i, c] = sum_j sf2 * Matern_nu(|xr_i - xc_j| / lx) * B[j, c],  i < nr, c < width.
 * The nr x nc Gram matrix is evaluated tile by tile and never stored.
 *   kernel            CAKF_MATERN12 | CAKF_MATERN32 | CAKF_MATERN52
 *   Xr, Xc            DEVICE arrays, nr*dim / nc*dim doubles, row-major coordinates (dim 1..3)
 *   B                 DEVICE, column-major nc x width (leading dimension ldb >= nc); double for
 *                     CAKF_FP64, float otherwise
 *   Out               DEVICE, column-major nr x width (ldo >= nr); same element type as B
 *   precision         CAKF_FP64 / CAKF_FP32: SIMT kernels; CAKF_BF16 / CAKF_FP16X3 / CAKF_TF32
 *                     / CAKF_TF32X3: tcgen05 tensor cores for columns 0..width-2 (bf16, fp16 hi +
 *                     lo, tf32, or tf32 hi + lo operands; fp32 accumulation) and fp32 CUDA-core
 *                     accumulation of the last column (width >= 2 and <= 513 for these paths)
 * Scratch is allocated on the first call per thread and kept (grown when needed).
 * Errors: CAKF_ERR_ARG (sizes, NULL, host pointers), CAKF_ERR_OOM, CAKF_ERR_CUDA.
 */
int cakf_gram_matmul(int32_t kernel, double log_lx, double log_sf2, int32_t dim, const double* Xr, int32_t nr,
                     const double* Xc, int32_t nc, const void* B, int32_t ldb, int32_t width, void* Out,
                     int32_t ldo, int32_t precision, void* cuda_stream);

/*
 * cakf_gram_matmul_noalloc -- cakf_gram_matmul (same arguments, same results, same kernels)
 * for callers that must not allocate device memory.  The paper has no counterpart: it is a
 * library integration variant, not part of the method.
 *
 * Who needs it: cakf_gram_matmul grows a per-thread scratch with cudaMalloc / cudaFree.  Those
 * calls synchronise the device and can fail when another allocator (a framework's caching
 * allocator, a pool sized at start-up) already holds almost all device memory; a caller in a
 * latency-bound loop, or one working inside a fixed memory plan, cannot accept either.  This
 * entry point performs no device allocation of its own: its scratch is one statically sized
 * device array of the library, CAKF_NOALLOC_SCRATCH_BYTES per device.  The CUDA runtime loads the
 * module that holds it lazily, so the array is reserved on a device by the first call of this
 * entry point there (and kept until the process exits); make that first call during set-up,
 * before a memory pool takes the rest of the device: if the reservation fails it returns
 * CAKF_ERR_OOM.
 *
 * Limit: the scratch must hold 256 bytes + (nr + nc) coordinate records (32 bytes each for
 * CAKF_FP64, 16 otherwise, rounded up to 256) and, for CAKF_BF16, the packed operand
 * (about 2 * nc * (width - 1) bytes plus 20 * nc; twice the operand bytes for CAKF_FP16X3 and
 * CAKF_TF32, four times for CAKF_TF32X3).
 * A call needing more returns CAKF_ERR_ARG with the required size in cakf_last_error, before
 * any device work; for example BF16 with nc = 32768, width = 513 fits, nc = 65536 needs
 * width <= 257 (FP16X3: nc = 32768 needs width <= 257).
 * Zero state: only the device error flag inside the scratch has to start at zero; the call
 * clears it on its stream before use.  All other scratch bytes are written before being read.
 * Concurrency: every call on a device uses the same scratch, so calls that overlap in time on
 * one device (other streams, other host threads) race and corrupt each other's results.  The
 * call synchronises its stream before returning; serialise calls across threads.
 * Setup: the first call on a device looks up the scratch address (cudaGetSymbolAddress, with
 * that device current) and sets kernel attributes; make that first call before any stream
 * capture begins on the device.
 * Arrays: Xr, Xc, B and Out must be device memory of the current device (CAKF_ERR_ARG otherwise);
 * their sizes cannot be checked here, so Xr must hold nr * dim and Xc nc * dim doubles.
 * Errors: as cakf_gram_matmul, with CAKF_ERR_ARG also for calls exceeding the scratch and
 * CAKF_ERR_OOM when the first call on a device cannot reserve the scratch.
 */
#define CAKF_NOALLOC_SCRATCH_BYTES ((size_t)64 << 20)
int cakf_gram_matmul_noalloc(int32_t kernel, double log_lx, double log_sf2, int32_t dim, const double* Xr,
                             int32_t nr, const double* Xc, int32_t nc, const void* B, int32_t ldb, int32_t width,
                             void* Out, int32_t ldo, int32_t precision, void* cuda_stream);

/*
 * cakf_factor_gemm -- the tall-skinny factor product of the filter and smoother on its own (the
 * products M^- (M_o^T [V v]), M_hat U of Truncate (Sec. 3.2), M^T X and the rotations of Alg. 3),
 * the same device code the filter and smoother run:
 *     C = alpha op(A) B + beta C,   op(A) = A (trans_a = 0) or A^T (trans_a = 1).
 *   A       DEVICE float, column-major: M x K (lda >= M) for trans_a = 0, K x M (lda >= K) for 1
 *   B       DEVICE float, column-major K x N (ldb >= K)
 *   C       DEVICE float, column-major M x N (ldc >= M), read when beta != 0
 *   precision  CAKF_FP32: FP32 SIMT kernels; a tensor-core mode (CAKF_TF32, CAKF_BF16, CAKF_FP16X3,
 *           CAKF_TF32X3): tcgen05 with split TF32 operands (hi + lo, three MMAs, FP32
 *           accumulation) for the large products, as in those modes' filter and smoother.
 * Its workspace is allocated on the first call per thread and kept (grown when needed).
 * Errors: CAKF_ERR_ARG, CAKF_ERR_OOM, CAKF_ERR_CUDA, CAKF_ERR_TIMEOUT.
 */
int cakf_factor_gemm(int32_t trans_a, int32_t M, int32_t N, int32_t K, double alpha, const float* A, int32_t lda,
                     const float* B, int32_t ldb, double beta, float* C, int32_t ldc, int32_t precision,
                     void* cuda_stream);

/*
 * cakf_eig_topk -- the FP64 symmetric eigensolver of Truncate (Sec. 3.2) on its own: the top
 * `keep` eigenpairs of the N x N symmetric matrix A (the Gram M^T M of a downdate factor in the
 * filter and smoother), the same device code the filter and smoother run.
 *   A       DEVICE, N*N doubles, column-major (only read; a copy is factorised)
 *   w_out   DEVICE, keep doubles: eigenvalues in descending order
 *   U_out   DEVICE, N*keep doubles, column-major: the matching orthonormal eigenvectors
 * Allocates and frees its workspace on every call (it is meant for verification and tools, not
 * for the hot loop).  Errors: CAKF_ERR_ARG, CAKF_ERR_OOM, CAKF_ERR_CUDA, CAKF_ERR_TIMEOUT,
 * CAKF_ERR_NUMERIC (secular iteration without convergence or non-finite values).
 */
int cakf_eig_topk(const double* A, int32_t N, int32_t keep, double* w_out, double* U_out, void* cuda_stream);

/*
 * cakf_eig_topk_mixed -- cakf_eig_topk as the FP32-based precision modes run it inside Truncate
 * (Sec. 3.2): the tridiagonalisation, divide and conquer and eigenvalues in FP64, the final product
 * of the Householder reflectors with the tridiagonal's eigenvectors in double-FP32 arithmetic
 * (pairs of FP32 numbers, about 48 significant bits; roughly 1e-14 relative error in U), because
 * those modes round U to FP32 right after.  Same arguments, layout, ownership and errors as
 * cakf_eig_topk.
 */
int cakf_eig_topk_mixed(const double* A, int32_t N, int32_t keep, double* w_out, double* U_out, void* cuda_stream);

/*
 * cakf_probe_peaks -- measured throughputs for the roofline denominators of the kernels that are
 * bound neither by HBM nor by the tensor cores (no counterpart in the paper: a measurement aid).
 *   mufu_ops_per_s    special-function results per second of the sqrt.approx + ex2.approx pair
 *                     that every kernel-matrix entry costs (both counted), over the whole device
 *   fp64_flops_per_s  FP64 fused multiply-add throughput (2 flops each) over the whole device
 * Plain kernels timed with CUDA events on cuda_stream after one warm-up launch each (a few ms);
 * the current device.  Errors: CAKF_ERR_ARG (NULL outputs), CAKF_ERR_OOM, CAKF_ERR_CUDA.
 */
int cakf_probe_peaks(double* mufu_ops_per_s, double* fp64_flops_per_s, void* cuda_stream);

/*
 * cakf_interpolate -- filter and smoother marginals at query times between (or after) the steps
 * (the temporal-interpolation corollary of the appendix in downdate form), for the OU prior:
 * for t_k <= t < t_{k+1} (t_k = k dt; k = T for t >= t_T), with A(t, s) = exp(-(t - s) / l_t),
 *   filter    m(t) = A(t, t_k) m_k + mu(t) - A(t, t_k) mu_k,  P(t) = K - A(t, t_k)^2 M_k M_k^T,
 *   smoother  m^s(t) = m(t) + P(t) A(t_{k+1}, t) ws_{k+1},
 *             P^s(t) = P(t) - P(t) A Ws_{k+1} (P(t) A Ws_{k+1})^T   (the filter's for t >= t_T),
 * with the smoother messages (Ws, ws) of Alg. 3.  Runs one smoother pass (the products come from
 * the stored factors and the smoother's K-recursion: no kernel evaluations).
 *   nq      number of query times, >= 1;  tq  nq times >= 0 (host)
 *   mu_q    NULL, or nq x n prior mean at the query times (required when the problem has a prior
 *           mean), host or device
 *   fmean, fvar, smean, svar   nq x n outputs (host or device, each may be NULL)
 * Errors: CAKF_ERR_STATE (no successful cakf_filter), CAKF_ERR_ARG, CAKF_ERR_OOM, CAKF_ERR_CUDA.
 */
int cakf_interpolate(cakf_ctx* ctx, int32_t nq, const double* tq, const double* mu_q, double* fmean, double* fvar,
                     double* smean, double* svar, void* cuda_stream);

/*
 * cakf_sample -- draws from the computation-aware posterior of the last cakf_filter (the CAKF/CAKS
 * sampler algorithm of the appendix: Matheron's rule in the modified model, with the smoother in
 * inverse-free form).  The filter's stored factors are reused: no kernel values are evaluated.
 * The random inputs are the caller's (e.g. random-Fourier-feature draws):
 *   x0    n x S  initial draw x_0 ~ N(mu_0, K), column s at x0[s * n]           (host or device)
 *   q     (T+1) x S x n dynamics noise q_{k-1} ~ N(0, (1 - a^2) K) of the transition into step
 *         k at q[(k * S + s) * n]; slot k = 0 is not read                          (host or device)
 *   eps   observation noise eps_k ~ N(0, sn2 I): for step k the m_k x S block (column-major) at
 *         eps[obs_ptr[k-1] * S]                                                    (host or device)
 * Outputs (T+1) x S x n, layout of q, host or device, either may be NULL:
 *   filter_out    x_k = x^-_k + P^-_k H^T V_k V_k^T (y_k - H x^-_k - eps_k), x^-_k = a x_{k-1} + b + q
 *   smoother_out  x^s_k = x_k + P_k a ws_{k+1}, ws_k = w_k + (I - W_k W_k^T P^-_k) a ws_{k+1}
 * With x0 = mu_0 and no noise the draws are the filter and smoother means.  1 <= S <= 1024.
 * Allocates its workspace per call.  Errors: CAKF_ERR_STATE, CAKF_ERR_ARG, CAKF_ERR_OOM, CAKF_ERR_CUDA.
 */
int cakf_sample(cakf_ctx* ctx, int32_t n_samples, const double* x0, const double* q, const double* eps,
                double* filter_out, double* smoother_out, void* cuda_stream);

/*
 * cakf_get_diagnostics -- per-step records of the last filter (and smoother) run on ctx, for
 * monitoring the approximation (the paper's update stops at the budget; these tell how far each
 * step got).  Each output is NULL or an array of T+1 entries (host); entry 0 is the prior (zeros).
 *   actions           i_k, the actions used (below the budget when the iteration broke down: an
 *                     action whose G-orthogonal part vanished, R2)
 *   rel_residual      |r_k| / |r0_k| of the step's final residual r = r0 - G v (the CG recursion's
 *                     residual; for the batch policies r0 - G S Ghat^-1 S^T r0)
 *   min_eta           the smallest eta_j = d_j^T G d_j of the step (the pivots of S^T G S)
 *   dropped_filter    trace(M^T M) minus the kept eigenvalues at the filter's truncation of step k
 *                     (the mass N N^T of Sec. 3.2 that is discarded); 0 without truncation
 *   dropped_smoother  the same for the smoother's truncation of Ws at step k (after cakf_smooth)
 * Errors: CAKF_ERR_STATE (no successful cakf_filter), CAKF_ERR_CUDA.
 */
int cakf_get_diagnostics(const cakf_ctx* ctx, int32_t* actions, double* rel_residual, double* min_eta,
                         double* dropped_filter, double* dropped_smoother);

/*
 * cakf_set_wait_limit -- iteration limit of every bounded device-side wait (the tensor-core
 * kernels' mbarrier waits, the tridiagonalisation's exchange polling) for the calls that follow,
 * process-wide; 0 restores each kernel's default (seconds of waiting).  A wait that runs out makes
 * its kernel stop cleanly and the call return CAKF_ERR_TIMEOUT; the context stays usable.  Meant
 * for tests of that path.  No counterpart in the paper.  Errors: CAKF_ERR_ARG (negative).
 */
int cakf_set_wait_limit(int64_t iterations);

/*
 * cakf_set_device_memory_limit -- cap (bytes) on the device memory one context may hold; a
 * cakf_filter that would exceed it returns CAKF_ERR_OOM before allocating.  0 = no cap (default).
 * Process-wide.  No counterpart in the paper (a resource guard, and the way tests reach the
 * out-of-memory path without exhausting the device).
 */
int cakf_set_device_memory_limit(uint64_t bytes);

/* cakf_get_stats -- timings and counters of the last filter / smooth calls (host output). */
int cakf_get_stats(const cakf_ctx* ctx, cakf_stats* out);

/* cakf_set_profiling -- when on, the hot kernels are bracketed by CUDA events on their stream
 * and their device times are summed into cakf_stats (adds one event pair per launch). */
int cakf_set_profiling(cakf_ctx* ctx, int on);

/* cakf_free -- release a context and all device memory it holds.  NULL is accepted. */
void cakf_free(cakf_ctx* ctx);

/* cakf_last_error -- message of the calling thread's last failed call ("" if none). */
const char* cakf_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* CAKF_H */
