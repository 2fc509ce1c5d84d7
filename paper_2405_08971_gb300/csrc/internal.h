// Internal declarations shared by the translation units of libcakf (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>
#include <algorithm>
#include "common.cuh"

namespace cakf {

// Count of kernels launched by this library (all threads); read by cakf_get_stats.
long long launch_count();
void note_launch(long long k = 1);

// Launch of a kernel that begins with pdl_wait(); pdl_trigger(); with programmatic stream
// serialisation, so that its launch overlaps the previous kernel in the stream (the chains of short
// dependent kernels of the CG loop and the eigensolver).  Counts the launch.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  note_launch();
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

template <class T> void prep_coords(const double* X, int n, int dim, double scale, C4<T>* out, cudaStream_t st);
template <class T> void gather_coords(const C4<T>* X, const int* idx, int m, C4<T>* out, cudaStream_t st);
template <class T>
// K(X_o, X_o) s into gram_matvec_slots(m) partial rows of part; with rp > 0 the same launch forms the
// partials of Mo^T s (Mo: m x rp, ld ldm) into tpart for cg_combine
void gram_matvec(int ker, const C4<T>* Xo, const T* s, int m, T sf2, T* part, const T* Mo, int ldm, int rp, T* tpart,
                 const int* active, cudaStream_t st);
// number of partial slots (rows of part, each m long) gram_matvec writes for m observations
int gram_matvec_slots(int m);
template <class T>
void gram_block_simt(int ker, const C4<T>* Xr, int nr, const C4<T>* Xc, int nc, const T* B, int ldb, int width,
                     T sf2, T* Out, int ldo, cudaStream_t st);
template <class T>
void gram_block_dlogl_simt(int ker, const C4<T>* Xr, int nr, const C4<T>* Xc, int nc, const T* B, int ldb, int width,
                           T sf2, T* Out, int ldo, cudaStream_t st);
// CG iteration j (non-FP64 modes skip cg_reorth; see the loop in cakf.cu):
//   cg_combine: g = K s + sn2 s - a2 Mo t, and per-block partials of the first-pass dots (dpart1)
//   cg_upd1:    first G-orthogonalisation pass, per-block partials of the second-pass dots (dpart2)
//   cg_upd2:    second pass, scalars, V/GV/v/r update; with Snext the next action s = r
template <class T>
void cg_combine(const T* part, int nsplit, const T* s, T sn2, const T* Mo, int ldm, int r, const T* t, T a2, int m,
                T* g, const T* V, int ldv, int j, const T* r0, const T* v, T* dpart1, const int* active,
                cudaStream_t st);
// elements needed for dpart1 followed by dpart2 at m observations and an action budget
size_t cg_dpart_elems(int m, int budget);
template <class T>
void cg_upd1(int j, const T* dpart1, double* dots1, T* V, T* GV, int ldv, const T* s, const T* g, int m,
             T* dpart2, const int* active, cudaStream_t st);
template <class T>
void cg_upd2(int j, const double* dots1, const T* dpart2, T* V, T* GV, int ldv, T* r, T* v, T* s, T* Q,
             int m, double bd_tol, double rtol2_r0sq, int use_rtol, int* active, double* eta, double* alpha,
             int* count, T* Snext, cudaStream_t st);
template <class T>
void cg_reorth(const T* Q, int ldq, int j, T* s, int m, double* qd, T* S, int lds, const int* active, cudaStream_t st);
template <class T>
void cg_select(int j, const T* r, const double* rep, int m, T* s, T* S, int lds, const int* active, cudaStream_t st);
template <class T>
void cg_init(const double* y, const double* mpred, const int* obs, int m, T* r, T* r0, T* v, double* r0sq,
             cudaStream_t st);
template <class T>
void gemm_tn(const T* A, int lda, int na, const T* B, int ldb, int nb, int K, double alpha, double beta, double* C,
             int ldc, double* part, size_t part_elems, cudaStream_t st);
template <class T, class TB>
void gemm_nn(int M, int N, int K, T alpha, const T* A, int lda, const TB* B, int ldb, T beta, T* C, int ldc,
             cudaStream_t st);
void gemm_small_f64(int ta, int tb, int M, int N, int K, double alpha, const double* A, int lda, const double* B,
                    int ldb, double beta, double* C, int ldc, cudaStream_t st);
template <class T> void gather_rows(const T* In, int ldi, const int* idx, int m, int cols, T* Out, int ldo, cudaStream_t st);
template <class T>
void scatter_add_rows(const T* In, int ldi, const int* idx, int m, int cols, T alpha, T* Out, int ldo, cudaStream_t st);
template <class T> void rowsumsq(const T* A, int lda, int n, int cols, double beta, double* rs, cudaStream_t st);
void predict_mean(const double* mprev, const double* mu_k, const double* mu_km1, double a, int n, double* mpred,
                  cudaStream_t st);
template <class T>
void filter_out(const double* mpred, const T* PVv, int ld, int ic, double sf2, double a2, const double* rs_plus, int n,
                double* mout, double* vout, double* rs_pw, cudaStream_t st);
// Two-block state of the Matern-3/2 temporal factor (rows [0, half) positions, [half, 2 half)
// velocities): Out = (C (x) I) In with C row-major 2 x 2 (In == Out allowed); the mean prediction
// m^- = A (m - (mu_{k-1}, 0)) + (mu_k, 0); out = a + b.
template <class T>
void mix2(const T* In, int ldi, T* Out, int ldo, int half, int cols, const double C[4], cudaStream_t st);
void predict_mean2(const double* mprev, const double* mu_k, const double* mu_km1, const double A[4], int n, int half,
                   double* mpred, cudaStream_t st);
template <class T> void add_vec(const double* a, const T* b, int n, double* out, cudaStream_t st);
template <class T> void scale_copy(const T* In, int ldi, int n, int cols, T alpha, T* Out, int ldo, cudaStream_t st);
template <class T>
void smooth_out(const double* mk, const double* vk, const T* Y, int ld, int cw, int n, double* ms, double* vs,
                cudaStream_t st);
template <class T> void ws_obs(const int* obs, int m, const T* vk, const T* Vz, T* ws, cudaStream_t st);
template <class T> void build_x(const T* Ws, int ldw, int cw, const T* ws, T alpha, int n, T* X, int ldx, cudaStream_t st);
void nll_step(const double* eta, const double* alpha, const int* count, double* SS, int ic, double* nll_k, int* err,
              cudaStream_t st);
void set_diag(double* G, int ld, const double* lam, double scale, int r, cudaStream_t st);
void nll_def(const int* count, double* Gh, double* SS, int ld, const double* yh, double* z, double* nll_k, int* err,
             cudaStream_t st);
void grad_small(int ic, int np, const double* Gh, const double* dGh, const double* yh, const double* dyh, double* L,
                double* Rinv, double* W, double* tmp, double* Q, double* u, double* grad, int* err, cudaStream_t st);
template <class T>
void gather_rows_f64(const double* In, int ld, const int* idx, int m, int cols, T* Out, int ldo, cudaStream_t st);
template <class T>
void tangent_mean(const double* dmpred, const T* E, size_t estride, int ecol, int lde, const T* t, int ldt, int n,
                  int np, double* dm, cudaStream_t st);
template <class T> void axpy_block(T alpha, const T* X, int ldx, int rows, int cols, T* Y, int ldy, cudaStream_t st);
template <class T> void scale_cols(T* A, int ld, int rows, int cols, T s, cudaStream_t st);
void tangent_predict(const double* mprev, const double* dmprev, const double* mu_km1, double a, double adot_lt, int n,
                     int np, double* dmpred, cudaStream_t st);
void put_block_sym(double* G, int ld, int row0, int col0, const double* B, int ldb, int nr, int nc, double scale,
                   cudaStream_t st);
void check_finite(const double* x, size_t n, int* err, cudaStream_t st);
void scale_f64(double* A, int ld, int rows, int cols, double s, cudaStream_t st);
template <class T>
void convert_from_f64(const double* In, int ldi, int rows, int cols, T* Out, int ldo, cudaStream_t st);
void convert_to_f64(const float* In, int ldi, int rows, int cols, double* Out, int ldo, cudaStream_t st);
void to_bf16(const float* In, int ldi, int rows, int cols, uint16_t* Out, int ldo, cudaStream_t st);
void from_bf16(const uint16_t* In, int ldi, int rows, int cols, float* Out, int ldo, cudaStream_t st);

// Batch update (Alg. 2): coordinate actions, Cholesky of the projected Gram with z = L^-1 S^T r0,
// and [V v] = [S L^-T, S L^-T z].  At most kBatchMaxActions actions per step.
constexpr int kBatchMaxActions = 160;
template <class T> void coord_actions(int m, int i, T* S, cudaStream_t st);
int batch_chol(const double* Gh, int i, const double* yh, double* L, double* z, double* eta, int* err,
               cudaStream_t st);
// Per-step diagnostics: *out += |x|^2; *out = trace(G); *out -= sum(w[0..keep)); *out += |r0 - GS L^-T z|^2
template <class T> void sqnorm_acc(const T* x, int m, double* out, cudaStream_t st);
void trace_into(const double* G, int N, int ld, double* out, cudaStream_t st);
void sub_sum(const double* w, int keep, double* out, cudaStream_t st);
template <class T>
void batch_resid(const T* GS, int m, int i, const double* L, const double* z, const T* r0, double* out, cudaStream_t st);
template <class T>
void batch_v(const T* S, int m, int i, const double* L, const double* z, T* Vv, cudaStream_t st);

// Posterior sampler helpers (S draws as columns): xp = a xprev + b + q; d = y - xp[obs] - eps;
// x = xa + alpha t.
void samp_predict(const double* xprev, const double* q, const double* mu_k, const double* mu_km1, double a, int n,
                  int S, double* xp, cudaStream_t st);
template <class T>
void samp_resid(const double* y, const double* xp, const int* obs, const double* eps, int m, int n, int S, T* d,
                cudaStream_t st);
template <class T>
void samp_add(const double* xa, const T* t, int ldt, double alpha, int n, int S, double* x, cudaStream_t st);

// Temporal interpolation: filter mean and variance at t_k + tau from step k's (at = A(t, t_k)).
void interp_filter(const double* mk, const double* vk, const double* mu_t, const double* mu_k, double at, double sf2,
                   int n, double* m, double* v, cudaStream_t st);

// Record msg as the calling thread's cakf_last_error message; returns code.
int set_last_error(int code, const char* msg);

// Device error-flag values (the flag is an int in device memory, 0 = ok)
constexpr int kErrNumeric = 1;     // a numeric failure without a more specific code
constexpr int kErrTimeout = 2;
constexpr int kErrNllChol = 3;     // S^T G S or S^T S of a step not positive definite (NLL term)
constexpr int kErrBatchChol = 4;   // the batch update's S^T G S not positive definite
constexpr int kErrSecular = 5;     // a secular equation of the eigensolver did not converge
constexpr int kErrNonFinite = 6;   // a non-finite output
constexpr int kErrGradChol = 7;    // the gradient pass's S^T G S not positive definite

// Switch for the FP32 GEMM launchers (gemm_nn / gemm_tn): 0 or 1 = own SIMT kernels (the plain
// FP32 path), 2 = own tensor-core kernels with split TF32 operands for the large products (the
// tensor-core modes).  Set by the orchestration per call (thread-local), with the device error
// flag the tensor-core kernels raise when a bounded wait runs out.
void set_gemm_mode(int mode);
int gemm_mode();
void set_gemm_err(int* err);
// Bounded device waits: the iteration limit to pass to a kernel (dflt unless cakf_set_wait_limit
// set another).
void set_wait_limit(long long it);
long long wait_limit(long long dflt);

// ---- FP64 symmetric eigensolver (eig.cu) ----
// Workspace bytes needed for matrices up to order nmax.
size_t eig_workspace_bytes(int nmax);
// Top-`nkeep` eigenpairs of the symmetric N x N matrix A (FP64, column-major, lda >= N; A is
// overwritten).  w: nkeep eigenvalues, descending (device).  U: N x nkeep eigenvectors
// (column-major, ld = ldu) in precision T.  err: device flag raised on timeout / non-finite.
// marks: NULL, or two events recorded after the tridiagonalisation and after divide & conquer.
// assembly: kAssemblyFP64, or kAssemblyFF for callers that round U to FP32 -- the final product of
// the Householder reflectors with the tridiagonal's eigenvectors then runs in double-FP32
// arithmetic (about 1e-14 relative in U) on the FP32 pipe; the tridiagonalisation, the divide and
// conquer and the eigenvalues stay FP64.  (T = double only.)
constexpr int kAssemblyFP64 = 0, kAssemblyFF = 1;
template <class T>
int eig_sym_topk(double* A, int lda, int N, int nkeep, double* w, T* U, int ldu, void* work, size_t work_bytes,
                 int* err, cudaStream_t st, cudaEvent_t* marks = nullptr, int assembly = kAssemblyFP64);

// ---- tensor-core Gram x block (gram_tc.cu) ----
// Out[nr x width] (FP32, column-major, ld = ldo) = sf2 K(Xr, Xc) B with B packed by gram_tc_pack_b.
// kind: 0 = BF16 operands (one MMA per slice), 1 = split BF16 (hi + lo parts, three MMAs).
int gram_block_tc(int ker, int kind, const C4<float>* Xr, int nr, const C4<float>* Xc, int nc, const void* B, int ldb,
                  int width, float sf2, float* Out, int ldo, int* err, cudaStream_t st);
// Tall-skinny FP32 products on the tensor cores with split TF32 operands (about 22 significant bits
// per product, FP32 accumulation):
//   gemm_tc_nn: C (M x N, float) = alpha A B + beta C, A M x K (lda), B K x N (ldb), column-major;
//   gemm_tc_tn: C (na x nb, double) = alpha A^T B + beta C, A K x na, B K x nb, with the K range
//               split over CTAs; part (part_bytes) holds the FP32 partial tiles, summed in FP64.
// Return 0 on success (launch errors otherwise); a timed-out wait raises the device flag err.
int gemm_tc_nn(int M, int N, int K, float alpha, const float* A, int lda, const float* B, int ldb, float beta,
               float* C, int ldc, int* err, cudaStream_t st);
int gemm_tc_tn(const float* A, int lda, int na, const float* B, int ldb, int nb, int K, double alpha, double beta,
               double* C, int ldc, void* part, size_t part_bytes, int* err, cudaStream_t st);
// Convert a column-major float block (rows x cols, ld) into the operand layout of gram_block_tc.
int gram_tc_pack_b(int kind, const float* B, int ldb, int rows, int cols, void* Bp, int ldp, cudaStream_t st);
size_t gram_tc_packed_ld(int rows);
int gram_tc_max_width();
// Staging bytes (packed operand part(s), mean column, padded coordinates) for a rows x width block.
size_t gram_tc_staging_bytes(int rows, int width, int kind);

}  // namespace cakf
