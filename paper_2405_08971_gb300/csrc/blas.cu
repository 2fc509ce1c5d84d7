// Plain tall-skinny GEMMs of the factor updates through cuBLAS (FP32 inputs and outputs).
// In the mixed-precision mode the products use cuBLAS's FP32 emulation on BF16 tensor cores
// (three-term bf16 splits, FP32-level accuracy); in the plain FP32 mode they use FP32 SIMT.
#include <cublas_v2.h>
#include <mutex>
#include "internal.h"

namespace cakf {
namespace {
thread_local cublasHandle_t t_handle = nullptr;
thread_local int t_device = -1;

cublasHandle_t handle() {
  int dev = 0;
  cudaGetDevice(&dev);
  if (t_handle && t_device == dev) return t_handle;
  if (t_handle) cublasDestroy(t_handle);
  t_handle = nullptr;
  if (cublasCreate(&t_handle) != CUBLAS_STATUS_SUCCESS) { t_handle = nullptr; return nullptr; }
  t_device = dev;
  return t_handle;
}
}  // namespace

// C (M x N) = alpha op(A) B + beta C, all column-major FP32; op(A) = A (M x K) or A^T (A is K x M).
int blas_gemm_f32(int emulate_bf16x9, int transA, int M, int N, int K, float alpha, const float* A, int lda,
                  const float* B, int ldb, float beta, float* C, int ldc, cudaStream_t st) {
  if (M <= 0 || N <= 0) return 0;
  cublasHandle_t h = handle();
  if (!h) return 1;
  cublasSetStream(h, st);
  cublasComputeType_t ct = CUBLAS_COMPUTE_32F;
  if (emulate_bf16x9) {
    ct = CUBLAS_COMPUTE_32F_EMULATED_16BFX9;
    cublasSetEmulationStrategy(h, CUBLAS_EMULATION_STRATEGY_EAGER);
  }
  cublasStatus_t s = cublasGemmEx(h, transA ? CUBLAS_OP_T : CUBLAS_OP_N, CUBLAS_OP_N, M, N, K, &alpha, A, CUDA_R_32F,
                                  lda, B, CUDA_R_32F, ldb, &beta, C, CUDA_R_32F, ldc, ct, CUBLAS_GEMM_DEFAULT);
  note_launch();
  return s == CUBLAS_STATUS_SUCCESS ? 0 : 2;
}

}  // namespace cakf
