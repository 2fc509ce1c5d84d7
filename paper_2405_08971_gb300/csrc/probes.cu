// Throughput probes for the roofline denominators that MEASURED_PEAKS-style copy / GEMM figures do
// not give: the special-function (MUFU) rate of the sqrt + exp2 pair that every kernel-matrix
// entry costs, and the FP64 FMA rate that bounds the eigensolver.  Plain kernels: every thread runs
// independent dependency chains (enough instruction-level parallelism to keep the pipe busy), the
// grid covers every SM several times, and the result is written so that nothing is optimised away.
#include <string>
#include "cakf.h"
#include "internal.h"

namespace cakf {
namespace {

constexpr int PROBE_CHAINS = 8;
constexpr int PROBE_THREADS = 256;

// Per iteration and chain: one sqrt.approx and one ex2.approx (the MUFU pair of a Matern entry),
// plus one FP32 multiply-add on the FMA pipe that keeps the value in [1, 2].
__global__ void __launch_bounds__(PROBE_THREADS) k_probe_mufu(int iters, float* out) {
  float v[PROBE_CHAINS];
#pragma unroll
  for (int c = 0; c < PROBE_CHAINS; ++c) v[c] = 1.0f + 0.01f * c + 1e-6f * threadIdx.x;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < PROBE_CHAINS; ++c) {
      float s, e;
      asm volatile("sqrt.approx.ftz.f32 %0, %1;" : "=f"(s) : "f"(v[c]));
      asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(e) : "f"(-s));
      v[c] = fmaf(e, 0.5f, 1.0f);
    }
  }
  float acc = 0.f;
#pragma unroll
  for (int c = 0; c < PROBE_CHAINS; ++c) acc += v[c];
  if (acc == 12345.678f) out[blockIdx.x * blockDim.x + threadIdx.x] = acc;   // never true; keeps the chains
}

// Per iteration and chain: one FP64 fused multiply-add.
__global__ void __launch_bounds__(PROBE_THREADS) k_probe_dfma(int iters, double* out) {
  double v[PROBE_CHAINS];
#pragma unroll
  for (int c = 0; c < PROBE_CHAINS; ++c) v[c] = 1.0 + 1e-3 * c + 1e-9 * threadIdx.x;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < PROBE_CHAINS; ++c) v[c] = fma(v[c], 0.9999999999, 1e-10);
  }
  double acc = 0.0;
#pragma unroll
  for (int c = 0; c < PROBE_CHAINS; ++c) acc += v[c];
  if (acc == 12345.678) out[blockIdx.x * blockDim.x + threadIdx.x] = acc;
}

template <class F>
double time_ms(F launch, cudaStream_t st) {
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  launch();   // warm-up
  cudaEventRecord(e0, st);
  launch();
  cudaEventRecord(e1, st);
  cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return ms;
}

}  // namespace
}  // namespace cakf

using namespace cakf;

extern "C" int cakf_probe_peaks(double* mufu_ops_per_s, double* fp64_flops_per_s, void* cuda_stream) {
  if (!mufu_ops_per_s || !fp64_flops_per_s) return set_last_error(CAKF_ERR_ARG, "cakf_probe_peaks: NULL output");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int blocks = sms * 8;               // eight 256-thread blocks per SM: 64 warps
  const int it_mufu = 4096, it_dfma = 512;
  void* sink = nullptr;                      // written only by a thread whose sum hits a sentinel
  if (cudaMalloc(&sink, (size_t)blocks * PROBE_THREADS * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return set_last_error(CAKF_ERR_OOM, "cakf_probe_peaks: sink allocation failed");
  }
  const double ms_mufu = time_ms([&] {
    k_probe_mufu<<<blocks, PROBE_THREADS, 0, st>>>(it_mufu, (float*)sink);
    note_launch();
  }, st);
  const double ms_dfma = time_ms([&] {
    k_probe_dfma<<<blocks, PROBE_THREADS, 0, st>>>(it_dfma, (double*)sink);
    note_launch();
  }, st);
  cudaError_t ce = cudaGetLastError();
  cudaFree(sink);
  if (ce != cudaSuccess)
    return set_last_error(CAKF_ERR_CUDA, (std::string("cakf_probe_peaks: ") + cudaGetErrorString(ce)).c_str());
  const double threads = (double)blocks * PROBE_THREADS;
  *mufu_ops_per_s = threads * it_mufu * PROBE_CHAINS * 2.0 / (ms_mufu * 1e-3);
  *fp64_flops_per_s = threads * it_dfma * PROBE_CHAINS * 2.0 / (ms_dfma * 1e-3);
  return CAKF_OK;
}
