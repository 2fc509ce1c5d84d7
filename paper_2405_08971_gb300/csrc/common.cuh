// Shared device helpers of libcakf: coordinate records, Matern kernel values, reductions and a
// bounded grid barrier.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <cmath>

namespace cakf {

// Grid coordinates, pre-scaled by c_nu / l_x (c = 1, sqrt(3), sqrt(5) for nu = 1/2, 3/2, 5/2), so
// that the Matern argument is the plain Euclidean distance s = |xs - xs'|.  w is padding.
template <class T> struct alignas(4 * sizeof(T)) C4 { T x, y, z, w; };

__device__ __forceinline__ float approx_sqrt(float v) {
  float r;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
  return r;
}
__device__ __forceinline__ float approx_exp_neg(float s) {   // exp(-s) via ex2.approx
  float r;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(-1.4426950408889634f * s));
  return r;
}

// ---- programmatic dependent launch.  A kernel started by launch_pdl may become resident while the
// kernel before it in the stream is still running; pdl_wait() returns once that kernel has completed
// and its writes are visible, so every such kernel calls it before it touches memory, and then
// pdl_trigger() so that the next kernel's launch overlaps this one.  (Without the launch attribute
// both are no-ops.)
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Matern correlation times sf2 of the scaled distance^2 (Rasmussen-Williams forms):
//   nu=1/2: e^-s,  nu=3/2: (1+s) e^-s,  nu=5/2: (1 + s + s^2/3) e^-s.
template <int KER> __device__ __forceinline__ float kval(float s2, float sf2) {
  float s = approx_sqrt(s2);
  float e = approx_exp_neg(s) * sf2;
  if (KER == 0) return e;
  if (KER == 1) return fmaf(s, e, e);
  return fmaf(fmaf(s, 0.33333333333333333f, 1.0f) * s, e, e);
}
template <int KER> __device__ __forceinline__ double kval(double s2, double sf2) {
  double s = sqrt(s2);
  double e = exp(-s) * sf2;
  if (KER == 0) return e;
  if (KER == 1) return fma(s, e, e);
  return fma(fma(s, 1.0 / 3.0, 1.0) * s, e, e);
}

// d/dlog(l_x) of the Matern value (s = scaled distance, ds/dlog l = -s):
//   nu=1/2: s e^-s,  nu=3/2: s^2 e^-s,  nu=5/2: s^2 (1 + s) e^-s / 3   (times sf2)
template <int KER> __device__ __forceinline__ float kval_dlogl(float s2, float sf2) {
  float s = approx_sqrt(s2);
  float e = approx_exp_neg(s) * sf2;
  if (KER == 0) return s * e;
  if (KER == 1) return s2 * e;
  return s2 * (1.0f + s) * e * 0.33333333333333333f;
}
template <int KER> __device__ __forceinline__ double kval_dlogl(double s2, double sf2) {
  double s = sqrt(s2);
  double e = exp(-s) * sf2;
  if (KER == 0) return s * e;
  if (KER == 1) return s2 * e;
  return s2 * (1.0 + s) * e / 3.0;
}

// ---- packed FP32 pairs (two columns of one row): f32x2 arithmetic on 64-bit registers
__device__ __forceinline__ uint64_t f2_make(float lo, float hi) {
  uint64_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void f2_split(uint64_t v, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ uint64_t f2_sub(uint64_t a, uint64_t b) {
  uint64_t r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ uint64_t f2_mul(uint64_t a, uint64_t b) {
  uint64_t r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ uint64_t f2_fma(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}
__device__ __forceinline__ float f2_sum(uint64_t v) {
  float lo, hi;
  f2_split(v, lo, hi);
  return lo + hi;
}
// Matern correlation (without sf2) of one row against a column pair.  Coordinates are pre-scaled
// by c_nu / l_x, so with s the Euclidean distance:  nu=1/2: e^-s,  nu=3/2: (1+s) e^-s,
// nu=5/2: (1 + s + s^2/3) e^-s.  sqrt and exp2 run on the MUFU unit (approximate, ftz).
template <int KER>
__device__ __forceinline__ uint64_t kpair(uint64_t rx, uint64_t ry, uint64_t rz, uint64_t cx, uint64_t cy,
                                          uint64_t cz) {
  const uint64_t dx = f2_sub(rx, cx), dy = f2_sub(ry, cy), dz = f2_sub(rz, cz);
  uint64_t d2 = f2_mul(dz, dz);
  d2 = f2_fma(dy, dy, d2);
  d2 = f2_fma(dx, dx, d2);
  float a, b;
  f2_split(d2, a, b);
  const uint64_t sd = f2_make(approx_sqrt(a), approx_sqrt(b));
  const uint64_t t = f2_mul(sd, f2_make(-1.4426950408889634f, -1.4426950408889634f));
  f2_split(t, a, b);
  float ea, eb;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(ea) : "f"(a));
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(eb) : "f"(b));
  const uint64_t e = f2_make(ea, eb);
  if (KER == 0) return e;
  if (KER == 1) return f2_fma(sd, e, e);
  const uint64_t p = f2_mul(f2_fma(sd, f2_make(0.33333333333333333f, 0.33333333333333333f),
                                   f2_make(1.0f, 1.0f)), sd);
  return f2_fma(p, e, e);
}

template <class T> __device__ __forceinline__ T dist2(const C4<T>& a, const C4<T>& b) {
  T dx = a.x - b.x, dy = a.y - b.y, dz = a.z - b.z;
  return fma(dx, dx, fma(dy, dy, dz * dz));
}

template <class T> __device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum (blockDim.x a multiple of 32, <= 1024); every thread gets the result.
template <class T> __device__ T block_sum(T v) {
  __shared__ T red[32];
  __syncthreads();
  v = warp_sum(v);
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) red[w] = v;
  __syncthreads();
  int nw = (blockDim.x + 31) >> 5;
  T t = (threadIdx.x < nw) ? red[threadIdx.x] : T(0);
  if (w == 0) t = warp_sum(t);
  if (threadIdx.x == 0) red[0] = t;
  __syncthreads();
  T r = red[0];
  __syncthreads();
  return r;
}


}  // namespace cakf
