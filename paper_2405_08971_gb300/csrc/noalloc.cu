// cakf_gram_matmul_noalloc: the Gram x matrix product of cakf_gram_matmul with every piece of
// scratch taken from one statically sized device array of this translation unit, so that the
// call itself never allocates device memory.  The paper has no counterpart; this is a library
// integration variant for callers that cannot allocate (see cakf.h).
//
// Scratch layout inside g_noalloc_scratch (offsets 256-byte aligned):
//   [0, 256)              device error flag (int), cleared on the call's stream before each use
//   [256, 256 + coords)   (nr + nc) pre-scaled coordinate records, C4<double> or C4<float>
//   [.., .. + staging)    tensor-core paths only: packed operand part(s), fp32 last column, padded
//                         coordinates (layout of gram_tc_pack_b / gram_block_tc)
// Every byte the kernels read from the coordinate and staging regions is written earlier on
// the same stream by the same call, so only the error flag has to start at zero.
#include <cmath>
#include <mutex>
#include <string>
#include "cakf.h"
#include "internal.h"

using namespace cakf;

namespace {

constexpr size_t kScratchBytes = CAKF_NOALLOC_SCRATCH_BYTES;   // 64 MiB per device
constexpr int kMaxDevices = 128;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_mu;
void* g_base[kMaxDevices] = {};

inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

double nu_scale_of(int kernel) { return kernel == 0 ? 1.0 : (kernel == 1 ? std::sqrt(3.0) : std::sqrt(5.0)); }

// True when p is device (or managed) memory of the current device: the kernels launched here run
// on the current device and must not be handed another device's allocation.
bool on_device(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) { cudaGetLastError(); return false; }
  if (at.type == cudaMemoryTypeManaged) return true;
  if (at.type != cudaMemoryTypeDevice) return false;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return false; }
  return at.device == dev;
}

int err(int code, const std::string& msg) { return set_last_error(code, msg.c_str()); }

// Device address of g_noalloc_scratch on the current device, looked up once per device.
int scratch_base(void** out) {
  int dev = -1;
  cudaError_t ce = cudaGetDevice(&dev);
  if (ce != cudaSuccess) return err(CAKF_ERR_CUDA, std::string("cakf_gram_matmul_noalloc: cudaGetDevice: ") +
                                                       cudaGetErrorString(ce));
  if (dev < 0 || dev >= kMaxDevices) return err(CAKF_ERR_CUDA, "cakf_gram_matmul_noalloc: device ordinal out of range");
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_base[dev]) {
    void* p = nullptr;
    // The first lookup on a device loads this module there, which reserves the static scratch:
    // next to a full memory pool that can fail with cudaErrorMemoryAllocation.
    ce = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (ce != cudaSuccess || !p) {
      cudaGetLastError();
      return err(ce == cudaErrorMemoryAllocation ? CAKF_ERR_OOM : CAKF_ERR_CUDA,
                 std::string("cakf_gram_matmul_noalloc: cudaGetSymbolAddress failed: ") + cudaGetErrorString(ce));
    }
    g_base[dev] = p;
  }
  *out = g_base[dev];
  return CAKF_OK;
}

}  // namespace

extern "C" int cakf_gram_matmul_noalloc(int32_t kernel, double log_lx, double log_sf2, int32_t dim, const double* Xr,
                                        int32_t nr, const double* Xc, int32_t nc, const void* B, int32_t ldb,
                                        int32_t width, void* Out, int32_t ldo, int32_t precision, void* cuda_stream) {
  if (kernel < 0 || kernel > 2 || dim < 1 || dim > 3 || nr < 1 || nc < 1 || width < 1 || ldb < nc || ldo < nr)
    return err(CAKF_ERR_ARG, "cakf_gram_matmul_noalloc: invalid sizes or kernel");
  if (!Xr || !Xc || !B || !Out) return err(CAKF_ERR_ARG, "cakf_gram_matmul_noalloc: NULL pointer");
  if (precision < CAKF_FP64 || precision > CAKF_TF32X3)
    return err(CAKF_ERR_ARG, "cakf_gram_matmul_noalloc: unknown precision");
  const int kind = precision == CAKF_BF16 ? 0 : precision == CAKF_FP16X3 ? 1 : precision == CAKF_TF32 ? 2
                 : precision == CAKF_TF32X3 ? 3 : -1;
  const bool tcp = kind >= 0;
  if (tcp && (width < 2 || width > gram_tc_max_width()))
    return err(CAKF_ERR_ARG, "cakf_gram_matmul_noalloc: the tensor-core paths need 2 <= width <= 513");
  if (!std::isfinite(log_lx) || !std::isfinite(log_sf2))
    return err(CAKF_ERR_ARG, "cakf_gram_matmul_noalloc: non-finite hyperparameters");

  // scratch demand, checked against the fixed capacity before anything touches the device
  const size_t rec = precision == CAKF_FP64 ? sizeof(C4<double>) : sizeof(C4<float>);
  const size_t off_coords = 256;
  const size_t off_stage = off_coords + align256(((size_t)nr + (size_t)nc) * rec);
  const size_t need = off_stage + (tcp ? align256(gram_tc_staging_bytes(nc, width, kind)) : 0);
  if (need > kScratchBytes)
    return err(CAKF_ERR_ARG, "cakf_gram_matmul_noalloc: this call needs " + std::to_string(need) +
                                 " bytes of scratch but the static scratch holds " + std::to_string(kScratchBytes) +
                                 " bytes; use cakf_gram_matmul, or split the rows / columns into smaller calls");
  if (!on_device(Xr) || !on_device(Xc) || !on_device(B) || !on_device(Out))
    return err(CAKF_ERR_ARG, "cakf_gram_matmul_noalloc: all arrays must be device arrays of the current device");

  void* base = nullptr;
  int rc = scratch_base(&base);
  if (rc) return rc;
  unsigned char* s = static_cast<unsigned char*>(base);
  int* dflag = reinterpret_cast<int*>(s);
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const double scale = nu_scale_of(kernel) / std::exp(log_lx);
  const double sf2 = std::exp(log_sf2);
  cudaError_t ce = cudaMemsetAsync(dflag, 0, sizeof(int), st);
  if (ce != cudaSuccess) return err(CAKF_ERR_CUDA, std::string("cakf_gram_matmul_noalloc: ") + cudaGetErrorString(ce));
  if (precision == CAKF_FP64) {
    C4<double>* xr = reinterpret_cast<C4<double>*>(s + off_coords);
    C4<double>* xc = xr + nr;
    prep_coords<double>(Xr, nr, dim, scale, xr, st);
    prep_coords<double>(Xc, nc, dim, scale, xc, st);
    gram_block_simt<double>(kernel, xr, nr, xc, nc, (const double*)B, ldb, width, sf2, (double*)Out, ldo, st);
  } else {
    C4<float>* xr = reinterpret_cast<C4<float>*>(s + off_coords);
    C4<float>* xc = xr + nr;
    prep_coords<float>(Xr, nr, dim, scale, xr, st);
    prep_coords<float>(Xc, nc, dim, scale, xc, st);
    if (precision == CAKF_FP32) {
      gram_block_simt<float>(kernel, xr, nr, xc, nc, (const float*)B, ldb, width, (float)sf2, (float*)Out, ldo, st);
    } else {
      void* stage = s + off_stage;
      const int ldp = (int)gram_tc_packed_ld(nc);
      int r2 = gram_tc_pack_b(kind, (const float*)B, ldb, nc, width, stage, ldp, st);
      if (!r2) r2 = gram_block_tc(kernel, kind, xr, nr, xc, nc, stage, ldp, width, (float)sf2, (float*)Out, ldo, dflag, st);
      if (r2)
        return err(CAKF_ERR_CUDA, "cakf_gram_matmul_noalloc: tensor-core Gram x block launch failed (code " +
                                      std::to_string(r2) + ")");
    }
  }
  ce = cudaStreamSynchronize(st);
  if (ce != cudaSuccess) return err(CAKF_ERR_CUDA, std::string("cakf_gram_matmul_noalloc: ") + cudaGetErrorString(ce));
  int e = 0;
  ce = cudaMemcpy(&e, dflag, sizeof(int), cudaMemcpyDeviceToHost);
  if (ce != cudaSuccess) return err(CAKF_ERR_CUDA, std::string("cakf_gram_matmul_noalloc: ") + cudaGetErrorString(ce));
  if (e == kErrTimeout) return err(CAKF_ERR_TIMEOUT, "cakf_gram_matmul_noalloc: a device-side wait exceeded its limit");
  if (e) return err(CAKF_ERR_NUMERIC, "cakf_gram_matmul_noalloc: numeric error");
  return CAKF_OK;
}
