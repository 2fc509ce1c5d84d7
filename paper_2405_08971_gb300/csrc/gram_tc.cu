// Tensor-core Gram x block product (placeholder until the tcgen05 kernel lands): reports no
// supported width, so callers use the SIMT kernel.
#include "internal.h"
namespace cakf {
int gram_block_tc(int, int, const C4<float>*, int, const C4<float>*, int, const void*, int, int, float, float*, int,
                  int*, cudaStream_t) { return 1; }
int gram_tc_pack_b(int, const float*, int, int, int, void*, int, cudaStream_t) { return 1; }
size_t gram_tc_packed_ld(int rows) { return (size_t)((rows + 127) / 128 * 128); }
int gram_tc_max_width() { return 0; }
}  // namespace cakf
