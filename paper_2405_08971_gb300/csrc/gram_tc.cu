// Tensor-core Gram x block product for sm_103a (tcgen05 + TMEM + TMA), the hot kernel of the CAKF / CAKS:
//
//   Out[i, c] = sf2 * sum_j corr(xr_i, xc_j) B[j, c]     (Out, B column-major; corr a Matern correlation)
//
// The kernel matrix is never stored.  The work is the sequence of (128-row tile, K slice) units,
// split evenly over a persistent grid of one CTA per SM.  Per slice, 16 producer warps evaluate the
// 128-row correlation tile from coordinates staged in shared memory and write it in the swizzled
// K-major layout the tensor core reads; a TMA warp stages the matching slice of the packed B
// operand; one thread issues tcgen05.mma (M = 128, N <= 256 per instruction, K = 16) accumulating
// in TMEM (up to 512 FP32 columns); the producer warps drain TMEM in the epilogue.  The last column
// of B (the mean vector of the filter / smoother) is not sent to the tensor core: the producers
// accumulate it in FP32 from the same correlation values.
//
// Four operand modes (template parameter MD):
//   BF16      one BF16 MMA per slice and N chunk (kind::f16); 64-column slices, 128-byte swizzle.
//   FP16 x3   every operand is carried as hi = fp16(x) plus lo = fp16(x - hi) (22 significant
//             bits; B is scaled per column by a power of two into [0.5, 1) first, undone in the
//             epilogue), and hi*hi + hi*lo + lo*hi accumulate in the same TMEM columns: FP32-class
//             products at three MMAs per slice; 32-column slices, 64-byte swizzle (the doubled
//             operands must still fit two pipeline stages in shared memory).
//   TF32      one kind::tf32 MMA per slice (operands rounded to TF32: 11 significant bits, FP32
//             exponent range); 32-column slices of 4-byte elements, 128-byte swizzle.
//   TF32 x3   hi = tf32(x), lo = tf32(x - hi) and three kind::tf32 MMAs (about 22 significant
//             bits, no scaling needed); 16-column slices, 64-byte swizzle.
// In every mode one MMA instruction consumes 32 bytes of K per operand row (16 16-bit or 8 32-bit
// elements), so the descriptors advance by 32 bytes per K step whatever the element type.
// Every mbarrier wait is bounded; on timeout the CTA raises the error flag and stops.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <mutex>
#include <map>
#include "internal.h"

namespace cakf {
namespace {

constexpr int BM = 128;          // rows per CTA (TMEM lanes)
constexpr int NPROD_WARPS = 16;  // kernel-tile producers (and epilogue)
constexpr int NQ = NPROD_WARPS / 4;   // producer warps per TMEM lane group (epilogue column split)
constexpr int TMA_WARP = NPROD_WARPS;
constexpr int MMA_WARP = NPROD_WARPS + 1;   // the remaining warp issues the MMAs
constexpr int NTHREADS = (NPROD_WARPS + 2) * 32;
constexpr int BK_MAX = 64;       // packed operands are padded to a multiple of the larger slice

// Operand modes (the kind argument of gram_block_tc / gram_tc_pack_b).
enum { MD_BF16 = 0, MD_F16X3 = 1, MD_TF32 = 2, MD_TF32X3 = 3 };

// Per-mode layout constants.
template <int MD> struct Mode {
  static constexpr bool SPLIT = (MD == MD_F16X3 || MD == MD_TF32X3);   // hi + lo parts, three MMAs
  static constexpr bool TF32 = (MD == MD_TF32 || MD == MD_TF32X3);     // kind::tf32, 4-byte elements
  static constexpr bool SCALED = (MD == MD_F16X3);                     // per-column power-of-two scale of B
  static constexpr int ES = TF32 ? 4 : 2;             // operand element bytes
  static constexpr int ROWB = SPLIT ? 64 : 128;       // bytes per tile row = swizzle span
  static constexpr int BK = ROWB / ES;                // kernel columns per pipeline stage
  static constexpr int NPART = SPLIT ? 2 : 1;         // operand parts (hi, lo)
  static constexpr int A_TILE = BM * ROWB;            // bytes per A part
  static constexpr int C_STAGE = BK * 16;             // column coordinates, pair layout
  static constexpr int W_STAGE = BK * 4;              // mean column
  static constexpr int CPT = BK / 8;                  // columns per producer thread and slice
  static constexpr uint32_t SBO = 8 * ROWB;           // 8-row group stride
  static constexpr uint64_t LAYOUT = SPLIT ? 4 : 2;   // descriptor swizzle: 64-byte / 128-byte
  // instruction descriptor format fields: FP32 accumulator (bit 4); A and B types in bits 7..9 and
  // 10..12: FP16 = 0, BF16 = 1 (kind::f16), TF32 = 2 (kind::tf32)
  static constexpr uint32_t FMT = (1u << 4) | (MD == MD_BF16 ? ((1u << 7) | (1u << 10)) : 0u) |
                                  (TF32 ? ((2u << 7) | (2u << 10)) : 0u);
};

constexpr long long WAIT_LIMIT = 20000000LL;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
// Bounded wait for the completion of the phase with the given parity.  Returns false on timeout
// or when another role of this CTA already aborted.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag, long long limit) {
  for (long long it = 0; it < limit; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
    if (*abort_flag) return false;
  }
  *abort_flag = 1;
  return false;
}

__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
      ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(dst), "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

// Shared-memory matrix descriptor: K-major, swizzled rows of ROWB bytes, 8-row groups SBO apart.
// The K step of an MMA (16 elements = 32 bytes) is taken by advancing the start address.
template <int MD>
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;                           // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(Mode<MD>::SBO >> 4) << 32;        // stride byte offset
  d |= (uint64_t)1 << 46;                           // descriptor version
  d |= Mode<MD>::LAYOUT << 61;                      // swizzle mode
  return d;
}

// Byte offset of byte `b` of row `row` in a swizzled tile: the 16-byte chunk index is XORed with
// the row's phase (row & 7 for 128-byte rows, (row >> 1) & 3 for 64-byte rows).
template <int MD>
__device__ __forceinline__ uint32_t sw_off(int row, int b) {
  constexpr int R = Mode<MD>::ROWB;
  const int chunk = b >> 4;
  const int phase = ((row * R) >> 7) & (R / 16 - 1);
  return (uint32_t)(row * R + ((chunk ^ phase) << 4) + (b & 15));
}

// Instruction descriptor, M = 128, N = n (K-major A and B).
template <int MD>
__host__ __device__ constexpr uint32_t idesc(int n) {
  return Mode<MD>::FMT | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

// D (TMEM) += A * B, or D = A * B when acc == 0; kind::tf32 for the TF32 modes, kind::f16 otherwise.
template <int MD>
__device__ __forceinline__ void mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  if constexpr (Mode<MD>::TF32) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
        ::"r"(d_tmem), "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
  } else {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
        ::"r"(d_tmem), "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
  }
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}

// (packed FP32 pair arithmetic f2_*: common.cuh)
__device__ __forceinline__ uint32_t f2_bf16(uint64_t v) {
  float lo, hi;
  f2_split(v, lo, hi);
  return pack_bf16(lo, hi);
}
__device__ __forceinline__ uint32_t f2_f16(uint64_t v) {
  float lo, hi;
  f2_split(v, lo, hi);
  __half2 h = __floats2half2_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&h);
}
// The two fp16 of a packed pair widened back to FP32 (exact).
__device__ __forceinline__ uint64_t f16x2_to_f2(uint32_t p) {
  const float2 f = __half22float2(*reinterpret_cast<const __half2*>(&p));
  return f2_make(f.x, f.y);
}

// FP32 -> TF32 (round to nearest, ties away from zero), kept in a 32-bit container.
__device__ __forceinline__ uint32_t tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

// (Matern correlation of a row against a column pair, kpair: common.cuh)

struct TcParams {
  const C4<float>* Xr;
  int nr;
  const C4<float>* Xc;     // nk * BK columns in pair layout (see k_pad_coords), sentinels beyond nc
  const float* wcol;       // padded mean column (zeros beyond nc), FP32
  const float* binv;       // FP16 x3: per-column factor undoing the operand scaling (else null)
  int nk;                  // number of K slices per row tile
  int ntiles;              // row tiles of BM rows
  int npad;                // accumulator columns (multiple of 16, <= 512)
  int nbox;                // TMA boxes per B slice
  int boxh;                // rows per TMA box
  int wtc;                 // valid tensor-core columns (<= npad)
  float sf2;
  float* Out;
  int ldo;
  int* err;
  int stages;
  int tmem_cols;
  uint32_t b_stage_bytes;
  long long wait_limit;    // iteration limit of every mbarrier wait
};

// Uniform vote over the producer warps (named barrier 1): true iff every producer passes true.
__device__ __forceinline__ bool producers_all(bool v) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.and.pred q, 1, %2, p;\n selp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"((uint32_t)v), "r"(NPROD_WARPS * 32)
      : "memory");
  return r != 0;
}

// Bounded wait that ignores the abort flag (used to let copies in flight land before exit).
__device__ __forceinline__ void mbar_drain(uint32_t bar, uint32_t parity) {
  for (long long it = 0; it < WAIT_LIMIT; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return;
  }
}

// Persistent schedule (stream-K): the work is the sequence of (row tile, K slice) units, tile-major;
// CTA b takes units [total*b/G, total*(b+1)/G).  With G <= ntiles every CTA covers at least one full
// tile's worth of slices, so a tile is shared by at most two CTAs; those add their partial sums
// into an output zeroed beforehand (two addends onto zero: the result does not depend on order).
template <int KER, int MD>
__global__ void __launch_bounds__(NTHREADS, 1)
k_gram_tc(const __grid_constant__ CUtensorMap tmapB, const TcParams P) {
  using M = Mode<MD>;
  extern __shared__ uint8_t smem_raw[];
  // 1024-byte aligned base for the swizzled tiles
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int S = P.stages;
  // per stage: A parts (NPART x A_TILE), then B parts (NPART x npad rows x ROWB bytes)
  uint8_t* A_base = smem;
  uint8_t* B_base = A_base + (size_t)S * M::NPART * M::A_TILE;
  uint8_t* C_base = B_base + (size_t)S * P.b_stage_bytes;            // coordinates
  uint8_t* W_base = C_base + (size_t)S * M::C_STAGE;                 // mean column
  uint64_t* bars = reinterpret_cast<uint64_t*>(W_base + (size_t)S * M::W_STAGE);
  uint64_t* fullA = bars;
  uint64_t* fullB = bars + S;
  uint64_t* fullC = bars + 2 * S;
  uint64_t* empty = bars + 3 * S;
  uint64_t* done = bars + 4 * S;           // MMA -> epilogue: a tile's accumulator is complete
  uint64_t* tfree = bars + 4 * S + 1;      // epilogue -> MMA: the accumulator has been read out
  uint64_t* fin = bars + 4 * S + 2;        // MMA issuer: all its MMAs have completed (exit)
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(bars + 4 * S + 3);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_holder + 1);
  float* mean_part = reinterpret_cast<float*>(tmem_holder + 4);     // [2][8][BM]

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long total = (long long)P.ntiles * P.nk;
  const long long u0 = total * blockIdx.x / gridDim.x;
  const long long u1 = total * (blockIdx.x + 1) / gridDim.x;

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(smem_u32(&fullA[s]), NPROD_WARPS);
      mbar_init(smem_u32(&fullB[s]), 1);
      mbar_init(smem_u32(&fullC[s]), 1);
      mbar_init(smem_u32(&empty[s]), 1);
    }
    mbar_init(smem_u32(done), 1);
    mbar_init(smem_u32(tfree), NPROD_WARPS);
    mbar_init(smem_u32(fin), 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 ::"r"(smem_u32(tmem_holder)), "r"(P.tmem_cols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_holder;

  if (warp < NPROD_WARPS) {
    // ------------------------------------------------------------ kernel-tile producers + epilogue
    // Producer role: warp w computes rows {rh*32 + lane, rh*32 + lane + 64} (rh = w & 1) for the
    // CPT-column group cg = w >> 1 of every slice, two columns at a time in packed f32x2
    // arithmetic.  Epilogue role: warp w reads TMEM lanes 32*(w & 3).. (the lane group it may
    // access) for the column chunks qt, qt + NQ, ... (qt = w >> 2).
    const int rh = warp & 1, cg = warp >> 1;
    const int lg = warp & 3;                        // TMEM lane group of this warp
    const int qt = warp >> 2;                       // which NQ-th of the 32-column epilogue chunks
    const int rl = lg * 32 + lane;                  // epilogue row within the tile (= TMEM lane)
    const int pr0 = rh * 32 + lane, pr1 = pr0 + 64; // producer rows within the tile
    long long u = u0;
    int tcount = 0;
    bool ok = true;
    while (u < u1) {
      const int tile = (int)(u / P.nk);
      const long long tbeg = (long long)tile * P.nk, tend = tbeg + P.nk;
      const long long uend = u1 < tend ? u1 : tend;
      const bool split = (u != tbeg) || (uend != tend);
      const int row = tile * BM + rl;
      uint64_t rx0, ry0, rz0, rx1, ry1, rz1;        // the two producer rows' coordinates, duplicated
      {
        C4<float> x0, x1;
        const int g0 = tile * BM + pr0, g1 = tile * BM + pr1;
        if (g0 < P.nr) x0 = P.Xr[g0]; else { x0.x = x0.y = x0.z = 1.0e6f; x0.w = 0.f; }
        if (g1 < P.nr) x1 = P.Xr[g1]; else { x1.x = x1.y = x1.z = 1.0e6f; x1.w = 0.f; }
        rx0 = f2_make(x0.x, x0.x); ry0 = f2_make(x0.y, x0.y); rz0 = f2_make(x0.z, x0.z);
        rx1 = f2_make(x1.x, x1.x); ry1 = f2_make(x1.y, x1.y); rz1 = f2_make(x1.z, x1.z);
      }
      uint64_t macc0 = 0ull, macc1 = 0ull;          // (even, odd column) partial means, FP32 pairs
      for (; u < uend; ++u) {
        const long long it = u - u0;
        const int s = (int)(it % S);
        const uint32_t n = (uint32_t)(it / S);
        // fullC completes only after the TMA warp saw empty[s] (the MMAs of this stage's previous
        // use are done) and its copies landed, so it also releases the A stage to the producers.
        ok = mbar_wait(smem_u32(&fullC[s]), n & 1, abort_flag, P.wait_limit);
        ok = __all_sync(0xffffffffu, ok);
        if (!ok) break;
        constexpr int NPAIR = M::CPT / 2;
        const uint8_t* cp = C_base + (size_t)s * M::C_STAGE + (size_t)cg * NPAIR * 32;
        const float* wc = reinterpret_cast<const float*>(W_base + (size_t)s * M::W_STAGE) + cg * M::CPT;
        // 16-bit modes: one packed word per column pair and part; TF32 modes: one word per column
        uint32_t pk0[2 * NPAIR], pk1[2 * NPAIR], pl0[2 * NPAIR], pl1[2 * NPAIR];
#pragma unroll
        for (int q = 0; q < NPAIR; ++q) {
          const ulonglong2 xy = *reinterpret_cast<const ulonglong2*>(cp + q * 32);
          const uint64_t cz = *reinterpret_cast<const uint64_t*>(cp + q * 32 + 16);
          const uint64_t w2 = *reinterpret_cast<const uint64_t*>(wc + 2 * q);
          const uint64_t k0 = kpair<KER>(rx0, ry0, rz0, xy.x, xy.y, cz);
          const uint64_t k1 = kpair<KER>(rx1, ry1, rz1, xy.x, xy.y, cz);
          macc0 = f2_fma(k0, w2, macc0);
          macc1 = f2_fma(k1, w2, macc1);
          if constexpr (M::TF32) {
            float a0, b0v, a1, b1v;
            f2_split(k0, a0, b0v);
            f2_split(k1, a1, b1v);
            pk0[2 * q] = tf32_rna(a0); pk0[2 * q + 1] = tf32_rna(b0v);
            pk1[2 * q] = tf32_rna(a1); pk1[2 * q + 1] = tf32_rna(b1v);
            if constexpr (M::SPLIT) {   // x - hi is exact in FP32; lo keeps its leading 11 bits
              pl0[2 * q] = tf32_rna(a0 - __uint_as_float(pk0[2 * q]));
              pl0[2 * q + 1] = tf32_rna(b0v - __uint_as_float(pk0[2 * q + 1]));
              pl1[2 * q] = tf32_rna(a1 - __uint_as_float(pk1[2 * q]));
              pl1[2 * q + 1] = tf32_rna(b1v - __uint_as_float(pk1[2 * q + 1]));
            }
          } else if constexpr (M::SPLIT) {
            pk0[q] = f2_f16(k0);
            pk1[q] = f2_f16(k1);
            pl0[q] = f2_f16(f2_sub(k0, f16x2_to_f2(pk0[q])));
            pl1[q] = f2_f16(f2_sub(k1, f16x2_to_f2(pk1[q])));
          } else {
            pk0[q] = f2_bf16(k0);
            pk1[q] = f2_bf16(k1);
          }
        }
        uint8_t* ast = A_base + (size_t)s * M::NPART * M::A_TILE;
        const int b0 = cg * M::CPT * M::ES;             // byte of this column group within a row
        const uint32_t o0 = sw_off<MD>(pr0, b0), o1 = sw_off<MD>(pr1, b0);
        if constexpr (M::SPLIT) {   // 8 bytes per row and part (4 fp16 or 2 tf32 values)
          *reinterpret_cast<uint2*>(ast + o0) = make_uint2(pk0[0], pk0[1]);
          *reinterpret_cast<uint2*>(ast + o1) = make_uint2(pk1[0], pk1[1]);
          *reinterpret_cast<uint2*>(ast + M::A_TILE + o0) = make_uint2(pl0[0], pl0[1]);
          *reinterpret_cast<uint2*>(ast + M::A_TILE + o1) = make_uint2(pl1[0], pl1[1]);
        } else {                    // 16 bytes per row (8 bf16 or 4 tf32 values)
          *reinterpret_cast<uint4*>(ast + o0) = make_uint4(pk0[0], pk0[1], pk0[2], pk0[3]);
          *reinterpret_cast<uint4*>(ast + o1) = make_uint4(pk1[0], pk1[1], pk1[2], pk1[3]);
        }
        fence_proxy_async();
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&fullA[s]));
      }
      // ---- end of this CTA's part of the tile: every producer warp arrives here, also on abort
      float* mp = mean_part + (tcount & 1) * (8 * BM);
      mp[cg * BM + pr0] = f2_sum(macc0);
      mp[cg * BM + pr1] = f2_sum(macc1);
      ok = producers_all(ok && !*abort_flag);
      if (!ok) break;
      if (qt == 0 && row < P.nr) {
        float m = mp[rl];
#pragma unroll
        for (int j = 1; j < 8; ++j) m += mp[j * BM + rl];
        m *= P.sf2;
        float* dst = P.Out + (size_t)P.wtc * P.ldo + row;
        if (split) atomicAdd(dst, m);
        else *dst = m;
      }
      ok = mbar_wait(smem_u32(done), tcount & 1, abort_flag, P.wait_limit);
      ok = __all_sync(0xffffffffu, ok);
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (ok) {
        const int nchunks = (P.npad + 31) / 32;   // TMEM holds >= 32 columns, so a 16-column tail is readable
        for (int ch = qt; ch < nchunks; ch += NQ) {
          uint32_t v[32];
          const uint32_t taddr = tmem + ((uint32_t)(lg * 32) << 16) + (uint32_t)(ch * 32);
          asm volatile(
              "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
              "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
              : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),
                "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]),
                "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
              : "r"(taddr)
              : "memory");
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
          if (row < P.nr) {
            float* o = P.Out + row;
#pragma unroll
            for (int j = 0; j < 32; ++j) {
              const int c = ch * 32 + j;
              if (c < P.wtc) {
                const float val = (M::SCALED ? P.sf2 * P.binv[c] : P.sf2) * __uint_as_float(v[j]);
                if (split) atomicAdd(o + (size_t)c * P.ldo, val);
                else o[(size_t)c * P.ldo] = val;
              }
            }
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(tfree));
      ++tcount;
      ok = producers_all(ok);
      if (!ok) break;
    }
  } else if (warp == TMA_WARP) {
    // ------------------------------------------------------------ TMA / bulk-copy producer
    if (lane == 0) {
      long long issued = 0;
      for (long long u = u0; u < u1; ++u) {
        const long long it = u - u0;
        const int s = (int)(it % S);
        const uint32_t n = (uint32_t)(it / S);
        const int kt = (int)(u % P.nk);
        if (!mbar_wait(smem_u32(&empty[s]), (n & 1) ^ 1, abort_flag, P.wait_limit)) break;
        const uint32_t cb = smem_u32(&fullC[s]);
        mbar_expect_tx(cb, M::C_STAGE + M::W_STAGE);
        bulk_load(smem_u32(C_base + (size_t)s * M::C_STAGE), P.Xc + (size_t)kt * M::BK, M::C_STAGE, cb);
        bulk_load(smem_u32(W_base + (size_t)s * M::W_STAGE), P.wcol + (size_t)kt * M::BK, M::W_STAGE, cb);
        const uint32_t bb = smem_u32(&fullB[s]);
        mbar_expect_tx(bb, P.b_stage_bytes);
        // B rows (operand columns) 0..npad-1 hold the hi part, npad..2 npad-1 the lo part
        for (int part = 0; part < M::NPART; ++part)
          for (int b = 0; b < P.nbox; ++b)
            tma_load_2d(smem_u32(B_base + (size_t)s * P.b_stage_bytes +
                                 ((size_t)part * P.npad + (size_t)b * P.boxh) * M::ROWB),
                        &tmapB, kt * M::BK, part * P.npad + b * P.boxh, bb);
        ++issued;
      }
      // on abort, let the copies possibly still in flight (the last S issued) land before exit
      if (*abort_flag) {
        for (long long it = issued > S ? issued - S : 0; it < issued; ++it) {
          const int s = (int)(it % S);
          const uint32_t par = (uint32_t)(it / S) & 1;
          mbar_drain(smem_u32(&fullB[s]), par);
          mbar_drain(smem_u32(&fullC[s]), par);
        }
      }
    }
  } else if (warp == MMA_WARP) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      bool ok = true;
      long long u = u0;
      int tcount = 0;
      while (u < u1 && ok) {
        const long long tend = (u / P.nk + 1) * P.nk;
        const long long uend = u1 < tend ? u1 : tend;
        if (tcount > 0) {   // the epilogue of the previous tile must have read the accumulator out
          ok = mbar_wait(smem_u32(tfree), (tcount - 1) & 1, abort_flag, P.wait_limit);
          if (!ok) break;
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        }
        bool first = true;
        for (; u < uend; ++u) {
          const long long it = u - u0;
          const int s = (int)(it % S);
          const uint32_t n = (uint32_t)(it / S);
          ok = mbar_wait(smem_u32(&fullA[s]), n & 1, abort_flag, P.wait_limit) && mbar_wait(smem_u32(&fullB[s]), n & 1, abort_flag, P.wait_limit);
          if (!ok) break;
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t a0 = smem_u32(A_base + (size_t)s * M::NPART * M::A_TILE);
          const uint32_t b0 = smem_u32(B_base + (size_t)s * P.b_stage_bytes);
          const uint32_t blo = (uint32_t)P.npad * M::ROWB;   // offset of the lo part of B
          for (int c0 = 0; c0 < P.npad; c0 += 256) {
            const int nn = min(256, P.npad - c0);
            const uint32_t id = idesc<MD>(nn);
            const uint32_t d = tmem + (uint32_t)c0;
#pragma unroll
            for (int kk = 0; kk < M::ROWB / 32; ++kk) {
              const uint64_t ah = sdesc<MD>(a0 + kk * 32);
              const uint64_t bh = sdesc<MD>(b0 + (uint32_t)c0 * M::ROWB + kk * 32);
              mma<MD>(d, ah, bh, id, (first && kk == 0) ? 0u : 1u);
              if constexpr (M::SPLIT) {
                mma<MD>(d, ah, sdesc<MD>(b0 + blo + (uint32_t)c0 * M::ROWB + kk * 32), id, 1u);
                mma<MD>(d, sdesc<MD>(a0 + M::A_TILE + kk * 32), bh, id, 1u);
              }
            }
          }
          first = false;
          mma_commit(smem_u32(&empty[s]));
        }
        if (!ok) break;
        mma_commit(smem_u32(done));
        ++tcount;
      }
      // every MMA issued above has completed before TMEM is released (also after an abort)
      mma_commit(smem_u32(fin));
      mbar_drain(smem_u32(fin), 0);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (*abort_flag && threadIdx.x == 0) atomicExch(P.err, kErrTimeout);
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(P.tmem_cols) : "memory");
  }
}

// ---------------------------------------------------------------------------- tall-skinny GEMM
// C (M x N) = alpha op(A) B + beta C for the factor products of the filter and smoother, on the
// tensor cores with split TF32 operands (MD_TF32X3: hi = tf32(x), lo = tf32(x - hi), three MMAs,
// about 22 significant bits per product, FP32 accumulation in TMEM).  op(A) = A (NN: A is M x K,
// column-major, M the long dimension) or A^T (TN: A is K x M, column-major, K the long dimension).
// B is K x N column-major.  The work is a list of units (128-row tile, N chunk <= 256 columns,
// K chunk); a persistent grid takes them round-robin.  Per K slice (16 values of K) the 16
// producer warps load the A and B tiles from global memory (coalesced), split them into hi / lo
// TF32 parts and write the swizzled K-major operand layout; one thread issues the MMAs; the
// producer warps drain TMEM.  A unit covering all of K writes alpha acc + beta C directly; with K
// split over chunks (and every TN product, whose output is FP64) each unit writes its FP32 partial
// tile and k_gemm_reduce sums the chunks in FP64.
struct GemmParams {
  const float* A;
  int lda, transA;
  const float* B;
  int ldb;
  int M, N, K;
  int ntiles, nchunks, cw, npad;   // row tiles, N chunks of cw columns (npad = cw rounded to 16)
  int nk, kslices, kchunks;        // K slices in all, per chunk, chunks
  int vecA, vecB;                  // 16-byte loads allowed along K
  float* C;
  int ldc;
  float alpha, beta;
  float* part;                     // non-null: part[(kc * N + col) * Mpad + row], else C directly
  int Mpad;
  int* err;
  int stages, tmem_cols;
  uint32_t b_stage_bytes;
  long long wait_limit;
  const uint8_t* Bpre;             // non-null: B already split and swizzled per (N chunk, K slice)
};

// Operand rows of B per producer thread and slice: a chunk has at most 256 columns (npad <= 256),
// 128 rows per pass of the 512 producer threads.
constexpr int GEMM_BROWS = 2;
constexpr int GEMM_PF = 3;   // slices of A in flight per producer thread
constexpr int GEMM_MAX_CHUNK = 128 * GEMM_BROWS;

// Global loads of one 16-wide K slice: A (128 rows) and B (npad operand rows) for this thread,
// zero outside the matrices.  Thread mapping: A of a TN product and B as (row tid / 4, quad tid % 4
// of 4 consecutive K values, one 16-byte load when aligned); A of an NN product as (row tid % 128,
// quad tid / 128), the lanes of a warp on consecutive rows.
__device__ __forceinline__ void load_slice(const GemmParams& P, int ks, int row0, int col0, int tid, float av[4],
                                           float bv[GEMM_BROWS][4], bool with_b, bool with_a = true) {
  const int k0 = ks * 16;
  if (!with_a) {
  } else if (P.transA) {
    const int r = tid >> 2, kq = tid & 3;
    const int row = row0 + r, k = k0 + kq * 4;
    const float* src = P.A + (size_t)row * P.lda + k;
    if (row < P.M && P.vecA && k + 3 < P.K) {
      const float4 q = *reinterpret_cast<const float4*>(src);
      av[0] = q.x; av[1] = q.y; av[2] = q.z; av[3] = q.w;
    } else {
#pragma unroll
      for (int e = 0; e < 4; ++e) av[e] = (row < P.M && k + e < P.K) ? src[e] : 0.f;
    }
  } else {
    const int r = tid & 127, kq = tid >> 7;
    const int row = row0 + r, k = k0 + kq * 4;
#pragma unroll
    for (int e = 0; e < 4; ++e) av[e] = (row < P.M && k + e < P.K) ? P.A[(size_t)(k + e) * P.lda + row] : 0.f;
  }
  if (!with_b) return;
#pragma unroll
  for (int b = 0; b < GEMM_BROWS; ++b) {
    const int jr = (tid >> 2) + 128 * b, kq = tid & 3, k = k0 + kq * 4;
    const int col = col0 + jr;
    const bool valid = jr < P.cw && col < P.N;
    const float* src = P.B + (size_t)col * P.ldb + k;
    if (valid && P.vecB && k + 3 < P.K) {
      const float4 q = *reinterpret_cast<const float4*>(src);
      bv[b][0] = q.x; bv[b][1] = q.y; bv[b][2] = q.z; bv[b][3] = q.w;
    } else {
#pragma unroll
      for (int e = 0; e < 4; ++e) bv[b][e] = (valid && k + e < P.K) ? src[e] : 0.f;
    }
  }
}

template <int MD>
__global__ void __launch_bounds__(NTHREADS, 1) k_gemm_tc(const GemmParams P) {
  using M = Mode<MD>;
  static_assert(M::BK == 16 && M::SPLIT && M::TF32, "the GEMM loaders assume 16-wide split-TF32 slices");
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int S = P.stages;
  uint8_t* A_base = smem;
  uint8_t* B_base = A_base + (size_t)S * M::NPART * M::A_TILE;
  uint64_t* bars = reinterpret_cast<uint64_t*>(B_base + (size_t)S * P.b_stage_bytes);
  uint64_t* fullA = bars;                  // producers -> MMA: the stage's A and B tiles are written
  uint64_t* empty = bars + S;              // MMA -> producers: the stage's MMAs are done
  uint64_t* done = bars + 2 * S;           // MMA -> epilogue: a unit's accumulator is complete
  uint64_t* tfree = bars + 2 * S + 1;      // epilogue -> MMA: the accumulator has been read out
  uint64_t* fin = bars + 2 * S + 2;        // MMA issuer: all its MMAs have completed (exit)
  uint64_t* fullB = bars + 2 * S + 3;      // bulk copy -> MMA: the stage's pre-split B slice landed
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(bars + 3 * S + 3);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_holder + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int units = P.ntiles * P.nchunks * P.kchunks;
  const bool preB = P.Bpre != nullptr;
  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(smem_u32(&fullA[s]), NPROD_WARPS);
      mbar_init(smem_u32(&empty[s]), 1);
      mbar_init(smem_u32(&fullB[s]), 1);
    }
    mbar_init(smem_u32(done), 1);
    mbar_init(smem_u32(tfree), NPROD_WARPS);
    mbar_init(smem_u32(fin), 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 ::"r"(smem_u32(tmem_holder)), "r"(P.tmem_cols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_holder;

  if (warp < NPROD_WARPS) {
    // ------------------------------------------------------------ operand producers + epilogue
    // With a pre-split B, thread 0 also copies each stage's B slice (one bulk copy onto fullB[s])
    // once the stage is free; the producers then load and split A only.
    const int tid = threadIdx.x;                    // 0 .. 511
    long long issued = 0;                           // B copies issued by thread 0
    const int lg = warp & 3, qt = warp >> 2;        // epilogue: TMEM lane group, column-chunk phase
    long long it = 0;                               // slices produced so far (stage counter)
    int tcount = 0;
    bool ok = true;
    for (int u = blockIdx.x; u < units && ok; u += gridDim.x) {
      const int t = u % P.ntiles;
      const int nc = (u / P.ntiles) % P.nchunks;
      const int kc = u / (P.ntiles * P.nchunks);
      const int row0 = t * BM, col0 = nc * P.cw;
      const int ks0 = kc * P.kslices, ks1 = min(P.nk, ks0 + P.kslices);
      // A is loaded GEMM_PF slices ahead (a ring of registers indexed statically: the loop over
      // the slices is unrolled GEMM_PF times), B one slice ahead when the producers split it, so
      // that the loads' latency overlaps the conversion, the stores and the waits for free stages
      float ar[GEMM_PF][4], bv[GEMM_BROWS][4];
      load_slice(P, ks0, row0, col0, tid, ar[0], bv, !preB);
#pragma unroll
      for (int q = 1; q < GEMM_PF; ++q)
        if (ks0 + q < ks1) load_slice(P, ks0 + q, row0, col0, tid, ar[q], bv, false);
      for (int kb = ks0; kb < ks1 && ok; kb += GEMM_PF) {
#pragma unroll
        for (int j = 0; j < GEMM_PF; ++j) {
          const int ks = kb + j;
          if (ks >= ks1) break;
          const int s = (int)(it % S);
          const uint32_t n = (uint32_t)(it / S);
          float bn[GEMM_BROWS][4];
          if (!preB && ks + 1 < ks1) load_slice(P, ks + 1, row0, col0, tid, ar[j], bn, true, false);
          ok = mbar_wait(smem_u32(&empty[s]), (n & 1) ^ 1, abort_flag, P.wait_limit);
          ok = __all_sync(0xffffffffu, ok);
          if (!ok) break;
          uint8_t* ast = A_base + (size_t)s * M::NPART * M::A_TILE;
          uint8_t* bst = B_base + (size_t)s * P.b_stage_bytes;
          if (preB && tid == 0) {
            mbar_expect_tx(smem_u32(&fullB[s]), P.b_stage_bytes);
            bulk_load(smem_u32(bst), P.Bpre + ((size_t)nc * P.nk + ks) * P.b_stage_bytes, P.b_stage_bytes,
                      smem_u32(&fullB[s]));
            ++issued;
          }
          {
            const int r = P.transA ? (tid >> 2) : (tid & 127);
            const int kq = P.transA ? (tid & 3) : (tid >> 7);
            uint32_t h[4], l[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) { h[e] = tf32_rna(ar[j][e]); l[e] = tf32_rna(ar[j][e] - __uint_as_float(h[e])); }
            const uint32_t o = sw_off<MD>(r, kq * 16);
            *reinterpret_cast<uint4*>(ast + o) = make_uint4(h[0], h[1], h[2], h[3]);
            *reinterpret_cast<uint4*>(ast + M::A_TILE + o) = make_uint4(l[0], l[1], l[2], l[3]);
          }
          if (ks + GEMM_PF < ks1) load_slice(P, ks + GEMM_PF, row0, col0, tid, ar[j], bn, false);
#pragma unroll
          for (int b = 0; b < GEMM_BROWS; ++b) {
            const int jr = (tid >> 2) + 128 * b;
            if (preB || jr >= P.npad) break;
            const int kq = tid & 3;
            uint32_t h[4], l[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) { h[e] = tf32_rna(bv[b][e]); l[e] = tf32_rna(bv[b][e] - __uint_as_float(h[e])); }
            const uint32_t o = sw_off<MD>(jr, kq * 16);
            *reinterpret_cast<uint4*>(bst + o) = make_uint4(h[0], h[1], h[2], h[3]);
            *reinterpret_cast<uint4*>(bst + (size_t)P.npad * M::ROWB + o) = make_uint4(l[0], l[1], l[2], l[3]);
          }
          if (!preB) {
#pragma unroll
            for (int b = 0; b < GEMM_BROWS; ++b)
#pragma unroll
              for (int e = 0; e < 4; ++e) bv[b][e] = bn[b][e];
          }
          fence_proxy_async();
          __syncwarp();
          if (lane == 0) mbar_arrive(smem_u32(&fullA[s]));
          ++it;
        }
      }
      ok = producers_all(ok && !*abort_flag);
      if (!ok) break;
      // ---- epilogue of the unit
      ok = mbar_wait(smem_u32(done), tcount & 1, abort_flag, P.wait_limit);
      ok = __all_sync(0xffffffffu, ok);
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (ok) {
        const int row = row0 + lg * 32 + lane;
        // TMEM is read 16 columns at a time; with beta != 0 the 16 matching C values are loaded
        // first, together, so they are in flight at once instead of one load per column
        const bool rdc = !P.part && P.beta != 0.f;
        const int nh = (P.npad + 15) / 16;
        for (int hc = qt; hc < nh; hc += NQ) {
          float cin[16];
          if (rdc && row < P.M) {
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              const int c = hc * 16 + j, col = col0 + c;
              cin[j] = (c < P.cw && col < P.N) ? P.C[(size_t)col * P.ldc + row] : 0.f;
            }
          }
          uint32_t v[16];
          const uint32_t taddr = tmem + ((uint32_t)(lg * 32) << 16) + (uint32_t)(hc * 16);
          asm volatile(
              "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
              : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                "=r"(v[15])
              : "r"(taddr)
              : "memory");
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
          if (row < P.M) {
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              const int c = hc * 16 + j;
              const int col = col0 + c;
              if (c < P.cw && col < P.N) {
                const float acc = __uint_as_float(v[j]);
                if (P.part) {
                  P.part[((size_t)kc * P.N + col) * P.Mpad + row] = acc;
                } else {
                  float* dst = P.C + (size_t)col * P.ldc + row;
                  *dst = rdc ? fmaf(P.alpha, acc, P.beta * cin[j]) : P.alpha * acc;
                }
              }
            }
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(tfree));
      ++tcount;
      ok = producers_all(ok);
    }
    if (preB && tid == 0) {
      // copy q went to stage q % S in phase q / S; after an abort the ones still in flight land
      // before the CTA exits (each has already completed in a run without abort)
      for (long long q = issued > S ? issued - S : 0; q < issued; ++q)
        mbar_drain(smem_u32(&fullB[(int)(q % S)]), (uint32_t)((q / S) & 1));
    }
  } else if (warp == MMA_WARP) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      bool ok = true;
      long long it = 0;
      int tcount = 0;
      for (int u = blockIdx.x; u < units && ok; u += gridDim.x) {
        const int kc = u / (P.ntiles * P.nchunks);
        const int ks0 = kc * P.kslices, ks1 = min(P.nk, ks0 + P.kslices);
        if (tcount > 0) {
          ok = mbar_wait(smem_u32(tfree), (tcount - 1) & 1, abort_flag, P.wait_limit);
          if (!ok) break;
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        }
        for (int ks = ks0; ks < ks1; ++ks, ++it) {
          const int s = (int)(it % S);
          const uint32_t n = (uint32_t)(it / S);
          ok = mbar_wait(smem_u32(&fullA[s]), n & 1, abort_flag, P.wait_limit);
          if (ok && preB) ok = mbar_wait(smem_u32(&fullB[s]), n & 1, abort_flag, P.wait_limit);
          if (!ok) break;
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t a0 = smem_u32(A_base + (size_t)s * M::NPART * M::A_TILE);
          const uint32_t b0 = smem_u32(B_base + (size_t)s * P.b_stage_bytes);
          const uint32_t blo = (uint32_t)P.npad * M::ROWB;
          for (int c0 = 0; c0 < P.npad; c0 += 256) {
            const int nn = min(256, P.npad - c0);
            const uint32_t id = idesc<MD>(nn);
            const uint32_t d = tmem + (uint32_t)c0;
#pragma unroll
            for (int kk = 0; kk < M::ROWB / 32; ++kk) {
              const uint64_t ah = sdesc<MD>(a0 + kk * 32);
              const uint64_t bh = sdesc<MD>(b0 + (uint32_t)c0 * M::ROWB + kk * 32);
              mma<MD>(d, ah, bh, id, (ks == ks0 && kk == 0) ? 0u : 1u);
              mma<MD>(d, ah, sdesc<MD>(b0 + blo + (uint32_t)c0 * M::ROWB + kk * 32), id, 1u);
              mma<MD>(d, sdesc<MD>(a0 + M::A_TILE + kk * 32), bh, id, 1u);
            }
          }
          mma_commit(smem_u32(&empty[s]));
        }
        if (!ok) break;
        mma_commit(smem_u32(done));
        ++tcount;
      }
      // every MMA issued above has completed before TMEM is released
      mma_commit(smem_u32(fin));
      mbar_drain(smem_u32(fin), 0);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (*abort_flag && threadIdx.x == 0) atomicExch(P.err, kErrTimeout);
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(P.tmem_cols) : "memory");
  }
}

// B of an NN product split into TF32 hi / lo parts once, in the swizzled stage layout k_gemm_tc's
// producers would write (same rounding, same zero padding): one b_stage_bytes block per (N chunk,
// K slice), hi part then lo part, so that the GEMM copies each stage's B with one bulk copy.
__global__ void __launch_bounds__(256)
k_gemm_prep_b(const float* __restrict__ B, int ldb, int K, int N, int cw, int npad, int nk, uint32_t b_stage_bytes,
              uint8_t* __restrict__ out) {
  using M = Mode<MD_TF32X3>;
  const int nc = blockIdx.x / nk, ks = blockIdx.x - nc * nk;
  uint8_t* bst = out + (size_t)blockIdx.x * b_stage_bytes;
  for (int idx = threadIdx.x; idx < npad * 4; idx += blockDim.x) {
    const int jr = idx >> 2, kq = idx & 3;
    const int col = nc * cw + jr, k = ks * 16 + kq * 4;
    const bool valid = jr < cw && col < N;
    uint32_t h[4], l[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const float b = (valid && k + e < K) ? B[(size_t)col * ldb + k + e] : 0.f;
      h[e] = tf32_rna(b);
      l[e] = tf32_rna(b - __uint_as_float(h[e]));
    }
    const uint32_t o = sw_off<MD_TF32X3>(jr, kq * 16);
    *reinterpret_cast<uint4*>(bst + o) = make_uint4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<uint4*>(bst + (size_t)npad * M::ROWB + o) = make_uint4(l[0], l[1], l[2], l[3]);
  }
}

// C[row + col * ldc] = alpha * sum_kc part[(kc * N + col) * Mpad + row] + beta * C  (FP64 sums)
template <class OutT>
__global__ void k_gemm_reduce(const float* __restrict__ part, int kchunks, int M, int N, int Mpad, double alpha,
                              double beta, OutT* __restrict__ C, int ldc) {
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  const int col = blockIdx.y;
  if (row >= M || col >= N) return;
  double acc = 0.0;
  for (int kc = 0; kc < kchunks; ++kc) acc += (double)part[((size_t)kc * N + col) * Mpad + row];
  OutT* c = C + (size_t)col * ldc + row;
  *c = OutT(alpha * acc + (beta != 0.0 ? beta * (double)*c : 0.0));
}

// ---------------------------------------------------------------------------- operand packing
// FP16 x3 mode: per column c < wtc of B, the power of two that brings max |B[:, c]| into [0.5, 1)
// (sc[c]) and its inverse (inv[c], applied in the epilogue).  One block per column.
__global__ void k_col_scale(const float* __restrict__ B, int ldb, int rows, int wtc, float* __restrict__ sc,
                            float* __restrict__ inv) {
  const int c = blockIdx.x;
  if (c >= wtc) return;
  float m = 0.f;
  for (int i = threadIdx.x; i < rows; i += blockDim.x) m = fmaxf(m, fabsf(B[(size_t)c * ldb + i]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  __shared__ float red[32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    m = red[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, red[w]);
    int e = 0;
    if (m > 0.f && isfinite(m)) frexpf(m, &e);     // m = f * 2^e, f in [0.5, 1)
    sc[c] = ldexpf(1.f, -e);
    inv[c] = ldexpf(1.f, e);
  }
}

// Bp (ld = ldp): rows 0..npad-1 hold the first wtc columns of B, zero-padded to ldp entries and
// npad rows, in the operand format of mode md: BF16; FP16 x3: hi = fp16(s_c B) with rows
// npad..2 npad-1 holding lo = fp16(s_c B - hi); TF32: tf32(B) in 4-byte words; TF32 x3: hi =
// tf32(B), lo = tf32(B - hi).  wp (fp32, ldp): column wtc of B (the mean column), zero-padded.
__global__ void k_pack_b(const float* __restrict__ B, int ldb, int rows, int wtc, int npad, int ldp, int md,
                         const float* __restrict__ sc, void* __restrict__ Bp, float* __restrict__ wp) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int c = blockIdx.y;
  if (i >= ldp) return;
  if (c < npad) {
    const float v = (c < wtc && i < rows) ? B[(size_t)c * ldb + i] : 0.f;
    if (md == MD_F16X3) {
      const float x = c < wtc ? v * sc[c] : 0.f;
      const __half hi = __float2half_rn(x);
      __half* h = reinterpret_cast<__half*>(Bp);
      h[(size_t)c * ldp + i] = hi;
      h[(size_t)(npad + c) * ldp + i] = __float2half_rn(x - __half2float(hi));
    } else if (md == MD_TF32 || md == MD_TF32X3) {
      uint32_t* w = reinterpret_cast<uint32_t*>(Bp);
      const uint32_t hi = tf32_rna(v);
      w[(size_t)c * ldp + i] = hi;
      if (md == MD_TF32X3) w[(size_t)(npad + c) * ldp + i] = tf32_rna(v - __uint_as_float(hi));
    } else {
      reinterpret_cast<__nv_bfloat16*>(Bp)[(size_t)c * ldp + i] = __float2bfloat16_rn(v);
    }
  } else {
    wp[i] = (i < rows) ? B[(size_t)wtc * ldb + i] : 0.f;
  }
}

// Xp holds the columns' coordinates in pairs: for columns 2p, 2p + 1 the 8 floats
// {x0, x1, y0, y1, z0, z1, 0, 0} (32 bytes), the layout the producers read as f32x2 operands.
__global__ void k_pad_coords(const C4<float>* __restrict__ X, int n, int ldp, float* __restrict__ Xp) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ldp) return;
  C4<float> c;
  if (i < n) c = X[i];
  else { c.x = c.y = c.z = 1.0e6f; c.w = 0.f; }
  float* o = Xp + (size_t)(i >> 1) * 8 + (i & 1);
  o[0] = c.x;
  o[2] = c.y;
  o[4] = c.z;
  o[6] = 0.f;
}

// ---------------------------------------------------------------------------- host side
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

inline int round_up(int x, int m) { return (x + m - 1) / m * m; }

// Multiprocessor count of the current device (cached per device).
int sm_count() {
  static int cache[128] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 128) return 1;
  if (!cache[dev]) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    cache[dev] = v > 0 ? v : 1;
  }
  return cache[dev];
}

struct Layout {
  int npad, nbox, boxh, stages, tmem_cols;
  uint32_t b_stage_bytes;
  size_t smem;
};

template <int MD>
Layout plan_layout(int wtc) {
  using M = Mode<MD>;
  Layout L;
  L.npad = std::max(16, round_up(wtc, 16));
  L.nbox = (L.npad + 255) / 256;           // npad <= 512: one or two boxes per part
  L.boxh = L.npad / L.nbox;                // a multiple of 8: boxes start on swizzle-atom boundaries
  L.b_stage_bytes = (uint32_t)(M::NPART * L.npad * M::ROWB);
  const size_t per_stage = (size_t)M::NPART * M::A_TILE + L.b_stage_bytes + M::C_STAGE + M::W_STAGE;
  const size_t fixed = 1024 /*alignment slack*/ + 64 * 8 + 64 + 2 * 8 * BM * 4;
  const size_t budget = 220 * 1024;
  L.stages = (int)std::min<size_t>(8, (budget - fixed) / per_stage);
  L.tmem_cols = 32;
  while (L.tmem_cols < L.npad) L.tmem_cols *= 2;
  L.smem = fixed + (size_t)L.stages * per_stage;
  // keep (CTAs per SM) x (TMEM columns) <= 512 by sizing shared memory
  const size_t smem_cap = 227 * 1024;
  const int max_ctas = 512 / L.tmem_cols;
  const size_t min_smem = max_ctas >= 6 ? 0 : smem_cap / (size_t)(max_ctas + 1) + 1024;
  L.smem = std::max(L.smem, min_smem);
  return L;
}

inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Staging layout: [B part(s), 2 bytes per element] [mean column, fp32] [coordinates, pair layout]
// [split mode: column scales sc and their inverses, fp32].
struct Staging {
  size_t wp, xc, sc, total;
};
Staging staging_layout(int rows, int width, int kind) {
  const size_t ldp = gram_tc_packed_ld(rows);
  const int wtc = std::max(width - 1, 1);
  const size_t npad = (size_t)std::max(16, round_up(wtc, 16));
  const size_t npart = (kind == MD_F16X3 || kind == MD_TF32X3) ? 2 : 1;
  const size_t es = (kind == MD_TF32 || kind == MD_TF32X3) ? 4 : 2;
  Staging g;
  g.wp = align256(npart * npad * ldp * es);
  g.xc = g.wp + align256(ldp * 4);
  g.sc = g.xc + align256(ldp * 16);
  g.total = g.sc + (kind == MD_F16X3 ? align256(2 * npad * 4) : 0) + 256;
  return g;
}

template <int MD>
const void* kernel_for(int ker) {
  return ker == 0 ? (const void*)k_gram_tc<0, MD>
                  : (ker == 1 ? (const void*)k_gram_tc<1, MD> : (const void*)k_gram_tc<2, MD>);
}

template <int MD>
int launch(int ker, const C4<float>* Xr, int nr, int nc, const void* Bp, int ldp, int width, float sf2, float* Out,
           int ldo, int* err, cudaStream_t st) {
  using M = Mode<MD>;
  auto encode = encode_fn();
  if (!encode) return 5;
  const int wtc = width - 1;
  const Layout L = plan_layout<MD>(wtc);
  const Staging g = staging_layout(nc, width, MD);
  const char* base = reinterpret_cast<const char*>(Bp);

  CUtensorMap map;
  cuuint64_t gdim[2] = {(cuuint64_t)ldp, (cuuint64_t)M::NPART * L.npad};
  cuuint64_t gstride[1] = {(cuuint64_t)ldp * M::ES};
  cuuint32_t box[2] = {(cuuint32_t)M::BK, (cuuint32_t)L.boxh};
  cuuint32_t estr[2] = {1, 1};
  const CUtensorMapDataType dt = M::TF32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                         : (MD == MD_F16X3 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                                           : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16);
  CUresult cr = encode(&map, dt, 2,
                       const_cast<void*>(Bp), gdim, gstride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                       M::SPLIT ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B,
                       CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (cr != CUDA_SUCCESS) return 6;

  TcParams P;
  P.Xr = Xr; P.nr = nr; P.Xc = reinterpret_cast<const C4<float>*>(base + g.xc);
  P.wcol = reinterpret_cast<const float*>(base + g.wp);
  P.binv = M::SCALED ? reinterpret_cast<const float*>(base + g.sc) + L.npad : nullptr;
  P.nk = ldp / M::BK; P.ntiles = (nr + BM - 1) / BM; P.npad = L.npad;
  P.nbox = L.nbox; P.boxh = L.boxh; P.wtc = wtc; P.sf2 = sf2; P.Out = Out; P.ldo = ldo; P.err = err;
  P.stages = L.stages; P.tmem_cols = L.tmem_cols; P.b_stage_bytes = L.b_stage_bytes;
  P.wait_limit = wait_limit(WAIT_LIMIT);

  const void* fn = kernel_for<MD>(ker);
  cudaError_t ce = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.smem);
  if (ce != cudaSuccess) return 8;
  int per_sm = 0;
  ce = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, NTHREADS, L.smem);
  if (ce != cudaSuccess || per_sm < 1) return 9;
  per_sm = std::min(per_sm, 512 / L.tmem_cols);   // every resident CTA holds tmem_cols TMEM columns
  const long long slots = (long long)sm_count() * per_sm;
  const int grid = (int)std::min<long long>(P.ntiles, slots);
  // tiles shared by two CTAs are accumulated with atomic adds onto zeros
  const long long total = (long long)P.ntiles * P.nk;
  bool split = false;
  for (int b = 1; b < grid && !split; ++b) split = (total * b / grid) % P.nk != 0;
  if (split) {
    ce = cudaMemset2DAsync(Out, (size_t)ldo * sizeof(float), 0, (size_t)nr * sizeof(float), (size_t)width, st);
    if (ce != cudaSuccess) return 10;
  }
  void* args[] = {&map, &P};
  ce = cudaLaunchKernel(fn, dim3(grid), dim3(NTHREADS), args, L.smem, st);
  note_launch();
  if (ce != cudaSuccess) { cudaGetLastError(); return 7; }
  return 0;
}

// Shared-memory bytes and stages of k_gemm_tc for a chunk of npad operand columns.
struct GemmLayout {
  int stages, tmem_cols;
  uint32_t b_stage_bytes;
  size_t smem;
};
GemmLayout gemm_layout(int npad) {
  using M = Mode<MD_TF32X3>;
  GemmLayout L;
  L.b_stage_bytes = (uint32_t)(M::NPART * npad * M::ROWB);
  const size_t per_stage = (size_t)M::NPART * M::A_TILE + L.b_stage_bytes;
  const size_t fixed = 1024 + 64 * 8 + 64;
  L.stages = (int)std::min<size_t>(6, (220 * 1024 - fixed) / per_stage);
  L.tmem_cols = 32;
  while (L.tmem_cols < npad) L.tmem_cols *= 2;
  L.smem = fixed + (size_t)L.stages * per_stage;
  const int max_ctas = 512 / L.tmem_cols;   // keep (CTAs per SM) x (TMEM columns) <= 512
  if (max_ctas < 6) L.smem = std::max(L.smem, (size_t)(227 * 1024) / (size_t)(max_ctas + 1) + 1024);
  return L;
}

// Launch k_gemm_tc; C_f32 receives alpha op(A) B + beta C directly when the K range is not split,
// otherwise part (part_floats capacity) takes the per-chunk partial sums and the caller reduces.
// Device scratch for the pre-split B of NN products (per host thread and current device, grown on
// demand; a few MB).
thread_local uint8_t* t_bpre = nullptr;
thread_local size_t t_bpre_bytes = 0;
thread_local int t_bpre_dev = -1;
uint8_t* bpre_scratch(size_t bytes) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return nullptr; }
  if (dev != t_bpre_dev) {            // a buffer of another device is not reachable from this one
    if (t_bpre) cudaFree(t_bpre);
    t_bpre = nullptr;
    t_bpre_bytes = 0;
    t_bpre_dev = dev;
  }
  if (bytes > t_bpre_bytes) {
    if (t_bpre) cudaFree(t_bpre);
    t_bpre = nullptr;
    t_bpre_bytes = 0;
    if (cudaMalloc(&t_bpre, bytes) != cudaSuccess) { cudaGetLastError(); return nullptr; }
    t_bpre_bytes = bytes;
  }
  return t_bpre;
}

int gemm_tc_launch(int transA, int Mr, int N, int K, float alpha, const float* A, int lda, const float* B, int ldb,
                   float beta, float* C_f32, int ldc, bool force_split, float* part, size_t part_floats,
                   int* kchunks_out, int* Mpad_out, int* err, cudaStream_t st) {
  using M = Mode<MD_TF32X3>;
  GemmParams P{};
  P.A = A; P.lda = lda; P.transA = transA; P.B = B; P.ldb = ldb; P.M = Mr; P.N = N; P.K = K;
  P.ntiles = (Mr + BM - 1) / BM;
  P.nchunks = (N + GEMM_MAX_CHUNK - 1) / GEMM_MAX_CHUNK;
  P.cw = (N + P.nchunks - 1) / P.nchunks;
  P.npad = round_up(P.cw, 16);
  P.nk = (K + M::BK - 1) / M::BK;
  P.Mpad = P.ntiles * BM;
  const GemmLayout L = gemm_layout(P.npad);
  const void* fn = (const void*)k_gemm_tc<MD_TF32X3>;
  cudaError_t ce = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.smem);
  if (ce != cudaSuccess) return 8;
  int per_sm = 0;
  ce = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, NTHREADS, L.smem);
  if (ce != cudaSuccess || per_sm < 1) return 9;
  per_sm = std::min(per_sm, 512 / L.tmem_cols);
  const int slots = sm_count() * per_sm;
  // split K when the row tiles alone cannot fill the GPU (long K, short M: the TN products)
  int kchunks = 1;
  const int base_units = P.ntiles * P.nchunks;
  if (force_split || base_units < slots) {
    const size_t per_chunk = (size_t)N * P.Mpad;
    const int cap = part ? (int)std::min<size_t>(4096, part_floats / std::max<size_t>(per_chunk, 1)) : 1;
    // enough chunks to fill the GPU, and at most 64 slices (1,024 K values) per chunk so that the
    // FP32 accumulation chains in TMEM stay short; the chunks are summed in FP64
    const int want = std::max((slots + base_units - 1) / base_units, (P.nk + 63) / 64);
    kchunks = std::max(1, std::min({want, cap, std::max(1, P.nk / 4)}));
    if (force_split && cap < 1) return 11;
  }
  P.kslices = (P.nk + kchunks - 1) / kchunks;
  P.kchunks = (P.nk + P.kslices - 1) / P.kslices;
  const bool split = force_split || P.kchunks > 1;
  if (split && !part) return 11;
  P.vecA = transA && lda % 4 == 0 && (reinterpret_cast<uintptr_t>(A) & 15) == 0;
  P.vecB = ldb % 4 == 0 && (reinterpret_cast<uintptr_t>(B) & 15) == 0;
  P.C = C_f32; P.ldc = ldc; P.alpha = alpha; P.beta = beta;
  P.part = split ? part : nullptr;
  P.err = err;
  P.stages = L.stages; P.tmem_cols = L.tmem_cols; P.b_stage_bytes = L.b_stage_bytes;
  P.wait_limit = wait_limit(WAIT_LIMIT);
  P.Bpre = nullptr;
  if (!transA && P.ntiles >= 64) {
    // B (K x N, small) is read by every row tile: split it once and copy it per stage in bulk
    const size_t bytes = (size_t)P.nchunks * P.nk * P.b_stage_bytes;
    if (uint8_t* bp = bpre_scratch(bytes)) {
      k_gemm_prep_b<<<P.nchunks * P.nk, 256, 0, st>>>(B, ldb, K, N, P.cw, P.npad, P.nk, P.b_stage_bytes, bp);
      note_launch();
      P.Bpre = bp;
    }
  }
  const int units = P.ntiles * P.nchunks * P.kchunks;
  const int grid = std::min(units, slots);
  void* args[] = {&P};
  ce = cudaLaunchKernel(fn, dim3(grid), dim3(NTHREADS), args, L.smem, st);
  note_launch();
  if (ce != cudaSuccess) { cudaGetLastError(); return 7; }
  *kchunks_out = P.kchunks;
  *Mpad_out = P.Mpad;
  return 0;
}

}  // namespace

int gemm_tc_nn(int M_, int N, int K, float alpha, const float* A, int lda, const float* B, int ldb, float beta,
               float* C, int ldc, int* err, cudaStream_t st) {
  if (M_ <= 0 || N <= 0 || K <= 0) return 3;
  int kc = 0, mp = 0;
  return gemm_tc_launch(0, M_, N, K, alpha, A, lda, B, ldb, beta, C, ldc, false, nullptr, 0, &kc, &mp, err, st);
}

int gemm_tc_tn(const float* A, int lda, int na, const float* B, int ldb, int nb, int K, double alpha, double beta,
               double* C, int ldc, void* part, size_t part_bytes, int* err, cudaStream_t st) {
  if (na <= 0 || nb <= 0 || K <= 0) return 3;
  int kc = 0, mp = 0;
  int rc = gemm_tc_launch(1, na, nb, K, 1.f, A, lda, B, ldb, 0.f, nullptr, 0, true, reinterpret_cast<float*>(part),
                          part_bytes / sizeof(float), &kc, &mp, err, st);
  if (rc) return rc;
  dim3 grid((na + 255) / 256, nb);
  k_gemm_reduce<double><<<grid, 256, 0, st>>>(reinterpret_cast<const float*>(part), kc, na, nb, mp, alpha, beta, C, ldc);
  note_launch();
  return cudaGetLastError() == cudaSuccess ? 0 : 1;
}

size_t gram_tc_packed_ld(int rows) { return (size_t)round_up(std::max(rows, 1), BK_MAX); }
int gram_tc_max_width() { return 513; }
size_t gram_tc_staging_bytes(int rows, int width, int kind) { return staging_layout(rows, width, kind).total; }

int gram_tc_pack_b(int kind, const float* B, int ldb, int rows, int cols, void* Bp, int ldp, cudaStream_t st) {
  if (kind < MD_BF16 || kind > MD_TF32X3) return 2;
  const int wtc = cols - 1;
  const int npad = std::max(16, round_up(std::max(wtc, 1), 16));
  const Staging g = staging_layout(rows, cols, kind);
  char* base = reinterpret_cast<char*>(Bp);
  float* wp = reinterpret_cast<float*>(base + g.wp);
  float* sc = kind == MD_F16X3 ? reinterpret_cast<float*>(base + g.sc) : nullptr;
  if (kind == MD_F16X3 && wtc > 0) {
    k_col_scale<<<wtc, 256, 0, st>>>(B, ldb, rows, wtc, sc, sc + npad);
    note_launch();
  }
  dim3 grid((ldp + 255) / 256, npad + 1);
  k_pack_b<<<grid, 256, 0, st>>>(B, ldb, rows, wtc, npad, ldp, kind, sc, Bp, wp);
  note_launch();
  return cudaGetLastError() == cudaSuccess ? 0 : 1;
}

int gram_block_tc(int ker, int kind, const C4<float>* Xr, int nr, const C4<float>* Xc, int nc, const void* Bp, int ldp,
                  int width, float sf2, float* Out, int ldo, int* err, cudaStream_t st) {
  if (kind < MD_BF16 || kind > MD_TF32X3) return 2;
  if (width < 2 || width > gram_tc_max_width() || nr <= 0 || nc <= 0) return 3;
  if (ldp % BK_MAX != 0 || ldp < nc) return 4;
  const Staging g = staging_layout(nc, width, kind);
  float* xcp = reinterpret_cast<float*>(reinterpret_cast<char*>(const_cast<void*>(Bp)) + g.xc);
  k_pad_coords<<<(ldp + 255) / 256, 256, 0, st>>>(Xc, nc, ldp, xcp);
  note_launch();
  switch (kind) {
    case MD_F16X3: return launch<MD_F16X3>(ker, Xr, nr, nc, Bp, ldp, width, sf2, Out, ldo, err, st);
    case MD_TF32: return launch<MD_TF32>(ker, Xr, nr, nc, Bp, ldp, width, sf2, Out, ldo, err, st);
    case MD_TF32X3: return launch<MD_TF32X3>(ker, Xr, nr, nc, Bp, ldp, width, sf2, Out, ldo, err, st);
    default: return launch<MD_BF16>(ker, Xr, nr, nc, Bp, ldp, width, sf2, Out, ldo, err, st);
  }
}

}  // namespace cakf
