// Tensor-core Gram x block product for sm_103a (tcgen05 + TMEM + TMA), the hot kernel of the CAKF / CAKS:
//
//   Out[i, c] = sum_j k(xr_i, xc_j) B[j, c]         (Out, B column-major; k a Matern kernel)
//
// The kernel matrix is never stored: each CTA owns 128 output rows and walks the columns j in
// slices of 64.  Per slice, 8 producer warps evaluate the 128 x 64 kernel tile from coordinates
// staged in shared memory and write it as BF16 in the 128-byte-swizzled K-major layout that the
// tensor core reads; a TMA warp stages the matching 64 x N slice of the packed B operand; a single
// thread issues tcgen05.mma (M = 128, N <= 256 per instruction, K = 16) accumulating in TMEM
// (up to 512 FP32 columns).  The last column of B (the mean vector of the filter / smoother) is
// not sent to the tensor core: the producers accumulate it in FP32 from the same kernel values.
// Every mbarrier wait is bounded; on timeout the CTA raises the error flag and stops.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <mutex>
#include <map>
#include "internal.h"

namespace cakf {
namespace {

constexpr int BM = 128;          // rows per CTA (TMEM lanes)
constexpr int BK = 64;           // kernel columns per pipeline stage (64 bf16 = one 128B swizzle row)
constexpr int NPROD_WARPS = 16;  // kernel-tile producers (and epilogue)
constexpr int NQ = NPROD_WARPS / 4;   // producer warps per TMEM lane group: each takes BK / NQ columns
constexpr int TMA_WARP = NPROD_WARPS;
constexpr int MMA_WARP = NPROD_WARPS + 1;   // the remaining warp issues the MMAs
constexpr int NTHREADS = (NPROD_WARPS + 2) * 32;
constexpr int A_STAGE_BYTES = BM * BK * 2;   // 16 KB
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
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag) {
  for (long long it = 0; it < WAIT_LIMIT; ++it) {
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

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;                 // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;       // stride byte offset
  d |= (uint64_t)1 << 46;                 // descriptor version
  d |= (uint64_t)2 << 61;                 // 128-byte swizzle
  return d;
}

// Instruction descriptor, kind::f16: BF16 A/B (K-major), FP32 accumulator, M = 128.
__host__ __device__ constexpr uint32_t idesc_bf16(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
      ::"r"(d_tmem), "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
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
__device__ __forceinline__ uint32_t f2_bf16(uint64_t v) {
  float lo, hi;
  f2_split(v, lo, hi);
  return pack_bf16(lo, hi);
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

struct TcParams {
  const C4<float>* Xr;
  int nr;
  const C4<float>* Xc;     // nk * BK columns in pair layout (see k_pad_coords), sentinels beyond nc
  const float* wcol;       // padded mean column (zeros beyond nc), FP32
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
template <int KER>
__global__ void __launch_bounds__(NTHREADS, 1)
k_gram_tc(const __grid_constant__ CUtensorMap tmapB, const TcParams P) {
  extern __shared__ uint8_t smem_raw[];
  // 1024-byte aligned base for the swizzled tiles
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int S = P.stages;
  uint8_t* A_base = smem;
  uint8_t* B_base = A_base + (size_t)S * A_STAGE_BYTES;
  uint8_t* C_base = B_base + (size_t)S * P.b_stage_bytes;            // coordinates, 1 KB per stage
  uint8_t* W_base = C_base + (size_t)S * (BK * 16);                  // mean column, 256 B per stage
  uint64_t* bars = reinterpret_cast<uint64_t*>(W_base + (size_t)S * (BK * 4));
  uint64_t* fullA = bars;
  uint64_t* fullB = bars + S;
  uint64_t* fullC = bars + 2 * S;
  uint64_t* empty = bars + 3 * S;
  uint64_t* done = bars + 4 * S;           // MMA -> epilogue: a tile's accumulator is complete
  uint64_t* tfree = bars + 4 * S + 1;      // epilogue -> MMA: the accumulator has been read out
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(bars + 4 * S + 2);
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
    // 8-column chunk c8 = w >> 1 of every slice, two columns at a time in packed f32x2 arithmetic.
    // Epilogue role: warp w reads TMEM lanes 32*(w & 3).. (the lane group it may access) for the
    // column chunks qt, qt + NQ, ... (qt = w >> 2).
    const int rh = warp & 1, c8 = warp >> 1;
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
        ok = mbar_wait(smem_u32(&fullC[s]), n & 1, abort_flag);
        ok = __all_sync(0xffffffffu, ok);
        if (!ok) break;
        const uint8_t* cp = C_base + (size_t)s * BK * 16 + (size_t)c8 * 4 * 32;   // 4 column pairs
        const float* wc = reinterpret_cast<const float*>(W_base + (size_t)s * BK * 4) + c8 * 8;
        uint32_t pk0[4], pk1[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const ulonglong2 xy = *reinterpret_cast<const ulonglong2*>(cp + q * 32);
          const uint64_t cz = *reinterpret_cast<const uint64_t*>(cp + q * 32 + 16);
          const uint64_t w2 = *reinterpret_cast<const uint64_t*>(wc + 2 * q);
          const uint64_t k0 = kpair<KER>(rx0, ry0, rz0, xy.x, xy.y, cz);
          const uint64_t k1 = kpair<KER>(rx1, ry1, rz1, xy.x, xy.y, cz);
          macc0 = f2_fma(k0, w2, macc0);
          macc1 = f2_fma(k1, w2, macc1);
          pk0[q] = f2_bf16(k0);
          pk1[q] = f2_bf16(k1);
        }
        uint8_t* ast = A_base + (size_t)s * A_STAGE_BYTES;
        const int chunk = c8 ^ (pr0 & 7);           // pr1 = pr0 + 64 has the same swizzle phase
        *reinterpret_cast<uint4*>(ast + pr0 * 128 + chunk * 16) = make_uint4(pk0[0], pk0[1], pk0[2], pk0[3]);
        *reinterpret_cast<uint4*>(ast + pr1 * 128 + chunk * 16) = make_uint4(pk1[0], pk1[1], pk1[2], pk1[3]);
        fence_proxy_async();
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&fullA[s]));
      }
      // ---- end of this CTA's part of the tile: every producer warp arrives here, also on abort
      float* mp = mean_part + (tcount & 1) * (8 * BM);
      mp[c8 * BM + pr0] = f2_sum(macc0);
      mp[c8 * BM + pr1] = f2_sum(macc1);
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
      ok = mbar_wait(smem_u32(done), tcount & 1, abort_flag);
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
                const float val = P.sf2 * __uint_as_float(v[j]);
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
        if (!mbar_wait(smem_u32(&empty[s]), (n & 1) ^ 1, abort_flag)) break;
        const uint32_t cb = smem_u32(&fullC[s]);
        mbar_expect_tx(cb, BK * 16 + BK * 4);
        bulk_load(smem_u32(C_base + (size_t)s * BK * 16), P.Xc + (size_t)kt * BK, BK * 16, cb);
        bulk_load(smem_u32(W_base + (size_t)s * BK * 4), P.wcol + (size_t)kt * BK, BK * 4, cb);
        const uint32_t bb = smem_u32(&fullB[s]);
        mbar_expect_tx(bb, P.b_stage_bytes);
        for (int b = 0; b < P.nbox; ++b)
          tma_load_2d(smem_u32(B_base + (size_t)s * P.b_stage_bytes + (size_t)b * P.boxh * 128), &tmapB, kt * BK,
                      b * P.boxh, bb);
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
          ok = mbar_wait(smem_u32(tfree), (tcount - 1) & 1, abort_flag);
          if (!ok) break;
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        }
        bool first = true;
        for (; u < uend; ++u) {
          const long long it = u - u0;
          const int s = (int)(it % S);
          const uint32_t n = (uint32_t)(it / S);
          ok = mbar_wait(smem_u32(&fullA[s]), n & 1, abort_flag) && mbar_wait(smem_u32(&fullB[s]), n & 1, abort_flag);
          if (!ok) break;
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t a0 = smem_u32(A_base + (size_t)s * A_STAGE_BYTES);
          const uint32_t b0 = smem_u32(B_base + (size_t)s * P.b_stage_bytes);
          for (int c0 = 0; c0 < P.npad; c0 += 256) {
            const int nn = min(256, P.npad - c0);
            const uint32_t idesc = idesc_bf16(nn);
#pragma unroll
            for (int kk = 0; kk < BK / 16; ++kk) {
              const uint64_t ad = sdesc_sw128(a0 + kk * 32);
              const uint64_t bd = sdesc_sw128(b0 + (uint32_t)c0 * 128 + kk * 32);
              mma_bf16(tmem + (uint32_t)c0, ad, bd, idesc, (first && kk == 0) ? 0u : 1u);
            }
          }
          first = false;
          mma_commit(smem_u32(&empty[s]));
        }
        if (!ok) break;
        mma_commit(smem_u32(done));
        ++tcount;
      }
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

// ---------------------------------------------------------------------------- operand packing
// Bp (bf16, column-major, ld = ldp): the first wtc columns of B, zero-padded to ldp rows and npad
// columns.  wp (fp32, ldp): column wtc of B (the mean column), zero-padded.  Xp: coordinates padded
// with far-away sentinels (kernel value 0).
__global__ void k_pack_b(const float* __restrict__ B, int ldb, int rows, int wtc, int npad, int ldp,
                         __nv_bfloat16* __restrict__ Bp, float* __restrict__ wp) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int c = blockIdx.y;
  if (i >= ldp) return;
  if (c < npad) {
    float v = (c < wtc && i < rows) ? B[(size_t)c * ldb + i] : 0.f;
    Bp[(size_t)c * ldp + i] = __float2bfloat16_rn(v);
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

Layout plan_layout(int wtc) {
  Layout L;
  L.npad = std::max(16, round_up(wtc, 16));
  L.boxh = L.npad <= 256 ? L.npad : 256;
  L.nbox = (L.npad + L.boxh - 1) / L.boxh;
  L.b_stage_bytes = (uint32_t)L.nbox * L.boxh * 128;
  const size_t per_stage = A_STAGE_BYTES + L.b_stage_bytes + BK * 16 + BK * 4;
  const size_t fixed = 1024 /*alignment slack*/ + 64 * 8 + 64 + 2 * 8 * BM * 4;
  const size_t budget = 220 * 1024;
  L.stages = (int)std::min<size_t>(4, (budget - fixed) / per_stage);
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

}  // namespace

size_t gram_tc_packed_ld(int rows) { return (size_t)round_up(std::max(rows, 1), BK); }
int gram_tc_max_width() { return 513; }

// Bytes of packed staging for a (rows x width) block: bf16 operand + fp32 mean column + padded coords.
static size_t packed_bytes(int rows, int width) {
  const size_t ldp = gram_tc_packed_ld(rows);
  const int wtc = std::max(width - 1, 1);
  const size_t npad = (size_t)std::max(16, round_up(wtc, 16));
  return ((npad * ldp * 2 + 255) & ~size_t(255)) + ((ldp * 4 + 255) & ~size_t(255)) + ldp * 16 + 256;
}

int gram_tc_pack_b(int kind, const float* B, int ldb, int rows, int cols, void* Bp, int ldp, cudaStream_t st) {
  (void)kind;
  const int wtc = cols - 1;
  const int npad = std::max(16, round_up(std::max(wtc, 1), 16));
  __nv_bfloat16* bp = reinterpret_cast<__nv_bfloat16*>(Bp);
  float* wp = reinterpret_cast<float*>(reinterpret_cast<char*>(Bp) + (((size_t)npad * ldp * 2 + 255) & ~size_t(255)));
  dim3 grid((ldp + 255) / 256, npad + 1);
  k_pack_b<<<grid, 256, 0, st>>>(B, ldb, rows, wtc, npad, ldp, bp, wp);
  note_launch();
  return cudaGetLastError() == cudaSuccess ? 0 : 1;
}

int gram_block_tc(int ker, int kind, const C4<float>* Xr, int nr, const C4<float>* Xc, int nc, const void* Bp, int ldp,
                  int width, float sf2, float* Out, int ldo, int* err, cudaStream_t st) {
  if (kind != 0) return 2;                 // bf16 only in this kernel
  if (width < 2 || width > gram_tc_max_width() || nr <= 0 || nc <= 0) return 3;
  if (ldp % BK != 0 || ldp < nc) return 4;
  auto encode = encode_fn();
  if (!encode) return 5;
  const int wtc = width - 1;
  const Layout L = plan_layout(wtc);
  const char* base = reinterpret_cast<const char*>(Bp);
  const size_t boff = (((size_t)L.npad * ldp * 2 + 255) & ~size_t(255));
  const float* wp = reinterpret_cast<const float*>(base + boff);
  C4<float>* xcp = reinterpret_cast<C4<float>*>(const_cast<char*>(base) + boff + (((size_t)ldp * 4 + 255) & ~size_t(255)));
  k_pad_coords<<<(ldp + 255) / 256, 256, 0, st>>>(Xc, nc, ldp, reinterpret_cast<float*>(xcp));
  note_launch();

  CUtensorMap map;
  cuuint64_t gdim[2] = {(cuuint64_t)ldp, (cuuint64_t)L.npad};
  cuuint64_t gstride[1] = {(cuuint64_t)ldp * 2};
  cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)L.boxh};
  cuuint32_t estr[2] = {1, 1};
  CUresult cr = encode(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(Bp), gdim, gstride, box, estr,
                       CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                       CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (cr != CUDA_SUCCESS) return 6;

  TcParams P;
  P.Xr = Xr; P.nr = nr; P.Xc = xcp; P.wcol = wp; P.nk = ldp / BK; P.ntiles = (nr + BM - 1) / BM; P.npad = L.npad;
  P.nbox = L.nbox; P.boxh = L.boxh; P.wtc = wtc; P.sf2 = sf2; P.Out = Out; P.ldo = ldo; P.err = err;
  P.stages = L.stages; P.tmem_cols = L.tmem_cols; P.b_stage_bytes = L.b_stage_bytes;

  const void* fn = ker == 0 ? (const void*)k_gram_tc<0> : (ker == 1 ? (const void*)k_gram_tc<1> : (const void*)k_gram_tc<2>);
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
  switch (ker) {
    case 0: k_gram_tc<0><<<grid, NTHREADS, L.smem, st>>>(map, P); break;
    case 1: k_gram_tc<1><<<grid, NTHREADS, L.smem, st>>>(map, P); break;
    default: k_gram_tc<2><<<grid, NTHREADS, L.smem, st>>>(map, P); break;
  }
  note_launch();
  ce = cudaGetLastError();
  return ce == cudaSuccess ? 0 : 7;
}

size_t gram_tc_staging_bytes(int rows, int width) { return packed_bytes(rows, width); }

}  // namespace cakf
