// SIMT kernels of the CAKF/CAKS hot path (FP32 and FP64 instantiations):
//   - Gram matvec of the CG loop:  part[p][i] = sum_{j in split p} k(xo_i, xo_j) s_j
//   - Gram x block (plain SIMT path): Out = K(Xr, Xc) B, evaluated tile by tile, never stored
//   - tall-skinny GEMMs (split-K transposed products, tiled NN products)
//   - the CG / Gram-Schmidt bookkeeping of the iterative update step
//   - gathers, scatters and row epilogues of the filter and smoother.
#include "common.cuh"
#include <cuda_bf16.h>
#include "internal.h"

#include <atomic>

namespace cakf {

static std::atomic<long long> g_launches{0};
static thread_local int t_gemm_mode = 0;
static thread_local int* t_gemm_err = nullptr;
void set_gemm_mode(int mode) { t_gemm_mode = mode; }
int gemm_mode() { return t_gemm_mode; }
void set_gemm_err(int* err) { t_gemm_err = err; }

// Iteration limits of the bounded device-side waits (0 = the defaults of each kernel); a
// diagnostic setting for tests of the timeout path.
static std::atomic<long long> g_wait_limit{0};
void set_wait_limit(long long it) { g_wait_limit.store(it < 0 ? 0 : it); }
long long wait_limit(long long dflt) {
  const long long v = g_wait_limit.load();
  return v > 0 ? v : dflt;
}
long long launch_count() { return g_launches.load(); }
void note_launch(long long k) { g_launches += k; }

// ------------------------------------------------------------------------------------------
// Coordinates
template <class T>
__global__ void k_prep_coords(const double* __restrict__ X, int n, int dim, double scale,
                              C4<T>* __restrict__ out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  C4<T> c;
  c.x = T(scale * X[(size_t)i * dim + 0]);
  c.y = dim > 1 ? T(scale * X[(size_t)i * dim + 1]) : T(0);
  c.z = dim > 2 ? T(scale * X[(size_t)i * dim + 2]) : T(0);
  c.w = T(0);
  out[i] = c;
}

template <class T>
__global__ void k_gather_coords(const C4<T>* __restrict__ X, const int* __restrict__ idx, int m,
                                C4<T>* __restrict__ out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m) out[i] = X[idx[i]];
}

// ------------------------------------------------------------------------------------------
// CG Gram matvec, split over columns; part is [nsplit][m].
// K(X_o, X_o) s for the CG actions, each kernel value evaluated once: the symmetric Gram is cut into
// MVS_T x MVS_T tiles and one block evaluates tile (I, J), I <= J.  Row sums (weights s_J) give tile
// I's share from J and, for I < J, column sums (weights s_I) give tile J's share from I.  The
// shares land in distinct slots -- part[J][rows of I] and part[I][rows of J] -- so every row has
// exactly nb = ceil(m / MVS_T) slots, each written once, summed in a fixed order by k_cg_combine.
// A lane owns MVS_R rows of the tile; each warp takes 32 of its columns (staged in shared memory)
// and reduces a column's MVS_R * 32 products with one warp sum.
// The first ngv blocks instead form the partials of t = Mo^T s (one warp per column of Mo and
// chunk of GV_CHUNK rows), which k_cg_combine needs next: one launch for both.
constexpr int MVS_T = 128, MVS_R = MVS_T / 32, MVS_W = MVS_T / 32;
constexpr int GV_CHUNK = 1024;
template <int KER, class T>
__global__ void __launch_bounds__(MVS_W * 32)
k_gram_matvec(const C4<T>* __restrict__ Xo, const T* __restrict__ s, int m, int nb, T sf2, T* __restrict__ part,
              const T* __restrict__ Mo, int ldm, int rp, int ngv, T* __restrict__ tpart,
              const int* __restrict__ active) {
  pdl_wait();
  pdl_trigger();
  if (active && !*active) return;
  __shared__ C4<T> xs[MVS_T];
  __shared__ T ss[MVS_T];
  __shared__ T racc[MVS_W][MVS_T];
  if ((int)blockIdx.x < ngv) {
    const int per_chunk = (rp + MVS_W - 1) / MVS_W;
    const int z = blockIdx.x / per_chunk;
    const int col = (blockIdx.x - z * per_chunk) * MVS_W + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (col >= rp) return;
    const int i0 = z * GV_CHUNK, i1 = min(m, i0 + GV_CHUNK);
    const T* a = Mo + (size_t)col * ldm;
    T acc = T(0);
#pragma unroll 8
    for (int i = i0 + lane; i < i1; i += 32) acc = fma(a[i], s[i], acc);
    acc = warp_sum(acc);
    if (lane == 0) tpart[(size_t)z * rp + col] = acc;
    return;
  }
  int idx = blockIdx.x - ngv, I = 0;
  while (idx >= nb - I) { idx -= nb - I; ++I; }
  const int J = I + idx;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int t = threadIdx.x; t < MVS_T; t += blockDim.x) {
    const int j = J * MVS_T + t;
    C4<T> x;
    x.x = x.y = x.z = x.w = T(0);
    T v = T(0);
    if (j < m) { x = Xo[j]; v = s[j]; }
    xs[t] = x;
    ss[t] = v;
  }
  C4<T> xi[MVS_R];
  T si[MVS_R], acc[MVS_R];
#pragma unroll
  for (int r = 0; r < MVS_R; ++r) {
    const int i = I * MVS_T + lane + 32 * r;
    xi[r].x = xi[r].y = xi[r].z = xi[r].w = T(0);
    si[r] = T(0);
    if (i < m) { xi[r] = Xo[i]; si[r] = s[i]; }
    acc[r] = T(0);
  }
  __syncthreads();
  T cacc = T(0);
  if (I == J) {
#pragma unroll 4
    for (int jj = 0; jj < 32; ++jj) {
      const C4<T> xj = xs[warp * 32 + jj];
      const T sj = ss[warp * 32 + jj];
#pragma unroll
      for (int r = 0; r < MVS_R; ++r) acc[r] = fma(kval<KER>(dist2(xi[r], xj), sf2), sj, acc[r]);
    }
  } else {
#pragma unroll 4
    for (int jj = 0; jj < 32; ++jj) {
      const C4<T> xj = xs[warp * 32 + jj];
      const T sj = ss[warp * 32 + jj];
      T cp = T(0);
#pragma unroll
      for (int r = 0; r < MVS_R; ++r) {
        const T kv = kval<KER>(dist2(xi[r], xj), sf2);
        acc[r] = fma(kv, sj, acc[r]);
        cp = fma(kv, si[r], cp);
      }
      cp = warp_sum(cp);
      if (lane == jj) cacc = cp;
    }
  }
#pragma unroll
  for (int r = 0; r < MVS_R; ++r) racc[warp][lane + 32 * r] = acc[r];
  __syncthreads();
  for (int t = threadIdx.x; t < MVS_T; t += blockDim.x) {
    const int i = I * MVS_T + t;
    if (i >= m) continue;
    T v = racc[0][t];
#pragma unroll
    for (int w = 1; w < MVS_W; ++w) v += racc[w][t];
    part[(size_t)J * m + i] = v;
  }
  if (I != J) {
    const int j = J * MVS_T + warp * 32 + lane;
    if (j < m) part[(size_t)I * m + j] = cacc;
  }
}

// The FP32 matvec on packed pairs of rows (f32x2 arithmetic): a lane owns MVS_R = 4 rows of tile I
// as two pairs, the column records of tile J are staged duplicated ({x,x},{y,y},{z,z},{w,w} with
// w = sf2 s_j), and a warp's 32 per-column sums over its lanes' rows are reduced by one butterfly
// reduce-scatter (31 shuffles) instead of one warp sum per column.  Same tiles, slots and Mo^T s
// blocks as k_gram_matvec.
template <int KER>
__global__ void __launch_bounds__(MVS_W * 32, 7)   // 7 blocks per SM (72 registers): 24.3 -> 23.9 us
k_gram_matvec_f2(const C4<float>* __restrict__ Xo, const float* __restrict__ s, int m, int nb, float sf2,
                 float* __restrict__ part, const float* __restrict__ Mo, int ldm, int rp, int ngv,
                 float* __restrict__ tpart, const int* __restrict__ active) {
  pdl_wait();
  pdl_trigger();
  if (active && !*active) return;
  __shared__ uint64_t xs2[MVS_T][4];
  __shared__ float racc[MVS_W][MVS_T];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if ((int)blockIdx.x < ngv) {
    const int per_chunk = (rp + MVS_W - 1) / MVS_W;
    const int z = blockIdx.x / per_chunk;
    const int col = (blockIdx.x - z * per_chunk) * MVS_W + warp;
    if (col >= rp) return;
    const int i0 = z * GV_CHUNK, i1 = min(m, i0 + GV_CHUNK);
    const float* a = Mo + (size_t)col * ldm;
    float acc = 0.f;
#pragma unroll 8
    for (int i = i0 + lane; i < i1; i += 32) acc = fmaf(a[i], s[i], acc);
    acc = warp_sum(acc);
    if (lane == 0) tpart[(size_t)z * rp + col] = acc;
    return;
  }
  int idx = blockIdx.x - ngv, I = 0;
  while (idx >= nb - I) { idx -= nb - I; ++I; }
  const int J = I + idx;
  for (int t = threadIdx.x; t < MVS_T; t += blockDim.x) {
    const int j = J * MVS_T + t;
    float x = 0.f, y = 0.f, zc = 0.f, w = 0.f;
    if (j < m) { const C4<float> c = Xo[j]; x = c.x; y = c.y; zc = c.z; w = sf2 * s[j]; }
    xs2[t][0] = f2_make(x, x);
    xs2[t][1] = f2_make(y, y);
    xs2[t][2] = f2_make(zc, zc);
    xs2[t][3] = f2_make(w, w);
  }
  uint64_t rx[2], ry[2], rz[2], rs[2], acc[2];
#pragma unroll
  for (int pr = 0; pr < 2; ++pr) {
    float xv[2] = {0.f, 0.f}, yv[2] = {0.f, 0.f}, zv[2] = {0.f, 0.f}, sv[2] = {0.f, 0.f};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int i = I * MVS_T + lane + 32 * (2 * pr + h);
      if (i < m) { const C4<float> c = Xo[i]; xv[h] = c.x; yv[h] = c.y; zv[h] = c.z; sv[h] = sf2 * s[i]; }
    }
    rx[pr] = f2_make(xv[0], xv[1]);
    ry[pr] = f2_make(yv[0], yv[1]);
    rz[pr] = f2_make(zv[0], zv[1]);
    rs[pr] = f2_make(sv[0], sv[1]);
    acc[pr] = f2_make(0.f, 0.f);
  }
  __syncthreads();
  const uint64_t(*xc)[4] = xs2 + warp * 32;
  float cacc = 0.f;
  if (I == J) {
#pragma unroll 8
    for (int jj = 0; jj < 32; ++jj) {
      const uint64_t cx = xc[jj][0], cy = xc[jj][1], cz = xc[jj][2], cw = xc[jj][3];
#pragma unroll
      for (int pr = 0; pr < 2; ++pr) acc[pr] = f2_fma(kpair<KER>(rx[pr], ry[pr], rz[pr], cx, cy, cz), cw, acc[pr]);
    }
  } else {
    float v[32];
#pragma unroll
    for (int jj = 0; jj < 32; ++jj) {
      const uint64_t cx = xc[jj][0], cy = xc[jj][1], cz = xc[jj][2], cw = xc[jj][3];
      const uint64_t k0 = kpair<KER>(rx[0], ry[0], rz[0], cx, cy, cz);
      const uint64_t k1 = kpair<KER>(rx[1], ry[1], rz[1], cx, cy, cz);
      acc[0] = f2_fma(k0, cw, acc[0]);
      acc[1] = f2_fma(k1, cw, acc[1]);
      v[jj] = f2_sum(f2_fma(k1, rs[1], f2_mul(k0, rs[0])));
    }
    // butterfly reduce-scatter: after the stage with offset o a lane keeps the half of its
    // column sums selected by its bit o; at the end lane l holds the sum for column l
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
      const bool up = (lane & o) != 0;
#pragma unroll
      for (int q = 0; q < o; ++q) {
        const float send = up ? v[q] : v[q + o];
        const float keep = up ? v[q + o] : v[q];
        v[q] = keep + __shfl_xor_sync(0xffffffffu, send, o);
      }
    }
    cacc = v[0];
  }
#pragma unroll
  for (int pr = 0; pr < 2; ++pr) {
    float lo, hi;
    f2_split(acc[pr], lo, hi);
    racc[warp][lane + 32 * (2 * pr)] = lo;
    racc[warp][lane + 32 * (2 * pr + 1)] = hi;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < MVS_T; t += blockDim.x) {
    const int i = I * MVS_T + t;
    if (i >= m) continue;
    float vv = racc[0][t];
#pragma unroll
    for (int w = 1; w < MVS_W; ++w) vv += racc[w][t];
    part[(size_t)J * m + i] = vv;
  }
  if (I != J) {
    const int j = J * MVS_T + warp * 32 + lane;
    if (j < m) part[(size_t)I * m + j] = cacc;
  }
}

// g = sum_p part[p] + sn2 * s - a2 * Mo t     (Mo: m x r col-major, ld = ldm).  t is summed from
// the row-chunk partials of the matvec launch's Mo^T s blocks (tz chunks) into shared memory
// first.  A block owns CB_ROWS rows: lane = row, each of the CB_WARPS warps takes every
// CB_WARPS-th column of Mo (coalesced
// 128-byte column segments, CB_UNROLL independent accumulators), and the warps' sums are added
// in shared memory.  The block then forms its rows' share of the first dot pass of CG iteration j
//   q < j: V[:, q] . g ;  j: s . g ;  j+1: s . r0 ;  j+2: g . v ;  j+3: s . s
// into dpart[q * gridDim.x + block] (summed by k_cg_upd1 in a fixed order, in the working precision:
// FP64 adds would cost more than the data they sum on this GPU).
constexpr int CB_ROWS = 32, CB_WARPS = 8, CB_UNROLL = 8;
template <class T>
__global__ void __launch_bounds__(CB_WARPS * 32)
k_cg_combine(const T* __restrict__ part, int nsplit, const T* __restrict__ s, T sn2,
             const T* __restrict__ Mo, int ldm, int r, const T* __restrict__ tpart, int tz, T a2,
             int m, T* __restrict__ g, const T* __restrict__ V, int ldv, int j, const T* __restrict__ r0,
             const T* __restrict__ v, T* __restrict__ dpart, const int* __restrict__ active) {
  pdl_wait();
  pdl_trigger();
  if (!*active) return;
  extern __shared__ unsigned char sm_raw[];
  T* t = reinterpret_cast<T*>(sm_raw);                 // r coefficients
  __shared__ T red[CB_WARPS][CB_ROWS], redk[CB_WARPS][CB_ROWS];
  __shared__ T gsh[CB_ROWS];
  // Every loop below loads a batch of independent values before it uses any of them, so a thread
  // waits for one L2 round trip per batch rather than one per value (the summation order is the
  // same as one value at a time).
  for (int l = threadIdx.x; l < r; l += blockDim.x) {
    T acc = T(0);
    int z = 0;
    for (; z + 8 <= tz; z += 8) {
      T x[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) x[u] = tpart[(size_t)(z + u) * r + l];
#pragma unroll
      for (int u = 0; u < 8; ++u) acc += x[u];
    }
    for (; z < tz; ++z) acc += tpart[(size_t)z * r + l];
    t[l] = acc;
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = blockIdx.x * CB_ROWS + lane;
  const bool valid = i < m;
  T acc[CB_UNROLL];
#pragma unroll
  for (int u = 0; u < CB_UNROLL; ++u) acc[u] = T(0);
  if (valid) {
    int l = warp;
    constexpr int CB_BATCH = 4;   // groups of CB_UNROLL columns loaded together
    for (; l + (CB_BATCH * CB_UNROLL - 1) * CB_WARPS < r; l += CB_BATCH * CB_UNROLL * CB_WARPS) {
      T x[CB_BATCH][CB_UNROLL];
#pragma unroll
      for (int b = 0; b < CB_BATCH; ++b)
#pragma unroll
        for (int u = 0; u < CB_UNROLL; ++u) x[b][u] = Mo[(size_t)(l + (b * CB_UNROLL + u) * CB_WARPS) * ldm + i];
#pragma unroll
      for (int b = 0; b < CB_BATCH; ++b)
#pragma unroll
        for (int u = 0; u < CB_UNROLL; ++u) acc[u] = fma(x[b][u], t[l + (b * CB_UNROLL + u) * CB_WARPS], acc[u]);
    }
    for (; l + (CB_UNROLL - 1) * CB_WARPS < r; l += CB_UNROLL * CB_WARPS) {
#pragma unroll
      for (int u = 0; u < CB_UNROLL; ++u) {
        const int lu = l + u * CB_WARPS;
        acc[u] = fma(Mo[(size_t)lu * ldm + i], t[lu], acc[u]);
      }
    }
    for (; l < r; l += CB_WARPS) acc[0] = fma(Mo[(size_t)l * ldm + i], t[l], acc[0]);
  }
  T lr = T(0);
#pragma unroll
  for (int u = 0; u < CB_UNROLL; ++u) lr += acc[u];
  red[warp][lane] = lr;
  // the Gram partials: warp w sums slots w, w + CB_WARPS, ...
  T kw = T(0);
  if (valid) {
    int p = warp;
    for (; p + 7 * CB_WARPS < nsplit; p += 8 * CB_WARPS) {
      T x[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) x[u] = part[(size_t)(p + u * CB_WARPS) * m + i];
#pragma unroll
      for (int u = 0; u < 8; ++u) kw += x[u];
    }
    for (; p < nsplit; p += CB_WARPS) kw += part[(size_t)p * m + i];
  }
  redk[warp][lane] = kw;
  __syncthreads();
  if (warp == 0) {
    T gv = T(0);
    if (valid) {
      T low = T(0), kv = T(0);
#pragma unroll
      for (int w = 0; w < CB_WARPS; ++w) { low += red[w][lane]; kv += redk[w][lane]; }
      kv = fma(sn2, s[i], kv);
      gv = fma(-a2, low, kv);
      g[i] = gv;
    }
    gsh[lane] = gv;
  }
  __syncthreads();
  const T gi = gsh[lane];
  const T si = valid ? s[i] : T(0);
  constexpr int CB_QB = 8;   // dots per warp whose loads are in flight together
  for (int q0 = warp; q0 < j + 4; q0 += CB_QB * CB_WARPS) {
    T pr[CB_QB];
#pragma unroll
    for (int u = 0; u < CB_QB; ++u) {
      const int q = q0 + u * CB_WARPS;
      T x = T(0);
      if (valid && q < j + 4) {
        if (q < j) x = V[(size_t)q * ldv + i] * gi;
        else if (q == j) x = si * gi;
        else if (q == j + 1) x = si * r0[i];
        else if (q == j + 2) x = gi * v[i];
        else x = si * si;
      }
      pr[u] = x;
    }
#pragma unroll
    for (int u = 0; u < CB_QB; ++u) {
      const int q = q0 + u * CB_WARPS;
      if (q >= j + 4) break;   // uniform across the warp
      const T tot = warp_sum(pr[u]);
      if (lane == 0) dpart[(size_t)q * gridDim.x + blockIdx.x] = tot;
    }
  }
}

// Per-thread share of a block-wide dot product a . b over m entries (strided by blockDim.x).
// FP32 data: four FP32 FMA chains combined in FP64, so the FP64 pipe (slow on this GPU) sees a
// handful of operations per thread; FP64 data: FP64 throughout.
template <class T> __device__ __forceinline__ double dot_part(const T* __restrict__ a, const T* __restrict__ b, int m) {
  const int st = blockDim.x;
  int i = threadIdx.x;
  if constexpr (sizeof(T) == 8) {
    double acc = 0.0;
    for (; i < m; i += st) acc = fma(a[i], b[i], acc);
    return acc;
  } else {
    float p0 = 0.f, p1 = 0.f, p2 = 0.f, p3 = 0.f;
    for (; i + 3 * st < m; i += 4 * st) {
      p0 = fmaf(a[i], b[i], p0);
      p1 = fmaf(a[i + st], b[i + st], p1);
      p2 = fmaf(a[i + 2 * st], b[i + 2 * st], p2);
      p3 = fmaf(a[i + 3 * st], b[i + 3 * st], p3);
    }
    for (; i < m; i += st) p0 = fmaf(a[i], b[i], p0);
    return (double(p0) + double(p1)) + (double(p2) + double(p3));
  }
}

// Sum of the per-block partials part[q * nblk + b] over b for q in [0, nq), in a fixed order, into
// out[q] (shared memory) -- and, if dots != null, into dots[q] in FP64.  Each warp takes UP_QB values
// of q at a time so that their loads are in flight together.
constexpr int UP_QB = 4;
template <class T>
__device__ __forceinline__ void sum_partials(const T* __restrict__ part, int nblk, int nq, T* out, double* dots) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  constexpr int BB = 8;   // partials per lane and value whose loads are in flight together
  for (int q0 = warp * UP_QB; q0 < nq; q0 += nw * UP_QB) {
    T acc[UP_QB];
#pragma unroll
    for (int u = 0; u < UP_QB; ++u) acc[u] = T(0);
    for (int b0 = lane; b0 < nblk; b0 += 32 * BB) {
      T x[UP_QB][BB];
#pragma unroll
      for (int u = 0; u < UP_QB; ++u)
#pragma unroll
        for (int e = 0; e < BB; ++e) {
          const int b = b0 + 32 * e;
          x[u][e] = (q0 + u < nq && b < nblk) ? part[(size_t)(q0 + u) * nblk + b] : T(0);
        }
#pragma unroll
      for (int u = 0; u < UP_QB; ++u)
#pragma unroll
        for (int e = 0; e < BB; ++e)
          if (b0 + 32 * e < nblk) acc[u] += x[u][e];
    }
#pragma unroll
    for (int u = 0; u < UP_QB; ++u) {
      const T t = warp_sum(acc[u]);
      if (lane == 0 && q0 + u < nq) {
        out[q0 + u] = t;
        if (dots) dots[q0 + u] = double(t);
      }
    }
  }
}

// Row block of the CG update kernels: UP_ROWS rows, UP_SPLIT threads per row, each summing every
// UP_SPLIT-th term of a row's sum over the previous directions (the loads of a warp stay coalesced:
// its 32 threads take 32 consecutive rows of one column).
constexpr int UP_THREADS = 256, UP_ROWS = 64, UP_SPLIT = UP_THREADS / UP_ROWS;
static_assert(UP_ROWS % 32 == 0, "rows per lane");
constexpr int UP_VB = 8;   // previous directions per thread whose V, GV loads are in flight together

// First G-orthogonalisation pass of CG iteration j.  The first-pass dots are summed from the
// combine blocks' partials (FP64, fixed order; block 0 also stores all j + 4 of them in dots1):
// c = V^T G s, then d = s - V c, G d = g - GV c, parked unnormalised in column j of V and GV.
// The block then forms its rows' share of the second-pass dots (q < j: V[:, q] . G d; j: d . G d)
// into dpart2[q * gridDim.x + block].
template <class T>
__global__ void __launch_bounds__(UP_THREADS)
k_cg_upd1(int j, const T* __restrict__ dpart1, int nblk1, double* __restrict__ dots1, T* __restrict__ V,
          T* __restrict__ GV, int ldv, const T* __restrict__ s, const T* __restrict__ g, int m,
          T* __restrict__ dpart2, const int* __restrict__ active) {
  pdl_wait();
  pdl_trigger();
  if (!*active) return;
  __shared__ T c[1024 + 4];
  __shared__ T sd[UP_SPLIT][UP_ROWS], sgd[UP_SPLIT][UP_ROWS];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  sum_partials(dpart1, nblk1, (blockIdx.x == 0) ? j + 4 : j, c, blockIdx.x == 0 ? dots1 : nullptr);
  __syncthreads();
  const int rl = threadIdx.x % UP_ROWS, sp = threadIdx.x / UP_ROWS;
  const int row0 = blockIdx.x * UP_ROWS;
  const int i = row0 + rl;
  T d = T(0), gd = T(0);
  if (i < m) {
    for (int q0 = sp; q0 < j; q0 += UP_SPLIT * UP_VB) {
      T xv[UP_VB], xg[UP_VB];
#pragma unroll
      for (int e = 0; e < UP_VB; ++e) {
        const int q = q0 + UP_SPLIT * e;
        xv[e] = q < j ? V[(size_t)q * ldv + i] : T(0);
        xg[e] = q < j ? GV[(size_t)q * ldv + i] : T(0);
      }
#pragma unroll
      for (int e = 0; e < UP_VB; ++e) {
        const int q = q0 + UP_SPLIT * e;
        if (q < j) {
          const T cq = c[q];
          d = fma(-xv[e], cq, d);
          gd = fma(-xg[e], cq, gd);
        }
      }
    }
  }
  sd[sp][rl] = d;
  sgd[sp][rl] = gd;
  __syncthreads();
  if (sp == 0) {
    d = T(0); gd = T(0);
    if (i < m) {
      d = s[i];
      gd = g[i];
#pragma unroll
      for (int u = 0; u < UP_SPLIT; ++u) { d += sd[u][rl]; gd += sgd[u][rl]; }
      V[(size_t)j * ldv + i] = d;
      GV[(size_t)j * ldv + i] = gd;
    }
    sd[0][rl] = d;
    sgd[0][rl] = gd;
  }
  __syncthreads();
  const int nrow = min(UP_ROWS, m - row0);
  constexpr int RT = UP_ROWS / 32;   // rows per lane
  for (int q0 = warp * UP_QB; q0 <= j; q0 += nw * UP_QB) {
    T acc[UP_QB];
#pragma unroll
    for (int u = 0; u < UP_QB; ++u) acc[u] = T(0);
    T x[UP_QB][RT];
#pragma unroll
    for (int u = 0; u < UP_QB; ++u)
#pragma unroll
      for (int e = 0; e < RT; ++e) {
        const int t = lane + 32 * e, q = q0 + u;
        x[u][e] = (t < nrow && q < j) ? V[(size_t)q * ldv + row0 + t] : T(0);
      }
#pragma unroll
    for (int e = 0; e < RT; ++e) {
      const int t = lane + 32 * e;
      if (t >= nrow) continue;
      const T gt = sgd[0][t];
#pragma unroll
      for (int u = 0; u < UP_QB; ++u) {
        const int q = q0 + u;
        if (q < j) acc[u] = fma(x[u][e], gt, acc[u]);
        else if (q == j) acc[u] = fma(sd[0][t], gt, acc[u]);
      }
    }
#pragma unroll
    for (int u = 0; u < UP_QB; ++u) {
      const T t = warp_sum(acc[u]);
      if (lane == 0 && q0 + u <= j) dpart2[(size_t)(q0 + u) * gridDim.x + blockIdx.x] = t;
    }
  }
}

// Second pass and the update of the iterative CAKF step (appendix algorithm):
//   c2 = V^T G d;  d <- d - V c2;  eta = d^T G d - |c2|^2;  alpha = s^T (r0 - G v) = s^T r0 - g^T v;
//   V[:, j] = d / sqrt(eta);  GV[:, j] = G d / sqrt(eta);  v += (alpha / eta) d;  r -= (alpha / eta) G d.
// Every block sums the second-pass dots from the k_cg_upd1 partials, recomputes the scalars and
// takes the same stop decision.  With Snext (CG policy, no re-orthogonalisation) the next action
// -- the updated residual -- is written to s and to column j + 1 of S here.
template <class T>
__global__ void __launch_bounds__(UP_THREADS)
k_cg_upd2(int j, const double* __restrict__ dots1, const T* __restrict__ dpart2, int nblk2,
          T* __restrict__ V, T* __restrict__ GV, int ldv, T* __restrict__ r, T* __restrict__ v,
          T* __restrict__ s, T* __restrict__ Q, int m,
          double bd_tol, double rtol2_r0sq, int use_rtol, int* __restrict__ active,
          double* __restrict__ eta_out, double* __restrict__ alpha_out, int* __restrict__ count,
          T* __restrict__ Snext) {
  pdl_wait();
  pdl_trigger();
  if (!*active) return;
  __shared__ T c[1024 + 4];
  __shared__ double sh[3];
  __shared__ T shc[3];             // 1 / sqrt(eta), alpha / eta, 1 / |s| (formed once, in FP64)
  __shared__ T sd[UP_SPLIT][UP_ROWS], sgd[UP_SPLIT][UP_ROWS];
  sum_partials(dpart2, nblk2, j + 1, c, nullptr);
  __syncthreads();
  double ccp = 0.0;
  for (int q = threadIdx.x; q < j; q += blockDim.x) ccp = fma(double(c[q]), double(c[q]), ccp);
  const double cc = block_sum(ccp);
  if (threadIdx.x == 0) {
    const double sg = dots1[j];
    const double eta = double(c[j]) - cc;
    const double alpha = dots1[j + 1] - dots1[j + 2];
    int stop = !(eta > bd_tol * sg) || !isfinite(eta) || !isfinite(alpha);
    if (use_rtol && dots1[j + 3] <= rtol2_r0sq) stop = 1;
    sh[0] = eta; sh[1] = alpha; sh[2] = stop;
    if (!stop) {
      shc[0] = T(1.0 / sqrt(eta));
      shc[1] = T(alpha / eta);
      shc[2] = T(1.0 / sqrt(dots1[j + 3]));
    }
  }
  __syncthreads();
  const double eta = sh[0], alpha = sh[1];
  const int rl = threadIdx.x % UP_ROWS, sp = threadIdx.x / UP_ROWS;
  const int i = blockIdx.x * UP_ROWS + rl;
  if (sh[2] != 0.0) {
    // breakdown / converged: this direction is not used; clear the parked column
    if (sp == 0 && i < m) { V[(size_t)j * ldv + i] = T(0); GV[(size_t)j * ldv + i] = T(0); }
    if (blockIdx.x == 0 && threadIdx.x == 0) *active = 0;
    return;
  }
  T d = T(0), gd = T(0);
  if (i < m) {
    for (int q0 = sp; q0 < j; q0 += UP_SPLIT * UP_VB) {
      T xv[UP_VB], xg[UP_VB];
#pragma unroll
      for (int e = 0; e < UP_VB; ++e) {
        const int q = q0 + UP_SPLIT * e;
        xv[e] = q < j ? V[(size_t)q * ldv + i] : T(0);
        xg[e] = q < j ? GV[(size_t)q * ldv + i] : T(0);
      }
#pragma unroll
      for (int e = 0; e < UP_VB; ++e) {
        const int q = q0 + UP_SPLIT * e;
        if (q < j) {
          const T cq = c[q];
          d = fma(-xv[e], cq, d);
          gd = fma(-xg[e], cq, gd);
        }
      }
    }
  }
  sd[sp][rl] = d;
  sgd[sp][rl] = gd;
  __syncthreads();
  if (sp == 0 && i < m) {
    d = V[(size_t)j * ldv + i];
    gd = GV[(size_t)j * ldv + i];
#pragma unroll
    for (int u = 0; u < UP_SPLIT; ++u) { d += sd[u][rl]; gd += sgd[u][rl]; }
    const T inv = shc[0];
    const T coef = shc[1];
    V[(size_t)j * ldv + i] = d * inv;
    GV[(size_t)j * ldv + i] = gd * inv;
    v[i] = fma(coef, d, v[i]);
    const T rn = fma(-coef, gd, r[i]);
    r[i] = rn;
    if (Q) Q[(size_t)j * ldv + i] = s[i] * shc[2];
    if (Snext) {
      s[i] = rn;
      Snext[i] = rn;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) { eta_out[j] = eta; alpha_out[j] = alpha; *count = j + 1; }
}

// Projection coefficients of the action on the orthonormal basis Q of the previous actions:
// qd[l] = Q[:, l] . s  (one block per l)
template <class T>
__global__ void k_cg_qdots(const T* __restrict__ Q, int ldq, int j, const T* __restrict__ s, int m,
                           double* __restrict__ qd, const int* __restrict__ active) {
  pdl_wait();
  pdl_trigger();
  if (!*active) return;
  const int l = blockIdx.x;
  const T* a = Q + (size_t)l * ldq;
  const double acc = block_sum(dot_part(a, s, m));
  if (threadIdx.x == 0) qd[l] = acc;
}
// s -= Q[:, :j] qd   (Gram-Schmidt against the previous actions; a no-op in exact arithmetic for CG
// residuals, which are mutually orthogonal).  On the last pass S[:, j] = s.
template <class T>
__global__ void k_cg_qorth(const T* __restrict__ Q, int ldq, int j, const double* __restrict__ qd, T* __restrict__ s,
                           int m, T* __restrict__ S, int lds, const int* __restrict__ active) {
  pdl_wait();
  pdl_trigger();
  if (!*active) return;
  __shared__ T c[1024];
  for (int q = threadIdx.x; q < j; q += blockDim.x) c[q] = T(qd[q]);
  __syncthreads();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  T v = s[i];
  for (int q = 0; q < j; ++q) v = fma(-Q[(size_t)q * ldq + i], c[q], v);
  s[i] = v;
  if (S) S[(size_t)j * lds + i] = v;
}

// s = r (CG policy: the current residual) or s = the replayed action; S[:, j] = s.
template <class T>
__global__ void k_cg_select(int j, const T* __restrict__ r, const double* __restrict__ rep, int m,
                            T* __restrict__ s, T* __restrict__ S, int lds, const int* __restrict__ active) {
  pdl_wait();
  pdl_trigger();
  if (!*active) return;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  T val = rep ? T(rep[(size_t)j * m + i]) : r[i];
  s[i] = val;
  S[(size_t)j * lds + i] = val;
}

// r0 = y - m_pred[obs] ; r = r0 ; v = 0 ; sum of squares of r0 accumulated by the caller
template <class T>
__global__ void k_cg_init(const double* __restrict__ y, const double* __restrict__ mpred,
                          const int* __restrict__ obs, int m, T* __restrict__ r, T* __restrict__ r0,
                          T* __restrict__ v, double* __restrict__ r0sq) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  double val = 0.0;
  if (i < m) {
    val = y[i] - mpred[obs[i]];
    r[i] = T(val);
    r0[i] = T(val);
    v[i] = T(0);
  }
  double sq = block_sum(val * val);
  if (threadIdx.x == 0) atomicAdd(r0sq, sq);
}

// ------------------------------------------------------------------------------------------
// Plain SIMT Gram x block:  Out[i, c] = sum_j k(xr_i, xc_j) B[j, c]   (Out, B column-major)
constexpr int GB_BM = 64, GB_BN = 64, GB_BK = 32, GB_THREADS = 256;

template <int KER, class T, bool DER = false>
__global__ void __launch_bounds__(GB_THREADS)
k_gram_block_simt(const C4<T>* __restrict__ Xr, int nr, const C4<T>* __restrict__ Xc, int nc,
                  const T* __restrict__ B, int ldb, int width, T sf2, T* __restrict__ Out, int ldo) {
  __shared__ T Ks[GB_BK][GB_BM + 1];
  __shared__ T Bs[GB_BK][GB_BN + 1];
  __shared__ C4<T> xr[GB_BM];
  const int r0 = blockIdx.x * GB_BM, n0 = blockIdx.y * GB_BN;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;   // 16 x 16 threads, 4 x 4 outputs each
  if (threadIdx.x < GB_BM) {
    int rr = r0 + threadIdx.x;
    if (rr < nr) xr[threadIdx.x] = Xr[rr]; else { C4<T> z; z.x = z.y = z.z = T(1e30); z.w = 0; xr[threadIdx.x] = z; }
  }
  T acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
  __syncthreads();
  for (int k0 = 0; k0 < nc; k0 += GB_BK) {
    // kernel tile 64 x 32: 2048 values, 8 per thread
    for (int e = threadIdx.x; e < GB_BM * GB_BK; e += GB_THREADS) {
      int rr = e % GB_BM, kk = e / GB_BM;
      int col = k0 + kk;
      T kvv = T(0);
      if (col < nc && r0 + rr < nr)
        kvv = DER ? kval_dlogl<KER>(dist2(xr[rr], Xc[col]), sf2) : kval<KER>(dist2(xr[rr], Xc[col]), sf2);
      Ks[kk][rr] = kvv;
    }
    for (int e = threadIdx.x; e < GB_BK * GB_BN; e += GB_THREADS) {
      int kk = e % GB_BK, cc = e / GB_BK;
      int col = k0 + kk, c = n0 + cc;
      Bs[kk][cc] = (col < nc && c < width) ? B[(size_t)c * ldb + col] : T(0);
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < GB_BK; ++kk) {
      T ka[4], bb[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) ka[a] = Ks[kk][ty + 16 * a];
#pragma unroll
      for (int b = 0; b < 4; ++b) bb[b] = Bs[kk][tx + 16 * b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = fma(ka[a], bb[b], acc[a][b]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    int rr = r0 + ty + 16 * a;
    if (rr >= nr) continue;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      int c = n0 + tx + 16 * b;
      if (c < width) Out[(size_t)c * ldo + rr] = acc[a][b];
    }
  }
}

// ------------------------------------------------------------------------------------------
// Split-K transposed product: part[z][a + b*na] = sum_{t in chunk z} A[t, a] B[t, b]
// (A: K x na, B: K x nb column-major), 64 x 64 output tiles, 4 x 4 per thread, K staged 32 at a time
// (rows of A and B are contiguous along K: each warp reads 32 consecutive K values of 8 columns).
// Accumulation in the working precision, partials in double; k_reduce_splits sums them.
constexpr int TN_T = 64, TN_K = 32;
template <class T>
__global__ void __launch_bounds__(256)
k_gemm_tn_part(const T* __restrict__ A, int lda, int na, const T* __restrict__ B, int ldb, int nb,
               int K, int chunk, double* __restrict__ part) {
  __shared__ T As[TN_K][TN_T + 1];
  __shared__ T Bs[TN_K][TN_T + 1];
  const int a0 = blockIdx.x * TN_T, b0 = blockIdx.y * TN_T;
  const int k_begin = blockIdx.z * chunk, k_end = min(K, k_begin + chunk);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  T acc[4][4];
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[p][q] = T(0);
  const int kk_ld = threadIdx.x & 31, cc_ld = threadIdx.x >> 5;   // 32 K values x 8 columns per pass
  for (int k0 = k_begin; k0 < k_end; k0 += TN_K) {
    const int t = k0 + kk_ld;
#pragma unroll
    for (int pass = 0; pass < TN_T / 8; ++pass) {
      const int cc = cc_ld + 8 * pass;
      As[kk_ld][cc] = (t < k_end && a0 + cc < na) ? A[(size_t)(a0 + cc) * lda + t] : T(0);
      Bs[kk_ld][cc] = (t < k_end && b0 + cc < nb) ? B[(size_t)(b0 + cc) * ldb + t] : T(0);
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < TN_K; ++kk) {
      T aa[4], bb[4];
#pragma unroll
      for (int p = 0; p < 4; ++p) aa[p] = As[kk][ty + 16 * p];
#pragma unroll
      for (int q = 0; q < 4; ++q) bb[q] = Bs[kk][tx + 16 * q];
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[p][q] = fma(aa[p], bb[q], acc[p][q]);
    }
    __syncthreads();
  }
  const size_t stride = (size_t)na * nb;
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int a = a0 + ty + 16 * p, b = b0 + tx + 16 * q;
      if (a < na && b < nb) part[blockIdx.z * stride + (size_t)b * na + a] = double(acc[p][q]);
    }
}

// C[a + b*ldc] = alpha * sum_z part[z][a + b*na]  (+ beta * C)
template <class OutT>
__global__ void k_reduce_splits(const double* __restrict__ part, int nsplit, int na, int nb, double alpha,
                                double beta, OutT* __restrict__ C, int ldc) {
  size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  size_t tot = (size_t)na * nb;
  if (e >= tot) return;
  double acc = 0.0;
  for (int z = 0; z < nsplit; ++z) acc += part[z * tot + e];
  int a = int(e % na), b = int(e / na);
  OutT* c = C + (size_t)b * ldc + a;
  *c = OutT(alpha * acc + (beta != 0.0 ? beta * double(*c) : 0.0));
}

// ------------------------------------------------------------------------------------------
// Tiled NN product for tall A: C[M x N] = alpha * A[M x K] * B[K x N] + beta * C (column-major).
// B may be double (small coefficient matrices); it is converted to T when staged.
constexpr int NN_BM = 64, NN_BN = 64, NN_BK = 16;
template <class T, class TB>
__global__ void __launch_bounds__(256)
k_gemm_nn(int M, int N, int K, T alpha, const T* __restrict__ A, int lda, const TB* __restrict__ B, int ldb,
          T beta, T* __restrict__ C, int ldc) {
  __shared__ T As[NN_BK][NN_BM + 1];
  __shared__ T Bs[NN_BK][NN_BN + 1];
  const int m0 = blockIdx.x * NN_BM, n0 = blockIdx.y * NN_BN;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  T acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
  for (int k0 = 0; k0 < K; k0 += NN_BK) {
    for (int e = threadIdx.x; e < NN_BM * NN_BK; e += 256) {
      int rr = e % NN_BM, kk = e / NN_BM;
      As[kk][rr] = (m0 + rr < M && k0 + kk < K) ? A[(size_t)(k0 + kk) * lda + m0 + rr] : T(0);
    }
    for (int e = threadIdx.x; e < NN_BK * NN_BN; e += 256) {
      int kk = e % NN_BK, cc = e / NN_BK;
      Bs[kk][cc] = (k0 + kk < K && n0 + cc < N) ? T(B[(size_t)(n0 + cc) * ldb + k0 + kk]) : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < NN_BK; ++kk) {
      T aa[4], bb[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) aa[a] = As[kk][ty + 16 * a];
#pragma unroll
      for (int b = 0; b < 4; ++b) bb[b] = Bs[kk][tx + 16 * b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = fma(aa[a], bb[b], acc[a][b]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    int rr = m0 + ty + 16 * a;
    if (rr >= M) continue;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      int c = n0 + tx + 16 * b;
      if (c >= N) continue;
      T* p = C + (size_t)c * ldc + rr;
      *p = (beta == T(0)) ? alpha * acc[a][b] : fma(alpha, acc[a][b], beta * *p);
    }
  }
}

// Small FP64 product with transposes: C = alpha op(A) op(B) + beta C  (sizes up to a few hundred)
__global__ void k_gemm_small_f64(int ta, int tb, int M, int N, int K, double alpha, const double* __restrict__ A,
                                 int lda, const double* __restrict__ B, int ldb, double beta, double* __restrict__ C,
                                 int ldc) {
  __shared__ double As[16][17], Bs[16][17];
  int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  int row = blockIdx.x * 16 + ty, col = blockIdx.y * 16 + tx;
  double acc = 0.0;
  for (int k0 = 0; k0 < K; k0 += 16) {
    int ka = k0 + tx, kb = k0 + ty;
    int ar = blockIdx.x * 16 + ty;
    As[ty][tx] = (ar < M && ka < K) ? (ta ? A[(size_t)ar * lda + ka] : A[(size_t)ka * lda + ar]) : 0.0;
    int bc = blockIdx.y * 16 + tx;
    Bs[ty][tx] = (bc < N && kb < K) ? (tb ? B[(size_t)kb * ldb + bc] : B[(size_t)bc * ldb + kb]) : 0.0;
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) acc = fma(As[ty][kk], Bs[kk][tx], acc);
    __syncthreads();
  }
  if (row < M && col < N) {
    double* c = C + (size_t)col * ldc + row;
    *c = alpha * acc + (beta != 0.0 ? beta * *c : 0.0);
  }
}

// ------------------------------------------------------------------------------------------
// Row kernels
// Out[i, c] = In[idx[i], c] for c < cols (column-major, gather rows)
template <class T>
__global__ void k_gather_rows(const T* __restrict__ In, int ldi, const int* __restrict__ idx, int m, int cols,
                              T* __restrict__ Out, int ldo) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int c = blockIdx.y;
  if (i < m && c < cols) Out[(size_t)c * ldo + i] = In[(size_t)c * ldi + idx[i]];
}

// Out[idx[i], c] += alpha * In[i, c]
template <class T>
__global__ void k_scatter_add_rows(const T* __restrict__ In, int ldi, const int* __restrict__ idx, int m, int cols,
                                   T alpha, T* __restrict__ Out, int ldo) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int c = blockIdx.y;
  if (i < m && c < cols) Out[(size_t)c * ldo + idx[i]] += alpha * In[(size_t)c * ldi + i];
}

// sum_c A[i, c]^2 for row i of a column-major block.  FP32 factors: four compensated (Kahan) FP32
// sums combined in FP64 -- relative error about 2^-24 whatever the column count, at FP32-pipe speed
// (an FP64 accumulation chain per row is bound by GB300's narrow FP64 pipe); FP64 factors: FP64.
template <class T>
__device__ __forceinline__ double row_sumsq(const T* __restrict__ A, int lda, int i, int cols) {
  double acc = 0.0;
  if constexpr (sizeof(T) == 4) {
    float s[4] = {0.f, 0.f, 0.f, 0.f}, e[4] = {0.f, 0.f, 0.f, 0.f};
    int c = 0;
    for (; c + 3 < cols; c += 4) {
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const float v = A[(size_t)(c + u) * lda + i];
        const float y = fmaf(v, v, -e[u]);
        const float t = s[u] + y;
        e[u] = (t - s[u]) - y;
        s[u] = t;
      }
    }
    for (; c < cols; ++c) {
      const float v = A[(size_t)c * lda + i];
      const float y = fmaf(v, v, -e[0]);
      const float t = s[0] + y;
      e[0] = (t - s[0]) - y;
      s[0] = t;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) acc += double(s[u]) - double(e[u]);
  } else {
    for (int c = 0; c < cols; ++c) { const double v = double(A[(size_t)c * lda + i]); acc += v * v; }
  }
  return acc;
}

// rs[i] = sum_c A[i, c]^2 (+ beta * rs[i])
template <class T>
__global__ void k_rowsumsq(const T* __restrict__ A, int lda, int n, int cols, double beta, double* __restrict__ rs) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double acc = row_sumsq(A, lda, i, cols);
  rs[i] = acc + (beta != 0.0 ? beta * rs[i] : 0.0);
}

// m_pred = a m_prev + (mu_k - a mu_{k-1})
__global__ void k_predict_mean(const double* __restrict__ mprev, const double* __restrict__ mu_k,
                               const double* __restrict__ mu_km1, double a, int n, double* __restrict__ mpred) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double b = mu_k ? (mu_k[i] - a * mu_km1[i]) : 0.0;
  mpred[i] = a * mprev[i] + b;
}

// Two-block state (Matern-3/2 temporal factor: positions in rows [0, half), velocities in rows
// [half, 2 half)): Out = (C (x) I) In for a 2 x 2 matrix C = [[c00, c01], [c10, c11]], i.e.
//   Out[i] = c00 In[i] + c01 In[half + i],  Out[half + i] = c10 In[i] + c11 In[half + i]
// per column.  In == Out is allowed: each thread reads its pair before writing it.
template <class T>
__global__ void k_mix2(const T* In, int ldi, T* Out, int ldo, int half, int cols, T c00, T c01, T c10, T c11) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int c = blockIdx.y;
  if (i >= half || c >= cols) return;
  const T x = In[(size_t)c * ldi + i], v = In[(size_t)c * ldi + half + i];
  Out[(size_t)c * ldo + i] = fma(c00, x, c01 * v);
  Out[(size_t)c * ldo + half + i] = fma(c10, x, c11 * v);
}

// Mean prediction of the two-block state with the prior mean (mu_k, 0) of the positions:
//   m^- = A (m - (mu_{k-1}, 0)) + (mu_k, 0)   (mu may be null: zero mean)
__global__ void k_predict_mean2(const double* __restrict__ mprev, const double* __restrict__ mu_k,
                                const double* __restrict__ mu_km1, double a00, double a01, double a10, double a11,
                                int n, int half, double* __restrict__ mpred) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double x = mprev[i] - (mu_km1 ? mu_km1[i] : 0.0), v = mprev[half + i];
  mpred[i] = fma(a00, x, a01 * v) + (mu_k ? mu_k[i] : 0.0);
  mpred[half + i] = fma(a10, x, a11 * v);
}

// out[i] = a[i] + b[i] (FP64 plus working precision), i < n
template <class T>
__global__ void k_add_vec(const double* __restrict__ a, const T* __restrict__ b, int n, double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = a[i] + double(b[i]);
}

// Filter outputs of step k:  m_k = m_pred + (P^- w);  var_k = sf2 - a^2 rs_plus - rowsumsq(P^- W)
template <class T>
__global__ void k_filter_out(const double* __restrict__ mpred, const T* __restrict__ PVv, int ld, int ic,
                             double sf2, double a2, const double* __restrict__ rs_plus, int n,
                             double* __restrict__ mout, double* __restrict__ vout, double* __restrict__ rs_pw) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double acc = ic > 0 ? row_sumsq(PVv, ld, i, ic) : 0.0;
  double pw = ic >= 0 ? double(PVv[(size_t)ic * ld + i]) : 0.0;
  mout[i] = mpred[i] + pw;
  vout[i] = sf2 - a2 * rs_plus[i] - acc;
  if (rs_pw) rs_pw[i] = acc;
}

// Copy of a scaled column block: Out[:, c] = alpha * In[:, c]
template <class T>
__global__ void k_scale_copy(const T* __restrict__ In, int ldi, int n, int cols, T alpha, T* __restrict__ Out, int ldo) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int c = blockIdx.y;
  if (i < n && c < cols) Out[(size_t)c * ldo + i] = alpha * In[(size_t)c * ldi + i];
}

// Smoother outputs at k: ms = m_k + Y[:, cw];  vs = v_k - rowsumsq(Y[:, 0:cw])
template <class T>
__global__ void k_smooth_out(const double* __restrict__ mk, const double* __restrict__ vk, const T* __restrict__ Y,
                             int ld, int cw, int n, double* __restrict__ ms, double* __restrict__ vs) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double acc = row_sumsq(Y, ld, i, cw);
  ms[i] = mk[i] + double(Y[(size_t)cw * ld + i]);
  vs[i] = vk[i] - acc;
}

// Dense vector from the sparse filter message:  out = x + scatter(v_obs - u_obs) ...
// ws_new[i] = X[i, cw] ; then ws_new[obs] += v - Vz (done by k_ws_obs)
template <class T>
__global__ void k_ws_obs(const int* __restrict__ obs, int m, const T* __restrict__ vk, const T* __restrict__ Vz,
                         T* __restrict__ ws) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m) ws[obs[i]] += vk[i] - Vz[i];
}

// Y[:, c] = alpha * [Ws, ws][:, c]   (X = A^T [Ws ws] in the smoother)
template <class T>
__global__ void k_build_x(const T* __restrict__ Ws, int ldw, int cw, const T* __restrict__ ws, T alpha, int n,
                          T* __restrict__ X, int ldx) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int c = blockIdx.y;
  if (i >= n || c > cw) return;
  X[(size_t)c * ldx + i] = alpha * (c < cw ? Ws[(size_t)c * ldw + i] : ws[i]);
}

// FP64 per-step NLL from the iteration: sum_j [ 1/2 log(2 pi eta_j) + 1/2 alpha_j^2 / eta_j ] - logdet(L)
// where L L^T = S^T S (Cholesky in FP64, in place on the i x i Gram).  One block.
__global__ void k_nll_step(const double* __restrict__ eta, const double* __restrict__ alpha,
                           const int* __restrict__ count, double* __restrict__ SS, int ic, double* __restrict__ nll_k,
                           int* __restrict__ err) {
  __shared__ double s_piv;
  __shared__ int s_bad;
  const int j = *count;
  if (threadIdx.x == 0) s_bad = 0;
  __syncthreads();
  // Cholesky of the leading j x j block (column-major, ld = ic), right-looking
  for (int p = 0; p < j; ++p) {
    if (threadIdx.x == 0) {
      double d = SS[(size_t)p * ic + p];
      if (!(d > 0.0) || !isfinite(d)) { s_bad = 1; d = 1.0; }
      s_piv = sqrt(d);
      SS[(size_t)p * ic + p] = s_piv;
    }
    __syncthreads();
    for (int q = p + 1 + threadIdx.x; q < j; q += blockDim.x) SS[(size_t)p * ic + q] /= s_piv;
    __syncthreads();
    for (int e = threadIdx.x; e < (j - p - 1) * (j - p - 1); e += blockDim.x) {
      int q = p + 1 + e % (j - p - 1), c = p + 1 + e / (j - p - 1);
      if (q >= c) SS[(size_t)c * ic + q] -= SS[(size_t)p * ic + q] * SS[(size_t)p * ic + c];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double acc = 0.0;
    const double l2pi = 1.8378770664093453;
    for (int q = 0; q < j; ++q) {
      acc += 0.5 * (l2pi + log(eta[q])) + 0.5 * alpha[q] * alpha[q] / eta[q];
      acc -= log(SS[(size_t)q * ic + q]);
    }
    *nll_k = acc;
    if (s_bad || !isfinite(acc)) atomicExch(err, kErrNllChol);
  }
}

// Per-step small FP64 algebra of the NLL tangent pass (one block).  With Gh = S^T G S = R^T R
// (R upper), beta = Gh^-1 yh and, per parameter p, W_p = R^-T dGh_p R^-1:
//   grad[p] += 1/2 tr(W_p) + beta^T dyh_p - 1/2 beta^T dGh_p beta
//   Q_p      = upper triangle of W_p with halved diagonal   (dR R^-1 of the Cholesky factor)
//   u_p      = R^-T (dyh_p - dGh_p beta)                    (R dbeta_p)
// Work arrays (global, ld = ic): L (ic x ic), Rinv (ic x ic), W (ic x ic), tmp (3 ic).
__global__ void k_grad_small(int ic, int np, const double* __restrict__ Gh, const double* __restrict__ dGh,
                             const double* __restrict__ yh, const double* __restrict__ dyh, double* __restrict__ L,
                             double* __restrict__ Rinv, double* __restrict__ W, double* __restrict__ tmp,
                             double* __restrict__ Q, double* __restrict__ u, double* __restrict__ grad,
                             int* __restrict__ err) {
  __shared__ double piv;
  __shared__ int bad;
  if (threadIdx.x == 0) bad = 0;
  for (int e = threadIdx.x; e < ic * ic; e += blockDim.x) L[e] = Gh[e];
  __syncthreads();
  // Cholesky Gh = L L^T (lower, in place, column-major)
  for (int p = 0; p < ic; ++p) {
    if (threadIdx.x == 0) {
      double d = L[(size_t)p * ic + p];
      if (!(d > 0.0) || !isfinite(d)) { bad = 1; d = 1.0; }
      piv = sqrt(d);
      L[(size_t)p * ic + p] = piv;
    }
    __syncthreads();
    for (int q = p + 1 + threadIdx.x; q < ic; q += blockDim.x) L[(size_t)p * ic + q] /= piv;
    __syncthreads();
    const int w = ic - p - 1;
    for (int e = threadIdx.x; e < w * w; e += blockDim.x) {
      int q = p + 1 + e % w, c = p + 1 + e / w;
      if (q >= c) L[(size_t)c * ic + q] -= L[(size_t)p * ic + q] * L[(size_t)p * ic + c];
    }
    __syncthreads();
  }
  // Rinv = (L^T)^-1 = upper triangular; column j solves L^T x = e_j by back substitution
  for (int j = threadIdx.x; j < ic; j += blockDim.x) {
    for (int i = ic - 1; i >= 0; --i) {
      double acc = (i == j) ? 1.0 : 0.0;
      for (int l = i + 1; l <= j; ++l) acc -= L[(size_t)i * ic + l] * Rinv[(size_t)j * ic + l];   // R_il = L_li
      Rinv[(size_t)j * ic + i] = (i > j) ? 0.0 : acc / L[(size_t)i * ic + i];
    }
  }
  __syncthreads();
  // beta = Rinv Rinv^T yh
  double* t1 = tmp;
  double* beta = tmp + ic;
  for (int i = threadIdx.x; i < ic; i += blockDim.x) {
    double acc = 0.0;
    for (int l = 0; l < ic; ++l) acc += Rinv[(size_t)i * ic + l] * yh[l];   // (Rinv^T yh)_i = sum_l Rinv[l, i] yh_l
    t1[i] = acc;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < ic; i += blockDim.x) {
    double acc = 0.0;
    for (int l = 0; l < ic; ++l) acc += Rinv[(size_t)l * ic + i] * t1[l];
    beta[i] = acc;
  }
  __syncthreads();
  double* t2 = tmp + 2 * ic;
  for (int p = 0; p < np; ++p) {
    const double* D = dGh + (size_t)p * ic * ic;
    // W = Rinv^T D Rinv : first Y = D Rinv (into Q_p as scratch), then W = Rinv^T Y
    double* Y = Q + (size_t)p * ic * ic;
    for (int e = threadIdx.x; e < ic * ic; e += blockDim.x) {
      int i = e % ic, j = e / ic;
      double acc = 0.0;
      for (int l = 0; l <= j; ++l) acc += D[(size_t)l * ic + i] * Rinv[(size_t)j * ic + l];
      Y[e] = acc;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < ic * ic; e += blockDim.x) {
      int i = e % ic, j = e / ic;
      double acc = 0.0;
      for (int l = 0; l <= i; ++l) acc += Rinv[(size_t)i * ic + l] * Y[(size_t)j * ic + l];
      W[e] = acc;
    }
    __syncthreads();
    // scalars
    double tr = 0.0, bdy = 0.0, bdb = 0.0;
    for (int i = threadIdx.x; i < ic; i += blockDim.x) {
      tr += W[(size_t)i * ic + i];
      bdy += beta[i] * dyh[(size_t)p * ic + i];
      double db = 0.0;
      for (int l = 0; l < ic; ++l) db += D[(size_t)l * ic + i] * beta[l];
      bdb += beta[i] * db;
      t2[i] = dyh[(size_t)p * ic + i] - db;
    }
    tr = block_sum(tr);
    bdy = block_sum(bdy);
    bdb = block_sum(bdb);
    if (threadIdx.x == 0) grad[p] += 0.5 * tr + bdy - 0.5 * bdb;
    // u_p = Rinv^T t2 ; Q_p = Phi(W)
    for (int i = threadIdx.x; i < ic; i += blockDim.x) {
      double acc = 0.0;
      for (int l = 0; l <= i; ++l) acc += Rinv[(size_t)i * ic + l] * t2[l];
      u[(size_t)p * ic + i] = acc;
    }
    for (int e = threadIdx.x; e < ic * ic; e += blockDim.x) {
      int i = e % ic, j = e / ic;
      Q[(size_t)p * ic * ic + e] = (i < j) ? W[e] : ((i == j) ? 0.5 * W[e] : 0.0);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0 && bad) atomicExch(err, kErrGradChol);
}

// out[i, p] = in[idx[i] + p * ld]   (gather rows of a double block into precision T)
template <class T>
__global__ void k_gather_rows_f64(const double* __restrict__ In, int ld, const int* __restrict__ idx, int m, int cols,
                                  T* __restrict__ Out, int ldo) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int c = blockIdx.y;
  if (i < m && c < cols) Out[(size_t)c * ldo + i] = T(In[(size_t)c * ld + idx[i]]);
}

// dm_new[:, p] = dmpred[:, p] + E[:, p][col] + t[:, p]    (tangent of the filter mean)
template <class T>
__global__ void k_tangent_mean(const double* __restrict__ dmpred, const T* __restrict__ E, size_t estride, int ecol,
                               int lde, const T* __restrict__ t, int ldt, int n, int np, double* __restrict__ dm) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int p = blockIdx.y;
  if (i >= n || p >= np) return;
  double v = dmpred[(size_t)p * n + i];
  if (E) v += double(E[p * estride + (size_t)ecol * lde + i]);
  if (t) v += double(t[(size_t)p * ldt + i]);
  dm[(size_t)p * n + i] = v;
}

// dmpred[:, p] = adot_p * m_prev + a * dm_prev[:, p] - adot_p * mu_{k-1}
__global__ void k_tangent_predict(const double* __restrict__ mprev, const double* __restrict__ dmprev,
                                  const double* __restrict__ mu_km1, double a, double adot_lt, int n, int np,
                                  double* __restrict__ dmpred) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int p = blockIdx.y;
  if (i >= n || p >= np) return;
  const double ad = (p == 1) ? adot_lt : 0.0;
  double v = a * dmprev[(size_t)p * n + i] + ad * mprev[i];
  if (mu_km1) v -= ad * mu_km1[i];
  dmpred[(size_t)p * n + i] = v;
}

template <class T>
__global__ void k_axpy_block(T alpha, const T* __restrict__ X, int ldx, int rows, int cols, T* __restrict__ Y, int ldy) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int c = blockIdx.y;
  if (i < rows && c < cols) Y[(size_t)c * ldy + i] += alpha * X[(size_t)c * ldx + i];
}
template <class T>
__global__ void k_scale_cols(T* A, int ld, int rows, int cols, T s) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int c = blockIdx.y;
  if (i < rows && c < cols) A[(size_t)c * ld + i] *= s;
}

// In-place Cholesky (lower) of the leading j x j block of a symmetric matrix (column-major, ld),
// symmetrised from both triangles first.  Block-wide; returns false (on all threads) if not PD.
__device__ bool block_cholesky(double* A, int ld, int j) {
  __shared__ double piv;
  __shared__ int bad;
  if (threadIdx.x == 0) bad = 0;
  for (int e = threadIdx.x; e < j * j; e += blockDim.x) {
    int r = e % j, c = e / j;
    if (r > c) {
      double v = 0.5 * (A[(size_t)c * ld + r] + A[(size_t)r * ld + c]);
      A[(size_t)c * ld + r] = v;
    }
  }
  __syncthreads();
  for (int p = 0; p < j; ++p) {
    if (threadIdx.x == 0) {
      double d = A[(size_t)p * ld + p];
      if (!(d > 0.0) || !isfinite(d)) { bad = 1; d = 1.0; }
      piv = sqrt(d);
      A[(size_t)p * ld + p] = piv;
    }
    __syncthreads();
    for (int q = p + 1 + threadIdx.x; q < j; q += blockDim.x) A[(size_t)p * ld + q] /= piv;
    __syncthreads();
    const int w = j - p - 1;
    for (int e = threadIdx.x; e < w * w; e += blockDim.x) {
      int q = p + 1 + e % w, c = p + 1 + e / w;
      if (q >= c) A[(size_t)c * ld + q] -= A[(size_t)p * ld + q] * A[(size_t)p * ld + c];
    }
    __syncthreads();
  }
  bool ok = bad == 0;
  __syncthreads();
  return ok;
}

// Per-step NLL from its definition (eq. proj-observation with the actions S of the step):
//   nll = 1/2 [ j log 2 pi + logdet(S^T G S) ] + 1/2 yh^T (S^T G S)^-1 yh - 1/2 logdet(S^T S),
// yh = S^T r0, with both log-determinants from FP64 Cholesky factors of the leading j x j blocks.
// z (length >= j) is scratch for the forward substitution.
__global__ void k_nll_def(const int* __restrict__ count, double* __restrict__ Gh, double* __restrict__ SS, int ld,
                          const double* __restrict__ yh, double* __restrict__ z, double* __restrict__ nll_k,
                          int* __restrict__ err) {
  const int j = *count;
  const bool ok1 = block_cholesky(Gh, ld, j);
  const bool ok2 = block_cholesky(SS, ld, j);
  if (threadIdx.x == 0) {
    double ld1 = 0.0, ld2 = 0.0, quad = 0.0;
    for (int q = 0; q < j; ++q) {
      ld1 += log(Gh[(size_t)q * ld + q]);
      ld2 += log(SS[(size_t)q * ld + q]);
    }
    for (int q = 0; q < j; ++q) {          // L z = yh, L = lower Cholesky factor of S^T G S
      double acc = yh[q];
      for (int l = 0; l < q; ++l) acc -= Gh[(size_t)l * ld + q] * z[l];
      z[q] = acc / Gh[(size_t)q * ld + q];
      quad += z[q] * z[q];
    }
    const double val = 0.5 * j * 1.8378770664093453 + ld1 + 0.5 * quad - ld2;
    *nll_k = val;
    if (!ok1 || !ok2 || !isfinite(val)) atomicExch(err, kErrNllChol);
  }
}

// The same NLL term with both j x j factorisations in shared memory, side by side (2 j^2 + 3 j
// doubles of dynamic shared memory).  GB300 issues a warp-wide FP64 instruction over 16 cycles, so
// the scalar work of a pivot (square root, reciprocal) is done once per matrix, by one lane of warp 0
// (S^T G S) and one lane of warp 1 (S^T S), and broadcast through shared memory; the column scale and
// the forward substitution multiply by the stored reciprocal, and the logarithms of the pivots are
// taken in parallel.
constexpr int NLL_THREADS = 256;
__global__ void __launch_bounds__(NLL_THREADS)
k_nll_def_smem(const int* __restrict__ count, const double* __restrict__ Gh, const double* __restrict__ SS, int ld,
               const double* __restrict__ yh, double* __restrict__ nll_k, int* __restrict__ err) {
  extern __shared__ double nsm[];
  const int j = min(*count, ld);
  double* S1 = nsm;                      // S^T G S, j x j (ld j), lower triangle used
  double* S2 = nsm + (size_t)j * j;      // S^T S
  double* inv1 = S2 + (size_t)j * j;     // reciprocal pivots of S1
  double* inv2 = inv1 + j;
  double* b = inv2 + j;                  // right-hand side of the forward substitution
  __shared__ int bad;
  __shared__ double red[NLL_THREADS / 32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  if (threadIdx.x == 0) bad = 0;
  for (int e = threadIdx.x; e < j * j; e += blockDim.x) {
    const int r = e % j, c = e / j;
    if (r >= c) {
      S1[c * j + r] = (r == c) ? Gh[(size_t)c * ld + r] : 0.5 * (Gh[(size_t)c * ld + r] + Gh[(size_t)r * ld + c]);
      S2[c * j + r] = (r == c) ? SS[(size_t)c * ld + r] : 0.5 * (SS[(size_t)c * ld + r] + SS[(size_t)r * ld + c]);
    }
  }
  for (int q = threadIdx.x; q < j; q += blockDim.x) b[q] = yh[q];
  __syncthreads();
  for (int p = 0; p < j; ++p) {
    if (lane == 0 && warp < 2) {
      double* S = warp == 0 ? S1 : S2;
      double d = S[p * j + p];
      if (!(d > 0.0) || !isfinite(d)) { bad = 1; d = 1.0; }
      const double piv = sqrt(d);
      S[p * j + p] = piv;
      (warp == 0 ? inv1 : inv2)[p] = 1.0 / piv;
    }
    __syncthreads();
    const double i1 = inv1[p], i2 = inv2[p];
    for (int q = p + 1 + threadIdx.x; q < j; q += blockDim.x) {
      S1[p * j + q] *= i1;
      S2[p * j + q] *= i2;
    }
    __syncthreads();
    // trailing updates: warps take the columns c of both matrices round robin, lanes the rows q >= c
    const int w = j - p - 1;
    for (int cc = warp; cc < 2 * w; cc += nw) {
      double* S = cc < w ? S1 : S2;
      const int c = p + 1 + (cc < w ? cc : cc - w);
      const double* lp = S + p * j;
      const double lc = lp[c];
      double* col = S + c * j;
      for (int q = c + lane; q < j; q += 32) col[q] = fma(-lp[q], lc, col[q]);
    }
    __syncthreads();
  }
  // L z = yh for the factor of S^T G S (column oriented)
  double quad = 0.0;
  for (int q = 0; q < j; ++q) {
    const double zq = b[q] * inv1[q];
    quad = fma(zq, zq, quad);
    for (int l = q + 1 + threadIdx.x; l < j; l += blockDim.x) b[l] = fma(-S1[q * j + l], zq, b[l]);
    __syncthreads();
  }
  // sum_q log L1_qq - sum_q log L2_qq, logarithms in parallel
  double lg = 0.0;
  for (int q = threadIdx.x; q < j; q += blockDim.x) lg += log(S1[q * j + q]) - log(S2[q * j + q]);
  lg = warp_sum(lg);
  if (lane == 0) red[warp] = lg;
  __syncthreads();
  if (threadIdx.x == 0) {
    double ldiff = 0.0;
    for (int w2 = 0; w2 < nw; ++w2) ldiff += red[w2];
    const double val = 0.5 * j * 1.8378770664093453 + ldiff + 0.5 * quad;
    *nll_k = val;
    if (bad || !isfinite(val)) atomicExch(err, kErrNllChol);
  }
}

__global__ void k_set_diag(double* __restrict__ G, int ld, const double* __restrict__ lam, double scale, int r) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < r) G[(size_t)i * ld + i] = scale * lam[i];
}

// Fill the upper-right / lower-left border of the truncation Gram from an r x i block B (double)
__global__ void k_put_block_sym(double* __restrict__ G, int ld, int row0, int col0, const double* __restrict__ B,
                                int ldb, int nr, int nc, double scale) {
  int a = blockIdx.x * blockDim.x + threadIdx.x;
  int b = blockIdx.y;
  if (a >= nr || b >= nc) return;
  double v = scale * B[(size_t)b * ldb + a];
  G[(size_t)(col0 + b) * ld + row0 + a] = v;
  G[(size_t)(row0 + a) * ld + col0 + b] = v;
}

__global__ void k_check_finite(const double* __restrict__ x, size_t n, int* __restrict__ err) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && !isfinite(x[i])) atomicExch(err, kErrNonFinite);
}


__global__ void k_scale_f64(double* __restrict__ A, int ld, int rows, int cols, double s) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int c = blockIdx.y;
  if (i < rows && c < cols) A[(size_t)c * ld + i] *= s;
}

template <class T>
__global__ void k_convert_from_f64(const double* __restrict__ In, int ldi, int rows, int cols, T* __restrict__ Out,
                                   int ldo) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int c = blockIdx.y;
  if (i < rows && c < cols) Out[(size_t)c * ldo + i] = T(In[(size_t)c * ldi + i]);
}

// ------------------------------------------------------------------------------------------
// Host-side launchers
static inline unsigned cdiv(size_t a, size_t b) { return unsigned((a + b - 1) / b); }

template <class T>
void prep_coords(const double* X, int n, int dim, double scale, C4<T>* out, cudaStream_t st) {
  if (n <= 0) return;
  k_prep_coords<T><<<cdiv(n, 256), 256, 0, st>>>(X, n, dim, scale, out); note_launch();
}
template <class T>
void gather_coords(const C4<T>* X, const int* idx, int m, C4<T>* out, cudaStream_t st) {
  if (m <= 0) return;
  k_gather_coords<T><<<cdiv(m, 256), 256, 0, st>>>(X, idx, m, out); note_launch();
}

int gram_matvec_slots(int m) { return std::max(1, (m + MVS_T - 1) / MVS_T); }

template <class T>
void gram_matvec(int ker, const C4<T>* Xo, const T* s, int m, T sf2, T* part, const T* Mo, int ldm, int rp, T* tpart,
                 const int* active, cudaStream_t st) {
  if (m <= 0) return;
  const int nb = gram_matvec_slots(m);
  const int ngv = rp > 0 ? (int)cdiv(m, GV_CHUNK) * (int)cdiv(rp, MVS_W) : 0;
  const int grid = ngv + nb * (nb + 1) / 2;
  if constexpr (sizeof(T) == 4) {
    switch (ker) {
      case 0: launch_pdl(k_gram_matvec_f2<0>, dim3(grid), dim3(MVS_W * 32), 0, st, Xo, s, m, nb, sf2, part, Mo, ldm, rp, ngv, tpart, active); break;
      case 1: launch_pdl(k_gram_matvec_f2<1>, dim3(grid), dim3(MVS_W * 32), 0, st, Xo, s, m, nb, sf2, part, Mo, ldm, rp, ngv, tpart, active); break;
      default: launch_pdl(k_gram_matvec_f2<2>, dim3(grid), dim3(MVS_W * 32), 0, st, Xo, s, m, nb, sf2, part, Mo, ldm, rp, ngv, tpart, active); break;
    }
  } else {
    switch (ker) {
      case 0: launch_pdl(k_gram_matvec<0, T>, dim3(grid), dim3(MVS_W * 32), 0, st, Xo, s, m, nb, sf2, part, Mo, ldm, rp, ngv, tpart, active); break;
      case 1: launch_pdl(k_gram_matvec<1, T>, dim3(grid), dim3(MVS_W * 32), 0, st, Xo, s, m, nb, sf2, part, Mo, ldm, rp, ngv, tpart, active); break;
      default: launch_pdl(k_gram_matvec<2, T>, dim3(grid), dim3(MVS_W * 32), 0, st, Xo, s, m, nb, sf2, part, Mo, ldm, rp, ngv, tpart, active); break;
    }
  }
}

template <class T>
void gram_block_simt(int ker, const C4<T>* Xr, int nr, const C4<T>* Xc, int nc, const T* B, int ldb, int width,
                     T sf2, T* Out, int ldo, cudaStream_t st) {
  if (nr <= 0 || width <= 0) return;
  dim3 grid(cdiv(nr, GB_BM), cdiv(width, GB_BN));
  switch (ker) {
    case 0: k_gram_block_simt<0, T><<<grid, GB_THREADS, 0, st>>>(Xr, nr, Xc, nc, B, ldb, width, sf2, Out, ldo); note_launch(); break;
    case 1: k_gram_block_simt<1, T><<<grid, GB_THREADS, 0, st>>>(Xr, nr, Xc, nc, B, ldb, width, sf2, Out, ldo); note_launch(); break;
    default: k_gram_block_simt<2, T><<<grid, GB_THREADS, 0, st>>>(Xr, nr, Xc, nc, B, ldb, width, sf2, Out, ldo); note_launch(); break;
  }
}

// Out = dK/dlog(l_x) (Xr, Xc) B  (the derivative Gram matrix, never stored)
template <class T>
void gram_block_dlogl_simt(int ker, const C4<T>* Xr, int nr, const C4<T>* Xc, int nc, const T* B, int ldb, int width,
                           T sf2, T* Out, int ldo, cudaStream_t st) {
  if (nr <= 0 || width <= 0) return;
  dim3 grid(cdiv(nr, GB_BM), cdiv(width, GB_BN));
  switch (ker) {
    case 0: k_gram_block_simt<0, T, true><<<grid, GB_THREADS, 0, st>>>(Xr, nr, Xc, nc, B, ldb, width, sf2, Out, ldo); note_launch(); break;
    case 1: k_gram_block_simt<1, T, true><<<grid, GB_THREADS, 0, st>>>(Xr, nr, Xc, nc, B, ldb, width, sf2, Out, ldo); note_launch(); break;
    default: k_gram_block_simt<2, T, true><<<grid, GB_THREADS, 0, st>>>(Xr, nr, Xc, nc, B, ldb, width, sf2, Out, ldo); note_launch(); break;
  }
}

template <class T>
void cg_combine(const T* part, int nsplit, const T* s, T sn2, const T* Mo, int ldm, int r, const T* t, T a2, int m,
                T* g, const T* V, int ldv, int j, const T* r0, const T* v, T* dpart1, const int* active,
                cudaStream_t st) {
  const int tz = std::max(1, (m + GV_CHUNK - 1) / GV_CHUNK);
  launch_pdl(k_cg_combine<T>, dim3(cdiv(m, CB_ROWS)), dim3(CB_WARPS * 32), std::max(r, 1) * sizeof(T), st, 
      part, nsplit, s, sn2, Mo, ldm, r, t, tz, a2, m, g, V, ldv, j, r0, v, dpart1, active);
}
size_t cg_dpart_elems(int m, int budget) {
  return (size_t)(budget + 4) * cdiv(std::max(m, 1), CB_ROWS) + (size_t)(budget + 1) * cdiv(std::max(m, 1), UP_ROWS);
}
template <class T>
void cg_upd1(int j, const T* dpart1, double* dots1, T* V, T* GV, int ldv, const T* s, const T* g, int m,
             T* dpart2, const int* active, cudaStream_t st) {
  launch_pdl(k_cg_upd1<T>, dim3(cdiv(m, UP_ROWS)), dim3(UP_THREADS), 0, st, j, dpart1, (int)cdiv(m, CB_ROWS), dots1, V, GV, ldv, s, g, m,
                                                        dpart2, active);
}
template <class T>
void cg_upd2(int j, const double* dots1, const T* dpart2, T* V, T* GV, int ldv, T* r, T* v, T* s, T* Q,
             int m, double bd_tol, double rtol2_r0sq, int use_rtol, int* active, double* eta, double* alpha,
             int* count, T* Snext, cudaStream_t st) {
  launch_pdl(k_cg_upd2<T>, dim3(cdiv(m, UP_ROWS)), dim3(UP_THREADS), 0, st, j, dots1, dpart2, (int)cdiv(m, UP_ROWS), V, GV, ldv, r, v,
                                                        s, Q, m, bd_tol, rtol2_r0sq, use_rtol, active, eta, alpha,
                                                        count, Snext);
}
template <class T>
void cg_reorth(const T* Q, int ldq, int j, T* s, int m, double* qd, T* S, int lds, const int* active, cudaStream_t st) {
  // two classical Gram-Schmidt passes against the previous (orthonormal) action basis
  for (int pass = 0; pass < 2; ++pass) {
    if (j > 0) {
      launch_pdl(k_cg_qdots<T>, dim3(j), dim3(256), 0, st, Q, ldq, j, s, m, qd, active);
    }
    launch_pdl(k_cg_qorth<T>, dim3(cdiv(m, 256)), dim3(256), 0, st, Q, ldq, j, qd, s, m, pass == 1 ? S : nullptr, lds, active);
  }
}
template <class T>
void cg_select(int j, const T* r, const double* rep, int m, T* s, T* S, int lds, const int* active, cudaStream_t st) {
  launch_pdl(k_cg_select<T>, dim3(cdiv(m, 256)), dim3(256), 0, st, j, r, rep, m, s, S, lds, active);
}
template <class T>
void cg_init(const double* y, const double* mpred, const int* obs, int m, T* r, T* r0, T* v, double* r0sq,
             cudaStream_t st) {
  k_cg_init<T><<<cdiv(m, 256), 256, 0, st>>>(y, mpred, obs, m, r, r0, v, r0sq); note_launch();
}

__global__ void k_axpby_f32_f64(const float* __restrict__ X, int ldx, int rows, int cols, double alpha, double beta,
                                double* __restrict__ C, int ldc) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int c = blockIdx.y;
  if (i >= rows || c >= cols) return;
  double* p = C + (size_t)c * ldc + i;
  *p = alpha * double(X[(size_t)c * ldx + i]) + (beta != 0.0 ? beta * *p : 0.0);
}

// FP32 <-> BF16 (round to nearest even) copies of column-major blocks, for the BF16 factor store
__global__ void k_to_bf16(const float* __restrict__ In, int ldi, int rows, int cols, uint16_t* __restrict__ Out,
                          int ldo) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int c = blockIdx.y;
  if (i >= rows || c >= cols) return;
  const __nv_bfloat16 b = __float2bfloat16_rn(In[(size_t)c * ldi + i]);
  Out[(size_t)c * ldo + i] = *reinterpret_cast<const uint16_t*>(&b);
}
__global__ void k_from_bf16(const uint16_t* __restrict__ In, int ldi, int rows, int cols, float* __restrict__ Out,
                            int ldo) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int c = blockIdx.y;
  if (i >= rows || c >= cols) return;
  Out[(size_t)c * ldo + i] = __uint_as_float((uint32_t)In[(size_t)c * ldi + i] << 16);
}
void to_bf16(const float* In, int ldi, int rows, int cols, uint16_t* Out, int ldo, cudaStream_t st) {
  if (rows <= 0 || cols <= 0) return;
  k_to_bf16<<<dim3(cdiv(rows, 256), cols), 256, 0, st>>>(In, ldi, rows, cols, Out, ldo); note_launch();
}
void from_bf16(const uint16_t* In, int ldi, int rows, int cols, float* Out, int ldo, cudaStream_t st) {
  if (rows <= 0 || cols <= 0) return;
  k_from_bf16<<<dim3(cdiv(rows, 256), cols), 256, 0, st>>>(In, ldi, rows, cols, Out, ldo); note_launch();
}

void convert_to_f64(const float* In, int ldi, int rows, int cols, double* Out, int ldo, cudaStream_t st) {
  if (rows <= 0 || cols <= 0) return;
  k_axpby_f32_f64<<<dim3(cdiv(rows, 256), cols), 256, 0, st>>>(In, ldi, rows, cols, 1.0, 0.0, Out, ldo); note_launch();
}

template <class T>
void gemm_tn(const T* A, int lda, int na, const T* B, int ldb, int nb, int K, double alpha, double beta, double* C,
             int ldc, double* part, size_t part_elems, cudaStream_t st) {
  if (na <= 0 || nb <= 0) return;
  if (sizeof(T) == 4 && t_gemm_mode == 2 && (double)na * nb * K > 2e7 && K >= 64) {
    // FP32 operands on the tensor cores (split TF32), FP32 partial tiles summed in FP64
    if (gemm_tc_tn((const float*)A, lda, na, (const float*)B, ldb, nb, K, alpha, beta, C, ldc, part,
                   part_elems * sizeof(double), t_gemm_err, st) == 0)
      return;
    cudaGetLastError();
  }
  const size_t tile_elems = (size_t)na * nb;
  int gx = cdiv(na, TN_T), gy = cdiv(nb, TN_T);
  int want = std::max(1, (int)(4 * 152 / std::max(1, gx * gy)));
  int chunk_min = 256;
  int nsplit = std::max(1, std::min(want, (K + chunk_min - 1) / chunk_min));
  nsplit = std::max(1, std::min<int>(nsplit, (int)(part_elems / tile_elems)));
  int chunk = (K + nsplit - 1) / nsplit;
  chunk = ((chunk + TN_K - 1) / TN_K) * TN_K;
  nsplit = std::max(1, (K + chunk - 1) / chunk);
  if (K <= 0) { nsplit = 1; chunk = TN_K; }
  k_gemm_tn_part<T><<<dim3(gx, gy, nsplit), 256, 0, st>>>(A, lda, na, B, ldb, nb, std::max(K, 0), chunk, part); note_launch();
  k_reduce_splits<double><<<cdiv(tile_elems, 256), 256, 0, st>>>(part, nsplit, na, nb, alpha, beta, C, ldc); note_launch();
}

// FP32 copy of a small double coefficient block for the tensor-core path (device scratch per host
// thread and current device)
static thread_local float* t_bscratch = nullptr;
static thread_local size_t t_bscratch_elems = 0;
static thread_local int t_bscratch_dev = -1;
static float* bscratch(size_t elems) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return nullptr; }
  if (dev != t_bscratch_dev) {        // a buffer of another device is not reachable from this one
    if (t_bscratch) cudaFree(t_bscratch);
    t_bscratch = nullptr;
    t_bscratch_elems = 0;
    t_bscratch_dev = dev;
  }
  if (elems > t_bscratch_elems) {
    if (t_bscratch) cudaFree(t_bscratch);
    t_bscratch = nullptr;
    t_bscratch_elems = 0;
    if (cudaMalloc(&t_bscratch, elems * sizeof(float)) != cudaSuccess) { cudaGetLastError(); return nullptr; }
    t_bscratch_elems = elems;
  }
  return t_bscratch;
}

template <class T, class TB>
void gemm_nn(int M, int N, int K, T alpha, const T* A, int lda, const TB* B, int ldb, T beta, T* C, int ldc,
             cudaStream_t st) {
  if (M <= 0 || N <= 0) return;
  if (K <= 0) {
    if (beta == T(1)) return;
  }
  if (sizeof(T) == 4 && t_gemm_mode == 2 && K >= 16 && M >= 4096 && (double)M * N * K > 2e7) {
    // tall factor times a small coefficient block on the tensor cores (split TF32)
    const float* Bf = reinterpret_cast<const float*>(B);
    int ldbf = ldb;
    if (sizeof(TB) == 8) {
      float* sb = bscratch((size_t)K * N);
      if (sb) {
        convert_from_f64<float>(reinterpret_cast<const double*>(B), ldb, K, N, sb, K, st);
        Bf = sb;
        ldbf = K;
      } else {
        Bf = nullptr;
      }
    }
    if (Bf && gemm_tc_nn(M, N, K, (float)alpha, (const float*)A, lda, Bf, ldbf, (float)beta, (float*)C, ldc,
                         t_gemm_err, st) == 0)
      return;
    cudaGetLastError();
  }
  k_gemm_nn<T, TB><<<dim3(cdiv(M, NN_BM), cdiv(N, NN_BN)), 256, 0, st>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc); note_launch();
}

void gemm_small_f64(int ta, int tb, int M, int N, int K, double alpha, const double* A, int lda, const double* B,
                    int ldb, double beta, double* C, int ldc, cudaStream_t st) {
  if (M <= 0 || N <= 0) return;
  k_gemm_small_f64<<<dim3(cdiv(M, 16), cdiv(N, 16)), 256, 0, st>>>(ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc); note_launch();
}

template <class T>
void gather_rows(const T* In, int ldi, const int* idx, int m, int cols, T* Out, int ldo, cudaStream_t st) {
  if (m <= 0 || cols <= 0) return;
  k_gather_rows<T><<<dim3(cdiv(m, 256), cols), 256, 0, st>>>(In, ldi, idx, m, cols, Out, ldo); note_launch();
}
template <class T>
void scatter_add_rows(const T* In, int ldi, const int* idx, int m, int cols, T alpha, T* Out, int ldo, cudaStream_t st) {
  if (m <= 0 || cols <= 0) return;
  k_scatter_add_rows<T><<<dim3(cdiv(m, 256), cols), 256, 0, st>>>(In, ldi, idx, m, cols, alpha, Out, ldo); note_launch();
}
template <class T>
void rowsumsq(const T* A, int lda, int n, int cols, double beta, double* rs, cudaStream_t st) {
  k_rowsumsq<T><<<cdiv(n, 256), 256, 0, st>>>(A, lda, n, cols, beta, rs); note_launch();
}
void predict_mean(const double* mprev, const double* mu_k, const double* mu_km1, double a, int n, double* mpred,
                  cudaStream_t st) {
  k_predict_mean<<<cdiv(n, 256), 256, 0, st>>>(mprev, mu_k, mu_km1, a, n, mpred); note_launch();
}
template <class T>
void mix2(const T* In, int ldi, T* Out, int ldo, int half, int cols, const double C[4], cudaStream_t st) {
  if (half <= 0 || cols <= 0) return;
  k_mix2<T><<<dim3(cdiv(half, 256), cols), 256, 0, st>>>(In, ldi, Out, ldo, half, cols, T(C[0]), T(C[1]), T(C[2]),
                                                         T(C[3])); note_launch();
}
void predict_mean2(const double* mprev, const double* mu_k, const double* mu_km1, const double A[4], int n, int half,
                   double* mpred, cudaStream_t st) {
  k_predict_mean2<<<cdiv(n, 256), 256, 0, st>>>(mprev, mu_k, mu_km1, A[0], A[1], A[2], A[3], n, half, mpred);
  note_launch();
}
template <class T>
void add_vec(const double* a, const T* b, int n, double* out, cudaStream_t st) {
  if (n <= 0) return;
  k_add_vec<T><<<cdiv(n, 256), 256, 0, st>>>(a, b, n, out); note_launch();
}
template <class T>
void filter_out(const double* mpred, const T* PVv, int ld, int ic, double sf2, double a2, const double* rs_plus, int n,
                double* mout, double* vout, double* rs_pw, cudaStream_t st) {
  k_filter_out<T><<<cdiv(n, 256), 256, 0, st>>>(mpred, PVv, ld, ic, sf2, a2, rs_plus, n, mout, vout, rs_pw); note_launch();
}
template <class T>
void scale_copy(const T* In, int ldi, int n, int cols, T alpha, T* Out, int ldo, cudaStream_t st) {
  if (n <= 0 || cols <= 0) return;
  k_scale_copy<T><<<dim3(cdiv(n, 256), cols), 256, 0, st>>>(In, ldi, n, cols, alpha, Out, ldo); note_launch();
}
template <class T>
void smooth_out(const double* mk, const double* vk, const T* Y, int ld, int cw, int n, double* ms, double* vs,
                cudaStream_t st) {
  k_smooth_out<T><<<cdiv(n, 256), 256, 0, st>>>(mk, vk, Y, ld, cw, n, ms, vs); note_launch();
}
template <class T>
void ws_obs(const int* obs, int m, const T* vk, const T* Vz, T* ws, cudaStream_t st) {
  if (m <= 0) return;
  k_ws_obs<T><<<cdiv(m, 256), 256, 0, st>>>(obs, m, vk, Vz, ws); note_launch();
}
template <class T>
void build_x(const T* Ws, int ldw, int cw, const T* ws, T alpha, int n, T* X, int ldx, cudaStream_t st) {
  k_build_x<T><<<dim3(cdiv(n, 256), cw + 1), 256, 0, st>>>(Ws, ldw, cw, ws, alpha, n, X, ldx); note_launch();
}
void nll_step(const double* eta, const double* alpha, const int* count, double* SS, int ic, double* nll_k, int* err,
              cudaStream_t st) {
  k_nll_step<<<1, 256, 0, st>>>(eta, alpha, count, SS, ic, nll_k, err); note_launch();
}
void grad_small(int ic, int np, const double* Gh, const double* dGh, const double* yh, const double* dyh, double* L,
                double* Rinv, double* W, double* tmp, double* Q, double* u, double* grad, int* err, cudaStream_t st) {
  k_grad_small<<<1, 256, 0, st>>>(ic, np, Gh, dGh, yh, dyh, L, Rinv, W, tmp, Q, u, grad, err); note_launch();
}
template <class T>
void gather_rows_f64(const double* In, int ld, const int* idx, int m, int cols, T* Out, int ldo, cudaStream_t st) {
  if (m <= 0 || cols <= 0) return;
  k_gather_rows_f64<T><<<dim3(cdiv(m, 256), cols), 256, 0, st>>>(In, ld, idx, m, cols, Out, ldo); note_launch();
}
template <class T>
void tangent_mean(const double* dmpred, const T* E, size_t estride, int ecol, int lde, const T* t, int ldt, int n,
                  int np, double* dm, cudaStream_t st) {
  k_tangent_mean<T><<<dim3(cdiv(n, 256), np), 256, 0, st>>>(dmpred, E, estride, ecol, lde, t, ldt, n, np, dm);
  note_launch();
}
void tangent_predict(const double* mprev, const double* dmprev, const double* mu_km1, double a, double adot_lt, int n,
                     int np, double* dmpred, cudaStream_t st) {
  k_tangent_predict<<<dim3(cdiv(n, 256), np), 256, 0, st>>>(mprev, dmprev, mu_km1, a, adot_lt, n, np, dmpred);
  note_launch();
}
template <class T>
void axpy_block(T alpha, const T* X, int ldx, int rows, int cols, T* Y, int ldy, cudaStream_t st) {
  if (rows <= 0 || cols <= 0) return;
  k_axpy_block<T><<<dim3(cdiv(rows, 256), cols), 256, 0, st>>>(alpha, X, ldx, rows, cols, Y, ldy); note_launch();
}
template <class T>
void scale_cols(T* A, int ld, int rows, int cols, T s, cudaStream_t st) {
  if (rows <= 0 || cols <= 0) return;
  k_scale_cols<T><<<dim3(cdiv(rows, 256), cols), 256, 0, st>>>(A, ld, rows, cols, s); note_launch();
}
template void axpy_block<float>(float, const float*, int, int, int, float*, int, cudaStream_t);
template void axpy_block<double>(double, const double*, int, int, int, double*, int, cudaStream_t);
template void scale_cols<float>(float*, int, int, int, float, cudaStream_t);
template void scale_cols<double>(double*, int, int, int, double, cudaStream_t);
template void gather_rows_f64<float>(const double*, int, const int*, int, int, float*, int, cudaStream_t);
template void gather_rows_f64<double>(const double*, int, const int*, int, int, double*, int, cudaStream_t);
template void tangent_mean<float>(const double*, const float*, size_t, int, int, const float*, int, int, int, double*,
                                  cudaStream_t);
template void tangent_mean<double>(const double*, const double*, size_t, int, int, const double*, int, int, int,
                                   double*, cudaStream_t);

void nll_def(const int* count, double* Gh, double* SS, int ld, const double* yh, double* z, double* nll_k, int* err,
             cudaStream_t st) {
  const size_t smem = (2 * (size_t)ld * ld + 3 * (size_t)ld) * sizeof(double);
  if (smem <= 200 * 1024) {
    if (smem > 40 * 1024) cudaFuncSetAttribute(k_nll_def_smem, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_nll_def_smem<<<1, NLL_THREADS, smem, st>>>(count, Gh, SS, ld, yh, nll_k, err); note_launch();
    return;
  }
  k_nll_def<<<1, 256, 0, st>>>(count, Gh, SS, ld, yh, z, nll_k, err); note_launch();
}

// ------------------------------------------------------------------------------------------
// Batch update (Alg. 2) helpers: the actions S are fixed up front, Ghat = S^T G S = L L^T,
// W = H^T S L^-T, w = H^T S Ghat^-1 S^T r0.

// Coordinate actions (reading R18 of the oracle): S = 0 except S[floor((q + 1/2) m / i), q] = 1.
template <class T>
__global__ void k_coord_actions(int m, int i, T* __restrict__ S) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= i) return;
  const int row = (int)(((double)q + 0.5) * (double)m / (double)i);
  S[(size_t)q * m + min(row, m - 1)] = T(1);
}

// Cholesky Ghat = L L^T (FP64, i x i, lower triangle of Ghat read symmetrised; L in shared memory,
// written to Lout with ld i) and z = L^-1 yh.  One block.  A non-positive or non-finite pivot
// raises the numeric error flag (the step's projected Gram must be positive definite).
constexpr int BCH_THREADS = 256;
__global__ void __launch_bounds__(BCH_THREADS)
k_batch_chol(const double* __restrict__ Gh, int i, const double* __restrict__ yh, double* __restrict__ Lout,
             double* __restrict__ z, double* __restrict__ eta, int* __restrict__ err) {
  extern __shared__ double bsm[];
  double* L = bsm;                  // i x i, column-major
  double* zz = bsm + (size_t)i * i;
  __shared__ double piv;
  __shared__ int bad;
  if (threadIdx.x == 0) bad = 0;
  for (int e = threadIdx.x; e < i * i; e += blockDim.x) {
    const int r = e % i, c = e / i;
    L[e] = r >= c ? 0.5 * (Gh[(size_t)c * i + r] + Gh[(size_t)r * i + c]) : 0.0;
  }
  for (int q = threadIdx.x; q < i; q += blockDim.x) zz[q] = yh[q];
  __syncthreads();
  for (int p = 0; p < i; ++p) {
    if (threadIdx.x == 0) {
      double d = L[(size_t)p * i + p];
      if (eta) eta[p] = d;            // the pivot: eta_j of the iterative form (S^T G S = U^-T diag(eta) U^-1)
      if (!(d > 0.0) || !isfinite(d)) { bad = 1; d = 1.0; }
      piv = sqrt(d);
      L[(size_t)p * i + p] = piv;
      zz[p] /= piv;
    }
    __syncthreads();
    const double ip = 1.0 / piv, zp = zz[p];
    for (int q = p + 1 + threadIdx.x; q < i; q += blockDim.x) {
      const double lq = L[(size_t)p * i + q] * ip;
      L[(size_t)p * i + q] = lq;
      zz[q] -= lq * zp;
    }
    __syncthreads();
    // trailing update of the lower triangle: column c, rows q >= c
    const int w = i - p - 1;
    for (int e = threadIdx.x; e < w * w; e += blockDim.x) {
      const int c = p + 1 + e / w, q = p + 1 + e % w;
      if (q >= c) L[(size_t)c * i + q] -= L[(size_t)p * i + q] * L[(size_t)p * i + c];
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < i * i; e += blockDim.x) Lout[e] = L[e];
  for (int q = threadIdx.x; q < i; q += blockDim.x) z[q] = zz[q];
  if (threadIdx.x == 0 && bad) atomicExch(err, kErrBatchChol);
}

// V = S L^-T (row by row: x L^T = s, forward substitution in FP64) into columns 0..i-1 of Vv, and
// v = V z into column i.  One thread per row of S.
template <class T>
__global__ void k_batch_v(const T* __restrict__ S, int m, int i, const double* __restrict__ L,
                          const double* __restrict__ z, T* __restrict__ Vv) {
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= m) return;
  double x[160];
  double v = 0.0;
  for (int j = 0; j < i; ++j) {
    double acc = (double)S[(size_t)j * m + row];
    for (int l = 0; l < j; ++l) acc = fma(-x[l], L[(size_t)l * i + j], acc);
    x[j] = acc / L[(size_t)j * i + j];
    Vv[(size_t)j * m + row] = T(x[j]);
    v = fma(x[j], z[j], v);
  }
  Vv[(size_t)i * m + row] = T(v);
}

template <class T>
void coord_actions(int m, int i, T* S, cudaStream_t st) {
  if (m <= 0 || i <= 0) return;
  cudaMemsetAsync(S, 0, (size_t)m * i * sizeof(T), st);
  k_coord_actions<T><<<cdiv(i, 128), 128, 0, st>>>(m, i, S); note_launch();
}
int batch_chol(const double* Gh, int i, const double* yh, double* L, double* z, double* eta, int* err,
               cudaStream_t st) {
  if (i <= 0) return 0;
  if (i > kBatchMaxActions) return 1;
  const size_t smem = ((size_t)i * i + i) * sizeof(double);
  if (smem > 48 * 1024) cudaFuncSetAttribute(k_batch_chol, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_batch_chol<<<1, BCH_THREADS, smem, st>>>(Gh, i, yh, L, z, eta, err); note_launch();
  return 0;
}
template <class T>
void batch_v(const T* S, int m, int i, const double* L, const double* z, T* Vv, cudaStream_t st) {
  if (m <= 0 || i <= 0) return;
  k_batch_v<T><<<cdiv(m, 128), 128, 0, st>>>(S, m, i, L, z, Vv); note_launch();
}
template void coord_actions<float>(int, int, float*, cudaStream_t);
template void coord_actions<double>(int, int, double*, cudaStream_t);
template void batch_v<float>(const float*, int, int, const double*, const double*, float*, cudaStream_t);
template void batch_v<double>(const double*, int, int, const double*, const double*, double*, cudaStream_t);

// ------------------------------------------------------------------------------------------
// Per-step diagnostics: the squared norm of a vector (the final residual of a step's update), the
// trace of the truncation Gram before the eigensolver and the discarded mass after it.
template <class T>
__global__ void k_sqnorm(const T* __restrict__ x, int m, double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const double v = i < m ? (double)x[i] : 0.0;
  const double s = block_sum(v * v);
  if (threadIdx.x == 0) atomicAdd(out, s);
}
__global__ void k_trace(const double* __restrict__ G, int N, int ld, double* __restrict__ out) {
  double acc = 0.0;
  for (int i = threadIdx.x; i < N; i += blockDim.x) acc += G[(size_t)i * ld + i];
  acc = block_sum(acc);
  if (threadIdx.x == 0) *out = acc;
}
__global__ void k_sub_sum(const double* __restrict__ w, int keep, double* __restrict__ out) {
  double acc = 0.0;
  for (int i = threadIdx.x; i < keep; i += blockDim.x) acc += w[i];
  acc = block_sum(acc);
  if (threadIdx.x == 0) *out -= acc;
}
// r_final = r0 - (G S) L^-T z for the batch update: squared norm accumulated into out
template <class T>
__global__ void k_batch_resid(const T* __restrict__ GS, int m, int i, const double* __restrict__ L,
                              const double* __restrict__ z, const T* __restrict__ r0, double* __restrict__ out) {
  extern __shared__ double yc[];   // L^-T z, by back substitution (thread 0), shared by the block
  if (threadIdx.x == 0) {
    for (int j = i - 1; j >= 0; --j) {
      double acc = z[j];
      for (int l = j + 1; l < i; ++l) acc = fma(-L[(size_t)j * i + l], yc[l], acc);
      yc[j] = acc / L[(size_t)j * i + j];
    }
  }
  __syncthreads();
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  double r = 0.0;
  if (row < m) {
    r = (double)r0[row];
    for (int j = 0; j < i; ++j) r = fma(-(double)GS[(size_t)j * m + row], yc[j], r);
  }
  const double s = block_sum(r * r);
  if (threadIdx.x == 0) atomicAdd(out, s);
}
template <class T> void sqnorm_acc(const T* x, int m, double* out, cudaStream_t st) {
  if (m <= 0) return;
  k_sqnorm<T><<<cdiv(m, 256), 256, 0, st>>>(x, m, out); note_launch();
}
void trace_into(const double* G, int N, int ld, double* out, cudaStream_t st) {
  k_trace<<<1, 256, 0, st>>>(G, N, ld, out); note_launch();
}
void sub_sum(const double* w, int keep, double* out, cudaStream_t st) {
  k_sub_sum<<<1, 256, 0, st>>>(w, keep, out); note_launch();
}
template <class T>
void batch_resid(const T* GS, int m, int i, const double* L, const double* z, const T* r0, double* out, cudaStream_t st) {
  if (m <= 0 || i <= 0) return;
  k_batch_resid<T><<<cdiv(m, 256), 256, i * sizeof(double), st>>>(GS, m, i, L, z, r0, out); note_launch();
}
template void sqnorm_acc<float>(const float*, int, double*, cudaStream_t);
template void sqnorm_acc<double>(const double*, int, double*, cudaStream_t);
template void batch_resid<float>(const float*, int, int, const double*, const double*, const float*, double*, cudaStream_t);
template void batch_resid<double>(const double*, int, int, const double*, const double*, const double*, double*,
                                  cudaStream_t);

// ------------------------------------------------------------------------------------------
// Posterior sampler (the CAKF/CAKS sampler algorithm): S draws as the columns of n x S blocks.
// xp = a xprev + (mu_k - a mu_{k-1}) + q   (FP64; mu pointers may be null)
__global__ void k_samp_predict(const double* __restrict__ xprev, const double* __restrict__ q,
                               const double* __restrict__ mu_k, const double* __restrict__ mu_km1, double a, int n,
                               int S, double* __restrict__ xp) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int s = blockIdx.y;
  if (j >= n || s >= S) return;
  const double b = mu_k ? mu_k[j] - a * mu_km1[j] : 0.0;
  xp[(size_t)s * n + j] = fma(a, xprev[(size_t)s * n + j], b + q[(size_t)s * n + j]);
}
// d = y - xp[obs] - eps  (m x S, precision T)
template <class T>
__global__ void k_samp_resid(const double* __restrict__ y, const double* __restrict__ xp, const int* __restrict__ obs,
                             const double* __restrict__ eps, int m, int n, int S, T* __restrict__ d) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int s = blockIdx.y;
  if (i >= m || s >= S) return;
  d[(size_t)s * m + i] = T(y[i] - xp[(size_t)s * n + obs[i]] - eps[(size_t)s * m + i]);
}
// x = xa + alpha * t  (x, xa FP64 n x S with ld n; t precision T with ld ldt)
template <class T>
__global__ void k_samp_add(const double* __restrict__ xa, const T* __restrict__ t, int ldt, double alpha, int n, int S,
                           double* __restrict__ x) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int s = blockIdx.y;
  if (j >= n || s >= S) return;
  x[(size_t)s * n + j] = fma(alpha, (double)t[(size_t)s * ldt + j], xa[(size_t)s * n + j]);
}
void samp_predict(const double* xprev, const double* q, const double* mu_k, const double* mu_km1, double a, int n,
                  int S, double* xp, cudaStream_t st) {
  k_samp_predict<<<dim3(cdiv(n, 256), S), 256, 0, st>>>(xprev, q, mu_k, mu_km1, a, n, S, xp); note_launch();
}
template <class T>
void samp_resid(const double* y, const double* xp, const int* obs, const double* eps, int m, int n, int S, T* d,
                cudaStream_t st) {
  if (m <= 0) return;
  k_samp_resid<T><<<dim3(cdiv(m, 256), S), 256, 0, st>>>(y, xp, obs, eps, m, n, S, d); note_launch();
}
template <class T>
void samp_add(const double* xa, const T* t, int ldt, double alpha, int n, int S, double* x, cudaStream_t st) {
  k_samp_add<T><<<dim3(cdiv(n, 256), S), 256, 0, st>>>(xa, t, ldt, alpha, n, S, x); note_launch();
}
template void samp_resid<float>(const double*, const double*, const int*, const double*, int, int, int, float*, cudaStream_t);
template void samp_resid<double>(const double*, const double*, const int*, const double*, int, int, int, double*,
                                 cudaStream_t);
template void samp_add<float>(const double*, const float*, int, double, int, int, double*, cudaStream_t);
template void samp_add<double>(const double*, const double*, int, double, int, int, double*, cudaStream_t);

// Filter marginal at a query time t_k + tau (the interpolation corollary, OU prior): m(t) = at m_k +
// mu(t) - at mu_k, var(t) = sf2 - at^2 (sf2 - var_k).
__global__ void k_interp_filter(const double* __restrict__ mk, const double* __restrict__ vk,
                                const double* __restrict__ mu_t, const double* __restrict__ mu_k, double at,
                                double sf2, int n, double* __restrict__ m, double* __restrict__ v) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const double b = mu_t ? mu_t[j] - (mu_k ? at * mu_k[j] : 0.0) : 0.0;
  m[j] = fma(at, mk[j], b);
  v[j] = sf2 - at * at * (sf2 - vk[j]);
}
void interp_filter(const double* mk, const double* vk, const double* mu_t, const double* mu_k, double at, double sf2,
                   int n, double* m, double* v, cudaStream_t st) {
  k_interp_filter<<<cdiv(n, 256), 256, 0, st>>>(mk, vk, mu_t, mu_k, at, sf2, n, m, v); note_launch();
}

void set_diag(double* G, int ld, const double* lam, double scale, int r, cudaStream_t st) {
  if (r <= 0) return;
  k_set_diag<<<cdiv(r, 256), 256, 0, st>>>(G, ld, lam, scale, r); note_launch();
}
void put_block_sym(double* G, int ld, int row0, int col0, const double* B, int ldb, int nr, int nc, double scale,
                   cudaStream_t st) {
  if (nr <= 0 || nc <= 0) return;
  k_put_block_sym<<<dim3(cdiv(nr, 256), nc), 256, 0, st>>>(G, ld, row0, col0, B, ldb, nr, nc, scale); note_launch();
}
void scale_f64(double* A, int ld, int rows, int cols, double s, cudaStream_t st) {
  if (rows <= 0 || cols <= 0) return;
  k_scale_f64<<<dim3(cdiv(rows, 256), cols), 256, 0, st>>>(A, ld, rows, cols, s); note_launch();
}
template <class T>
void convert_from_f64(const double* In, int ldi, int rows, int cols, T* Out, int ldo, cudaStream_t st) {
  if (rows <= 0 || cols <= 0) return;
  k_convert_from_f64<T><<<dim3(cdiv(rows, 256), cols), 256, 0, st>>>(In, ldi, rows, cols, Out, ldo); note_launch();
}
template void convert_from_f64<float>(const double*, int, int, int, float*, int, cudaStream_t);
template void convert_from_f64<double>(const double*, int, int, int, double*, int, cudaStream_t);

void check_finite(const double* x, size_t n, int* err, cudaStream_t st) {
  if (n == 0) return;
  k_check_finite<<<cdiv(n, 256), 256, 0, st>>>(x, n, err); note_launch();
}

#define INST(T)                                                                                                  \
  template void prep_coords<T>(const double*, int, int, double, C4<T>*, cudaStream_t);                           \
  template void gather_coords<T>(const C4<T>*, const int*, int, C4<T>*, cudaStream_t);                          \
  template void gram_matvec<T>(int, const C4<T>*, const T*, int, T, T*, const T*, int, int, T*, const int*,     \
                               cudaStream_t);                                                                   \
  template void gram_block_simt<T>(int, const C4<T>*, int, const C4<T>*, int, const T*, int, int, T, T*, int,    \
                                   cudaStream_t);                                                                \
  template void gram_block_dlogl_simt<T>(int, const C4<T>*, int, const C4<T>*, int, const T*, int, int, T, T*,   \
                                         int, cudaStream_t);                                                     \
  template void cg_combine<T>(const T*, int, const T*, T, const T*, int, int, const T*, T, int, T*, const T*,     \
                              int, int, const T*, const T*, T*, const int*, cudaStream_t);                       \
  template void cg_upd1<T>(int, const T*, double*, T*, T*, int, const T*, const T*, int, T*,                    \
                           const int*, cudaStream_t);                                                            \
  template void cg_upd2<T>(int, const double*, const T*, T*, T*, int, T*, T*, T*, T*, int, double, double,       \
                           int, int*, double*, double*, int*, T*, cudaStream_t);                                 \
  template void cg_reorth<T>(const T*, int, int, T*, int, double*, T*, int, const int*, cudaStream_t);          \
  template void cg_select<T>(int, const T*, const double*, int, T*, T*, int, const int*, cudaStream_t);          \
  template void cg_init<T>(const double*, const double*, const int*, int, T*, T*, T*, double*, cudaStream_t);    \
  template void gemm_tn<T>(const T*, int, int, const T*, int, int, int, double, double, double*, int, double*,   \
                           size_t, cudaStream_t);                                                                \
  template void gemm_nn<T, T>(int, int, int, T, const T*, int, const T*, int, T, T*, int, cudaStream_t);         \
  template void gather_rows<T>(const T*, int, const int*, int, int, T*, int, cudaStream_t);                      \
  template void scatter_add_rows<T>(const T*, int, const int*, int, int, T, T*, int, cudaStream_t);              \
  template void rowsumsq<T>(const T*, int, int, int, double, double*, cudaStream_t);                             \
  template void filter_out<T>(const double*, const T*, int, int, double, double, const double*, int, double*,   \
                              double*, double*, cudaStream_t);                                                   \
  template void scale_copy<T>(const T*, int, int, int, T, T*, int, cudaStream_t);                                \
  template void smooth_out<T>(const double*, const double*, const T*, int, int, int, double*, double*,           \
                              cudaStream_t);                                                                     \
  template void ws_obs<T>(const int*, int, const T*, const T*, T*, cudaStream_t);                                \
  template void build_x<T>(const T*, int, int, const T*, T, int, T*, int, cudaStream_t);                        \
  template void mix2<T>(const T*, int, T*, int, int, int, const double*, cudaStream_t);                          \
  template void add_vec<T>(const double*, const T*, int, double*, cudaStream_t);

INST(float)
INST(double)
template void gemm_nn<float, double>(int, int, int, float, const float*, int, const double*, int, float, float*, int,
                                     cudaStream_t);

}  // namespace cakf
