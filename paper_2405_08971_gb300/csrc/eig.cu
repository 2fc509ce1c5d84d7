// FP64 symmetric eigensolver for the truncation step (Truncate, Sec. 3.2: the top-r eigen-directions
// of the (r+i) x (r+i) Gram of the downdate factor).
//
//   1. Householder tridiagonalisation, one cooperative kernel; the blocks exchange each column's
//      matvec and pivot column through epoch-tagged words (no grid barrier), with bounded polling.
//   2. Divide and conquer on the tridiagonal (Cuppen's tearing; deflation of small z components and
//      close poles by Givens rotations; secular roots by a two-pole rational model guarded by
//      bisection; eigenvectors from the Loewner-corrected z (Gu-Eisenstat), which keeps them
//      orthogonal without re-orthogonalisation).
//   3. Back-transformation of the wanted columns through the Householder reflectors.
// All arithmetic is FP64; only the final eigenvector block is stored in the caller's precision.
#include <vector>
#include <map>
#include <mutex>
#include "internal.h"

namespace cakf {

namespace {

constexpr double kEps = 2.220446049250313e-16;

// Reciprocal by Newton-Raphson: an FP32 seed (rcp.approx, ~2^-23 relative) refined by two FP64
// Newton steps r <- r + r (1 - x r), which square the relative error each time (2^-46, 2^-92), so
// the result is accurate to the last bit or two of FP64.  Falls back to division outside the FP32
// exponent range.
__device__ __forceinline__ double nr_rcp(double x) {
  const float xf = (float)x;
  const float ax = fabsf(xf);
  if (!(ax > 1e-36f && ax < 1e36f)) return 1.0 / x;
  float rf;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(rf) : "f"(xf));
  double r = (double)rf;
  r = fma(r, fma(-x, r, 1.0), r);
  r = fma(r, fma(-x, r, 1.0), r);
  return r;
}

// Per-step exchange without a grid barrier: every word a block publishes for step k carries the
// step's epoch (k mod 4), and the consumers poll the words themselves until all carry the epoch they
// wait for.  A value x travels as a pair of 8-byte words: hi is the bit pattern of x with its two
// lowest bits replaced by the epoch, lo holds those two original bits in bits 0-1 and the epoch in
// bits 2-3.  The reader accepts the pair when both epochs match and rebuilds x bit for bit from hi
// and lo with integer operations (no FP64 arithmetic, nothing lost).  Each 8-byte word is written
// and read as one access, so a reader sees either the old or the new word; the data dependence of
// the recursion (no block can publish step k + 2 before every block has published step k + 1, which
// needs step k consumed) makes two buffers enough.
__device__ __forceinline__ int epoch_hi(long long h) { return (int)(h & 3LL); }
__device__ __forceinline__ int epoch_lo(long long l) { return (int)((l >> 2) & 3LL); }
__device__ __forceinline__ void publish_pair(double* p, double x, int ep) {
  const long long b = __double_as_longlong(x);
  const long long hi = (b & ~3LL) | (long long)ep;
  const long long lo = (b & 3LL) | ((long long)ep << 2);
  asm volatile("st.relaxed.gpu.global.v2.b64 [%0], {%1, %2};" ::"l"(p), "l"(hi), "l"(lo) : "memory");
}
__device__ __forceinline__ void ld_pair(const double* p, long long& hi, long long& lo) {
  asm volatile("ld.relaxed.gpu.global.v2.b64 {%0, %1}, [%2];" : "=l"(hi), "=l"(lo) : "l"(p) : "memory");
}
__device__ __forceinline__ double pair_value(long long hi, long long lo) {
  return __longlong_as_double((hi & ~3LL) | (lo & 3LL));
}
__device__ __forceinline__ int ld_relaxed_int(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
constexpr long long kPollLimit = 4000000LL;


// ---------------------------------------------------------------------------------- tridiagonal
// Householder tridiagonalisation (lower), one exchange of epoch-tagged words per column.  Columns
// of the trailing block are owned by (block, warp) round-robin and stay resident in shared memory.
// At step k every block reads p_k = tau_k A22 v_k and the pre-update pivot column k+1 from double
// buffers the owners published during step k-1, forms w_k = p_k - 1/2 tau_k (p_k . v_k) v_k, the
// updated pivot column and from it v_{k+1}, tau_{k+1} (all redundantly, so nothing else has to be
// exchanged); the owners then update their columns and, in the same pass, compute their entries of
// p_{k+1} and publish the next pivot column.  Reflector v_k is stored in column k below the
// subdiagonal (v_k[0] = 1).  Block reductions go through shared memory and one warp (the FP64 pipe
// is narrow on this GPU, so a shuffle tree in every warp would cost more than the data it sums).
constexpr int TD_THREADS = 160;      // warp 0: reductions and Householder scalars; warps 1-4: columns
constexpr int TD_MAX_SLOTS = 64;     // owned columns per block
constexpr int TD_BATCH = 5;     // exchange entries a thread polls with their loads in flight together

// Householder scalars for x (x[0] = alpha, sum of the squares of x[1..] = sigma): H x = beta e_1,
// H = I - tau v v^T with v[0] = 1 and v[t] = x[t] * scal.
__device__ __forceinline__ void house_scalars(double alpha, double sigma, double& tau, double& beta, double& scal) {
  if (sigma == 0.0) { tau = 0.0; beta = alpha; scal = 0.0; return; }
  beta = -copysign(sqrt(alpha * alpha + sigma), alpha);
  tau = (beta - alpha) * nr_rcp(beta);
  scal = nr_rcp(alpha - beta);
}

// Sum of red[0 .. blockDim.x) by warp 0 (called by warp 0 only); the result is in every lane.
__device__ __forceinline__ double warp0_sum(const double* red) {
  const int lane = threadIdx.x & 31;
  double s = 0.0;
  for (int i = lane; i < (int)blockDim.x; i += 32) s += red[i];
  return warp_sum(s);
}

__global__ void __launch_bounds__(TD_THREADS)
k_tridiag(double* __restrict__ A, int lda, int N, double* __restrict__ d, double* __restrict__ e,
          double* __restrict__ tau, double* __restrict__ Pbuf, double* __restrict__ Cbuf, int* err,
          long long poll_limit) {
  extern __shared__ double sm[];
  // sm[0, N) and sm[N, 2N): v_k and v_{k+1}, swapped every step
  double* w = sm + 2 * N;           // w_k
  double* c = sm + 3 * N;           // updated pivot column k+1
  double* cols = sm + 4 * N;        // owned columns (full length N), resident for the whole reduction
  __shared__ double red[TD_THREADS];
  __shared__ double bc[4];          // broadcast scalars
  __shared__ double colS[TD_MAX_SLOTS], colF[TD_MAX_SLOTS];   // owner warps' parts of p_{k+1}
  const int G = gridDim.x, tid = threadIdx.x, TB = blockDim.x;
  const int warp = tid >> 5, lane = tid & 31, nw = TB >> 5;
  const int nslot = (N + G - 1) / G;   // column j lives in block j % G, slot j / G
  // The block owning the last column writes the outputs (d, e, tau, reflectors): it publishes
  // exchange words at every step.  Every other block leaves once it owns no column >= k + 2 (it
  // would publish nothing more), so each block still reading step k's words publishes words for
  // step k + 1 -- which is what keeps two exchange buffers safe: no block can publish step k + 2
  // before every running block has consumed step k.
  const int ob = (N - 1) % G;
  const int maxcol = (int)blockIdx.x + G * ((N - 1 - (int)blockIdx.x) / G);
  if (N <= 2) {
    if (blockIdx.x == 0 && tid == 0) {
      d[0] = A[0];
      if (N == 2) { e[0] = A[1]; d[1] = A[(size_t)lda + 1]; tau[0] = 0.0; }
    }
    return;
  }
  for (int q = 0; q < nslot; ++q) {
    const int j = q * G + blockIdx.x;
    if (j >= N) break;
    for (int t = tid; t < N; t += TB) cols[(size_t)q * N + t] = A[(size_t)j * lda + t];
  }
  // ---- prologue: v_0 from column 0; p_0; publish column 1
  double tk, bk;
  {
    const int L = N - 1;
    double part = 0.0;
    for (int t = tid; t < L; t += TB) {
      const double x = A[1 + t];
      c[t] = x;
      if (t >= 1) part = fma(x, x, part);
    }
    red[tid] = part;
    __syncthreads();
    if (warp == 0) {
      const double sigma = warp0_sum(red);
      if (lane == 0) {
        double ta, be, sc;
        house_scalars(c[0], sigma, ta, be, sc);
        bc[0] = ta; bc[1] = be; bc[2] = sc;
      }
    }
    __syncthreads();
    tk = bc[0]; bk = bc[1];
    const double sc = bc[2];
    double* v = sm;
    for (int t = tid; t < L; t += TB) v[t] = (t == 0) ? 1.0 : c[t] * sc;
    __syncthreads();
    for (int q = warp; q < nslot; q += nw) {
      const int j = q * G + blockIdx.x;
      if (j < 1 || j >= N) continue;
      const double* col = cols + (size_t)q * N + 1;
      double acc = 0.0;
      for (int t = lane; t < L; t += 32) acc = fma(col[t], v[t], acc);
      acc = warp_sum(acc);
      if (lane == 0) publish_pair(Pbuf + 2 * (j - 1), tk * acc, 0);
      if (j == 1) for (int t = lane; t < L; t += 32) publish_pair(Cbuf + 2 * t, col[t], 0);
    }
    if (blockIdx.x == ob && tid == 0) d[0] = A[0];
    __syncthreads();
  }
  for (int k = 0; k + 2 < N; ++k) {
    if ((int)blockIdx.x != ob && maxcol < k + 2) return;
    const int L = N - k - 1;
    const double* Pk = Pbuf + (size_t)(k & 1) * 2 * N;
    double* Pn = Pbuf + (size_t)((k + 1) & 1) * 2 * N;
    const double* Ck = Cbuf + (size_t)(k & 1) * 2 * N;
    double* Cn = Cbuf + (size_t)((k + 1) & 1) * 2 * N;
    const double* v = sm + (size_t)(k & 1) * N;
    double* v2 = sm + (size_t)((k + 1) & 1) * N;
    const bool next = (k + 3 < N);      // a reflector for column k+1 exists
    // (1) p_k . v_k; the pivot column C_k is fetched in the same pass (into c).  Each thread polls
    // its entries of P_k and C_k, up to TD_BATCH of them with their loads in flight together, until
    // all carry epoch k mod 4 (bounded; a timeout or another block's error ends the kernel).
    const int ek = k & 3;
    double part = 0.0;
    bool ok = true;
    for (int t0 = tid; t0 < L && ok; t0 += TB * TD_BATCH) {
      long long ph[TD_BATCH], pl[TD_BATCH], ch[TD_BATCH], cl[TD_BATCH];
      unsigned pend = 0;
#pragma unroll
      for (int u = 0; u < TD_BATCH; ++u)
        if (t0 + u * TB < L) pend |= 1u << u;
      long long spins = 0;
      while (pend) {
#pragma unroll
        for (int u = 0; u < TD_BATCH; ++u)
          if ((pend >> u) & 1u) {
            const int t = t0 + u * TB;
            ld_pair(Pk + 2 * t, ph[u], pl[u]);
            ld_pair(Ck + 2 * t, ch[u], cl[u]);
          }
#pragma unroll
        for (int u = 0; u < TD_BATCH; ++u)
          if (((pend >> u) & 1u) && epoch_hi(ph[u]) == ek && epoch_lo(pl[u]) == ek && epoch_hi(ch[u]) == ek &&
              epoch_lo(cl[u]) == ek)
            pend &= ~(1u << u);
        if (!pend) break;
        if (++spins > poll_limit) { atomicExch(err, kErrTimeout); ok = false; break; }
        if ((spins & 255) == 0 && ld_relaxed_int(err)) { ok = false; break; }
      }
      if (!ok) break;
#pragma unroll
      for (int u = 0; u < TD_BATCH; ++u) {
        const int t = t0 + u * TB;
        if (t < L) {
          const double pt = pair_value(ph[u], pl[u]), ct = pair_value(ch[u], cl[u]);
          c[t] = ct;
          w[t] = pt;
          part = fma(pt, v[t], part);
        }
      }
    }
    red[tid] = part;
    if (!__syncthreads_and(ok)) return;
    if (warp == 0) {
      const double pv = warp0_sum(red);
      if (lane == 0) {
        const double kc = 0.5 * tk * pv;
        bc[0] = kc;
        bc[1] = w[0] - kc;               // w_k[0] (v_k[0] = 1)
      }
    }
    __syncthreads();
    const double kc = bc[0], w0 = bc[1];
    // (2) w_k and the updated pivot column c = C_k - v w0 - w v0 (v0 = 1); sum of squares of c[2..]
    part = 0.0;
    for (int t = tid; t < L; t += TB) {
      const double wt = fma(-kc, v[t], w[t]);
      w[t] = wt;
      const double ct = fma(-v[t], w0, c[t]) - wt;
      c[t] = ct;
      if (t >= 2) part = fma(ct, ct, part);
    }
    red[tid] = part;
    __syncthreads();
    // (3) warp 0 sums sigma and forms the Householder scalars of column k+1 while the owner warps
    // update their columns, A22 -= v w^T + w v^T (rows k+1..), publish the next pivot column
    // (column k+2) as it is formed, and sum their parts of p_{k+1} = tau_{k+1} A22 v_{k+1}:
    // nv[1] + scn * sum_{t >= 2} nv[t] c[t]  (v_{k+1}[0] = 1, v_{k+1}[t-1] = c[t] scn), finished
    // once scn is known.
    if (warp == 0) {
      const double sigma = warp0_sum(red);
      if (lane == 0) {
        double ta = 0.0, be = 0.0, sc = 0.0;
        if (next) house_scalars(c[1], sigma, ta, be, sc);
        bc[2] = ta; bc[3] = be; bc[0] = sc;
        if (blockIdx.x == ob) {
          d[k + 1] = c[0];
          e[k] = bk;
          tau[k] = tk;
          if (!next) { e[k + 1] = c[1]; tau[k + 1] = 0.0; }
        }
      }
    } else {
      for (int q = warp - 1; q < nslot; q += nw - 1) {
        const int j = q * G + blockIdx.x;
        if (j < k + 1 || j >= N) continue;
        const int tj = j - (k + 1);
        double* col = cols + (size_t)q * N + k + 1;
        const double vj = v[tj], wj = w[tj];
        const bool publish = next && tj == 1;       // column k+2 becomes the next pivot column
        double a0 = 0.0, a1 = 0.0, first = 0.0;
        for (int t = lane; t < L; t += 64) {
          const double nv = fma(-v[t], wj, fma(-w[t], vj, col[t]));
          col[t] = nv;
          if (publish && t >= 1) publish_pair(Cn + 2 * (t - 1), nv, (k + 1) & 3);
          if (t >= 2) a0 = fma(nv, c[t], a0);
          else if (t == 1) first = nv;
          const int t2 = t + 32;
          if (t2 < L) {
            const double nv2 = fma(-v[t2], wj, fma(-w[t2], vj, col[t2]));
            col[t2] = nv2;
            if (publish) publish_pair(Cn + 2 * (t2 - 1), nv2, (k + 1) & 3);
            a1 = fma(nv2, c[t2], a1);
          }
        }
        const double S = warp_sum(a0 + a1);
        const double F = warp_sum(first);
        if (lane == 0) { colS[q] = S; colF[q] = F; }
        if (k + 3 == N && j == N - 1) {                  // last diagonal entry (written by lane L-1)
          __syncwarp();
          if (lane == 0) d[N - 1] = col[L - 1];
        }
      }
    }
    __syncthreads();
    const double tn = bc[2], bn = bc[3], scn = bc[0];
    // (4) the owners publish their entries of p_{k+1} (lane 0 reads back its own colS, colF);
    // every thread writes v_{k+1}
    if (warp > 0 && lane == 0 && next) {
      for (int q = warp - 1; q < nslot; q += nw - 1) {
        const int j = q * G + blockIdx.x;
        if (j < k + 2 || j >= N) continue;
        publish_pair(Pn + 2 * (j - k - 2), tn * fma(scn, colS[q], colF[q]), (k + 1) & 3);
      }
    }
    if (next)
      for (int t = tid; t < L - 1; t += TB) v2[t] = (t == 0) ? 1.0 : c[t + 1] * scn;
    // (5) store the reflector v_k below the subdiagonal of column k (for the back-transformation)
    if (blockIdx.x == ob)
      for (int t = tid; t < L; t += TB) A[(size_t)k * lda + k + 1 + t] = v[t];
    tk = tn;
    bk = bn;
    __syncthreads();
  }
}

// ------------------------------------------------------------------------------ divide & conquer
struct MergeDesc { int lo, mid, hi; };

struct DcWork {
  double *lam, *lamk, *lamtmp, *Dw, *Zw, *Dk, *Zk, *Dd, *Q, *Qtmp, *Delta, *rho, *rot, *z2, *Tm;
  int *colk, *cold, *perm, *Kp, *nrot, *mergeof, *gperm, *gcnt;
};

__global__ void k_dc_init(const double* __restrict__ d, const double* __restrict__ e, int N, double* lam,
                          double* Q) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= N) return;
  double v = d[j];
  if (j > 0) v -= fabs(e[j - 1]);
  if (j + 1 < N) v -= fabs(e[j]);
  lam[j] = v;
  Q[(size_t)j * N + j] = 1.0;
}

// Order-preserving integer key of a double (IEEE bit pattern; negative values mirrored), so the
// sorting below compares on the integer units instead of the FP64 pipe.
__device__ __forceinline__ long long order_key(double x) {
  const long long b = __double_as_longlong(x);
  return b >= 0 ? b : (b ^ 0x7FFFFFFFFFFFFFFFLL);
}

// Block-wide maximum (every thread gets the result).
__device__ double block_max(double v) {
  __shared__ double red[32];
  __syncthreads();
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = (blockDim.x + 31) >> 5;
  if (l == 0) red[w] = v;
  __syncthreads();
  double t = (l < nw) ? red[l] : 0.0;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) t = fmax(t, __shfl_xor_sync(0xffffffffu, t, o));
  __syncthreads();
  return t;
}

// Block-wide exclusive prefix sum of one int per thread (thread order); *total gets the sum.
__device__ int block_excl_scan(int v, int* total) {
  __shared__ int ws[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  __syncthreads();
  if (lane == 31) ws[wid] = x;
  __syncthreads();
  if (wid == 0) {
    int t = (lane < nw) ? ws[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    ws[lane] = t;
  }
  __syncthreads();
  const int before = (wid > 0 ? ws[wid - 1] : 0) + x - v;
  *total = ws[nw - 1];
  __syncthreads();
  return before;
}

constexpr int DC_THREADS = 256;

// Shared memory of k_dc_prep for a merge of order K: four FP64 arrays, one int64 key array, six int arrays.
inline size_t prep_smem_bytes(int K) { return (size_t)K * (4 * sizeof(double) + sizeof(long long) + 6 * sizeof(int)); }

// Phase 1 of a merge: z vector, sorted poles, deflation.  One block per merge.
//   1. The two ascending child spectra are merged by rank (each entry's position is its index
//      plus the number of entries of the other list before it, found by binary search).
//   2. Small z components are deflated (all entries in parallel).
//   3. Close poles are deflated by a Givens rotation: a scan in pole order, since a rotation changes
//      the entries the next test reads; one thread, operands carried in registers.  The rotations
//      are written to W.rot and applied to the eigenvector rows by k_dc_rot.
//   4. Kept and deflated entries are compacted (block prefix sums); the kept poles are re-sorted
//      by rank when a rotation moved one.
//   5. The kept columns are grouped by their row support (child 1 only, both, child 2 only) for the
//      eigenvector product of phase 5.
// (device function: every thread of the block calls it; psm holds prep_smem_bytes(K))
__device__ void dc_prep(const MergeDesc mg, const double* __restrict__ e, int N, DcWork W, double* psm) {
  const int lo = mg.lo, mid = mg.mid, K = mg.hi - mg.lo, n1 = mg.mid - mg.lo;
  double* sLam = psm;
  double* sZr = psm + K;
  double* sD = psm + 2 * K;
  double* sZ = psm + 3 * K;
  long long* sKey = reinterpret_cast<long long*>(psm + 4 * K);
  int* sPerm = reinterpret_cast<int*>(psm + 5 * K);
  int* sStat = sPerm + K;       // 0 kept, 1 deflated (small z), 2 deflated (rotated away)
  int* sType = sStat + K;       // row support: 1 child 1, 3 child 2, 2 both
  int* sKeep = sType + K;
  int* sDefl = sKeep + K;
  int* sSort = sDefl + K;
  __shared__ int s_nrot;
  const double rho0 = e[mid - 1];
  const double sgn = rho0 >= 0.0 ? 1.0 : -1.0;
  double zz = 0.0;
  for (int t = threadIdx.x; t < K; t += blockDim.x) {
    const double z = (t < n1) ? W.Q[(size_t)(lo + t) * N + (mid - 1)] : sgn * W.Q[(size_t)(lo + t) * N + mid];
    sZr[t] = z;
    const double l = W.lam[lo + t];
    sLam[t] = l;
    sKey[t] = order_key(l);
    sPerm[t] = t;
    zz += z * z;
  }
  zz = block_sum(zz);
  const double zn = sqrt(zz);
  const double rho = fabs(rho0) * zz;
  // 1. merge by rank (ties: child 1 first)
  for (int t = threadIdx.x; t < K; t += blockDim.x) {
    const long long kt = sKey[t];
    int pos;
    if (t < n1) {
      int a = n1, b = K;
      while (a < b) { const int m = (a + b) >> 1; if (sKey[m] < kt) a = m + 1; else b = m; }
      pos = t + (a - n1);
    } else {
      int a = 0, b = n1;
      while (a < b) { const int m = (a + b) >> 1; if (sKey[m] <= kt) a = m + 1; else b = m; }
      pos = (t - n1) + a;
    }
    sPerm[pos] = t;
    sD[pos] = sLam[t];
    sZ[pos] = sZr[t] / zn;
    sType[pos] = (t < n1) ? 1 : 3;
  }
  __syncthreads();
  // 2. tolerance and small-z deflation
  double dm = 0.0;
  for (int t = threadIdx.x; t < K; t += blockDim.x) dm = fmax(dm, fabs(sD[t]));
  dm = block_max(dm);
  const double tol = 8.0 * kEps * fmax(dm, rho);
  for (int t = threadIdx.x; t < K; t += blockDim.x) sStat[t] = (rho * fabs(sZ[t]) <= tol) ? 1 : 0;
  __syncthreads();
  // 3. close poles.  The test |(D_j - D_l) c s| <= tol with c s = -z_l z_j / t^2 is evaluated
  // without the division, as |D_j - D_l| |z_l z_j| <= tol t^2; c and s are formed only for a
  // rotation.  The pairs of consecutive candidates (entries not deflated by small z) are first tested
  // in parallel on the merged values; a pair's test can only change after a rotation, so the
  // sequential scan starts at the first pair that fires (in the common case none does).
  const int ch0 = (K + (int)blockDim.x - 1) / (int)blockDim.x;
  const int a0 = min(K, (int)threadIdx.x * ch0), a1 = min(K, a0 + ch0);
  int ncl = 0;
  for (int t = a0; t < a1; ++t) ncl += (sStat[t] == 0);
  int nc = 0;
  int oc = block_excl_scan(ncl, &nc);
  int* sCand = sSort;                 // free until the kept poles are re-sorted below
  for (int t = a0; t < a1; ++t)
    if (sStat[t] == 0) sCand[oc++] = t;
  __shared__ int s_first;
  if (threadIdx.x == 0) s_first = nc;
  __syncthreads();
  for (int u = 1 + threadIdx.x; u < nc; u += blockDim.x) {
    const int l = sCand[u - 1], jj = sCand[u];
    const double zl = sZ[l], zj = sZ[jj];
    const double t2 = fma(zl, zl, zj * zj);
    if (fabs(sD[jj] - sD[l]) * fabs(zl * zj) <= tol * t2) atomicMin(&s_first, u);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int nrot = 0;
    const int first = s_first;
    if (first < nc) {
      int last = sCand[first - 1];
      double zl = sZ[last], dl = sD[last];
      for (int u = first; u < nc; ++u) {
        const int j = sCand[u];
        double zj = sZ[j], dj = sD[j];
        const double t2 = fma(zl, zl, zj * zj);
        if (fabs(dj - dl) * fabs(zl * zj) <= tol * t2) {
          const double t = sqrt(t2);
          const double c = zj / t, sn = -zl / t;
          double* rr = W.rot + (size_t)4 * (lo + nrot);
          rr[0] = (double)(lo + sPerm[last]);
          rr[1] = (double)(lo + sPerm[j]);
          rr[2] = c;
          rr[3] = sn;
          ++nrot;
          sD[last] = c * c * dl + sn * sn * dj;
          dj = sn * sn * dl + c * c * dj;
          sD[j] = dj;
          sZ[last] = 0.0;
          sZ[j] = t;
          zj = t;
          sStat[last] = 2;
          if (sType[last] != sType[j]) sType[j] = 2;
        }
        last = j;
        zl = zj;
        dl = dj;
      }
    }
    s_nrot = nrot;
    W.nrot[lo] = nrot;
  }
  __syncthreads();
  const int nrot = s_nrot;
  // 4. compaction: kept and deflated entries in pole order
  const int ch = (K + (int)blockDim.x - 1) / (int)blockDim.x;
  const int c0 = min(K, (int)threadIdx.x * ch), c1 = min(K, c0 + ch);
  int nk = 0;
  for (int t = c0; t < c1; ++t) nk += (sStat[t] == 0);
  int kp = 0;
  int ok = block_excl_scan(nk, &kp);
  int od = c0 - ok;
  for (int t = c0; t < c1; ++t) {
    if (sStat[t] == 0) sKeep[ok++] = t;
    else sDefl[od++] = t;
  }
  __syncthreads();
  const int* keep = sKeep;
  if (nrot > 0) {
    // a rotation can move a kept pole past its neighbours: rank sort by (value, position)
    for (int q = threadIdx.x; q < kp; q += blockDim.x) sKey[q] = order_key(sD[sKeep[q]]);
    __syncthreads();
    for (int q = threadIdx.x; q < kp; q += blockDim.x) {
      const long long kq = sKey[q];
      int rank = 0;
      for (int u = 0; u < kp; ++u) {
        const long long ku = sKey[u];
        rank += (ku < kq) || (ku == kq && u < q);
      }
      sSort[rank] = sKeep[q];
    }
    __syncthreads();
    keep = sSort;
  }
  for (int q = threadIdx.x; q < kp; q += blockDim.x) {
    const int j = keep[q];
    W.Dk[lo + q] = sD[j];
    W.Zk[lo + q] = sZ[j];
    W.z2[lo + q] = rho * sZ[j] * sZ[j];
    W.colk[lo + q] = lo + sPerm[j];
  }
  for (int q = threadIdx.x; q < K - kp; q += blockDim.x) {
    const int j = sDefl[q];
    W.Dd[lo + q] = sD[j];
    W.cold[lo + q] = lo + sPerm[j];
  }
  // 5. kept columns grouped by row support: child 1 only, both children, child 2 only
  {
    const int kc = (kp + (int)blockDim.x - 1) / (int)blockDim.x;
    const int q0 = min(kp, (int)threadIdx.x * kc), q1 = min(kp, q0 + kc);
    int cnt[3] = {0, 0, 0};
    for (int q = q0; q < q1; ++q) ++cnt[sType[keep[q]] - 1];
    int tot[3];
    int off[3];
    for (int g = 0; g < 3; ++g) off[g] = block_excl_scan(cnt[g], &tot[g]);
    off[1] += tot[0];
    off[2] += tot[0] + tot[1];
    for (int q = q0; q < q1; ++q) W.gperm[lo + off[sType[keep[q]] - 1]++] = q;
    if (threadIdx.x == 0) {
      W.gcnt[2 * lo] = tot[0];
      W.gcnt[2 * lo + 1] = tot[1];
      W.rho[lo] = rho;
      W.Kp[lo] = kp;
    }
  }
}
__global__ void __launch_bounds__(DC_THREADS)
k_dc_prep(const MergeDesc* __restrict__ merges, const double* __restrict__ e, int N, DcWork W) {
  extern __shared__ double psm[];
  dc_prep(merges[blockIdx.x], e, N, W, psm);
}

// Phase 1b: the deflation rotations applied to the child eigenvector columns, one thread per row of
// the merge.  Rotation q acts on (a_q, b_q) with b_q a column no earlier rotation touched, and a_q
// either untouched as well or equal to b_{q-1}; so each group of RG rotations loads its operands up
// front (independent loads), and the a_q = b_{q-1} chain is carried in a register.
__device__ void dc_rot_row(const MergeDesc mg, int N, DcWork W, int row) {
  const int lo = mg.lo, K = mg.hi - mg.lo;
  if (row >= K) return;
  const int nrot = W.nrot[lo];
  if (nrot == 0) return;
  const double* rot = W.rot + (size_t)4 * lo;
  double* qrow = W.Q + lo + row;
  constexpr int RG = 8;
  double carry = 0.0;
  int carry_col = -1;
  for (int q0 = 0; q0 < nrot; q0 += RG) {
    const int nq = min(RG, nrot - q0);
    int ca[RG], cb[RG];
    double xa[RG], xb[RG];
#pragma unroll
    for (int u = 0; u < RG; ++u) {
      if (u >= nq) break;
      const double* rr = rot + 4 * (q0 + u);
      ca[u] = (int)rr[0];
      cb[u] = (int)rr[1];
      const int prev = (u == 0) ? carry_col : cb[u - 1];
      xb[u] = qrow[(size_t)cb[u] * N];
      xa[u] = (ca[u] == prev) ? 0.0 : qrow[(size_t)ca[u] * N];
    }
#pragma unroll
    for (int u = 0; u < RG; ++u) {
      if (u >= nq) break;
      const double* rr = rot + 4 * (q0 + u);
      const double c = rr[2], sn = rr[3];
      const int prev = (u == 0) ? carry_col : cb[u - 1];
      const double a = (ca[u] == prev) ? carry : xa[u];
      const double na = c * a + sn * xb[u];
      const double nb = -sn * a + c * xb[u];
      qrow[(size_t)ca[u] * N] = na;
      qrow[(size_t)cb[u] * N] = nb;
      carry = nb;
      carry_col = cb[u];
    }
  }
}
__global__ void __launch_bounds__(128)
k_dc_rot(const MergeDesc* __restrict__ merges, int N, DcWork W) {
  dc_rot_row(merges[blockIdx.y], N, W, blockIdx.x * blockDim.x + threadIdx.x);
}

// Sum over the LANES lanes that share one root (LANES = 32: a warp; LANES = 1: one thread; in
// between, an aligned group of lanes of a warp named by mask, which lets the groups of one warp
// run different iteration counts).
template <int LANES> __device__ __forceinline__ double group_sum(double v, unsigned mask = 0xffffffffu) {
  if constexpr (LANES == 32) return warp_sum(v);
  else if constexpr (LANES == 1) return v;
  else {
#pragma unroll
    for (int o = LANES / 2; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o);
    return v;
  }
}

// Phase 2: secular roots, LANES lanes per (merge, root) -- a warp for large merges, one thread for
// small ones; the sums over poles are split across the lanes.
// delta column i: Delta[(lo+i)*N + lo + j] = Dk_j - lam_i, computed from the origin pole.
template <int LANES>
__device__ void dc_secular_root(int lo, int i, int N, DcWork W, int* err, int lane, unsigned gmask) {
  const int Kp = W.Kp[lo];
  if (i >= Kp) return;
  const double* Dk = W.Dk + lo;
  const double* Zk = W.Zk + lo;
  const double* z2 = W.z2 + lo;
  const double rho = W.rho[lo];
  double* delta = W.Delta + (size_t)(lo + i) * N + lo;
  // For an inner root the sums are first evaluated at the midpoint of (D_i, D_{i+1}): the sign of f
  // there picks the origin pole (the nearer end of the root's half interval), and the same sums give
  // the first rational-model step from the midpoint.  The last root starts from its bracket midpoint.
  int org;
  double tlo, thi, tau;
  double psi = 0.0, dpsi = 0.0, phi = 0.0, dphi = 0.0;
  bool have = false;            // sums already evaluated at tau
  if (i < Kp - 1) {
    const double mid = 0.5 * (Dk[i] + Dk[i + 1]);
    for (int j = lane; j < Kp; j += LANES) {
      const double rinv = nr_rcp(Dk[j] - mid);
      const double tv = z2[j] * rinv;
      if (j <= i) { psi += tv; dpsi += tv * rinv; }
      else { phi += tv; dphi += tv * rinv; }
    }
    psi = group_sum<LANES>(psi, gmask); dpsi = group_sum<LANES>(dpsi, gmask);
    phi = group_sum<LANES>(phi, gmask); dphi = group_sum<LANES>(dphi, gmask);
    if (1.0 + psi + phi >= 0.0) { org = i; tlo = 0.0; thi = mid - Dk[i]; tau = thi; }
    else { org = i + 1; tlo = mid - Dk[i + 1]; thi = 0.0; tau = tlo; }
    have = true;
  } else {
    org = i;
    double zz = 0.0;
    for (int j = lane; j < Kp; j += LANES) zz += Zk[j] * Zk[j];
    tlo = 0.0;
    thi = rho * group_sum<LANES>(zz, gmask);
    tau = 0.5 * (tlo + thi);
  }
  const double Dorg = Dk[org];
  bool conv = false;
  for (int it = 0; it < 200 && !conv; ++it) {
    if (!have) {
      psi = 0.0; dpsi = 0.0; phi = 0.0; dphi = 0.0;
      for (int j = lane; j < Kp; j += LANES) {
        const double dl = (Dk[j] - Dorg) - tau;
        const double rinv = nr_rcp(dl);
        const double tv = z2[j] * rinv;
        if (j <= i) { psi += tv; dpsi += tv * rinv; }
        else { phi += tv; dphi += tv * rinv; }
      }
      psi = group_sum<LANES>(psi, gmask); dpsi = group_sum<LANES>(dpsi, gmask);
      phi = group_sum<LANES>(phi, gmask); dphi = group_sum<LANES>(dphi, gmask);
    }
    have = false;
    const double f = 1.0 + psi + phi;
    if (f == 0.0) break;
    // residual test: f is as small as rounding of its terms allows (psi < 0 < phi term-wise)
    if (fabs(f) <= 8.0 * kEps * (1.0 - psi + phi)) break;
    if (f > 0.0) thi = tau; else tlo = tau;
    // The model step is a guess (the bracket and the residual test decide convergence), so its
    // quotients are taken as products with Newton reciprocals (about 1 ulp; an FP64 division has a
    // much longer dependency chain on this GPU).
    const double Dl = (Dk[i] - Dorg) - tau;
    const double sl = Dl * Dl * dpsi;
    double nt = NAN;
    if (i < Kp - 1) {
      const double Dr = (Dk[i + 1] - Dorg) - tau;
      const double sr = Dr * Dr * dphi;
      const double c = f - sl * nr_rcp(Dl) - sr * nr_rcp(Dr);
      const double A2 = c, B2 = -(c * (Dl + Dr) + sl + sr), C2 = c * Dl * Dr + sl * Dr + sr * Dl;
      double c1 = NAN, c2 = NAN;
      if (A2 == 0.0) { if (B2 != 0.0) c1 = -C2 * nr_rcp(B2); }
      else {
        double disc = B2 * B2 - 4.0 * A2 * C2;
        if (disc < 0.0) disc = 0.0;
        const double q = -0.5 * (B2 + copysign(sqrt(disc), B2));
        c1 = q * nr_rcp(A2);
        if (q != 0.0) c2 = C2 * nr_rcp(q);
      }
      if (isfinite(c1) && tau + c1 > tlo && tau + c1 < thi) nt = tau + c1;
      else if (isfinite(c2) && tau + c2 > tlo && tau + c2 < thi) nt = tau + c2;
    } else {
      const double c = f - sl * nr_rcp(Dl);
      if (c != 0.0) {
        const double t2 = tau + Dl + sl * nr_rcp(c);
        if (isfinite(t2) && t2 > tlo && t2 < thi) nt = t2;
      }
    }
    if (!isfinite(nt)) nt = 0.5 * (tlo + thi);
    conv = fabs(nt - tau) <= 2.0 * kEps * fmax(fabs(nt), fabs(tau)) ||
           (thi - tlo) <= 4.0 * kEps * fmax(fabs(tlo), fabs(thi));
    tau = nt;
    if (it == 199 && !conv && lane == 0) atomicExch(err, kErrSecular);
  }
  for (int j = lane; j < Kp; j += LANES) delta[j] = (Dk[j] - Dorg) - tau;
  if (lane == 0) W.lamk[lo + i] = Dorg + tau;
}
template <int LANES>
__global__ void k_dc_secular(const MergeDesc* __restrict__ merges, const int* __restrict__ mergeof, int N, DcWork W,
                             int* err) {
  const int p = (blockIdx.x * blockDim.x + threadIdx.x) / LANES;
  const int lane = threadIdx.x % LANES;
  if (p >= N) return;
  const int mi = mergeof[p];
  if (mi < 0) return;
  const int lo = merges[mi].lo;
  dc_secular_root<LANES>(lo, p - lo, N, W, err, lane, 0xffffffffu);
}

// Phase 3: Loewner-corrected z (one warp per j):
//   zhat_j^2 = (lam_last - D_j)/rho * prod_{i<j} (lam_i - D_j)/(D_i - D_j) * prod_{i>j} (lam_{i-1} - D_j)/(D_i - D_j)
// The product is formed as a sum of logarithms of the (positive) factors split across lanes.
template <int LANES>
__device__ void dc_zhat_one(int lo, int j, int N, DcWork W, int lane, unsigned gmask) {
  const int Kp = W.Kp[lo];
  if (j >= Kp) return;
  const double* Dk = W.Dk + lo;
  const double rho = W.rho[lo];
  const double Dj = Dk[j];
  // each lane multiplies its factors and takes one logarithm (more only if the product leaves
  // [1e-150, 1e150]); the lanes' logarithms are summed
  double lg = 0.0, prod = 1.0;
  for (int i = lane; i < Kp; i += LANES) {
    if (i == j) continue;
    const int ii = (i < j) ? i : i - 1;                       // lam_i for i < j, lam_{i-1} for i > j
    const double num = -W.Delta[(size_t)(lo + ii) * N + lo + j];
    prod *= fabs(num / (Dk[i] - Dj));
    if (!(prod > 1e-150 && prod < 1e150)) { lg += log(prod); prod = 1.0; }
  }
  lg += log(prod);
  lg = group_sum<LANES>(lg, gmask);
  if (lane == 0) {
    const double last = -W.Delta[(size_t)(lo + Kp - 1) * N + lo + j] / rho;
    W.Zw[lo + j] = copysign(sqrt(fabs(last)) * exp(0.5 * lg), W.Zk[lo + j]);
  }
}
template <int LANES>
__global__ void k_dc_zhat(const MergeDesc* __restrict__ merges, const int* __restrict__ mergeof, int N, DcWork W) {
  const int p = (blockIdx.x * blockDim.x + threadIdx.x) / LANES;
  const int lane = threadIdx.x % LANES;
  if (p >= N) return;
  const int mi = mergeof[p];
  if (mi < 0) return;
  const int lo = merges[mi].lo;
  dc_zhat_one<LANES>(lo, p - lo, N, W, lane, 0xffffffffu);
}

// Phase 4: eigenvector columns u_i = zhat / delta_i, normalised, written over Delta (one warp per i).
template <int LANES>
__device__ void dc_vecs_one(int lo, int i, int N, DcWork W, int lane, unsigned gmask) {
  const int Kp = W.Kp[lo];
  if (i >= Kp) return;
  double* col = W.Delta + (size_t)(lo + i) * N + lo;
  double nrm = 0.0;
  for (int j = lane; j < Kp; j += LANES) { double u = W.Zw[lo + j] * nr_rcp(col[j]); col[j] = u; nrm += u * u; }
  nrm = group_sum<LANES>(nrm, gmask);
  const double inv = 1.0 / sqrt(nrm);
  for (int j = lane; j < Kp; j += LANES) col[j] *= inv;
}
template <int LANES>
__global__ void k_dc_vecs(const MergeDesc* __restrict__ merges, const int* __restrict__ mergeof, int N, DcWork W) {
  const int p = (blockIdx.x * blockDim.x + threadIdx.x) / LANES;
  const int lane = threadIdx.x % LANES;
  if (p >= N) return;
  const int mi = mergeof[p];
  if (mi < 0) return;
  const int lo = merges[mi].lo;
  dc_vecs_one<LANES>(lo, p - lo, N, W, lane, 0xffffffffu);
}

// Phase 5: Qtmp[lo:hi, lo+i] = Q[lo:hi, colk] U[:, i] (i < Kp); deflated columns copied after them.
// The sum over kept poles runs in the support order of phase 1 (gperm): a row tile inside child 1
// skips the columns supported on child 2 only and vice versa, about half of the products.
constexpr int DG_T = 32;
// (device function: every thread of a 256-thread block calls it with the same tile)
__device__ void dc_gemm_tile(const MergeDesc mg, int N, DcWork W, int r0, int c0) {
  const int lo = mg.lo, K = mg.hi - mg.lo, n1 = mg.mid - mg.lo;
  const int Kp = W.Kp[lo];
  if (r0 >= K || c0 >= K) return;
  __shared__ double As[DG_T][DG_T + 1], Bs[DG_T][DG_T + 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int g1 = W.gcnt[2 * lo], g2 = W.gcnt[2 * lo + 1];
  int kb = 0, ke = Kp;
  if (r0 + DG_T <= n1) ke = g1 + g2;        // rows of child 1 only
  else if (r0 >= n1) kb = g1;               // rows of child 2 only
  const int* gp = W.gperm + lo;
  double acc[2][2] = {{0, 0}, {0, 0}};
  if (c0 < Kp) {
    for (int k0 = kb; k0 < ke; k0 += DG_T) {
      for (int e2 = threadIdx.x; e2 < DG_T * DG_T; e2 += 256) {
        const int i32 = e2 % DG_T, o32 = e2 / DG_T;
        // A tile: consecutive threads take consecutive rows of one column
        {
          const int row = r0 + i32, kidx = k0 + o32;
          As[o32][i32] = (row < K && kidx < ke) ? W.Q[(size_t)W.colk[lo + gp[kidx]] * N + lo + row] : 0.0;
        }
        // B tile: consecutive threads take consecutive poles of one eigenvector column
        {
          const int kidx = k0 + i32, ci = c0 + o32;
          Bs[i32][o32] = (ci < Kp && kidx < ke) ? W.Delta[(size_t)(lo + ci) * N + lo + gp[kidx]] : 0.0;
        }
      }
      __syncthreads();
#pragma unroll 8
      for (int kk = 0; kk < DG_T; ++kk)
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
          for (int b = 0; b < 2; ++b) acc[a][b] = fma(As[kk][ty + 16 * a], Bs[kk][tx + 16 * b], acc[a][b]);
      __syncthreads();
    }
  }
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      int row = r0 + ty + 16 * a, c = c0 + tx + 16 * b;
      if (row >= K || c >= K) continue;
      double val;
      if (c < Kp) val = acc[a][b];
      else val = W.Q[(size_t)W.cold[lo + (c - Kp)] * N + lo + row];
      W.Qtmp[(size_t)(lo + c) * N + lo + row] = val;
    }
}
__global__ void __launch_bounds__(256)
k_dc_gemm(const MergeDesc* __restrict__ merges, int N, DcWork W) {
  dc_gemm_tile(merges[blockIdx.z], N, W, blockIdx.x * DG_T, blockIdx.y * DG_T);
}

// Phase 6a: order the merged spectrum ascending (one block per merge): W.lam and the column
// permutation W.perm (relative to lo) for phase 6b.  Rank sort on (value key, position): the kept
// roots come before deflated poles of equal value.
__device__ void dc_finish(const MergeDesc mg, int N, DcWork W, double* fsm) {
  const int lo = mg.lo, K = mg.hi - mg.lo;
  const int Kp = W.Kp[lo];
  double* sl = fsm;                                          // K merged eigenvalues (kept roots, deflated poles)
  long long* key = reinterpret_cast<long long*>(fsm + K);
  for (int t = threadIdx.x; t < K; t += blockDim.x) {
    const double v = (t < Kp) ? W.lamk[lo + t] : W.Dd[lo + t - Kp];
    sl[t] = v;
    key[t] = order_key(v);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < K; t += blockDim.x) {
    const long long kt = key[t];
    int rank = 0;
    for (int u = 0; u < K; ++u) {
      const long long ku = key[u];
      rank += (ku < kt) || (ku == kt && u < t);
    }
    W.lam[lo + rank] = sl[t];
    W.perm[lo + rank] = t;
  }
}
__global__ void __launch_bounds__(256)
k_dc_finish(const MergeDesc* __restrict__ merges, int N, DcWork W) {
  extern __shared__ double fsm[];
  dc_finish(merges[blockIdx.x], N, W, fsm);
}

// Phase 6b: move the merged eigenvector columns back into Q in ascending order
// (grid: column groups of 8 x merges).
__device__ void dc_copy_cols(const MergeDesc mg, int N, DcWork W, int c0) {
  const int lo = mg.lo, K = mg.hi - mg.lo;
  if (c0 >= K) return;
  const int c1 = min(K, c0 + 8);
  for (int c = c0; c < c1; ++c) {
    const double* src = W.Qtmp + (size_t)(lo + W.perm[lo + c]) * N + lo;
    double* dst = W.Q + (size_t)(lo + c) * N + lo;
    for (int row = threadIdx.x; row < K; row += blockDim.x) dst[row] = src[row];
  }
}
__global__ void __launch_bounds__(256)
k_dc_copy(const MergeDesc* __restrict__ merges, int N, DcWork W) {
  dc_copy_cols(merges[blockIdx.y], N, W, blockIdx.x * 8);
}

// All phases of a merge of order at most DC_SMALL_K in one block (one block per merge of the level):
// the levels near the leaves have many small merges, where eight launches per level cost more than
// the work.  The phases run in the order of the per-phase kernels, separated by block barriers;
// every phase touches only the merge's own rows and columns.  Roots, z entries and eigenvector
// columns are taken by groups of DC_SMALL_LANES lanes.
constexpr int DC_SMALL_K = 40;
constexpr int DC_SMALL_LANES = 8;
inline size_t small_smem_bytes(int K) {
  return std::max(prep_smem_bytes(K), (size_t)K * (sizeof(double) + sizeof(long long)));
}
__global__ void __launch_bounds__(DC_THREADS)
k_dc_small(const MergeDesc* __restrict__ merges, const double* __restrict__ e, int N, DcWork W, int* err) {
  extern __shared__ double ssm[];
  constexpr int L = DC_SMALL_LANES;
  const MergeDesc mg = merges[blockIdx.x];
  const int lo = mg.lo, K = mg.hi - mg.lo;
  dc_prep(mg, e, N, W, ssm);
  __syncthreads();
  for (int row = threadIdx.x; row < K; row += blockDim.x) dc_rot_row(mg, N, W, row);
  __syncthreads();
  const int Kp = W.Kp[lo];
  const int grp = threadIdx.x / L, lane = threadIdx.x % L, ngrp = blockDim.x / L;
  const unsigned gmask = ((1u << L) - 1u) << ((threadIdx.x & 31) & ~(L - 1));
  for (int i = grp; i < Kp; i += ngrp) dc_secular_root<L>(lo, i, N, W, err, lane, gmask);
  __syncthreads();
  for (int j = grp; j < Kp; j += ngrp) dc_zhat_one<L>(lo, j, N, W, lane, gmask);
  __syncthreads();
  for (int i = grp; i < Kp; i += ngrp) dc_vecs_one<L>(lo, i, N, W, lane, gmask);
  __syncthreads();
  const int nt = (K + DG_T - 1) / DG_T;
  for (int t = 0; t < nt * nt; ++t) dc_gemm_tile(mg, N, W, (t / nt) * DG_T, (t % nt) * DG_T);
  __syncthreads();
  dc_finish(mg, N, W, ssm);
  __syncthreads();
  for (int c0 = 0; c0 < K; c0 += 8) dc_copy_cols(mg, N, W, c0);
}

// ---- double-FP32 arithmetic (pairs hi + lo of FP32 numbers).  The _rn intrinsics keep the compiler
// from contracting the error-free transformations into FMAs.
__device__ __forceinline__ float2 ff_from_double(double x) {
  const float h = __double2float_rn(x);
  return make_float2(h, __double2float_rn(x - (double)h));
}
// (s, c) <- (s, c) + (s2, c2): two_sum of the leading terms (Knuth), errors into the compensation
__device__ __forceinline__ void ff_acc_add(float& s, float& c, float s2, float c2) {
  const float t = __fadd_rn(s, s2);
  const float bb = __fsub_rn(t, s);
  const float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bb)), __fsub_rn(s2, bb));
  s = t;
  c = __fadd_rn(__fadd_rn(c, c2), e);
}
// (s, c) <- (s, c) + a b: the product of the leading parts exactly (its error by FMA), the cross
// terms into its error, the lo * lo term (2^-48 relative) dropped
__device__ __forceinline__ void ff_fma_acc(float& s, float& c, float2 a, float2 b) {
  const float p = __fmul_rn(a.x, b.x);
  float pe = __fmaf_rn(a.x, b.x, -p);
  pe = __fmaf_rn(a.x, b.y, pe);
  pe = __fmaf_rn(a.y, b.x, pe);
  ff_acc_add(s, c, p, pe);
}
// normalised pair of s + c (two_sum, valid for any magnitudes)
__device__ __forceinline__ float2 ff_norm(float s, float c) {
  const float h = __fadd_rn(s, c);
  const float bb = __fsub_rn(h, s);
  const float l = __fadd_rn(__fsub_rn(s, __fsub_rn(h, bb)), __fsub_rn(c, bb));
  return make_float2(h, l);
}
// z - (s + c)
__device__ __forceinline__ float2 ff_sub(float2 z, float s, float c) {
  float hs = z.x, cs = z.y;
  ff_acc_add(hs, cs, -s, -c);
  return ff_norm(hs, cs);
}

// Back-transformation of the top columns through the reflectors, RB reflectors at a time in the
// compact WY form: H_k0 H_k0+1 ... H_k0+RB-1 = I - V T V^T (V the RB reflectors, T upper
// triangular).  A block owns CB output columns; per group it stages V in shared memory once for
// all its columns, forms Y = V^T Z (RB x CB dots), Y <- T Y, and Z -= V Y.
constexpr int RB = 16;
constexpr int CB = 4;

// T of every group (one block per group): T_ii = tau_i, T[0:i, i] = -tau_i T[0:i, 0:i] V[:, 0:i]^T v_i.
// The RB (RB - 1) / 2 reflector dots are spread over the warps.
__global__ void __launch_bounds__(256)
k_bt_tmat(const double* __restrict__ A, int lda, const double* __restrict__ tau, int N,
          double* __restrict__ Tm, float2* __restrict__ Vff, float2* __restrict__ Tff) {
  const int g = blockIdx.x, warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int nref = N - 2;
  const int k0 = g * RB, nb = min(RB, nref - k0);
  __shared__ double vv[RB][RB];
  for (int pr = warp; pr < RB * RB; pr += nw) {
    const int a = pr / RB, b = pr - a * RB;
    if (!(a < b && b < nb)) continue;
    const double* va = A + (size_t)(k0 + a) * lda;
    const double* vb = A + (size_t)(k0 + b) * lda;
    double acc = 0.0;
    for (int row = k0 + b + 1 + lane; row < N; row += 32) acc = fma(va[row], vb[row], acc);
    acc = warp_sum(acc);
    if (lane == 0) vv[a][b] = acc;
  }
  __syncthreads();
  // T column by column: thread r < i forms T[r][i] from the finished columns 0 .. i-1
  __shared__ double Ts[RB][RB];
  for (int e = threadIdx.x; e < RB * RB; e += blockDim.x) Ts[e / RB][e % RB] = 0.0;
  __syncthreads();
  for (int i = 0; i < nb; ++i) {
    const double ti = tau[k0 + i];
    const int r = threadIdx.x;
    if (r < i) {
      double acc = 0.0;
      for (int c = r; c < i; ++c) acc = fma(Ts[r][c], vv[c][i], acc);
      Ts[r][i] = -ti * acc;
    } else if (r == i) {
      Ts[i][i] = ti;
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < RB * RB; e += blockDim.x) Tm[(size_t)g * RB * RB + e] = Ts[e / RB][e % RB];
  if (Vff) {
    // the group's reflectors (zero outside their support) and T as double-FP32 pairs, for
    // k_backtransform_ff: converted once here instead of in every block of the back-transform
    for (int e = threadIdx.x; e < RB * RB; e += blockDim.x) Tff[(size_t)g * RB * RB + e] = ff_from_double(Ts[e / RB][e % RB]);
    for (int e = threadIdx.x; e < RB * N; e += blockDim.x) {
      const int a = e / N, row = e - a * N;
      const double x = (a < nb && row >= k0 + a + 1) ? A[(size_t)(k0 + a) * lda + row] : 0.0;
      Vff[((size_t)g * RB + a) * N + row] = ff_from_double(x);
    }
  }
}

// One block per CB output columns (descending eigenvalue order: column c holds Q[:, N-1-c]).
template <class T>
__global__ void __launch_bounds__(256)
k_backtransform(const double* __restrict__ A, int lda, const double* __restrict__ Tm, int N,
                const double* __restrict__ Q, const double* __restrict__ lam, int nkeep,
                double* __restrict__ w, T* __restrict__ U, int ldu) {
  extern __shared__ double bsm[];
  double* Vs = bsm;                      // RB x N, the group's reflectors (zero outside support)
  double* Z = bsm + (size_t)RB * N;      // CB x N, the columns being transformed
  __shared__ double Y[RB][CB], Yt[RB][CB];
  const int c0 = blockIdx.x * CB;
  const int ncol = min(CB, nkeep - c0);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int e = threadIdx.x; e < CB * N; e += blockDim.x) {
    const int c = e / N, t = e - c * N;
    Z[e] = (c < ncol) ? Q[(size_t)(N - 1 - (c0 + c)) * N + t] : 0.0;
  }
  const int nref = N - 2, ng = (nref + RB - 1) / RB;
  for (int g = ng - 1; g >= 0; --g) {
    const int k0 = g * RB, nb = min(RB, nref - k0), r0 = k0 + 1, L = N - r0;
    __syncthreads();
    for (int e = threadIdx.x; e < RB * L; e += blockDim.x) {
      const int a = e / L, row = r0 + (e - a * L);
      Vs[(size_t)a * N + row] = (a < nb && row >= k0 + a + 1) ? A[(size_t)(k0 + a) * lda + row] : 0.0;
    }
    __syncthreads();
    // Y = V^T Z: warp w takes reflectors 2w, 2w + 1 for all CB columns, 2 * CB = 8 partial dots
    // per lane, summed over the warp by a transposing butterfly (each exchange halves the values a
    // lane holds; 9 adds per lane instead of 5 per dot)
    {
      static_assert(RB == 16 && CB == 4, "the butterfly assumes 16 reflectors over 8 warps and 4 columns");
      const int a0 = 2 * warp;
      double acc[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) acc[u] = 0.0;
      const double* va0 = Vs + (size_t)a0 * N;
      const double* va1 = va0 + N;
      for (int row = r0 + lane; row < N; row += 32) {
        const double x0 = va0[row], x1 = va1[row];
#pragma unroll
        for (int c = 0; c < CB; ++c) {
          const double z = Z[(size_t)c * N + row];
          acc[c] = fma(x0, z, acc[c]);
          acc[CB + c] = fma(x1, z, acc[CB + c]);
        }
      }
      const bool b16 = lane & 16, b8 = lane & 8, b4 = lane & 4;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const double send = b16 ? acc[u] : acc[u + 4];
        const double keep = b16 ? acc[u + 4] : acc[u];
        acc[u] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
      }
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const double send = b8 ? acc[u] : acc[u + 2];
        const double keep = b8 ? acc[u + 2] : acc[u];
        acc[u] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
      }
      {
        const double send = b4 ? acc[0] : acc[1];
        const double keep = b4 ? acc[1] : acc[0];
        acc[0] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
      }
      acc[0] += __shfl_xor_sync(0xffffffffu, acc[0], 2);
      acc[0] += __shfl_xor_sync(0xffffffffu, acc[0], 1);
      if ((lane & 3) == 0) {
        const int idx = (b16 ? 4 : 0) + (b8 ? 2 : 0) + (b4 ? 1 : 0);   // = 4 * (a - a0) + c
        Y[a0 + (idx >> 2)][idx & 3] = acc[0];
      }
    }
    __syncthreads();
    // Yt = T Y (T upper triangular), then Z -= V Yt
    if (threadIdx.x < RB * CB) {
      const int i = threadIdx.x / CB, c = threadIdx.x - i * CB;
      const double* Tg = Tm + (size_t)g * RB * RB + i * RB;
      double acc = 0.0;
      for (int j = i; j < RB; ++j) acc = fma(Tg[j], Y[j][c], acc);
      Yt[i][c] = acc;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < CB * L; e += blockDim.x) {
      const int c = e / L, row = r0 + (e - c * L);
      double upd = 0.0;
#pragma unroll
      for (int a = 0; a < RB; ++a) upd = fma(Vs[(size_t)a * N + row], Yt[a][c], upd);
      Z[(size_t)c * N + row] -= upd;
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < ncol * N; e += blockDim.x) {
    const int c = e / N, t = e - c * N;
    U[(size_t)(c0 + c) * ldu + t] = T(Z[e]);
  }
  if (threadIdx.x < ncol) w[c0 + threadIdx.x] = lam[N - 1 - (c0 + threadIdx.x)];
}

// The same back-transformation in double-FP32 arithmetic, for callers that round U to FP32: every
// value is an unevaluated pair hi + lo of FP32 numbers (about 48 significant bits), products are
// formed exactly by FMA and sums carry their rounding errors in a compensation term (the Dot2 scheme
// of Ogita, Rump and Oishi), so each dot product is as accurate as if computed in twice FP32's
// precision.  It runs on the FP32 pipe (128 lanes per SM per clock against FP64's 1.67 FMA), so it
// is several times faster than the FP64 kernel; its error in U (about 1e-14 relative) stays far
// below the FP32 rounding that the FP32-based modes apply to U next.  Same grouping as
// k_backtransform (RB reflectors in compact WY form per group, CB output columns per block); the
// next group's reflectors are copied into the other half of a double buffer (cp.async) while the
// current group is applied, and in Z -= V Yt each thread owns rows and updates all CB columns of a
// row together (CB independent accumulations sharing the V loads).
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void cp_async8(void* sdst, const void* gsrc) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_addr(sdst)), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int PENDING> __device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(PENDING) : "memory");
}

__global__ void __launch_bounds__(256)
k_backtransform_ff(const float2* __restrict__ Vff, const float2* __restrict__ Tff, int N,
                   const double* __restrict__ Q, const double* __restrict__ lam, int nkeep,
                   double* __restrict__ w, double* __restrict__ U, int ldu) {
  extern __shared__ float2 bsf[];
  // bsf: two buffers of RB x N (the reflectors of a group), then Z
  float2* Z = bsf + (size_t)2 * RB * N;            // CB x N, the columns being transformed
  __shared__ float2 Y[RB][CB], Yt[RB][CB];
  const int c0 = blockIdx.x * CB;
  const int ncol = min(CB, nkeep - c0);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nref = N - 2, ng = (nref + RB - 1) / RB;
  // rows [g RB + 1, N) of the RB reflectors of group g into buffer b (the rest of the group's
  // column range is zero and never read)
  auto stage = [&](int g, int b) {
    const int r0 = g * RB + 1, L = N - r0;
    float2* dst = bsf + (size_t)b * RB * N;
    for (int e = threadIdx.x; e < RB * L; e += blockDim.x) {
      const int a = e / L, row = r0 + (e - a * L);
      cp_async8(dst + (size_t)a * N + row, Vff + ((size_t)g * RB + a) * N + row);
    }
    cp_async_commit();
  };
  stage(ng - 1, (ng - 1) & 1);
  for (int e = threadIdx.x; e < CB * N; e += blockDim.x) {
    const int c = e / N, t = e - c * N;
    Z[e] = (c < ncol) ? ff_from_double(Q[(size_t)(N - 1 - (c0 + c)) * N + t]) : make_float2(0.f, 0.f);
  }
  for (int g = ng - 1; g >= 0; --g) {
    const int k0 = g * RB, r0 = k0 + 1;
    const float2* Vs = bsf + (size_t)(g & 1) * RB * N;
    if (g > 0) {
      stage(g - 1, (g - 1) & 1);   // its buffer was last read in the previous iteration (synced below)
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    // Y = V^T Z: warp w takes reflectors 2w, 2w + 1 for all CB columns; the 8 (sum, compensation)
    // pairs of a lane are combined over the warp by a transposing butterfly
    {
      static_assert(RB == 16 && CB == 4, "the butterfly assumes 16 reflectors over 8 warps and 4 columns");
      const int a0 = 2 * warp;
      float sa[8], ca[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) { sa[u] = 0.f; ca[u] = 0.f; }
      const float2* va0 = Vs + (size_t)a0 * N;
      const float2* va1 = va0 + N;
      for (int row = r0 + lane; row < N; row += 32) {
        const float2 x0 = va0[row], x1 = va1[row];
#pragma unroll
        for (int c = 0; c < CB; ++c) {
          const float2 z = Z[(size_t)c * N + row];
          ff_fma_acc(sa[c], ca[c], x0, z);
          ff_fma_acc(sa[CB + c], ca[CB + c], x1, z);
        }
      }
      const bool b16 = lane & 16, b8 = lane & 8, b4 = lane & 4;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const float ss = b16 ? sa[u] : sa[u + 4], cs = b16 ? ca[u] : ca[u + 4];
        const float sk = b16 ? sa[u + 4] : sa[u], ck = b16 ? ca[u + 4] : ca[u];
        sa[u] = sk; ca[u] = ck;
        ff_acc_add(sa[u], ca[u], __shfl_xor_sync(0xffffffffu, ss, 16), __shfl_xor_sync(0xffffffffu, cs, 16));
      }
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const float ss = b8 ? sa[u] : sa[u + 2], cs = b8 ? ca[u] : ca[u + 2];
        const float sk = b8 ? sa[u + 2] : sa[u], ck = b8 ? ca[u + 2] : ca[u];
        sa[u] = sk; ca[u] = ck;
        ff_acc_add(sa[u], ca[u], __shfl_xor_sync(0xffffffffu, ss, 8), __shfl_xor_sync(0xffffffffu, cs, 8));
      }
      {
        const float ss = b4 ? sa[0] : sa[1], cs = b4 ? ca[0] : ca[1];
        const float sk = b4 ? sa[1] : sa[0], ck = b4 ? ca[1] : ca[0];
        sa[0] = sk; ca[0] = ck;
        ff_acc_add(sa[0], ca[0], __shfl_xor_sync(0xffffffffu, ss, 4), __shfl_xor_sync(0xffffffffu, cs, 4));
      }
      ff_acc_add(sa[0], ca[0], __shfl_xor_sync(0xffffffffu, sa[0], 2), __shfl_xor_sync(0xffffffffu, ca[0], 2));
      ff_acc_add(sa[0], ca[0], __shfl_xor_sync(0xffffffffu, sa[0], 1), __shfl_xor_sync(0xffffffffu, ca[0], 1));
      if ((lane & 3) == 0) {
        const int idx = (b16 ? 4 : 0) + (b8 ? 2 : 0) + (b4 ? 1 : 0);   // = 4 * (a - a0) + c
        Y[a0 + (idx >> 2)][idx & 3] = ff_norm(sa[0], ca[0]);
      }
    }
    __syncthreads();
    // Yt = T Y (T upper triangular): output (i, c) by the 4 threads of a quad, each summing every
    // fourth term, combined by two shuffles
    {
      const int o = threadIdx.x >> 2, part = threadIdx.x & 3;   // 64 outputs x 4 parts = 256 threads
      const int i = o / CB, c = o - i * CB;
      const float2* Tg = Tff + (size_t)g * RB * RB + i * RB;
      float sacc = 0.f, cacc = 0.f;
      for (int j = i + part; j < RB; j += 4) ff_fma_acc(sacc, cacc, Tg[j], Y[j][c]);
      ff_acc_add(sacc, cacc, __shfl_xor_sync(0xffffffffu, sacc, 1), __shfl_xor_sync(0xffffffffu, cacc, 1));
      ff_acc_add(sacc, cacc, __shfl_xor_sync(0xffffffffu, sacc, 2), __shfl_xor_sync(0xffffffffu, cacc, 2));
      if (part == 0) Yt[i][c] = ff_norm(sacc, cacc);
    }
    __syncthreads();
    // Z -= V Yt: two rows per thread at a time, CB columns each (2 CB independent accumulations)
    for (int row = r0 + threadIdx.x; row < N; row += 2 * blockDim.x) {
      const int row2 = row + blockDim.x;
      const bool two = row2 < N;
      float sacc[2][CB], cacc[2][CB];
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int c = 0; c < CB; ++c) { sacc[h][c] = 0.f; cacc[h][c] = 0.f; }
#pragma unroll
      for (int a = 0; a < RB; ++a) {
        const float2 v0 = Vs[(size_t)a * N + row];
        const float2 v1 = two ? Vs[(size_t)a * N + row2] : make_float2(0.f, 0.f);
#pragma unroll
        for (int c = 0; c < CB; ++c) {
          const float2 y = Yt[a][c];
          ff_fma_acc(sacc[0][c], cacc[0][c], v0, y);
          ff_fma_acc(sacc[1][c], cacc[1][c], v1, y);
        }
      }
#pragma unroll
      for (int c = 0; c < CB; ++c) {
        float2& z = Z[(size_t)c * N + row];
        z = ff_sub(z, sacc[0][c], cacc[0][c]);
        if (two) {
          float2& z2 = Z[(size_t)c * N + row2];
          z2 = ff_sub(z2, sacc[1][c], cacc[1][c]);
        }
      }
    }
    __syncthreads();   // every thread is done with Vs before it is refilled two groups later
  }
  for (int e = threadIdx.x; e < ncol * N; e += blockDim.x) {
    const int c = e / N, t = e - c * N;
    const float2 z = Z[e];
    U[(size_t)(c0 + c) * ldu + t] = (double)z.x + (double)z.y;   // exact: 48 bits fit in FP64
  }
  if (threadIdx.x < ncol) w[c0 + threadIdx.x] = lam[N - 1 - (c0 + threadIdx.x)];
}

// ------------------------------------------------------------------------------------ host side
struct Plan {
  std::vector<MergeDesc> merges;      // all levels, deepest first
  std::vector<int> level_off;         // offsets into merges per level (+ end)
  std::vector<int> mergeof;           // per level: N entries
};

void build_plan(int N, Plan& pl) {
  std::vector<std::vector<MergeDesc>> by_depth;
  struct Node { int lo, hi, depth; };
  std::vector<Node> stack{{0, N, 0}};
  while (!stack.empty()) {
    Node nd = stack.back();
    stack.pop_back();
    if (nd.hi - nd.lo <= 1) continue;
    int mid = (nd.lo + nd.hi) / 2;
    if ((int)by_depth.size() <= nd.depth) by_depth.resize(nd.depth + 1);
    by_depth[nd.depth].push_back({nd.lo, mid, nd.hi});
    stack.push_back({nd.lo, mid, nd.depth + 1});
    stack.push_back({mid, nd.hi, nd.depth + 1});
  }
  pl.merges.clear();
  pl.level_off.clear();
  pl.mergeof.clear();
  for (int dpt = (int)by_depth.size() - 1; dpt >= 0; --dpt) {
    pl.level_off.push_back((int)pl.merges.size());
    std::vector<int> mo(N, -1);
    int base = (int)pl.merges.size();
    for (size_t q = 0; q < by_depth[dpt].size(); ++q) {
      const MergeDesc& m = by_depth[dpt][q];
      for (int t = m.lo; t < m.hi; ++t) mo[t] = (int)q;
      pl.merges.push_back(m);
    }
    (void)base;
    pl.mergeof.insert(pl.mergeof.end(), mo.begin(), mo.end());
  }
  pl.level_off.push_back((int)pl.merges.size());
}

struct PlanCacheEntry {
  MergeDesc* d_merges = nullptr;
  int* d_mergeof = nullptr;
  Plan plan;
};

std::mutex g_plan_mu;
std::map<std::pair<int, int>, PlanCacheEntry> g_plans;   // (device, N)

const PlanCacheEntry* get_plan(int N) {
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(g_plan_mu);
  auto key = std::make_pair(dev, N);
  auto it = g_plans.find(key);
  if (it != g_plans.end()) return &it->second;
  PlanCacheEntry ent;
  build_plan(N, ent.plan);
  size_t nm = std::max<size_t>(1, ent.plan.merges.size());
  size_t nmo = std::max<size_t>(1, ent.plan.mergeof.size());
  if (cudaMalloc(&ent.d_merges, nm * sizeof(MergeDesc)) != cudaSuccess) return nullptr;
  if (cudaMalloc(&ent.d_mergeof, nmo * sizeof(int)) != cudaSuccess) return nullptr;
  if (!ent.plan.merges.empty())
    cudaMemcpy(ent.d_merges, ent.plan.merges.data(), ent.plan.merges.size() * sizeof(MergeDesc), cudaMemcpyHostToDevice);
  if (!ent.plan.mergeof.empty())
    cudaMemcpy(ent.d_mergeof, ent.plan.mergeof.data(), ent.plan.mergeof.size() * sizeof(int), cudaMemcpyHostToDevice);
  auto res = g_plans.emplace(key, std::move(ent));
  return &res.first->second;
}

inline size_t align_up(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

size_t eig_workspace_bytes(int nmax) {
  size_t N = std::max(nmax, 1);
  size_t b = 0;
  b += align_up(3 * N * sizeof(double));          // d, e, tau
  b += 2 * align_up(4 * N * sizeof(double));      // P, C (double buffered (hi, lo) pairs)
  b += 3 * align_up(N * N * sizeof(double));      // Q, Qtmp, Delta
  b += 10 * align_up(N * sizeof(double));         // lam, lamk, lamtmp, Dw, Zw, Dk, Zk, Dd, rho, spare
  b += align_up(4 * N * sizeof(double));          // rot
  b += align_up((N / RB + 2) * RB * RB * sizeof(double));   // back-transform T blocks
  b += align_up((N / RB + 2) * RB * RB * sizeof(float2));   // T blocks as double-FP32 pairs
  b += align_up((N / RB + 2) * RB * N * sizeof(float2));    // reflector groups as double-FP32 pairs
  b += 7 * align_up(N * sizeof(int));             // colk, cold, perm, Kp, nrot, gperm, spare
  b += align_up(2 * N * sizeof(int));             // gcnt
  return b + 4096;
}

template <class T>
int eig_sym_topk(double* A, int lda, int N, int nkeep, double* w, T* U, int ldu, void* work, size_t work_bytes,
                 int* err, cudaStream_t st, cudaEvent_t* marks, int assembly) {
  if (N <= 0 || nkeep <= 0) return 0;
  if (nkeep > N) nkeep = N;
  if (work_bytes < eig_workspace_bytes(N)) return 1;
  const PlanCacheEntry* pe = get_plan(N);
  if (!pe) return 2;
  char* p = (char*)work;
  auto take = [&](size_t bytes) { void* q = p; p += align_up(bytes); return q; };
  double* d = (double*)take(3 * N * sizeof(double));
  double* e = d + N;
  double* tau = e + N;
  double* P = (double*)take(4 * N * sizeof(double));
  double* Cb = (double*)take(4 * N * sizeof(double));
  DcWork W;
  W.Q = (double*)take((size_t)N * N * sizeof(double));
  W.Qtmp = (double*)take((size_t)N * N * sizeof(double));
  W.Delta = (double*)take((size_t)N * N * sizeof(double));
  W.lam = (double*)take(N * sizeof(double));
  W.lamk = (double*)take(N * sizeof(double));
  W.lamtmp = (double*)take(N * sizeof(double));
  W.Dw = (double*)take(N * sizeof(double));
  W.Zw = (double*)take(N * sizeof(double));
  W.Dk = (double*)take(N * sizeof(double));
  W.Zk = (double*)take(N * sizeof(double));
  W.Dd = (double*)take(N * sizeof(double));
  W.rho = (double*)take(N * sizeof(double));
  W.z2 = (double*)take(N * sizeof(double));
  W.rot = (double*)take(4 * N * sizeof(double));
  W.Tm = (double*)take(((size_t)N / RB + 2) * RB * RB * sizeof(double));
  float2* Tff = (float2*)take(((size_t)N / RB + 2) * RB * RB * sizeof(float2));
  float2* Vff = (float2*)take(((size_t)N / RB + 2) * RB * (size_t)N * sizeof(float2));
  W.colk = (int*)take(N * sizeof(int));
  W.cold = (int*)take(N * sizeof(int));
  W.perm = (int*)take(N * sizeof(int));
  W.Kp = (int*)take(N * sizeof(int));
  W.nrot = (int*)take(N * sizeof(int));
  W.gperm = (int*)take(N * sizeof(int));
  W.gcnt = (int*)take(2 * N * sizeof(int));
  W.mergeof = nullptr;

  // exchange buffers of the tridiagonalisation: every byte 0x0f, i.e. pairs whose both words carry
  // epoch 3, which no consumer waits for before the buffer has been rewritten
  cudaMemsetAsync(P, 0x0f, 4 * N * sizeof(double), st);
  cudaMemsetAsync(Cb, 0x0f, 4 * N * sizeof(double), st);
  cudaMemsetAsync(W.Q, 0, (size_t)N * N * sizeof(double), st);
  cudaMemsetAsync(d, 0, 3 * N * sizeof(double), st);

  // 1. tridiagonalisation (cooperative: all blocks co-resident)
  {
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    int G = N >= 3 ? std::max(1, std::min(nsm, (N + 3) / 4)) : 1;
    cudaFuncSetAttribute(k_tridiag, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    size_t smem = 0;
    for (int attempt = 0; attempt < 8; ++attempt) {
      const int nslot = (N + G - 1) / G;
      smem = (4 + (size_t)nslot) * N * sizeof(double);
      cudaFuncSetAttribute(k_tridiag, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)std::max<size_t>(smem, 48 * 1024));
      int occ = 0;
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_tridiag, TD_THREADS, smem);
      if ((long long)occ * nsm >= G) break;
      G = std::max(1, occ * nsm);     // fewer blocks own more columns each
      if (occ == 0) { cudaGetLastError(); return 1000 + (int)cudaErrorCooperativeLaunchTooLarge; }
    }
    if ((N + G - 1) / G > TD_MAX_SLOTS) return 1000 + (int)cudaErrorInvalidValue;
    long long poll_limit = wait_limit(kPollLimit);
    void* args[] = {&A, &lda, &N, &d, &e, &tau, &P, &Cb, &err, &poll_limit};
    cudaError_t ce = cudaLaunchCooperativeKernel((void*)k_tridiag, dim3(G), dim3(TD_THREADS), args, smem, st);
    note_launch();
    if (ce != cudaSuccess) return 1000 + (int)ce;
  }
  if (marks) cudaEventRecord(marks[0], st);
  // 2. divide and conquer
  k_dc_init<<<(N + 255) / 256, 256, 0, st>>>(d, e, N, W.lam, W.Q); note_launch();
  const Plan& pl = pe->plan;
  const int nlev = (int)pl.level_off.size() - 1;
  for (int lv = 0; lv < nlev; ++lv) {
    const int m0 = pl.level_off[lv], m1 = pl.level_off[lv + 1];
    const int nm = m1 - m0;
    if (nm <= 0) continue;
    const MergeDesc* dm = pe->d_merges + m0;
    const int* dmo = pe->d_mergeof + (size_t)lv * N;
    int kmax = 0;
    for (int q = m0; q < m1; ++q) kmax = std::max(kmax, pl.merges[q].hi - pl.merges[q].lo);
    if (kmax <= DC_SMALL_K) {
      k_dc_small<<<nm, DC_THREADS, small_smem_bytes(kmax), st>>>(dm, e, N, W, err); note_launch();
      continue;
    }
    const size_t psmem = prep_smem_bytes(kmax);
    if (psmem > 40 * 1024) cudaFuncSetAttribute(k_dc_prep, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)psmem);
    k_dc_prep<<<nm, DC_THREADS, psmem, st>>>(dm, e, N, W); note_launch();
    k_dc_rot<<<dim3((kmax + 127) / 128, nm), 128, 0, st>>>(dm, N, W); note_launch();
    // The per-root work is FP64-bound (2 FMA/clk/SM), so the grids use two-warp blocks (one warp per
    // root) to spread the roots over all SMs.  (One thread per root for the small merges measured
    // 3x slower: one warp per SM leaves its FP64 dependency chains uncovered.)
    k_dc_secular<32><<<(N + 1) / 2, 64, 0, st>>>(dm, dmo, N, W, err); note_launch();
    k_dc_zhat<32><<<(N + 1) / 2, 64, 0, st>>>(dm, dmo, N, W); note_launch();
    k_dc_vecs<32><<<(N + 1) / 2, 64, 0, st>>>(dm, dmo, N, W); note_launch();
    dim3 gg((kmax + DG_T - 1) / DG_T, (kmax + DG_T - 1) / DG_T, nm);
    k_dc_gemm<<<gg, 256, 0, st>>>(dm, N, W); note_launch();
    const size_t fsmem = (size_t)kmax * (sizeof(double) + sizeof(long long));
    if (fsmem > 40 * 1024) cudaFuncSetAttribute(k_dc_finish, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsmem);
    k_dc_finish<<<nm, 256, fsmem, st>>>(dm, N, W); note_launch();
    k_dc_copy<<<dim3((kmax + 7) / 8, nm), 256, 0, st>>>(dm, N, W); note_launch();
  }
  if (marks) cudaEventRecord(marks[1], st);
  // 3. back-transformation of the top nkeep columns (descending eigenvalues)
  {
    const int ng = std::max(1, (N - 2 + RB - 1) / RB);
    if constexpr (sizeof(T) == sizeof(double)) {
      // (larger orders than the double-buffered staging fits in shared memory take the FP64 kernel)
      if (assembly == kAssemblyFF && N >= 3 && (size_t)(2 * RB + CB) * N * sizeof(float2) <= 227 * 1024) {
        k_bt_tmat<<<ng, 256, 0, st>>>(A, lda, tau, N, W.Tm, Vff, Tff); note_launch();
        const size_t smem = (size_t)(2 * RB + CB) * N * sizeof(float2);
        if (smem > 40 * 1024) cudaFuncSetAttribute(k_backtransform_ff, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_backtransform_ff<<<(nkeep + CB - 1) / CB, 256, smem, st>>>(Vff, Tff, N, W.Q, W.lam, nkeep, w, U, ldu); note_launch();
        return cudaGetLastError() == cudaSuccess ? 0 : 4;
      }
    }
    if (N >= 3) {
      k_bt_tmat<<<ng, 256, 0, st>>>(A, lda, tau, N, W.Tm, nullptr, nullptr); note_launch();
    }
    const size_t smem = (size_t)(RB + CB) * N * sizeof(double);
    if (smem > 40 * 1024) cudaFuncSetAttribute(k_backtransform<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_backtransform<T><<<(nkeep + CB - 1) / CB, 256, smem, st>>>(A, lda, W.Tm, N, W.Q, W.lam, nkeep, w, U, ldu); note_launch();
  }
  return cudaGetLastError() == cudaSuccess ? 0 : 4;
}

template int eig_sym_topk<float>(double*, int, int, int, double*, float*, int, void*, size_t, int*, cudaStream_t,
                                  cudaEvent_t*, int);
template int eig_sym_topk<double>(double*, int, int, int, double*, double*, int, void*, size_t, int*, cudaStream_t,
                                   cudaEvent_t*, int);

}  // namespace cakf
