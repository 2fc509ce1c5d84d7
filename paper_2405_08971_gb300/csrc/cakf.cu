// Host orchestration of the CAKF forward pass and CAKS backward pass behind the C ABI of cakf.h.
//
// Device data layout (all factors column-major, leading dimension ldn = n rounded up to 128):
//   X        n coordinate records (C4<T>, pre-scaled by c_nu / l_x)
//   Mplus[k] n x c_k truncated downdate factor M+_k, k = 0..T (c_k <= r); its columns are kept
//            orthogonal with squared norms lam_k (every truncation rotates onto the eigenbasis),
//            so the leading block of the next truncation Gram is diag(a^2 lam_k)
//   PVv[k]   n x (i_k + 1): [P^-_k W_k, P^-_k w_k]  (the new factor columns and the mean shift)
//   Vv[k]    m_k x (i_k + 1): [V_k, v_k] -- G-orthonormal directions and solution coefficients
//   S[k]     m_k x i_k actions
//   mf, vf   (T+1) x n filter means / variances (FP64)
#include <atomic>
#include <type_traits>
#include <cstring>
#include <cstdio>
#include <string>
#include <vector>
#include <memory>
#include <cmath>
#include "cakf.h"
#include "internal.h"

using namespace cakf;

namespace {

thread_local std::string g_err;
std::atomic<unsigned long long> g_mem_limit{0};   // cap on a context's device bytes (0 = none)

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

// Where a caller's pointer lives: host memory (pageable or pinned), device memory of the current
// device, or device memory of another device (which the kernels here must not be given).
enum PtrKind { kHost = 0, kDevice = 1, kOtherDevice = 2 };

PtrKind ptr_kind(const void* p) {
  if (!p) return kHost;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) { cudaGetLastError(); return kHost; }
  if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) return kHost;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return kOtherDevice; }
  return (at.type == cudaMemoryTypeManaged || at.device == dev) ? kDevice : kOtherDevice;
}

bool is_device_ptr(const void* p) { return ptr_kind(p) == kDevice; }

inline int round_up(int x, int m) { return (x + m - 1) / m * m; }

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

}  // namespace

struct cakf_ctx {
  // problem
  int n = 0, dim = 0, kernel = 1, T = 0, budget = 0, rank_r = 0, precision = 1;
  double lx = 1, lt = 1, sf2 = 1, sn2 = 1, dt = 1, a = 1, cg_rtol = 0;
  // temporal factor: dprime = 1 (OU: the factors are propagated lazily by the scalar a) or 2
  // (Matern-3/2: two row blocks of ldn rows, positions then velocities; the prediction M^- =
  // (A^t (x) I) M+ is applied in place, after which the step runs with the scalar 1).  At and
  // Pt are A^t and P^t_inf, row-major.
  int dprime = 1;
  double At[4] = {1, 0, 0, 1}, Pt[4] = {1, 0, 0, 1};
  // the scalar the lazily propagated factors carry (a for OU, 1 once the two-block prediction has
  // been applied)
  double a_lazy() const { return dprime == 2 ? 1.0 : a; }
  bool has_mu = false, replay = false;
  std::vector<int> obs_ptr, icap, mcols, replay_counts;
  // sizes: ldn rows per block, ldf = dprime * ldn rows of a factor column, mstride = the stride
  // of the per-step state means in mf (n for OU, ldf for the two-block state)
  int ldn = 0, ldf = 0, mstride = 0, mmax = 0, rmax = 0, imax = 0, nmax_eig = 0, cwmax = 0;
  std::vector<size_t> off_M, off_PV, off_KV, off_V, off_S;
  // device memory
  std::vector<DevBuf> bufs;
  size_t dev_bytes = 0;
  void* X = nullptr;       // C4<T>
  int* obs = nullptr;
  double* y = nullptr;
  double* mu = nullptr;
  double* mf = nullptr;
  double* vf = nullptr;
  void* Mpool = nullptr;
  void* PVpool = nullptr;
  void* KVpool = nullptr;     // K(X, X_o)[V v] per step (PV before its low-rank correction)
  void* Vpool = nullptr;
  void* Spool = nullptr;
  double* rep = nullptr;   // replayed actions (device, double)
  std::vector<size_t> off_rep;
  double* nll = nullptr;   // T+1
  double* eta = nullptr;   // (T+1) * budget
  double* alpha = nullptr;
  int* count = nullptr;    // T+1
  int* err = nullptr;      // device error flag
  int* active = nullptr;
  double* r0sq = nullptr;     // (T+1) |r0|^2 per step
  double* rfin = nullptr;     // (T+1) |r|^2 of the final residual per step
  double* dropped_f = nullptr;   // (T+1) discarded eigenvalue mass of the filter truncation per step
  double* dropped_s = nullptr;   // (T+1) the same for the smoother truncation
  // workspace
  double *mpred = nullptr, *rs_plus = nullptr, *rs_pw = nullptr, *lam = nullptr, *lam2 = nullptr;
  void *Xo = nullptr, *Mo = nullptr, *rv = nullptr, *r0v = nullptr, *sv = nullptr, *gv = nullptr, *GV = nullptr,
       *part = nullptr, *tv = nullptr, *GS = nullptr, *Qa = nullptr;
  double* dots = nullptr;
  double* dots2 = nullptr;
  double* dpart = nullptr;     // per-block partials of the CG dot passes
  double* part64 = nullptr;
  size_t part64_elems = 0;
  double* gram = nullptr;
  double* small = nullptr;   // scratch for small FP64 matrices
  size_t small_elems = 0;
  // the per-step NLL term runs on a side stream, overlapped with the truncation eigensolver
  cudaStream_t st_nll = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  double* small_nll = nullptr;
  double* part_nll = nullptr;
  size_t part_nll_elems = 0;
  double* U64 = nullptr;
  void* UT = nullptr;
  void* eigw = nullptr;
  size_t eigw_bytes = 0;
  double* wv = nullptr;
  // smoother
  void *KWa = nullptr, *KWb = nullptr;   // smoother: K [Ws, ws] (ldn x (cw + 1)), double buffered
  void *WsA = nullptr, *WsB = nullptr, *wsA = nullptr, *wsB = nullptr, *Xs = nullptr, *Y = nullptr, *Xobs = nullptr,
       *Fb = nullptr;
  void* KX = nullptr;   // two-block smoother: K A^T [Ws ws] (ldf x (cw + 1))
  double* Gws = nullptr;
  double* Gws2 = nullptr;
  // tensor-core operand staging (bf16 / tf32 paths)
  void* Bpack = nullptr;
  size_t Bpack_bytes = 0;
  double* coords64 = nullptr;
  // truncation rotations per step (for the NLL tangent pass) and tangent workspace
  double* Upool = nullptr;
  std::vector<size_t> off_U;
  std::vector<int> Urows;
  void *dMa = nullptr, *dMb = nullptr, *Eg = nullptr, *KS = nullptr, *KlS = nullptr, *dmo = nullptr, *tvec = nullptr;
  double *dmA = nullptr, *dmB = nullptr, *dmpred = nullptr, *gsmall = nullptr, *grad = nullptr;
  size_t gsmall_elems = 0;
  double* ms_dev = nullptr;   // smoother outputs when the caller passes host arrays
  double* vs_dev = nullptr;
  // factor storage between the filter and the smoother / gradient pass: seg_c = 0 keeps every step
  // resident; otherwise the pools are rings of seg_c steps (M: seg_c + 1 slots) and the steps
  // [res_a, res_b] are resident; RECOMPUTE keeps M+ and lam at every segment start, STORE_BF16
  // keeps BF16 copies of every step's factors
  int storage = CAKF_STORE_FP32, ckpt_req = 0, seg_c = 0, res_a = 1, res_b = 0;
  int policy = CAKF_POLICY_CG;
  bool freeze = false;     // truncate with the stored rotations of the previous run
  void* GSb = nullptr;     // batch policies: G [S r0] (m x (i + 1))
  double* Lb = nullptr;    // batch policies: Cholesky factor of S^T G S and z = L^-1 S^T r0
  void* ckptM = nullptr;
  double* ckpt_lam = nullptr;
  void *Mh = nullptr, *PVh = nullptr, *KVh = nullptr, *Vh = nullptr;
  // state
  bool filtered = false;
  long long launch_base = 0;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  bool profiling = false;
  cakf_stats stats{};
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> prof_gb, prof_mv, prof_eig, prof_eig_tri, prof_eig_dc, prof_eig_bt;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> prof_phase;
  std::vector<double> prof_gb_flops, prof_gb_evals, prof_mv_evals;
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;

  ~cakf_ctx() { release(); }

  void release() {
    for (auto& b : bufs) if (b.p) cudaFree(b.p);
    bufs.clear();
    dev_bytes = 0;
    for (auto e : ev_pool) cudaEventDestroy(e);
    ev_pool.clear();
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
    ev0 = ev1 = nullptr;
    if (ev_fork) cudaEventDestroy(ev_fork);
    if (ev_join) cudaEventDestroy(ev_join);
    ev_fork = ev_join = nullptr;
    if (st_nll) cudaStreamDestroy(st_nll);
    st_nll = nullptr;
  }

  template <class P> int alloc(P*& out, size_t bytes) {
    void* p = nullptr;
    bytes = std::max<size_t>(bytes, 16);
    const unsigned long long cap = g_mem_limit.load();
    if (cap && dev_bytes + bytes > cap) {
      out = nullptr;
      return fail(CAKF_ERR_OOM, "device memory limit of " + std::to_string(cap) + " bytes reached (cakf_set_device_memory_limit)");
    }
    cudaError_t ce = cudaMalloc(&p, bytes);
    if (ce != cudaSuccess) {
      cudaGetLastError();
      out = nullptr;
      return fail(CAKF_ERR_OOM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed: " + cudaGetErrorString(ce));
    }
    bufs.push_back({p, bytes});
    dev_bytes += bytes;
    out = (P*)p;
    return CAKF_OK;
  }

  cudaEvent_t ev() {
    if (ev_used >= ev_pool.size()) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      ev_pool.push_back(e);
    }
    return ev_pool[ev_used++];
  }
};

namespace {

size_t elem_size(int precision) { return precision == CAKF_FP64 ? 8 : 4; }

// Operand mode of the tensor-core Gram x block for a precision (gram_block_tc's kind), -1 for the
// SIMT paths.
int tc_kind_of(int precision) {
  switch (precision) {
    case CAKF_BF16: return 0;
    case CAKF_FP16X3: return 1;
    case CAKF_TF32: return 2;
    case CAKF_TF32X3: return 3;
    default: return -1;
  }
}

// ------------------------------------------------------------------------------------ planning
int plan_and_alloc(cakf_ctx* c, const cakf_problem* p) {
  const int T = p->T;
  c->obs_ptr.assign(p->obs_ptr, p->obs_ptr + T + 1);
  c->icap.assign(T + 1, 0);
  c->mcols.assign(T + 1, 0);
  c->mmax = 0;
  for (int k = 1; k <= T; ++k) {
    int mk = c->obs_ptr[k] - c->obs_ptr[k - 1];
    c->mmax = std::max(c->mmax, mk);
    int ic = c->replay ? c->replay_counts[k] : std::min(c->budget, mk);
    if (mk == 0) ic = 0;
    c->icap[k] = ic;
    int prev = c->mcols[k - 1];
    c->mcols[k] = (c->rank_r > 0) ? std::min(c->rank_r, prev + ic) : prev + ic;
  }
  c->imax = 0;
  c->rmax = 0;
  for (int k = 0; k <= T; ++k) { c->imax = std::max(c->imax, c->icap[k]); c->rmax = std::max(c->rmax, c->mcols[k]); }
  c->ldn = round_up(std::max(c->n, 1), 128);
  c->ldf = c->dprime * c->ldn;
  c->mstride = c->dprime == 1 ? c->n : c->ldf;
  // smoother width bound: rank (after truncation) or the untruncated accumulation
  int cw = 0, cwmax = 0;
  for (int k = T; k >= 1; --k) {
    cw = (k == T) ? c->icap[T] : ((c->rank_r > 0) ? std::min(c->rank_r, cw + c->icap[k]) : cw + c->icap[k]);
    cwmax = std::max(cwmax, cw);
    // the pre-truncation width at step k is icap[k] + previous cw
  }
  int cwfull = 0;
  {
    int cc = c->icap[T];
    cwfull = cc;
    for (int k = T - 1; k >= 1; --k) {
      int full = c->icap[k] + cc;
      cwfull = std::max(cwfull, full);
      cc = (c->rank_r > 0) ? std::min(c->rank_r, full) : full;
    }
  }
  c->cwmax = std::max(cwmax, 1);
  int Nf = 0;
  for (int k = 1; k <= T; ++k) Nf = std::max(Nf, c->mcols[k - 1] + c->icap[k]);
  c->nmax_eig = std::max({Nf, cwfull, 1});
  const int wmax = std::max(c->cwmax, cwfull) + 1;   // width of the smoother Gram x block

  const size_t es = elem_size(c->precision);
  const size_t ldn = c->ldn, ldf = c->ldf;
  c->storage = p->factor_storage;
  c->ckpt_req = p->checkpoint_every;
  c->policy = p->policy;
  c->seg_c = 0;
  if (c->storage != CAKF_STORE_FP32) {
    const int seg = p->checkpoint_every > 0 ? p->checkpoint_every : 20;
    c->seg_c = seg < T ? seg : 0;   // a segment as long as the series keeps every step resident
  }
  // per-step pools
  c->off_M.assign(T + 2, 0);
  c->off_PV.assign(T + 2, 0);
  c->off_KV.assign(T + 2, 0);
  c->off_V.assign(T + 2, 0);
  c->off_S.assign(T + 2, 0);
  for (int k = 0; k <= T; ++k) {
    int mk = (k == 0) ? 0 : c->obs_ptr[k] - c->obs_ptr[k - 1];
    c->off_M[k + 1] = c->off_M[k] + ldf * c->mcols[k];
    c->off_PV[k + 1] = c->off_PV[k] + (c->icap[k] ? ldf * (c->icap[k] + 1) : 0);
    c->off_KV[k + 1] = c->off_KV[k] + (c->icap[k] ? ldn * (c->icap[k] + 1) : 0);
    c->off_V[k + 1] = c->off_V[k] + (size_t)mk * (c->icap[k] + 1);
    c->off_S[k + 1] = c->off_S[k] + (size_t)mk * c->icap[k];
  }
  const size_t Ntot = c->obs_ptr[T];
  int rc;
  const size_t n = c->n;
  if ((rc = c->alloc(c->X, n * 4 * es))) return rc;
  if ((rc = c->alloc(c->coords64, n * 3 * sizeof(double)))) return rc;
  if ((rc = c->alloc(c->obs, std::max<size_t>(Ntot, 1) * sizeof(int)))) return rc;
  if ((rc = c->alloc(c->y, std::max<size_t>(Ntot, 1) * sizeof(double)))) return rc;
  if (c->has_mu && (rc = c->alloc(c->mu, (size_t)(T + 1) * n * sizeof(double)))) return rc;
  if ((rc = c->alloc(c->mf, (size_t)(T + 1) * c->mstride * sizeof(double)))) return rc;
  if ((rc = c->alloc(c->vf, (size_t)(T + 1) * n * sizeof(double)))) return rc;
  if (c->seg_c == 0) {
    if ((rc = c->alloc(c->Mpool, c->off_M[T + 1] * es))) return rc;
    if ((rc = c->alloc(c->PVpool, c->off_PV[T + 1] * es))) return rc;
    if ((rc = c->alloc(c->KVpool, c->off_KV[T + 1] * es))) return rc;
    if ((rc = c->alloc(c->Vpool, c->off_V[T + 1] * es))) return rc;
  } else {
    const size_t sc = c->seg_c, rmx = std::max(c->rmax, 1), ip = c->imax + 1;
    if ((rc = c->alloc(c->Mpool, (sc + 1) * ldn * rmx * es))) return rc;
    if ((rc = c->alloc(c->PVpool, sc * ldn * ip * es))) return rc;
    if ((rc = c->alloc(c->KVpool, sc * ldn * ip * es))) return rc;
    if ((rc = c->alloc(c->Vpool, sc * (size_t)std::max(c->mmax, 1) * ip * es))) return rc;
    if (c->storage == CAKF_RECOMPUTE) {
      const size_t nck = (size_t)(T - 1) / sc + 1;
      if ((rc = c->alloc(c->ckptM, nck * ldn * rmx * es))) return rc;
      if ((rc = c->alloc(c->ckpt_lam, nck * rmx * sizeof(double)))) return rc;
    } else {
      if ((rc = c->alloc(c->Mh, c->off_M[T + 1] * 2))) return rc;
      if ((rc = c->alloc(c->PVh, c->off_PV[T + 1] * 2))) return rc;
      if ((rc = c->alloc(c->KVh, c->off_PV[T + 1] * 2))) return rc;
      if ((rc = c->alloc(c->Vh, c->off_V[T + 1] * 2))) return rc;
    }
  }
  if ((rc = c->alloc(c->Spool, c->off_S[T + 1] * es))) return rc;
  if (c->policy != CAKF_POLICY_CG) {
    const size_t ib = std::max(c->imax, 1);
    if ((rc = c->alloc(c->GSb, (size_t)std::max(c->mmax, 1) * (ib + 1) * es))) return rc;
    if ((rc = c->alloc(c->Lb, (2 * ib * ib + 2 * ib + 16) * sizeof(double)))) return rc;
  }
  if (c->replay) {
    c->off_rep.assign(T + 2, 0);
    for (int k = 0; k <= T; ++k) {
      int mk = (k == 0) ? 0 : c->obs_ptr[k] - c->obs_ptr[k - 1];
      c->off_rep[k + 1] = c->off_rep[k] + (size_t)mk * c->icap[k];
    }
    if ((rc = c->alloc(c->rep, c->off_rep[T + 1] * sizeof(double)))) return rc;
  }
  const int B = std::max(c->budget, c->imax);
  if ((rc = c->alloc(c->nll, (T + 1) * sizeof(double)))) return rc;
  if ((rc = c->alloc(c->eta, (size_t)(T + 1) * B * sizeof(double)))) return rc;
  if ((rc = c->alloc(c->alpha, (size_t)(T + 1) * B * sizeof(double)))) return rc;
  if ((rc = c->alloc(c->count, (T + 1) * sizeof(int)))) return rc;
  if ((rc = c->alloc(c->err, 16))) return rc;
  if ((rc = c->alloc(c->active, 16))) return rc;
  if ((rc = c->alloc(c->r0sq, (T + 1) * sizeof(double)))) return rc;
  if ((rc = c->alloc(c->rfin, (T + 1) * sizeof(double)))) return rc;
  if ((rc = c->alloc(c->dropped_f, (T + 1) * sizeof(double)))) return rc;
  if ((rc = c->alloc(c->dropped_s, (T + 1) * sizeof(double)))) return rc;
  if ((rc = c->alloc(c->mpred, c->mstride * sizeof(double)))) return rc;
  if ((rc = c->alloc(c->rs_plus, n * sizeof(double)))) return rc;
  if ((rc = c->alloc(c->rs_pw, n * sizeof(double)))) return rc;
  const size_t NE = c->nmax_eig;
  if ((rc = c->alloc(c->lam, NE * sizeof(double)))) return rc;
  if ((rc = c->alloc(c->lam2, NE * sizeof(double)))) return rc;
  const size_t mm = std::max(c->mmax, 1);
  if ((rc = c->alloc(c->Xo, mm * 4 * es))) return rc;
  if ((rc = c->alloc(c->Mo, mm * std::max(c->rmax, 1) * es))) return rc;
  if ((rc = c->alloc(c->rv, mm * es))) return rc;
  if ((rc = c->alloc(c->r0v, mm * es))) return rc;
  if ((rc = c->alloc(c->sv, mm * es))) return rc;
  if ((rc = c->alloc(c->gv, mm * es))) return rc;
  if ((rc = c->alloc(c->GV, mm * std::max(B, 1) * es))) return rc;
  if ((rc = c->alloc(c->GS, mm * std::max(B, 1) * es))) return rc;
  if ((rc = c->alloc(c->Qa, mm * std::max(B, 1) * es))) return rc;
  if ((rc = c->alloc(c->part, mm * std::max(32, gram_matvec_slots((int)mm)) * es))) return rc;
  if ((rc = c->alloc(c->tv, std::max<size_t>(c->rmax, 1) * ((mm + 1023) / 1024 + 1) * es))) return rc;
  if ((rc = c->alloc(c->dots, (B + 8) * sizeof(double)))) return rc;
  if ((rc = c->alloc(c->dots2, (B + 8) * sizeof(double)))) return rc;
  if ((rc = c->alloc(c->dpart, cg_dpart_elems((int)mm, B) * sizeof(double)))) return rc;
  c->part64_elems = std::max<size_t>(size_t(1) << 24, NE * NE * 4);   // partial tiles of the split-K products
  if ((rc = c->alloc(c->part64, c->part64_elems * sizeof(double)))) return rc;
  if ((rc = c->alloc(c->gram, NE * NE * sizeof(double)))) return rc;
  c->small_elems = 8 * (NE * (size_t)wmax + NE * NE) + 64;
  if ((rc = c->alloc(c->small, c->small_elems * sizeof(double)))) return rc;
  if ((rc = c->alloc(c->small_nll, (2 * (size_t)B * B + 4 * (size_t)B + 16) * sizeof(double)))) return rc;
  c->part_nll_elems = std::max<size_t>(size_t(1) << 18, (size_t)B * B * 64);
  if ((rc = c->alloc(c->part_nll, c->part_nll_elems * sizeof(double)))) return rc;
  if (!c->st_nll && cudaStreamCreateWithFlags(&c->st_nll, cudaStreamNonBlocking) != cudaSuccess)
    return fail(CAKF_ERR_CUDA, "cudaStreamCreateWithFlags failed");
  if (!c->ev_fork && cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess)
    return fail(CAKF_ERR_CUDA, "cudaEventCreate failed");
  if (!c->ev_join && cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess)
    return fail(CAKF_ERR_CUDA, "cudaEventCreate failed");
  if ((rc = c->alloc(c->U64, NE * NE * sizeof(double)))) return rc;
  if ((rc = c->alloc(c->UT, NE * NE * es))) return rc;
  if ((rc = c->alloc(c->wv, NE * sizeof(double)))) return rc;
  c->eigw_bytes = eig_workspace_bytes((int)NE);
  if ((rc = c->alloc(c->eigw, c->eigw_bytes))) return rc;
  const size_t wsw = std::max(c->cwmax, cwfull);
  if ((rc = c->alloc(c->WsA, ldf * std::max<size_t>(wsw, 1) * es))) return rc;
  if ((rc = c->alloc(c->WsB, ldf * std::max<size_t>(wsw, 1) * es))) return rc;
  if ((rc = c->alloc(c->wsA, ldf * es))) return rc;
  if ((rc = c->alloc(c->wsB, ldf * es))) return rc;
  if ((rc = c->alloc(c->KWa, ldf * (wsw + 1) * es))) return rc;
  if ((rc = c->alloc(c->KWb, ldf * (wsw + 1) * es))) return rc;
  const size_t wfin = std::max<size_t>(wmax, c->imax + 1);
  if ((rc = c->alloc(c->Xs, ldf * wfin * es))) return rc;
  if ((rc = c->alloc(c->Y, ldf * wfin * es))) return rc;
  if (c->dprime == 2 && (rc = c->alloc(c->KX, ldf * wfin * es))) return rc;
  if ((rc = c->alloc(c->Xobs, mm * wfin * es))) return rc;
  if ((rc = c->alloc(c->Fb, mm * std::max<size_t>(NE, 1) * es))) return rc;
  if ((rc = c->alloc(c->Gws, NE * NE * sizeof(double)))) return rc;
  if ((rc = c->alloc(c->Gws2, NE * NE * sizeof(double)))) return rc;
  // truncation rotations U_k (N_k x c_k, FP64) of every step, kept for the gradient pass
  c->off_U.assign(T + 2, 0);
  c->Urows.assign(T + 1, 0);
  for (int k = 1; k <= T; ++k) {
    const bool trunc = c->rank_r > 0 && c->icap[k] > 0;
    c->Urows[k] = trunc ? c->mcols[k - 1] + c->icap[k] : 0;
    c->off_U[k + 1] = c->off_U[k] + (trunc ? (size_t)c->Urows[k] * c->mcols[k] : 0);
  }
  c->off_U[1] = 0;
  for (int k = 1; k <= T; ++k) c->off_U[k + 1] = c->off_U[k] + (size_t)c->Urows[k] * (c->Urows[k] ? c->mcols[k] : 0);
  if ((rc = c->alloc(c->Upool, std::max<size_t>(c->off_U[T + 1], 1) * sizeof(double)))) return rc;
  if (tc_kind_of(c->precision) >= 0) {
    c->Bpack_bytes = gram_tc_staging_bytes(std::max(c->n, c->mmax), (int)wfin, tc_kind_of(c->precision)) + 4096;
    if ((rc = c->alloc(c->Bpack, c->Bpack_bytes))) return rc;
  }
  if (!c->ev0) { cudaEventCreate(&c->ev0); cudaEventCreate(&c->ev1); }
  return CAKF_OK;
}

int copy_in(void* dst, const void* src, size_t bytes, cudaStream_t st) {
  if (bytes == 0) return CAKF_OK;
  const PtrKind kind = ptr_kind(src);
  if (kind == kOtherDevice) return fail(CAKF_ERR_ARG, "an input array lives on another device than the current one");
  cudaError_t ce = cudaMemcpyAsync(dst, src, bytes, kind == kDevice ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st);
  return ce == cudaSuccess ? CAKF_OK : fail(CAKF_ERR_CUDA, std::string("copy in: ") + cudaGetErrorString(ce));
}

int copy_out(double* dst, const double* src, size_t elems, cudaStream_t st) {
  if (!dst || elems == 0) return CAKF_OK;
  const PtrKind kind = ptr_kind(dst);
  if (kind == kOtherDevice) return fail(CAKF_ERR_ARG, "an output array lives on another device than the current one");
  cudaError_t ce = cudaMemcpyAsync(dst, src, elems * sizeof(double),
                                   kind == kDevice ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st);
  return ce == cudaSuccess ? CAKF_OK : fail(CAKF_ERR_CUDA, std::string("copy out: ") + cudaGetErrorString(ce));
}

// ------------------------------------------------------------------------------------ runner
template <class T>
struct Runner {
  cakf_ctx* c;
  cudaStream_t st;
  bool tc;      // tensor-core Gram x block
  int tc_kind;  // 0 BF16, 1 split FP16 (three MMAs per slice)

  // phase timers (profiling on): begin returns the start event, end records the pair
  bool quiet = false;   // no phase timers (recomputation inside the smoother or gradient pass)
  // temporal interpolation queries (cakf_interpolate): per step k the query indices with
  // t_k <= t < t_{k+1}; outputs nq x n (device, FP64); mu_q nq x n or null
  struct Queries {
    std::vector<std::vector<int>> at_k;
    std::vector<double> tq;
    const double* mu_q = nullptr;
    double *fm = nullptr, *fv = nullptr, *sm = nullptr, *sv = nullptr;
  };
  const Queries* qs = nullptr;
  cudaEvent_t ph_begin() {
    if (!c->profiling || quiet) return nullptr;
    cudaEvent_t e = c->ev();
    cudaEventRecord(e, st);
    return e;
  }
  void ph_end(int id, cudaEvent_t e0) {
    if (!e0) return;
    cudaEvent_t e1 = c->ev();
    cudaEventRecord(e1, st);
    c->prof_phase.push_back({id, {e0, e1}});
  }

  // per-step factors: exact offsets when every step is resident, ring slots otherwise
  T* Mk(int k) {
    return c->seg_c ? (T*)c->Mpool + (size_t)(k % (c->seg_c + 1)) * c->ldn * std::max(c->rmax, 1)
                    : (T*)c->Mpool + c->off_M[k];
  }
  T* PV(int k) {
    return c->seg_c ? (T*)c->PVpool + (size_t)(k % c->seg_c) * c->ldn * (c->imax + 1) : (T*)c->PVpool + c->off_PV[k];
  }
  T* KV(int k) {
    return c->seg_c ? (T*)c->KVpool + (size_t)(k % c->seg_c) * c->ldn * (c->imax + 1) : (T*)c->KVpool + c->off_KV[k];
  }
  T* Vk(int k) {
    return c->seg_c ? (T*)c->Vpool + (size_t)(k % c->seg_c) * std::max(c->mmax, 1) * (c->imax + 1)
                    : (T*)c->Vpool + c->off_V[k];
  }

  // ---------------------------------------------------------------- factor storage
  // M+_k and its eigenvalues at the start of a RECOMPUTE segment (k = a - 1, a multiple of seg_c)
  void save_checkpoint(int k) {
    const size_t j = (size_t)k / c->seg_c, rmx = std::max(c->rmax, 1);
    const int cols = c->mcols[k];
    if (cols > 0) {
      cudaMemcpyAsync((T*)c->ckptM + j * c->ldn * rmx, Mk(k), (size_t)c->ldn * cols * sizeof(T),
                      cudaMemcpyDeviceToDevice, st);
      cudaMemcpyAsync(c->ckpt_lam + j * rmx, c->lam, cols * sizeof(double), cudaMemcpyDeviceToDevice, st);
    }
  }
  // BF16 copies of step k's factors (STORE_BF16)
  void pack_history(int k) {
    if (sizeof(T) != 4) return;
    const int ldn = c->ldn, ic = c->icap[k];
    if (k == 1) pack_one(0);
    pack_one(k);
    if (mk(k) > 0 && ic > 0) {
      to_bf16((const float*)PV(k), ldn, c->n, ic + 1, (uint16_t*)c->PVh + c->off_PV[k], ldn, st);
      to_bf16((const float*)KV(k), ldn, c->n, ic + 1, (uint16_t*)c->KVh + c->off_PV[k], ldn, st);
      to_bf16((const float*)Vk(k), mk(k), mk(k), ic + 1, (uint16_t*)c->Vh + c->off_V[k], mk(k), st);
    }
  }
  void pack_one(int k) {
    if (c->mcols[k] > 0)
      to_bf16((const float*)Mk(k), c->ldn, c->n, c->mcols[k], (uint16_t*)c->Mh + c->off_M[k], c->ldn, st);
  }
  // Make the factors of filter step k (1..T) and M+_{k-1} resident in the rings: the segment of
  // seg_c steps holding k is recomputed from its checkpoint with the stored actions (RECOMPUTE)
  // or unpacked from the BF16 copies (STORE_BF16).
  int restore(int k) {
    if (!c->seg_c || (k >= c->res_a && k <= c->res_b)) return CAKF_OK;
    const int sc = c->seg_c;
    const int a0 = ((k - 1) / sc) * sc + 1, b0 = std::min(c->T, a0 + sc - 1);
    cudaEvent_t ph7 = ph_begin();
    const bool q = quiet;
    quiet = true;
    if (c->storage == CAKF_RECOMPUTE) {
      const size_t j = (size_t)(a0 - 1) / sc, rmx = std::max(c->rmax, 1);
      const int cols = c->mcols[a0 - 1];
      if (cols > 0) {
        cudaMemcpyAsync(Mk(a0 - 1), (T*)c->ckptM + j * c->ldn * rmx, (size_t)c->ldn * cols * sizeof(T),
                        cudaMemcpyDeviceToDevice, st);
        cudaMemcpyAsync(c->lam, c->ckpt_lam + j * rmx, cols * sizeof(double), cudaMemcpyDeviceToDevice, st);
        rowsumsq<T>(Mk(a0 - 1), c->ldn, c->n, cols, 0.0, c->rs_plus, st);
      } else {
        cudaMemsetAsync(c->rs_plus, 0, c->n * sizeof(double), st);
      }
      for (int kk = a0; kk <= b0; ++kk) {
        int rc = filter_step(kk, true, nullptr);
        if (rc) { quiet = q; return rc; }
      }
    } else if (sizeof(T) == 4) {
      const int ldn = c->ldn;
      for (int kk = a0 - 1; kk <= b0; ++kk)
        if (c->mcols[kk] > 0)
          from_bf16((const uint16_t*)c->Mh + c->off_M[kk], ldn, c->n, c->mcols[kk], (float*)Mk(kk), ldn, st);
      for (int kk = a0; kk <= b0; ++kk) {
        const int ic = c->icap[kk];
        if (mk(kk) == 0 || ic == 0) continue;
        from_bf16((const uint16_t*)c->PVh + c->off_PV[kk], ldn, c->n, ic + 1, (float*)PV(kk), ldn, st);
        from_bf16((const uint16_t*)c->KVh + c->off_PV[kk], ldn, c->n, ic + 1, (float*)KV(kk), ldn, st);
        from_bf16((const uint16_t*)c->Vh + c->off_V[kk], mk(kk), mk(kk), ic + 1, (float*)Vk(kk), mk(kk), st);
      }
    }
    quiet = q;
    ph_end(7, ph7);
    c->res_a = a0;
    c->res_b = b0;
    cudaError_t ce = cudaGetLastError();
    return ce == cudaSuccess ? CAKF_OK : fail(CAKF_ERR_CUDA, std::string("restoring factors: ") + cudaGetErrorString(ce));
  }
  T* Sk(int k) { return (T*)c->Spool + c->off_S[k]; }
  int mk(int k) { return c->obs_ptr[k] - c->obs_ptr[k - 1]; }
  const int* obs(int k) { return c->obs + c->obs_ptr[k - 1]; }
  C4<T>* X() { return (C4<T>*)c->X; }

  // Out (nr x width, ld ldo) = K(Xr, Xc) B  -- the hot Gram x block product.  On the tensor-core
  // path the first width-1 columns go through tcgen05 (bf16 operands, fp32 accumulation) and the
  // last column (the mean vector) is accumulated in fp32 by the tile producers.
  int gram_block(const C4<T>* Xr, int nr, const C4<T>* Xc, int nc, const T* B, int ldb, int width, T* Out, int ldo) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (c->profiling) { e0 = c->ev(); e1 = c->ev(); cudaEventRecord(e0, st); }
    const bool on_tc = tc && sizeof(T) == 4 && width >= 2 && width <= gram_tc_max_width();
    if (on_tc) {
      size_t ldp = gram_tc_packed_ld(nc);
      int rc = gram_tc_pack_b(tc_kind, (const float*)B, ldb, nc, width, c->Bpack, (int)ldp, st);
      if (!rc)
        rc = gram_block_tc(c->kernel, tc_kind, (const C4<float>*)Xr, nr, (const C4<float>*)Xc, nc, c->Bpack, (int)ldp,
                           width, (float)c->sf2, (float*)Out, ldo, c->err, st);
      if (rc) return fail(CAKF_ERR_CUDA, "tensor-core Gram x block launch failed (code " + std::to_string(rc) + ")");
    } else {
      gram_block_simt<T>(c->kernel, Xr, nr, Xc, nc, B, ldb, width, T(c->sf2), Out, ldo, st);
    }
    if (c->profiling) {
      cudaEventRecord(e1, st);
      c->prof_gb.push_back({e0, e1});
      // tensor-core path: the flops of the width-1 tensor-core columns (the last column runs on the
      // CUDA cores); the bracket also holds the operand packing, so the rate is conservative
      c->prof_gb_flops.push_back(2.0 * nr * (double)nc * (on_tc ? width - 1 : width));
      c->prof_gb_evals.push_back((double)nr * nc);
    }
    return CAKF_OK;
  }

  // ---------------------------------------------------------------- filter (Alg. 1)
  int filter() {
    const int n = c->n, T_ = c->T;
    cudaMemsetAsync(c->err, 0, sizeof(int), st);
    cudaMemsetAsync(c->rs_plus, 0, n * sizeof(double), st);
    cudaMemsetAsync(c->nll, 0, (T_ + 1) * sizeof(double), st);
    cudaMemsetAsync(c->count, 0, (T_ + 1) * sizeof(int), st);
    cudaMemsetAsync(c->r0sq, 0, (T_ + 1) * sizeof(double), st);
    cudaMemsetAsync(c->rfin, 0, (T_ + 1) * sizeof(double), st);
    cudaMemsetAsync(c->dropped_f, 0, (T_ + 1) * sizeof(double), st);
    cudaMemsetAsync(c->Spool, 0, c->off_S[T_ + 1] * sizeof(T), st);
    // state 0: prior (the two-block state starts with zero velocities)
    if (c->dprime == 2) cudaMemsetAsync(c->mf, 0, (size_t)(T_ + 1) * c->mstride * sizeof(double), st);
    if (c->has_mu) cudaMemcpyAsync(c->mf, c->mu, n * sizeof(double), cudaMemcpyDeviceToDevice, st);
    else cudaMemsetAsync(c->mf, 0, n * sizeof(double), st);
    {
      std::vector<double> sfv(n, c->sf2);
      cudaMemcpyAsync(c->vf, sfv.data(), n * sizeof(double), cudaMemcpyHostToDevice, st);
      cudaStreamSynchronize(st);
    }
    bool nll_pending = false;   // an NLL term is in flight on the side stream
    c->res_a = 1;
    c->res_b = 0;
    for (int k = 1; k <= T_; ++k) {
      if (nll_pending) {
        cudaStreamWaitEvent(st, c->ev_join, 0);
        nll_pending = false;
      }
      if (c->seg_c && c->storage == CAKF_RECOMPUTE && (k - 1) % c->seg_c == 0) save_checkpoint(k - 1);
      int rc = filter_step(k, false, &nll_pending);
      if (rc) return rc;
      if (c->seg_c && c->storage == CAKF_STORE_BF16) pack_history(k);
      cudaError_t ce = cudaGetLastError();
      if (ce != cudaSuccess) return fail(CAKF_ERR_CUDA, std::string("filter step: ") + cudaGetErrorString(ce));
    }
    if (nll_pending) cudaStreamWaitEvent(st, c->ev_join, 0);
    if (c->seg_c && c->storage == CAKF_RECOMPUTE) {   // the ring holds the last segment
      c->res_a = T_ >= 1 ? ((T_ - 1) / c->seg_c) * c->seg_c + 1 : 1;
      c->res_b = T_;
    } else if (c->seg_c) {   // BF16 store: every segment is read back from the BF16 copies
      c->res_a = 1;
      c->res_b = 0;
    } else {
      c->res_a = 1;
      c->res_b = T_;
    }
    return CAKF_OK;
  }

  // One filter step k (Alg. 1: predict, iterative update, finalize, Truncate).  With recompute the
  // step is re-run from the actions stored by the first pass (replayed from the action pool, no
  // NLL term, no phase timers): the same kernels on the same inputs give the same factors.
  int filter_step(int k, bool recompute, bool* nll_pending) {
    const int n = c->n, ldn = c->ldn, ldf = c->ldf;
    const bool two = c->dprime == 2;
    const int rows = two ? ldf : n;    // factor rows the products run over
    const double a = c->a_lazy(), a2 = a * a;
    const int B = std::max(c->budget, c->imax);
    const double bd_tol = (sizeof(T) == 8) ? 1e-12 : 1e-6;
    {
      const int m = mk(k), ic = c->icap[k], rp = c->mcols[k - 1];
      const double* mprev = c->mf + (size_t)(k - 1) * c->mstride;
      double* mout = c->mf + (size_t)k * c->mstride;
      double* vout = c->vf + (size_t)k * n;
      if (two) {
        // predict the two-block state: m^- = A m + b, and M^- = (A^t (x) I) M+_{k-1} in place (the
        // slot of M+_{k-1} holds M^-_k from here on, which is what the smoother reads); the
        // positions' part of rowsumsq(M^-) enters the variances
        predict_mean2(mprev, c->has_mu ? c->mu + (size_t)k * n : nullptr,
                      c->has_mu ? c->mu + (size_t)(k - 1) * n : nullptr, c->At, n, ldn, c->mpred, st);
        if (rp > 0) {
          mix2<T>(Mk(k - 1), ldf, Mk(k - 1), ldf, ldn, rp, c->At, st);
          rowsumsq<T>(Mk(k - 1), ldf, n, rp, 0.0, c->rs_plus, st);
        }
      } else {
        predict_mean(mprev, c->has_mu ? c->mu + (size_t)k * n : nullptr,
                     c->has_mu ? c->mu + (size_t)(k - 1) * n : nullptr, a, n, c->mpred, st);
      }
      if (m == 0 || ic == 0) {
        // no data at this step: m = m^-, M = M^- = a M+_{k-1}; no truncation needed (c_k = c_{k-1})
        filter_out<T>(c->mpred, (const T*)nullptr, ldn, -1, c->sf2, a2, c->rs_plus, n, mout, vout, nullptr, st);
        if (two) cudaMemcpyAsync(mout + ldn, c->mpred + ldn, n * sizeof(double), cudaMemcpyDeviceToDevice, st);
        scale_copy<T>(Mk(k - 1), ldf, rows, rp, T(a), Mk(k), ldf, st);
        if (rp > 0 && !two) rowsumsq<T>(Mk(k), ldn, n, rp, 0.0, c->rs_plus, st);
        scale_f64(c->lam, rp, rp, 1, a2, st);   // lam_k = a^2 lam_{k-1}
        return CAKF_OK;
      }
      const int* ob = obs(k);
      C4<T>* Xo = (C4<T>*)c->Xo;
      T* Mo = (T*)c->Mo;
      T* V = Vk(k);
      T* vcol = V + (size_t)ic * m;
      T* r = (T*)c->rv;
      T* s = (T*)c->sv;
      T* GV = (T*)c->GV;
      T* GSk = (T*)c->GS;      // G s_j of every iteration (column j), for the NLL
      cudaEvent_t ph0 = ph_begin();
      gather_coords<T>(X(), ob, m, Xo, st);
      gather_rows<T>(Mk(k - 1), ldf, ob, m, rp, Mo, m, st);   // H M^-: the position rows
      cudaMemsetAsync(c->r0sq + k, 0, sizeof(double), st);
      cudaMemsetAsync(c->rfin + k, 0, sizeof(double), st);
      cg_init<T>(c->y + c->obs_ptr[k - 1], c->mpred, ob, m, r, (T*)c->r0v, vcol, c->r0sq + k, st);
      cudaMemsetAsync(V, 0, (size_t)m * ic * sizeof(T), st);
      cudaMemsetAsync(GV, 0, (size_t)m * std::max(ic, 1) * sizeof(T), st);
      cudaMemsetAsync(GSk, 0, (size_t)m * std::max(ic, 1) * sizeof(T), st);
      {
        int one = 1;
        cudaMemcpyAsync(c->active, &one, sizeof(int), cudaMemcpyHostToDevice, st);
      }
      if (c->policy != CAKF_POLICY_CG) {
        if (int rcb = batch_update(k, m, ic, rp, Xo, Mo, V, GSk, recompute)) return rcb;
      } else {
      // rtol threshold needs ||r0||^2: read back once per step only when requested
      double rtol2 = 0.0;
      int use_rtol = 0;
      if (c->cg_rtol > 0 && !c->replay && !recompute) {
        double r0sq = 0;
        cudaMemcpyAsync(&r0sq, c->r0sq + k, sizeof(double), cudaMemcpyDeviceToHost, st);
        cudaStreamSynchronize(st);
        rtol2 = c->cg_rtol * c->cg_rtol * r0sq;
        use_rtol = 1;
      }
      const int nsplit = gram_matvec_slots(m);
      const double* rep = (c->replay && !recompute) ? c->rep + c->off_rep[k] : nullptr;
      T* Qa = (T*)c->Qa;       // orthonormal basis of the previous actions (CG policy only)
      // Re-orthogonalising each action against the previous ones leaves span(S) -- and so every
      // output -- unchanged; it keeps S^T S well conditioned for the NLL's FP64 Cholesky, which the
      // FP64 mode's 1e-9 agreement needs.  The FP32-based modes need it only when the budget is a
      // large share of the observations (4 i >= m): there CG can converge within the budget and
      // the later residuals, at FP32 rounding level, are no longer independent of the earlier ones.
      // (a recomputed step takes every action from its stored column: no selection, no reorth)
      const bool reorth = !rep && !recompute && (sizeof(T) == 8 || 4 * ic >= m);
      // CG policy without re-orthogonalisation: k_cg_upd2 writes the next action (the updated
      // residual) itself, so the selection runs only for the first action
      const bool fused_select = !rep && !reorth && !recompute;
      T* dpart1 = (T*)c->dpart;
      T* dpart2 = dpart1 + (size_t)(B + 4) * ((m + 31) / 32);
      for (int j = 0; j < ic; ++j) {
        T* g = GSk + (size_t)j * m;
        if (recompute) cg_select<T>(j, Sk(k) + (size_t)j * m, nullptr, m, s, Sk(k), m, c->active, st);
        else if (!fused_select || j == 0) cg_select<T>(j, r, rep, m, s, Sk(k), m, c->active, st);
        if (reorth) cg_reorth<T>(Qa, m, j, s, m, c->dots2, Sk(k), m, c->active, st);
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        bool prof = c->profiling && !recompute && (j % 8 == 0);
        if (prof) { e0 = c->ev(); e1 = c->ev(); cudaEventRecord(e0, st); }
        gram_matvec<T>(c->kernel, Xo, s, m, T(c->sf2), (T*)c->part, Mo, m, rp, (T*)c->tv, c->active, st);
        if (prof) {
          cudaEventRecord(e1, st);
          c->prof_mv.push_back({e0, e1});
          c->prof_mv_evals.push_back(0.5 * (double)m * (m + 1));   // unique entries of K(X_o, X_o)
        }
        cg_combine<T>((const T*)c->part, nsplit, s, T(c->sn2), Mo, m, rp, (const T*)c->tv, T(a2), m, g, V, m, j,
                      (const T*)c->r0v, vcol, dpart1, c->active, st);
        cg_upd1<T>(j, dpart1, c->dots, V, GV, m, s, g, m, dpart2, c->active, st);
        T* snext = (fused_select && j + 1 < ic) ? Sk(k) + (size_t)(j + 1) * m : nullptr;
        cg_upd2<T>(j, c->dots, dpart2, V, GV, m, r, vcol, s, reorth ? Qa : nullptr, m, bd_tol, rtol2, use_rtol,
                   c->active, c->eta + (size_t)k * B, c->alpha + (size_t)k * B, c->count + k, snext, st);
      }
      sqnorm_acc<T>(r, m, c->rfin + k, st);   // the final (updated) residual
      }
      ph_end(0, ph0);
      // finalize: [P^- W, P^- w] = K(X, X_o) [V v] - a^2 M+ (M+_o^T [V v])
      cudaEvent_t ph1 = ph_begin();
      T* PVk = PV(k);
      // K(X, X_o)[V v] is kept (the smoother propagates K [Ws, ws] from it); P^- [W w] = that minus
      // the low-rank part
      if (int rcg = gram_block(X(), n, Xo, m, V, m, ic + 1, KV(k), ldn)) return rcg;
      if (two) {
        // Sigma H^T [V v] = (P^t_inf[:, 0] (x) K(X, X_o)) [V v]: P^t_inf[1][0] = 0 for the stationary
        // Matern-3/2 factor, so the velocity rows start at zero
        cudaMemsetAsync(PVk, 0, (size_t)ldf * (ic + 1) * sizeof(T), st);
        cudaMemcpy2DAsync(PVk, ldf * sizeof(T), KV(k), ldn * sizeof(T), n * sizeof(T), ic + 1,
                          cudaMemcpyDeviceToDevice, st);
      } else {
        cudaMemcpyAsync(PVk, KV(k), (size_t)ldn * (ic + 1) * sizeof(T), cudaMemcpyDeviceToDevice, st);
      }
      if (rp > 0) {
        double* t2 = c->small;
        gemm_tn<T>(Mo, m, rp, V, m, ic + 1, m, 1.0, 0.0, t2, rp, c->part64, c->part64_elems, st);
        gemm_nn<T, double>(rows, ic + 1, rp, T(-a2), Mk(k - 1), ldf, t2, rp, T(1), PVk, ldf, st);
      }
      filter_out<T>(c->mpred, PVk, ldf, ic, c->sf2, a2, c->rs_plus, n, mout, vout, c->rs_pw, st);
      if (two) add_vec<T>(c->mpred + ldn, PVk + (size_t)ic * ldf + ldn, n, mout + ldn, st);
      ph_end(1, ph1);
      // NLL term from its definition: S^T G S (with the stored G s_j), S^T S and S^T r0, FP64 Cholesky.
      // It reads only this step's actions, G S and r0, so it runs on the side stream while the
      // truncation below runs here; the next step waits for it before the CG reuses those buffers.
      if (!recompute) {
        cudaEventRecord(c->ev_fork, st);
        cudaStreamWaitEvent(c->st_nll, c->ev_fork, 0);
        cudaStream_t s2 = c->st_nll;
        cudaEvent_t ph6 = nullptr;
        if (c->profiling) { ph6 = c->ev(); cudaEventRecord(ph6, s2); }
        double* SS = c->small_nll;
        double* Gh = SS + (size_t)ic * ic;
        double* yh = Gh + (size_t)ic * ic;
        double* zs = yh + ic;
        // The term depends on the actions only through their span.  The CG policy evaluates it on
        // the G-orthonormal directions V_k (same span, with G V_k kept by the iteration): when CG
        // converges within the budget the late residual actions are numerically dependent, and
        // S^T G S formed from working-precision G s products is no longer positive definite, while
        // V^T V and V^T G V stay well conditioned.  Given actions (batch policies) are used as they
        // are.
        const bool cg = c->policy == CAKF_POLICY_CG;
        const T* Sa = cg ? (const T*)V : Sk(k);
        const T* GSa = cg ? (const T*)GV : GSk;
        const int mode = gemm_mode();
        set_gemm_mode(0);   // own kernels only: the library GEMM handle belongs to the main stream
        gemm_tn<T>(Sa, m, ic, Sa, m, ic, m, 1.0, 0.0, SS, ic, c->part_nll, c->part_nll_elems, s2);
        gemm_tn<T>(Sa, m, ic, GSa, m, ic, m, 1.0, 0.0, Gh, ic, c->part_nll, c->part_nll_elems, s2);
        gemm_tn<T>(Sa, m, ic, (const T*)c->r0v, m, 1, m, 1.0, 0.0, yh, ic, c->part_nll, c->part_nll_elems, s2);
        set_gemm_mode(mode);
        nll_def(c->count + k, Gh, SS, ic, yh, zs, c->nll + k, c->err, s2);
        if (ph6) {
          cudaEvent_t e1 = c->ev();
          cudaEventRecord(e1, s2);
          c->prof_phase.push_back({6, {ph6, e1}});
        }
        cudaEventRecord(c->ev_join, s2);
        *nll_pending = true;
      }
      // Truncate (Sec. 3.2)
      cudaEvent_t ph2 = ph_begin();
      int rc = truncate_filter(k, rp, ic);
      if (rc) return rc;
      ph_end(2, ph2);
      cudaError_t ce = cudaGetLastError();
      if (ce != cudaSuccess) return fail(CAKF_ERR_CUDA, std::string("filter step: ") + cudaGetErrorString(ce));
    }
    return CAKF_OK;
  }

  // Batch update (Alg. 2) of step k: the ic actions S are fixed up front (coordinate actions, or
  // the given ones; a recomputed step reuses the stored ones), G [S r0] = K(X_o, X_o)[S r0] + sn2 S -
  // a^2 M_o (M_o^T S) with the Gram x block product (tensor cores in those modes), S^T G S = L L^T
  // and z = L^-1 S^T r0 in FP64, then [V v] = [S L^-T, S L^-T z].  G S is kept for the NLL term.
  int batch_update(int k, int m, int ic, int rp, const C4<T>* Xo, const T* Mo, T* V, T* GSk, bool recompute) {
    const double a2 = c->a_lazy() * c->a_lazy();
    T* S = Sk(k);
    if (!recompute) {
      if (c->policy == CAKF_POLICY_COORDINATE) coord_actions<T>(m, ic, S, st);
      else convert_from_f64<T>(c->rep + c->off_rep[k], m, m, ic, S, m, st);
    }
    T* Bsr = (T*)c->Xobs;
    cudaMemcpyAsync(Bsr, S, (size_t)m * ic * sizeof(T), cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(Bsr + (size_t)ic * m, c->r0v, (size_t)m * sizeof(T), cudaMemcpyDeviceToDevice, st);
    T* GSb = (T*)c->GSb;
    if (int rcg = gram_block(Xo, m, Xo, m, Bsr, m, ic + 1, GSb, m)) return rcg;
    if (rp > 0) {
      double* t = c->small;
      gemm_tn<T>(Mo, m, rp, S, m, ic, m, 1.0, 0.0, t, rp, c->part64, c->part64_elems, st);
      gemm_nn<T, double>(m, ic, rp, T(-a2), Mo, m, t, rp, T(1), GSb, m, st);
    }
    axpy_block<T>(T(c->sn2), S, m, m, ic, GSb, m, st);
    cudaMemcpyAsync(GSk, GSb, (size_t)m * ic * sizeof(T), cudaMemcpyDeviceToDevice, st);
    const size_t ii = (size_t)ic * ic;
    double* Gh = c->Lb;
    double* L = Gh + ii;
    double* yh = L + ii;
    double* z = yh + ic;
    gemm_tn<T>(S, m, ic, GSb, m, ic, m, 1.0, 0.0, Gh, ic, c->part64, c->part64_elems, st);
    gemm_tn<T>(S, m, ic, (const T*)c->r0v, m, 1, m, 1.0, 0.0, yh, ic, c->part64, c->part64_elems, st);
    const int B = std::max(c->budget, c->imax);
    if (batch_chol(Gh, ic, yh, L, z, c->eta + (size_t)k * B, c->err, st))
      return fail(CAKF_ERR_ARG, "too many actions for the batch update");
    batch_v<T>(S, m, ic, L, z, V, st);
    batch_resid<T>(GSb, m, ic, L, z, (const T*)c->r0v, c->rfin + k, st);
    cudaMemcpyAsync(c->count + k, &ic, sizeof(int), cudaMemcpyHostToDevice, st);
    return CAKF_OK;
  }

  int truncate_filter(int k, int rp, int ic) {
    const int n = c->n, ldn = c->ldn, ldf = c->ldf;
    const bool two = c->dprime == 2;
    const int rows = two ? ldf : n;
    const double a = c->a_lazy(), a2 = a * a;
    T* PVk = PV(k);
    if (c->rank_r <= 0) {
      // M+_k = M_k = (a M+_{k-1}, P^- W_k)
      scale_copy<T>(Mk(k - 1), ldf, rows, rp, T(a), Mk(k), ldf, st);
      scale_copy<T>(PVk, ldf, rows, ic, T(1), Mk(k) + (size_t)rp * ldf, ldf, st);
      if (!two) rowsumsq<T>(Mk(k), ldn, n, rp + ic, 0.0, c->rs_plus, st);
      return CAKF_OK;
    }
    if (two) return truncate_filter2(k, rp, ic);
    const int N = rp + ic;
    const int keep = std::min(c->rank_r, N);
    T* U = (T*)c->UT;
    if (c->freeze) {
      // the rotation of the previous run at this step (the frozen modified model)
      convert_from_f64<T>(c->Upool + c->off_U[k], N, N, keep, U, N, st);
      if (rp > 0) gemm_nn<T, T>(n, keep, rp, T(a), Mk(k - 1), ldn, U, N, T(0), Mk(k), ldn, st);
      gemm_nn<T, T>(n, keep, ic, T(1), PVk, ldn, U + rp, N, rp > 0 ? T(1) : T(0), Mk(k), ldn, st);
      rowsumsq<T>(Mk(k), ldn, n, keep, 0.0, c->rs_plus, st);
      return CAKF_OK;
    }
    double* G = c->gram;
    cudaMemsetAsync(G, 0, (size_t)N * N * sizeof(double), st);
    set_diag(G, N, c->lam, a2, rp, st);
    if (rp > 0) {
      double* Bm = c->small;
      gemm_tn<T>(Mk(k - 1), ldn, rp, PVk, ldn, ic, n, a, 0.0, Bm, rp, c->part64, c->part64_elems, st);
      put_block_sym(G, N, 0, rp, Bm, rp, rp, ic, 1.0, st);
    }
    gemm_tn<T>(PVk, ldn, ic, PVk, ldn, ic, n, 1.0, 0.0, G + (size_t)rp * N + rp, N, c->part64, c->part64_elems, st);
    trace_into(G, N, N, c->dropped_f + k, st);   // discarded mass = trace - kept eigenvalues
    int rc = eig(G, N, keep);
    if (rc) return rc;
    sub_sum(c->wv, keep, c->dropped_f + k, st);
    // M+_k = a M+_{k-1} U[0:rp, :] + P^- W U[rp:N, :]
    if (rp > 0) gemm_nn<T, T>(n, keep, rp, T(a), Mk(k - 1), ldn, U, N, T(0), Mk(k), ldn, st);
    gemm_nn<T, T>(n, keep, ic, T(1), PVk, ldn, U + rp, N, rp > 0 ? T(1) : T(0), Mk(k), ldn, st);
    cudaMemcpyAsync(c->lam, c->wv, keep * sizeof(double), cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(c->Upool + c->off_U[k], c->U64, (size_t)N * keep * sizeof(double), cudaMemcpyDeviceToDevice, st);
    rowsumsq<T>(Mk(k), ldn, n, keep, 0.0, c->rs_plus, st);
    return CAKF_OK;
  }

  // Truncate for the two-block state: the columns of M^-_k = (A^t (x) I) M+_{k-1} are not
  // orthogonal, so the whole Gram of M_k = (M^-_k, P^- W_k) is formed over its ldf rows (three
  // products: M^-T M^-, M^-T P^-W, (P^-W)^T P^-W), eigendecomposed in FP64 and rotated.
  int truncate_filter2(int k, int rp, int ic) {
    const int ldf = c->ldf;
    T* PVk = PV(k);
    const int N = rp + ic;
    const int keep = std::min(c->rank_r, N);
    T* U = (T*)c->UT;
    double* G = c->gram;
    cudaMemsetAsync(G, 0, (size_t)N * N * sizeof(double), st);
    if (rp > 0) {
      gemm_tn<T>(Mk(k - 1), ldf, rp, Mk(k - 1), ldf, rp, ldf, 1.0, 0.0, G, N, c->part64, c->part64_elems, st);
      double* Bm = c->small;
      gemm_tn<T>(Mk(k - 1), ldf, rp, PVk, ldf, ic, ldf, 1.0, 0.0, Bm, rp, c->part64, c->part64_elems, st);
      put_block_sym(G, N, 0, rp, Bm, rp, rp, ic, 1.0, st);
    }
    gemm_tn<T>(PVk, ldf, ic, PVk, ldf, ic, ldf, 1.0, 0.0, G + (size_t)rp * N + rp, N, c->part64, c->part64_elems, st);
    trace_into(G, N, N, c->dropped_f + k, st);   // discarded mass = trace - kept eigenvalues
    int rc = eig(G, N, keep);
    if (rc) return rc;
    sub_sum(c->wv, keep, c->dropped_f + k, st);
    if (rp > 0) gemm_nn<T, T>(ldf, keep, rp, T(1), Mk(k - 1), ldf, U, N, T(0), Mk(k), ldf, st);
    gemm_nn<T, T>(ldf, keep, ic, T(1), PVk, ldf, U + rp, N, rp > 0 ? T(1) : T(0), Mk(k), ldf, st);
    cudaMemcpyAsync(c->lam, c->wv, keep * sizeof(double), cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(c->Upool + c->off_U[k], c->U64, (size_t)N * keep * sizeof(double), cudaMemcpyDeviceToDevice, st);
    return CAKF_OK;
  }

  // eigen-decomposition of the FP64 Gram G (N x N): top `keep` pairs -> wv, U64 (double), UT (T)
  int eig(double* G, int N, int keep) {
    cudaEvent_t e0 = nullptr, e1 = nullptr, mk[2] = {nullptr, nullptr};
    if (c->profiling) { e0 = c->ev(); e1 = c->ev(); mk[0] = c->ev(); mk[1] = c->ev(); cudaEventRecord(e0, st); }
    // U feeds FP32 products in the FP32-based modes: its final assembly runs in double-FP32 there
    int rc = eig_sym_topk<double>(G, N, N, keep, c->wv, c->U64, N, c->eigw, c->eigw_bytes, c->err, st,
                                  c->profiling ? mk : nullptr, sizeof(T) == 4 ? kAssemblyFF : kAssemblyFP64);
    if (rc) {
      cudaGetLastError();
      std::string why = rc >= 1000 ? cudaGetErrorString((cudaError_t)(rc - 1000)) : std::to_string(rc);
      return fail(CAKF_ERR_CUDA, "eigensolver launch failed (N = " + std::to_string(N) + "): " + why);
    }
    convert_from_f64<T>(c->U64, N, N, keep, (T*)c->UT, N, st);
    if (c->profiling) {
      cudaEventRecord(e1, st);
      c->stats.eig_calls++;
      c->stats.eig_flops[0] += 4.0 / 3.0 * (double)N * N * N;
      c->stats.eig_flops[1] += 2.0 * (double)N * N * keep;
      c->prof_eig.push_back({e0, e1});
      c->prof_eig_tri.push_back({e0, mk[0]});
      c->prof_eig_dc.push_back({mk[0], mk[1]});
      c->prof_eig_bt.push_back({mk[1], e1});
    }
    return CAKF_OK;
  }

  // K ws_new = K w_k + a KW[:, cw] - K W_k Z[:, cw] into out (n), with KVk = K [W_k w_k] (ic + 1
  // columns) and Z (ic x (cw + 1), FP64) from the smoother step.
  void kws_update(const T* KVk, int ic, const T* KW, int cw, const double* Z, T* out) {
    const int n = c->n, ldn = c->ldn;
    scale_copy<T>(KW + (size_t)cw * ldn, ldn, n, 1, T(c->a), out, ldn, st);
    axpy_block<T>(T(1), KVk + (size_t)ic * ldn, ldn, n, 1, out, ldn, st);
    gemm_nn<T, double>(n, 1, ic, T(-1), KVk, ldn, Z + (size_t)cw * ic, ic, T(1), out, ldn, st);
  }

  // ---------------------------------------------------------------- smoother, two-block state
  // Alg. 3 for the Matern-3/2 temporal factor.  As in the OU smoother, KW = (I_2 (x) K) [Ws ws] is
  // carried through the recursion from the filter's K(X, X_o)[V v] blocks, so for X = A^T [Ws ws]
  //   K X = (A^t^T (x) I) KW   and   Sigma X = (P^t_inf A^t^T (x) I) KW
  // need no kernel evaluations.  W_k = H^T V_k lives in the position rows.  The Gram of the new
  // Ws (whose predicted part has no orthogonal columns here) is formed from its ldf rows.
  int smooth2(double* ms, double* vs) {
    const int n = c->n, T_ = c->T, ldn = c->ldn, ldf = c->ldf;
    cudaMemcpyAsync(ms + (size_t)T_ * n, c->mf + (size_t)T_ * c->mstride, n * sizeof(double), cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(vs + (size_t)T_ * n, c->vf + (size_t)T_ * n, n * sizeof(double), cudaMemcpyDeviceToDevice, st);
    cudaMemsetAsync(c->dropped_s, 0, (T_ + 1) * sizeof(double), st);
    if (T_ == 0) return CAKF_OK;
    const double AT[4] = {c->At[0], c->At[2], c->At[1], c->At[3]};   // (A^t)^T, row-major
    const double PAT[4] = {c->Pt[0] * AT[0] + c->Pt[1] * AT[2], c->Pt[0] * AT[1] + c->Pt[1] * AT[3],
                           c->Pt[2] * AT[0] + c->Pt[3] * AT[2], c->Pt[2] * AT[1] + c->Pt[3] * AT[3]};
    T* Ws = (T*)c->WsA;
    T* Wn = (T*)c->WsB;
    T* ws = (T*)c->wsA;
    T* wn = (T*)c->wsB;
    T* KW = (T*)c->KWa;
    T* KWn = (T*)c->KWb;
    T* Xs = (T*)c->Xs;
    T* Y = (T*)c->Y;
    T* KX = (T*)c->KX;
    const size_t es = sizeof(T);
    int cw = c->icap[T_];
    cudaMemsetAsync(ws, 0, ldf * es, st);
    cudaMemsetAsync(KW, 0, (size_t)ldf * (cw + 1) * es, st);
    if (cw > 0) {
      const int m = mk(T_);
      cudaMemsetAsync(Ws, 0, (size_t)ldf * cw * es, st);
      scatter_add_rows<T>(Vk(T_), m, obs(T_), m, cw, T(1), Ws, ldf, st);
      scatter_add_rows<T>(Vk(T_) + (size_t)cw * m, m, obs(T_), m, 1, T(1), ws, ldf, st);
      cudaMemcpy2DAsync(KW, ldf * es, KV(T_), ldn * es, n * es, cw + 1, cudaMemcpyDeviceToDevice, st);
    }
    for (int k = T_ - 1; k >= 0; --k) {
      cudaEvent_t ph3 = ph_begin();
      // X = A^T [Ws ws];  K X and Y = Sigma X from KW
      mix2<T>(Ws, ldf, Xs, ldf, ldn, cw, AT, st);
      mix2<T>(ws, ldf, Xs + (size_t)cw * ldf, ldf, ldn, 1, AT, st);
      mix2<T>(KW, ldf, KX, ldf, ldn, cw + 1, AT, st);
      mix2<T>(KW, ldf, Y, ldf, ldn, cw + 1, PAT, st);
      // Y = P^-_k X = Sigma X - M^-_k (M^-_k^T X)  (the slot of M+_{k-1} holds M^-_k)
      const int rp = (k >= 1) ? c->mcols[k - 1] : 0;
      if (rp > 0) {
        double* t = c->small;
        gemm_tn<T>(Mk(k - 1), ldf, rp, Xs, ldf, cw + 1, ldf, 1.0, 0.0, t, rp, c->part64, c->part64_elems, st);
        gemm_nn<T, double>(ldf, cw + 1, rp, T(-1), Mk(k - 1), ldf, t, rp, T(1), Y, ldf, st);
      }
      ph_end(3, ph3);
      cudaEvent_t ph4 = ph_begin();
      const int ic = (k >= 1) ? c->icap[k] : 0;
      const int m = (k >= 1) ? mk(k) : 0;
      double* Z = c->small;                       // ic x (cw + 1)
      if (ic > 0) {
        // Z = W_k^T P^- X = V_k^T Y[obs];  Y <- P_k X = Y - (P^- W_k) Z
        T* Xo = (T*)c->Xobs;
        gather_rows<T>(Y, ldf, obs(k), m, cw + 1, Xo, m, st);
        gemm_tn<T>(Vk(k), m, ic, Xo, m, cw + 1, m, 1.0, 0.0, Z, ic, c->part64, c->part64_elems, st);
        gemm_nn<T, double>(ldf, cw + 1, ic, T(-1), PV(k), ldf, Z, ic, T(1), Y, ldf, st);
      }
      smooth_out<T>(c->mf + (size_t)k * c->mstride, c->vf + (size_t)k * n, Y, ldf, cw, n, ms + (size_t)k * n,
                    vs + (size_t)k * n, st);
      if (k == 0) break;
      if (ic == 0) {
        // no update at k: [Ws ws]_k = A^T [Ws ws]_{k+1}, K [Ws ws]_k = K X
        cudaMemcpyAsync(wn, Xs + (size_t)cw * ldf, ldf * es, cudaMemcpyDeviceToDevice, st);
        cudaMemcpyAsync(Wn, Xs, (size_t)ldf * cw * es, cudaMemcpyDeviceToDevice, st);
        cudaMemcpyAsync(KWn, KX, (size_t)ldf * (cw + 1) * es, cudaMemcpyDeviceToDevice, st);
        std::swap(Ws, Wn); std::swap(ws, wn); std::swap(KW, KWn);
        ph_end(4, ph4);
        continue;
      }
      T* Vkk = Vk(k);
      const T* KVk = KV(k);
      // ws_k = w_k + X[:, cw] - W_k Z[:, cw]
      cudaMemcpyAsync(wn, Xs + (size_t)cw * ldf, ldf * es, cudaMemcpyDeviceToDevice, st);
      T* vz = (T*)c->Fb;
      gemm_nn<T, double>(m, 1, ic, T(1), Vkk, m, Z + (size_t)cw * ic, ic, T(0), vz, m, st);
      ws_obs<T>(obs(k), m, Vkk + (size_t)ic * m, vz, wn, st);
      ph_end(4, ph4);
      cudaEvent_t ph5 = ph_begin();
      // Ws_full = [W_k, X[:, :cw] - W_k Z[:, :cw]] and K Ws_full = [K W_k, K X[:, :cw] - K W_k Z[:, :cw]],
      // with K ws_k = K w_k + K X[:, cw] - K W_k Z[:, cw] in column N
      const int N = ic + cw;
      cudaMemsetAsync(Wn, 0, (size_t)ldf * N * es, st);
      scatter_add_rows<T>(Vkk, m, obs(k), m, ic, T(1), Wn, ldf, st);
      cudaMemsetAsync(KWn, 0, (size_t)ldf * ic * es, st);
      cudaMemcpy2DAsync(KWn, ldf * es, KVk, ldn * es, n * es, ic, cudaMemcpyDeviceToDevice, st);
      cudaMemcpyAsync(KWn + (size_t)ic * ldf, KX, (size_t)ldf * (cw + 1) * es, cudaMemcpyDeviceToDevice, st);
      if (cw > 0) {
        cudaMemcpyAsync(Wn + (size_t)ic * ldf, Xs, (size_t)ldf * cw * es, cudaMemcpyDeviceToDevice, st);
        T* F = (T*)c->Fb;
        gemm_nn<T, double>(m, cw, ic, T(1), Vkk, m, Z, ic, T(0), F, m, st);
        scatter_add_rows<T>(F, m, obs(k), m, cw, T(-1), Wn + (size_t)ic * ldf, ldf, st);
      }
      axpy_block<T>(T(1), KVk + (size_t)ic * ldn, ldn, n, 1, KWn + (size_t)N * ldf, ldf, st);
      gemm_nn<T, double>(n, cw + 1, ic, T(-1), KVk, ldn, Z, ic, T(1), KWn + (size_t)ic * ldf, ldf, st);
      if (c->rank_r > 0) {
        const int keep = std::min(c->rank_r, N);
        double* G = c->gram;
        gemm_tn<T>(Wn, ldf, N, Wn, ldf, N, ldf, 1.0, 0.0, G, N, c->part64, c->part64_elems, st);
        trace_into(G, N, N, c->dropped_s + k, st);
        int rc = eig(G, N, keep);
        if (rc) return rc;
        sub_sum(c->wv, keep, c->dropped_s + k, st);
        T* U = (T*)c->UT;
        // Ws = Ws_full U, K Ws = (K Ws_full) U  (into the buffers of step k + 1, no longer needed)
        gemm_nn<T, T>(ldf, keep, N, T(1), Wn, ldf, U, N, T(0), Ws, ldf, st);
        gemm_nn<T, T>(ldf, keep, N, T(1), KWn, ldf, U, N, T(0), KW, ldf, st);
        cudaMemcpyAsync(KW + (size_t)keep * ldf, KWn + (size_t)N * ldf, ldf * es, cudaMemcpyDeviceToDevice, st);
        cw = keep;
      } else {
        std::swap(Ws, Wn);
        std::swap(KW, KWn);
        cw = N;
      }
      std::swap(ws, wn);
      ph_end(5, ph5);
      cudaError_t ce = cudaGetLastError();
      if (ce != cudaSuccess) return fail(CAKF_ERR_CUDA, std::string("smoother step: ") + cudaGetErrorString(ce));
    }
    return CAKF_OK;
  }

  // ---------------------------------------------------------------- smoother (Alg. 3)
  int smooth(double* ms, double* vs) {
    if (c->dprime == 2) return smooth2(ms, vs);
    const int n = c->n, T_ = c->T, ldn = c->ldn;
    const double a = c->a, a2 = a * a;
    cudaMemcpyAsync(ms + (size_t)T_ * n, c->mf + (size_t)T_ * n, n * sizeof(double), cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(vs + (size_t)T_ * n, c->vf + (size_t)T_ * n, n * sizeof(double), cudaMemcpyDeviceToDevice, st);
    cudaMemsetAsync(c->dropped_s, 0, (T_ + 1) * sizeof(double), st);
    if (T_ == 0) return CAKF_OK;
    T* Ws = (T*)c->WsA;
    T* Wn = (T*)c->WsB;
    T* ws = (T*)c->wsA;
    T* wn = (T*)c->wsB;
    double* Gw = c->Gws;
    double* Gn = c->Gws2;
    if (int rc = restore(T_)) return rc;
    // Ws_T = H^T V_T, ws_T = H^T v_T
    int cw = c->icap[T_];
    cudaMemsetAsync(ws, 0, ldn * sizeof(T), st);
    if (cw > 0) {
      const int m = mk(T_);
      cudaMemsetAsync(Ws, 0, (size_t)ldn * cw * sizeof(T), st);
      scatter_add_rows<T>(Vk(T_), m, obs(T_), m, cw, T(1), Ws, ldn, st);
      scatter_add_rows<T>(Vk(T_) + (size_t)cw * m, m, obs(T_), m, 1, T(1), ws, ldn, st);
      gemm_tn<T>(Vk(T_), m, cw, Vk(T_), m, cw, m, 1.0, 0.0, Gw, cw, c->part64, c->part64_elems, st);
    } else if (T_ >= 1 && mk(T_) > 0) {
      // no actions at T
    }
    T* Xs = (T*)c->Xs;
    T* Y = (T*)c->Y;
    // KW = K [Ws ws] is carried along with [Ws ws] through the same linear recursion, starting from
    // the filter's K(X, X_o)[V_T v_T]; so K X = a KW needs no kernel evaluations in the smoother.
    T* KW = (T*)c->KWa;
    T* KWn = (T*)c->KWb;
    if (cw > 0) cudaMemcpyAsync(KW, KV(T_), (size_t)ldn * (cw + 1) * sizeof(T), cudaMemcpyDeviceToDevice, st);
    else cudaMemsetAsync(KW, 0, (size_t)ldn * sizeof(T), st);
    if (qs) interp_at(T_, cw, Ws, ws, KW);
    for (int k = T_ - 1; k >= 0; --k) {
      if (k >= 1)
        if (int rc = restore(k)) return rc;
      if (qs) interp_at(k, cw, Ws, ws, KW);
      // X = A^T [Ws ws] = a [Ws ws]
      cudaEvent_t ph3 = ph_begin();
      build_x<T>(Ws, ldn, cw, ws, T(a), n, Xs, ldn, st);
      // Y = P^-_k X = K X - a^2 M+_{k-1} (M+_{k-1}^T X),  K X = a KW
      scale_copy<T>(KW, ldn, n, cw + 1, T(a), Y, ldn, st);
      const int rp = (k >= 1) ? c->mcols[k - 1] : 0;
      if (rp > 0) {
        double* t = c->small;
        gemm_tn<T>(Mk(k - 1), ldn, rp, Xs, ldn, cw + 1, n, 1.0, 0.0, t, rp, c->part64, c->part64_elems, st);
        gemm_nn<T, double>(n, cw + 1, rp, T(-a2), Mk(k - 1), ldn, t, rp, T(1), Y, ldn, st);
      }
      ph_end(3, ph3);
      cudaEvent_t ph4 = ph_begin();
      const int ic = (k >= 1) ? c->icap[k] : 0;
      const int m = (k >= 1) ? mk(k) : 0;
      double* Z = c->small;                       // ic x (cw+1)
      double* VtV = Z + (size_t)ic * (cw + 1);    // ic x ic
      double* Bx = VtV + (size_t)ic * ic;         // ic x cw
      double* Vz = Bx + (size_t)ic * std::max(cw, 1);   // scratch
      if (ic > 0) {
        // Z = W_k^T P^- X = V_k^T Y[obs];  Y <- P_k X = Y - (P^- W_k) Z
        T* Xo = (T*)c->Xobs;
        gather_rows<T>(Y, ldn, obs(k), m, cw + 1, Xo, m, st);
        gemm_tn<T>(Vk(k), m, ic, Xo, m, cw + 1, m, 1.0, 0.0, Z, ic, c->part64, c->part64_elems, st);
        gemm_nn<T, double>(n, cw + 1, ic, T(-1), PV(k), ldn, Z, ic, T(1), Y, ldn, st);
      }
      smooth_out<T>(c->mf + (size_t)k * n, c->vf + (size_t)k * n, Y, ldn, cw, n, ms + (size_t)k * n,
                    vs + (size_t)k * n, st);
      if (k == 0) break;
      if (ic == 0) {
        // no update at k: ws_k = a ws_{k+1}, Ws_k = a Ws_{k+1}
        scale_copy<T>(Xs + (size_t)cw * ldn, ldn, n, 1, T(1), wn, ldn, st);
        scale_copy<T>(Xs, ldn, n, cw, T(1), Wn, ldn, st);
        scale_copy<T>(KW, ldn, n, cw + 1, T(a), KWn, ldn, st);      // K [Wn wn] = a K [Ws ws]
        if (cw > 0) {
          cudaMemcpyAsync(Gn, Gw, (size_t)cw * cw * sizeof(double), cudaMemcpyDeviceToDevice, st);
          scale_f64(Gn, cw * cw, cw * cw, 1, a2, st);
        }
        std::swap(Ws, Wn); std::swap(ws, wn); std::swap(Gw, Gn); std::swap(KW, KWn);
        continue;
      }
      T* Vkk = Vk(k);
      // ws_k = w_k + X[:, cw] - W_k Z[:, cw]
      scale_copy<T>(Xs + (size_t)cw * ldn, ldn, n, 1, T(1), wn, ldn, st);
      T* vz = (T*)c->Fb;
      gemm_nn<T, double>(m, 1, ic, T(1), Vkk, m, Z + (size_t)cw * ic, ic, T(0), vz, m, st);
      ws_obs<T>(obs(k), m, Vkk + (size_t)ic * m, vz, wn, st);
      T* KVk = KV(k);
      ph_end(4, ph4);
      cudaEvent_t ph5 = ph_begin();
      // Gram of Ws_full = [W_k, X'] with X' = X[:, :cw] - W_k Z[:, :cw]  (small-matrix identities)
      const int N = ic + cw;
      double* G = c->gram;
      gemm_tn<T>(Vkk, m, ic, Vkk, m, ic, m, 1.0, 0.0, VtV, ic, c->part64, c->part64_elems, st);
      if (cw > 0) {
        T* Xo = (T*)c->Xobs;
        gather_rows<T>(Xs, ldn, obs(k), m, cw, Xo, m, st);
        gemm_tn<T>(Vkk, m, ic, Xo, m, cw, m, 1.0, 0.0, Bx, ic, c->part64, c->part64_elems, st);
      }
      // G = [[VtV, Bx - VtV Z], [., a^2 Gw - Z^T Bx - Bx^T Z + Z^T VtV Z]]
      cudaMemsetAsync(G, 0, (size_t)N * N * sizeof(double), st);
      copy_block(VtV, ic, ic, ic, G, N);
      if (cw > 0) {
        double* TR = Vz;                          // ic x cw
        copy_block(Bx, ic, ic, cw, TR, ic);
        gemm_small_f64(0, 0, ic, cw, ic, -1.0, VtV, ic, Z, ic, 1.0, TR, ic, st);
        put_block_sym(G, N, 0, ic, TR, ic, ic, cw, 1.0, st);
        double* BR = G + (size_t)ic * N + ic;     // cw x cw block, ld N
        copy_block_scaled(Gw, cw, cw, cw, BR, N, a2);
        gemm_small_f64(1, 0, cw, cw, ic, -1.0, Z, ic, Bx, ic, 1.0, BR, N, st);
        gemm_small_f64(1, 0, cw, cw, ic, -1.0, Bx, ic, Z, ic, 1.0, BR, N, st);
        double* VZ = TR + (size_t)ic * cw;        // ic x cw = VtV Z
        gemm_small_f64(0, 0, ic, cw, ic, 1.0, VtV, ic, Z, ic, 0.0, VZ, ic, st);
        gemm_small_f64(1, 0, cw, cw, ic, 1.0, Z, ic, VZ, ic, 1.0, BR, N, st);
      }
      if (c->rank_r > 0) {
        const int keep = std::min(c->rank_r, N);
        trace_into(G, N, N, c->dropped_s + k, st);
        int rc = eig(G, N, keep);
        if (rc) return rc;
        sub_sum(c->wv, keep, c->dropped_s + k, st);
        T* U = (T*)c->UT;
        // Ws_new = X[:, :cw] U[ic:, :] + scatter_obs( V_k (U[:ic, :] - Z[:, :cw] U[ic:, :]) )
        if (cw > 0) gemm_nn<T, T>(n, keep, cw, T(1), Xs, ldn, U + ic, N, T(0), Wn, ldn, st);
        else cudaMemsetAsync(Wn, 0, (size_t)ldn * keep * sizeof(T), st);
        double* E = Vz;   // ic x keep
        copy_block(c->U64, N, ic, keep, E, ic);
        if (cw > 0) gemm_small_f64(0, 0, ic, keep, cw, -1.0, Z, ic, c->U64 + ic, N, 1.0, E, ic, st);
        T* F = (T*)c->Fb;
        gemm_nn<T, double>(m, keep, ic, T(1), Vkk, m, E, ic, T(0), F, m, st);
        scatter_add_rows<T>(F, m, obs(k), m, keep, T(1), Wn, ldn, st);
        // K Ws_new = a KW[:, :cw] U_bot + K W_k E
        if (cw > 0) gemm_nn<T, T>(n, keep, cw, T(a), KW, ldn, U + ic, N, T(0), KWn, ldn, st);
        gemm_nn<T, double>(n, keep, ic, T(1), KVk, ldn, E, ic, cw > 0 ? T(1) : T(0), KWn, ldn, st);
        kws_update(KVk, ic, KW, cw, Z, KWn + (size_t)keep * ldn);
        // Gram of the new Ws is diag(lam)
        cudaMemsetAsync(Gn, 0, (size_t)keep * keep * sizeof(double), st);
        set_diag(Gn, keep, c->wv, 1.0, keep, st);
        cw = keep;
      } else {
        // no truncation: Ws_new = [W_k, X[:, :cw] - W_k Z[:, :cw]] explicitly
        cudaMemsetAsync(Wn, 0, (size_t)ldn * N * sizeof(T), st);
        scatter_add_rows<T>(Vkk, m, obs(k), m, ic, T(1), Wn, ldn, st);
        if (cw > 0) {
          scale_copy<T>(Xs, ldn, n, cw, T(1), Wn + (size_t)ic * ldn, ldn, st);
          T* F = (T*)c->Fb;
          gemm_nn<T, double>(m, cw, ic, T(1), Vkk, m, Z, ic, T(0), F, m, st);
          scatter_add_rows<T>(F, m, obs(k), m, cw, T(-1), Wn + (size_t)ic * ldn, ldn, st);
        }
        // K Ws_full = [K W_k, a KW[:, :cw] - K W_k Z[:, :cw]]
        scale_copy<T>(KVk, ldn, n, ic, T(1), KWn, ldn, st);
        if (cw > 0) {
          scale_copy<T>(KW, ldn, n, cw, T(a), KWn + (size_t)ic * ldn, ldn, st);
          gemm_nn<T, double>(n, cw, ic, T(-1), KVk, ldn, Z, ic, T(1), KWn + (size_t)ic * ldn, ldn, st);
        }
        kws_update(KVk, ic, KW, cw, Z, KWn + (size_t)N * ldn);
        cudaMemcpyAsync(Gn, G, (size_t)N * N * sizeof(double), cudaMemcpyDeviceToDevice, st);
        cw = N;
      }
      ph_end(5, ph5);
      std::swap(Ws, Wn); std::swap(ws, wn); std::swap(Gw, Gn); std::swap(KW, KWn);
      cudaError_t ce = cudaGetLastError();
      if (ce != cudaSuccess) return fail(CAKF_ERR_CUDA, std::string("smoother step: ") + cudaGetErrorString(ce));
    }
    return CAKF_OK;
  }

  // ---------------------------------------------------------------- temporal interpolation
  // Queries t_k <= t < t_{k+1} (the interpolation corollary in downdate form, OU prior): with
  // at = A(t, t_k), a2 = A(t_{k+1}, t), M_k = (a M+_{k-1}, [P^-W]_k) the updated factor,
  //   filter   m(t) = at m_k + b(t, t_k), var(t) = sf2 - at^2 (sf2 - var_k),
  //   smoother Y = P(t) a2 [Ws ws]_{k+1} = a2 (K[Ws ws] - at^2 M_k (M_k^T [Ws ws])) with K[Ws ws]
  //            carried by the smoother's recursion, m^s(t) = m(t) + Y[:, cw],
  //            var^s(t) = var(t) - rowsumsq(Y[:, :cw]);  at k = T the smoother output is the filter's.
  void interp_at(int k, int cw, const T* Ws, const T* ws, const T* KW) {
    const std::vector<int>& ids = qs->at_k[k];
    if (ids.empty()) return;
    const int n = c->n, ldn = c->ldn;
    const double dt = c->dt, lt = c->lt;
    T* Xs = (T*)c->Xs;
    T* Y = (T*)c->Y;
    const int rp = k >= 1 ? c->mcols[k - 1] : 0;
    const int ic = (k >= 1 && mk(k) > 0) ? c->icap[k] : 0;
    if (k < c->T) build_x<T>(Ws, ldn, cw, ws, T(1), n, Xs, ldn, st);   // [Ws ws] of step k + 1
    double* u1 = c->small;
    double* u2 = u1 + (size_t)std::max(rp, 1) * (cw + 1);
    for (int q : ids) {
      const double tau = qs->tq[q] - k * dt;
      const double at = std::exp(-tau / lt);
      double* fm = qs->fm + (size_t)q * n;
      double* fv = qs->fv + (size_t)q * n;
      interp_filter(c->mf + (size_t)k * n, c->vf + (size_t)k * n, qs->mu_q ? qs->mu_q + (size_t)q * n : nullptr,
                    c->has_mu ? c->mu + (size_t)k * n : nullptr, at, c->sf2, n, fm, fv, st);
      double* sm = qs->sm + (size_t)q * n;
      double* sv = qs->sv + (size_t)q * n;
      if (k == c->T) {
        cudaMemcpyAsync(sm, fm, n * sizeof(double), cudaMemcpyDeviceToDevice, st);
        cudaMemcpyAsync(sv, fv, n * sizeof(double), cudaMemcpyDeviceToDevice, st);
        continue;
      }
      const double ar = std::exp(-(dt - tau) / lt);     // A(t_{k+1}, t)
      scale_copy<T>(KW, ldn, n, cw + 1, T(ar), Y, ldn, st);
      if (rp > 0) {
        gemm_tn<T>(Mk(k - 1), ldn, rp, Xs, ldn, cw + 1, n, 1.0, 0.0, u1, rp, c->part64, c->part64_elems, st);
        gemm_nn<T, double>(n, cw + 1, rp, T(-ar * at * at * c->a * c->a), Mk(k - 1), ldn, u1, rp, T(1), Y, ldn, st);
      }
      if (ic > 0) {
        gemm_tn<T>(PV(k), ldn, ic, Xs, ldn, cw + 1, n, 1.0, 0.0, u2, ic, c->part64, c->part64_elems, st);
        gemm_nn<T, double>(n, cw + 1, ic, T(-ar * at * at), PV(k), ldn, u2, ic, T(1), Y, ldn, st);
      }
      smooth_out<T>(fm, fv, Y, ldn, cw, n, sm, sv, st);
    }
  }

  // ---------------------------------------------------------------- posterior sampler
  // The CAKF/CAKS sampler (appendix algorithm) for S draws, with the filter's stored factors: no
  // kernel values are evaluated.  Filter: x^-_k = a x_{k-1} + b + q_k, c_k = V_k^T (y_k - x^-_k[obs]
  // - eps_k), x_k = x^-_k + [P^-W]_k c_k.  Smoother: t = a ws_{k+1}, with K t carried by the same
  // recursion the smoother uses (K ws_T = K(X, X_o) V_T c_T, K ws_k = K t + K(X, X_o) V_k (c_k - z)):
  // P^- t = K t - a^2 M+_{k-1}(M+_{k-1}^T t), z = V_k^T (P^- t)[obs], x^s_k = x_k + P^- t - [P^-W]_k z,
  // ws_k = t + H^T V_k (c_k - z).  xf (T+1) x S x n holds the filter draws (x0 in slot 0); q and eps
  // are device arrays laid out like the outputs / like y with S columns per step.
  int sample(int S, double* xf, double* xs, const double* q, const double* eps, T* work, size_t work_elems,
             double* small, size_t small_elems) {
    const int n = c->n, T_ = c->T, ldn = c->ldn;
    const double a = c->a, a2 = a * a;
    const size_t blk = (size_t)n * S;
    // work layout (precision T): tmp (ldn x S), t (ldn x S), Kt (ldn x S), ws (ldn x S), Kws (ldn x S),
    // gathered rows (mmax x S) x 2
    const size_t lS = (size_t)ldn * S, mS = (size_t)std::max(c->mmax, 1) * S;
    if (work_elems < 5 * lS + 2 * mS) return fail(CAKF_ERR_ARG, "sampler workspace too small");
    T* tmp = work;
    T* t = tmp + lS;
    T* Kt = t + lS;
    T* ws = Kt + lS;
    T* Kws = ws + lS;
    T* dm = Kws + lS;
    T* dm2 = dm + mS;
    const size_t ii = (size_t)std::max(c->imax, 1) * S;
    double* cc = small;                       // c_k for every step: (T+1) x imax x S
    double* u = cc + (size_t)(T_ + 1) * ii;   // rmax x S
    double* z = u + (size_t)std::max(c->rmax, 1) * S;
    double* e = z + ii;
    if ((size_t)(e + ii - small) > small_elems) return fail(CAKF_ERR_ARG, "sampler scratch too small");
    cudaMemsetAsync(cc, 0, (size_t)(T_ + 1) * ii * sizeof(double), st);
    // ---- filter draws
    for (int k = 1; k <= T_; ++k) {
      if (int rc = restore(k)) return rc;
      double* xk = xf + (size_t)k * blk;
      samp_predict(xf + (size_t)(k - 1) * blk, q + (size_t)k * blk, c->has_mu ? c->mu + (size_t)k * n : nullptr,
                   c->has_mu ? c->mu + (size_t)(k - 1) * n : nullptr, a, n, S, xk, st);
      const int m = mk(k), ic = c->icap[k];
      if (m == 0 || ic == 0) continue;
      samp_resid<T>(c->y + c->obs_ptr[k - 1], xk, obs(k), eps + (size_t)c->obs_ptr[k - 1] * S, m, n, S, dm, st);
      double* ck = cc + (size_t)k * ii;
      gemm_tn<T>(Vk(k), m, ic, dm, m, S, m, 1.0, 0.0, ck, ic, c->part64, c->part64_elems, st);
      gemm_nn<T, double>(n, S, ic, T(1), PV(k), ldn, ck, ic, T(0), tmp, ldn, st);
      samp_add<T>(xk, tmp, ldn, 1.0, n, S, xk, st);
    }
    // ---- smoother draws
    cudaMemcpyAsync(xs + (size_t)T_ * blk, xf + (size_t)T_ * blk, blk * sizeof(double), cudaMemcpyDeviceToDevice, st);
    cudaMemsetAsync(ws, 0, lS * sizeof(T), st);
    cudaMemsetAsync(Kws, 0, lS * sizeof(T), st);
    if (T_ >= 1 && mk(T_) > 0 && c->icap[T_] > 0) {
      const int m = mk(T_), ic = c->icap[T_];
      if (int rc = restore(T_)) return rc;
      const double* cT = cc + (size_t)T_ * ii;
      gemm_nn<T, double>(m, S, ic, T(1), Vk(T_), m, cT, ic, T(0), dm, m, st);
      scatter_add_rows<T>(dm, m, obs(T_), m, S, T(1), ws, ldn, st);
      gemm_nn<T, double>(n, S, ic, T(1), KV(T_), ldn, cT, ic, T(0), Kws, ldn, st);
    }
    for (int k = T_ - 1; k >= 0; --k) {
      if (k >= 1)
        if (int rc = restore(k)) return rc;
      scale_copy<T>(ws, ldn, n, S, T(a), t, ldn, st);
      scale_copy<T>(Kws, ldn, n, S, T(a), Kt, ldn, st);
      // P^- t into Kt (in place)
      const int rp = (k >= 1) ? c->mcols[k - 1] : 0;
      if (rp > 0) {
        gemm_tn<T>(Mk(k - 1), ldn, rp, t, ldn, S, n, 1.0, 0.0, u, rp, c->part64, c->part64_elems, st);
        gemm_nn<T, double>(n, S, rp, T(-a2), Mk(k - 1), ldn, u, rp, T(1), Kt, ldn, st);
      }
      const int m = (k >= 1) ? mk(k) : 0, ic = (k >= 1) ? c->icap[k] : 0;
      double* xsk = xs + (size_t)k * blk;
      if (m == 0 || ic == 0) {
        samp_add<T>(xf + (size_t)k * blk, Kt, ldn, 1.0, n, S, xsk, st);
        if (k == 0) break;
        // no update at k: ws_k = t; K ws_k = K t (before the low-rank part)
        cudaMemcpyAsync(ws, t, lS * sizeof(T), cudaMemcpyDeviceToDevice, st);
        scale_copy<T>(Kws, ldn, n, S, T(a), Kws, ldn, st);
        continue;
      }
      // z = V_k^T (P^- t)[obs];  x^s_k = x_k + P^- t - [P^-W]_k z
      gather_rows<T>(Kt, ldn, obs(k), m, S, dm2, m, st);
      gemm_tn<T>(Vk(k), m, ic, dm2, m, S, m, 1.0, 0.0, z, ic, c->part64, c->part64_elems, st);
      gemm_nn<T, double>(n, S, ic, T(-1), PV(k), ldn, z, ic, T(1), Kt, ldn, st);
      samp_add<T>(xf + (size_t)k * blk, Kt, ldn, 1.0, n, S, xsk, st);
      // e = c_k - z;  ws_k = t + H^T V_k e;  K ws_k = a K ws_{k+1} + K(X, X_o) V_k e
      const double* ck = cc + (size_t)k * ii;
      copy_block(ck, ic, ic, S, e, ic);
      axpy_f64(-1.0, z, e, (size_t)ic * S);
      cudaMemcpyAsync(ws, t, lS * sizeof(T), cudaMemcpyDeviceToDevice, st);
      gemm_nn<T, double>(m, S, ic, T(1), Vk(k), m, e, ic, T(0), dm, m, st);
      scatter_add_rows<T>(dm, m, obs(k), m, S, T(1), ws, ldn, st);
      scale_copy<T>(Kws, ldn, n, S, T(a), Kws, ldn, st);
      gemm_nn<T, double>(n, S, ic, T(1), KV(k), ldn, e, ic, T(1), Kws, ldn, st);
    }
    cudaError_t ce = cudaGetLastError();
    return ce == cudaSuccess ? CAKF_OK : fail(CAKF_ERR_CUDA, std::string("sampler: ") + cudaGetErrorString(ce));
  }

  // ---------------------------------------------------------------- NLL gradient (tangent pass)
  // Forward-mode derivatives of the filter with the actions S_k and truncation rotations U_k of the
  // last filter run held fixed, for the four log-hyperparameters at once (p = 0: log l_x,
  // 1: log l_t, 2: log sf2, 3: log sn2).  Per step, with S the basis V_k of span(S_k) (below) and
  // Gh = S^T G S = R^T R:
  //   dGh_p = S^T dK_oo S - sym(...) + dsn2 S^T S,  dyh_p = -S^T dm^-_p[obs],
  //   dNLL_p = 1/2 tr(Gh^-1 dGh_p) + beta^T dyh_p - 1/2 beta^T dGh_p beta,
  //   d(P^-W)_p = dP^-_{:,obs} V - (P^-W) Phi(R^-T dGh_p R^-1),
  //   dm_p = dm^-_p + dP^-_{:,obs} v + (P^-W) R^-T (dyh_p - dGh_p beta),
  //   dM+_p = [dM^-_p, d(P^-W)_p] U_k.
  int nll_grad(const std::vector<int>& cnt) {
    const int n = c->n, T_ = c->T, ldn = c->ldn, NP = 4;
    const double a = c->a, a2 = a * a, adot = a * c->dt / c->lt;   // da / dlog l_t
    const size_t msz = (size_t)ldn * std::max(c->rmax, 1);
    T* dMprev = (T*)c->dMa;
    T* dMnew = (T*)c->dMb;
    double* dm = c->dmA;
    double* dmn = c->dmB;
    cudaMemsetAsync(c->grad, 0, 4 * sizeof(double), st);
    cudaMemsetAsync(dm, 0, (size_t)NP * n * sizeof(double), st);
    const size_t estride = (size_t)ldn * (c->imax + 1);
    for (int k = 1; k <= T_; ++k) {
      if (int rc = restore(k)) return rc;
      const int m = mk(k), icap = c->icap[k], rp = c->mcols[k - 1];
      const int ic = (m > 0 && icap > 0) ? cnt[k] : 0;
      const double* mprev = c->mf + (size_t)(k - 1) * n;
      tangent_predict(mprev, dm, c->has_mu ? c->mu + (size_t)(k - 1) * n : nullptr, a, adot, n, NP, c->dmpred, st);
      if (m == 0 || icap == 0) {
        // dM+_k = dM^-_k = adot M+ + a dM+ (only p = 1 carries adot)
        for (int p = 0; p < NP; ++p) scale_copy<T>(dMprev + p * msz, ldn, n, rp, T(a), dMnew + p * msz, ldn, st);
        if (rp > 0) axpy_cols(T(adot), Mk(k - 1), ldn, n, rp, dMnew + 1 * msz, ldn);
        cudaMemcpyAsync(dmn, c->dmpred, (size_t)NP * n * sizeof(double), cudaMemcpyDeviceToDevice, st);
        std::swap(dMprev, dMnew);
        std::swap(dm, dmn);
        continue;
      }
      const int* ob = obs(k);
      C4<T>* Xo = (C4<T>*)c->Xo;
      gather_coords<T>(X(), ob, m, Xo, st);
      // The derivatives depend on the actions only through span(S_k), so the products below use
      // the stored G-orthonormal directions V_k as the basis of that span: with B = V_k the
      // Cholesky factor of B^T G B is R = R_S R_S0^-1 at every theta, and H^T B R^-1 = H^T S_k R_S^-1,
      // the same W as with S_k itself, while B^T G B stays well conditioned where CG converged
      // within the budget (the NLL term uses the same basis).
      T* S = Vk(k);
      T* V = Vk(k);                       // m x (icap + 1): V (ic valid columns), zero columns, v
      T* PVk = PV(k);                     // n x (icap + 1): P^- W, P^- w
      T* Mo = (T*)c->Mo;
      gather_rows<T>(Mk(k - 1), ldn, ob, m, rp, Mo, m, st);
      double* G = c->gsmall;              // small FP64 matrices
      const size_t ii = (size_t)ic * ic;
      double* Gh = G;
      double* dGh = Gh + ii;              // NP blocks
      double* SS = dGh + NP * ii;
      double* SKS = SS + ii;
      double* SKlS = SKS + ii;
      double* Ao = SKlS + ii;             // rp x ic
      double* dAo = Ao + (size_t)rp * ic; // NP blocks rp x ic
      double* yh = dAo + (size_t)NP * rp * ic;
      double* dyh = yh + ic;              // NP x ic
      double* L = dyh + (size_t)NP * ic;
      double* Rinv = L + ii;
      double* W = Rinv + ii;
      double* tmp = W + ii;               // 3 ic
      double* Qm = tmp + 3 * (size_t)ic;  // NP blocks
      double* u = Qm + NP * ii;           // NP x ic
      double* to = u + (size_t)NP * ic;   // rp x (icap+1): M+_o^T [V v]
      double* dto = to + (size_t)rp * (icap + 1);   // NP blocks
      double* coef = dto + (size_t)NP * rp * (icap + 1);
      // K_oo S and dK_oo/dlog l S (SIMT, precision T)
      T* KS = (T*)c->KS;
      T* KlS = (T*)c->KlS;
      gram_block_simt<T>(c->kernel, Xo, m, Xo, m, S, m, ic, T(c->sf2), KS, m, st);
      gram_block_dlogl_simt<T>(c->kernel, Xo, m, Xo, m, S, m, ic, T(c->sf2), KlS, m, st);
      gemm_tn<T>(S, m, ic, S, m, ic, m, 1.0, 0.0, SS, ic, c->part64, c->part64_elems, st);
      gemm_tn<T>(S, m, ic, KS, m, ic, m, 1.0, 0.0, SKS, ic, c->part64, c->part64_elems, st);
      gemm_tn<T>(S, m, ic, KlS, m, ic, m, 1.0, 0.0, SKlS, ic, c->part64, c->part64_elems, st);
      if (rp > 0) {
        gemm_tn<T>(Mo, m, rp, S, m, ic, m, 1.0, 0.0, Ao, rp, c->part64, c->part64_elems, st);
        for (int p = 0; p < NP; ++p) {
          gather_rows<T>(dMprev + p * msz, ldn, ob, m, rp, (T*)c->Xobs, m, st);
          gemm_tn<T>((T*)c->Xobs, m, rp, S, m, ic, m, 1.0, 0.0, dAo + (size_t)p * rp * ic, rp, c->part64,
                     c->part64_elems, st);
        }
      }
      // Gh = S^T K S + sn2 S^T S - a^2 Ao^T Ao
      copy_block(SKS, ic, ic, ic, Gh, ic);
      axpy_f64(c->sn2, SS, Gh, ii);
      if (rp > 0) gemm_small_f64(1, 0, ic, ic, rp, -a2, Ao, rp, Ao, rp, 1.0, Gh, ic, st);
      for (int p = 0; p < NP; ++p) {
        double* D = dGh + p * ii;
        cudaMemsetAsync(D, 0, ii * sizeof(double), st);
        if (p == 0) copy_block(SKlS, ic, ic, ic, D, ic);
        if (p == 2) copy_block(SKS, ic, ic, ic, D, ic);
        if (p == 3) axpy_f64(c->sn2, SS, D, ii);
        if (rp > 0) {
          if (p == 1) gemm_small_f64(1, 0, ic, ic, rp, -2.0 * a * adot, Ao, rp, Ao, rp, 1.0, D, ic, st);
          gemm_small_f64(1, 0, ic, ic, rp, -a2, dAo + (size_t)p * rp * ic, rp, Ao, rp, 1.0, D, ic, st);
          gemm_small_f64(1, 0, ic, ic, rp, -a2, Ao, rp, dAo + (size_t)p * rp * ic, rp, 1.0, D, ic, st);
        }
      }
      // yh = S^T r0, dyh_p = -S^T dm^-_p[obs]
      T* r0 = (T*)c->r0v;
      predict_mean(mprev, c->has_mu ? c->mu + (size_t)k * n : nullptr, c->has_mu ? c->mu + (size_t)(k - 1) * n : nullptr,
                   a, n, c->mpred, st);
      cudaMemsetAsync(c->r0sq, 0, sizeof(double), st);   // element 0 (no data at state 0): scratch
      cg_init<T>(c->y + c->obs_ptr[k - 1], c->mpred, ob, m, (T*)c->rv, r0, (T*)c->sv, c->r0sq, st);
      gemm_tn<T>(S, m, ic, r0, m, 1, m, 1.0, 0.0, yh, ic, c->part64, c->part64_elems, st);
      T* dmo = (T*)c->dmo;
      gather_rows_f64<T>(c->dmpred, n, ob, m, NP, dmo, m, st);
      gemm_tn<T>(S, m, ic, dmo, m, NP, m, -1.0, 0.0, dyh, ic, c->part64, c->part64_elems, st);
      grad_small(ic, NP, Gh, dGh, yh, dyh, L, Rinv, W, tmp, Qm, u, c->grad, c->err, st);
      // E_p = dP^-_{:,obs} [V v]  for the icap + 1 stored columns
      T* E = (T*)c->Eg;
      const int w1 = icap + 1;
      if (rp > 0) {
        gemm_tn<T>(Mo, m, rp, V, m, w1, m, 1.0, 0.0, to, rp, c->part64, c->part64_elems, st);
        for (int p = 0; p < NP; ++p) {
          gather_rows<T>(dMprev + p * msz, ldn, ob, m, rp, (T*)c->Xobs, m, st);
          gemm_tn<T>((T*)c->Xobs, m, rp, V, m, w1, m, 1.0, 0.0, dto + (size_t)p * rp * w1, rp, c->part64,
                     c->part64_elems, st);
        }
      }
      for (int p = 0; p < NP; ++p) {
        T* Ep = E + p * estride;
        if (p == 0) gram_block_dlogl_simt<T>(c->kernel, X(), n, Xo, m, V, m, w1, T(c->sf2), Ep, ldn, st);
        else if (p == 2) scale_copy<T>(PVk, ldn, n, w1, T(1), Ep, ldn, st);
        else cudaMemsetAsync(Ep, 0, (size_t)ldn * w1 * sizeof(T), st);
        if (rp > 0) {
          // E_p += M+ (alpha_p to - a^2 dto_p) - a^2 dM+_p to,  alpha_p = -2 a adot [p=1] + a^2 [p=2]
          const double alpha_p = (p == 1 ? -2.0 * a * adot : 0.0) + (p == 2 ? a2 : 0.0);
          copy_block(dto + (size_t)p * rp * w1, rp, rp, w1, coef, rp);
          scale_f64(coef, rp, rp, w1, -a2, st);
          if (alpha_p != 0.0) axpy_f64(alpha_p, to, coef, (size_t)rp * w1);
          gemm_nn<T, double>(n, w1, rp, T(1), Mk(k - 1), ldn, coef, rp, T(1), Ep, ldn, st);
          gemm_nn<T, double>(n, w1, rp, T(-a2), dMprev + p * msz, ldn, to, rp, T(1), Ep, ldn, st);
        }
        // d(P^-W)_p = E_p[:, :ic] - (P^-W) Q_p   (in place in E_p)
        gemm_nn<T, double>(n, ic, ic, T(-1), PVk, ldn, Qm + p * ii, ic, T(1), Ep, ldn, st);
      }
      // dm_p = dm^-_p + E_p[:, icap] + (P^-W) u_p
      T* tv = (T*)c->tvec;
      for (int p = 0; p < NP; ++p)
        gemm_nn<T, double>(n, 1, ic, T(1), PVk, ldn, u + (size_t)p * ic, ic, T(0), tv + (size_t)p * ldn, ldn, st);
      tangent_mean<T>(c->dmpred, E, estride, icap, ldn, tv, ldn, n, NP, dmn, st);
      // dM^-_p = a dM+_p + adot [p=1] M+ ;  dM+_k = [dM^-_p, d(P^-W)_p] U_k
      const int keep = c->mcols[k];
      for (int p = 0; p < NP; ++p) {
        T* dMp = dMprev + p * msz;
        if (rp > 0) {
          scale_cols<T>(dMp, ldn, n, rp, T(a), st);
          if (p == 1) axpy_cols(T(adot), Mk(k - 1), ldn, n, rp, dMp, ldn);
        }
        T* out = dMnew + p * msz;
        T* Ep = E + p * estride;
        if (c->rank_r > 0) {
          const double* U = c->Upool + c->off_U[k];
          const int N = c->Urows[k];
          if (rp > 0) gemm_nn<T, double>(n, keep, rp, T(1), dMp, ldn, U, N, T(0), out, ldn, st);
          gemm_nn<T, double>(n, keep, icap, T(1), Ep, ldn, U + rp, N, rp > 0 ? T(1) : T(0), out, ldn, st);
        } else {
          scale_copy<T>(dMp, ldn, n, rp, T(1), out, ldn, st);
          scale_copy<T>(Ep, ldn, n, icap, T(1), out + (size_t)rp * ldn, ldn, st);
        }
      }
      std::swap(dMprev, dMnew);
      std::swap(dm, dmn);
      cudaError_t ce = cudaGetLastError();
      if (ce != cudaSuccess) return fail(CAKF_ERR_CUDA, std::string("gradient step: ") + cudaGetErrorString(ce));
    }
    return CAKF_OK;
  }
  void axpy_cols(T alpha, const T* X_, int ldx, int rows, int cols, T* Y_, int ldy) {
    axpy_block<T>(alpha, X_, ldx, rows, cols, Y_, ldy, st);
  }
  void axpy_f64(double alpha, const double* x, double* y, size_t len) { axpy_block<double>(alpha, x, (int)len, (int)len, 1, y, (int)len, st); }

  void copy_block(const double* src, int lds, int rows, int cols, double* dst, int ldd) {
    if (rows <= 0 || cols <= 0) return;
    cudaMemcpy2DAsync(dst, ldd * sizeof(double), src, lds * sizeof(double), rows * sizeof(double), cols,
                      cudaMemcpyDeviceToDevice, st);
  }
  void copy_block_scaled(const double* src, int lds, int rows, int cols, double* dst, int ldd, double s) {
    copy_block(src, lds, rows, cols, dst, ldd);
    scale_f64(dst, ldd, rows, cols, s, st);
  }
};

}  // namespace


namespace {

// ------------------------------------------------------------------------------------ validation
int validate(const cakf_problem* p) {
  if (!p) return fail(CAKF_ERR_ARG, "problem is NULL");
  if (p->abi_version != CAKF_ABI_VERSION) return fail(CAKF_ERR_ARG, "abi_version mismatch");
  if (p->n < 1) return fail(CAKF_ERR_ARG, "n must be >= 1");
  if (p->dim < 1 || p->dim > 3) return fail(CAKF_ERR_ARG, "dim must be 1..3");
  if (!p->coords) return fail(CAKF_ERR_ARG, "coords is NULL");
  if (p->kernel < 0 || p->kernel > 2) return fail(CAKF_ERR_ARG, "unknown kernel");
  if (p->T < 0) return fail(CAKF_ERR_ARG, "T must be >= 0");
  if (!p->obs_ptr) return fail(CAKF_ERR_ARG, "obs_ptr is NULL");
  if (is_device_ptr(p->obs_ptr)) return fail(CAKF_ERR_ARG, "obs_ptr must be a host array");
  if (p->obs_ptr[0] != 0) return fail(CAKF_ERR_ARG, "obs_ptr[0] must be 0");
  for (int k = 1; k <= p->T; ++k) {
    if (p->obs_ptr[k] < p->obs_ptr[k - 1]) return fail(CAKF_ERR_ARG, "obs_ptr must be non-decreasing");
    if (p->obs_ptr[k] - p->obs_ptr[k - 1] > p->n) return fail(CAKF_ERR_ARG, "more observations than grid points in a step");
  }
  const int N = p->obs_ptr[p->T];
  if (N > 0 && (!p->obs_idx || !p->y)) return fail(CAKF_ERR_ARG, "obs_idx / y is NULL");
  if (p->budget_i < 1 || p->budget_i > 1024) return fail(CAKF_ERR_ARG, "budget_i must be in 1..1024");
  if (p->precision < CAKF_FP64 || p->precision > CAKF_TF32X3) return fail(CAKF_ERR_ARG, "unknown precision");
  const double hp[4] = {p->log_lx, p->log_lt, p->log_sf2, p->log_sn2};
  for (double h : hp)
    if (!std::isfinite(h) || std::fabs(h) > 80) return fail(CAKF_ERR_ARG, "hyperparameters must be finite");
  if (!(p->dt > 0) || !std::isfinite(p->dt)) return fail(CAKF_ERR_ARG, "dt must be > 0");
  if (!(p->cg_rtol >= 0)) return fail(CAKF_ERR_ARG, "cg_rtol must be >= 0");
  if (p->factor_storage < CAKF_STORE_FP32 || p->factor_storage > CAKF_RECOMPUTE)
    return fail(CAKF_ERR_ARG, "unknown factor_storage");
  if (p->factor_storage == CAKF_STORE_BF16 && p->precision == CAKF_FP64)
    return fail(CAKF_ERR_ARG, "CAKF_STORE_BF16 needs an FP32-based precision");
  if (p->checkpoint_every < 0) return fail(CAKF_ERR_ARG, "checkpoint_every must be >= 0");
  if (p->policy < CAKF_POLICY_CG || p->policy > CAKF_POLICY_BATCH) return fail(CAKF_ERR_ARG, "unknown policy");
  if (p->temporal != CAKF_TEMPORAL_OU && p->temporal != CAKF_TEMPORAL_MATERN32)
    return fail(CAKF_ERR_ARG, "unknown temporal factor");
  if (p->temporal == CAKF_TEMPORAL_MATERN32 && p->factor_storage != CAKF_STORE_FP32)
    return fail(CAKF_ERR_ARG, "the Matern-3/2 temporal factor keeps its factors resident (CAKF_STORE_FP32)");
  if (p->temporal == CAKF_TEMPORAL_MATERN32 && p->freeze_truncation)
    return fail(CAKF_ERR_ARG, "freeze_truncation is not available with the Matern-3/2 temporal factor");
  if (p->policy == CAKF_POLICY_BATCH && !p->replay_actions)
    return fail(CAKF_ERR_ARG, "CAKF_POLICY_BATCH takes its actions from replay_actions");
  if (p->policy == CAKF_POLICY_COORDINATE && p->replay_actions)
    return fail(CAKF_ERR_ARG, "CAKF_POLICY_COORDINATE chooses its own actions (replay_actions must be NULL)");
  if (p->policy == CAKF_POLICY_COORDINATE && p->budget_i > kBatchMaxActions)
    return fail(CAKF_ERR_ARG, "the batch policies take at most 160 actions per step");
  if (p->replay_actions && !p->replay_counts) return fail(CAKF_ERR_ARG, "replay_actions without replay_counts");
  if (p->replay_counts) {
    for (int k = 1; k <= p->T; ++k) {
      int c = p->replay_counts[k], mk = p->obs_ptr[k] - p->obs_ptr[k - 1];
      if (c < 0 || c > mk || c > 1024) return fail(CAKF_ERR_ARG, "replay_counts out of range");
      if (p->policy == CAKF_POLICY_BATCH && c > kBatchMaxActions)
        return fail(CAKF_ERR_ARG, "the batch policies take at most 160 actions per step");
    }
  }
  // host inputs are checked for non-finite values here (device inputs surface as CAKF_ERR_NUMERIC
  // through the outputs' finiteness check)
  if (ptr_kind(p->coords) == kHost)
    for (size_t q = 0; q < (size_t)p->n * p->dim; ++q)
      if (!std::isfinite(p->coords[q])) return fail(CAKF_ERR_ARG, "non-finite coordinate");
  if (N > 0 && ptr_kind(p->y) == kHost)
    for (int q = 0; q < N; ++q)
      if (!std::isfinite(p->y[q])) return fail(CAKF_ERR_ARG, "non-finite observation");
  // observation indices: range and distinctness per step (checked on a host copy)
  if (N > 0) {
    std::vector<int> idx(N);
    if (is_device_ptr(p->obs_idx)) {
      if (cudaMemcpy(idx.data(), p->obs_idx, N * sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        return fail(CAKF_ERR_CUDA, "reading obs_idx");
    } else {
      std::memcpy(idx.data(), p->obs_idx, N * sizeof(int));
    }
    std::vector<int> mark(p->n, -1);
    for (int k = 1; k <= p->T; ++k)
      for (int q = p->obs_ptr[k - 1]; q < p->obs_ptr[k]; ++q) {
        int v = idx[q];
        if (v < 0 || v >= p->n) return fail(CAKF_ERR_ARG, "obs_idx out of range");
        if (mark[v] == k) return fail(CAKF_ERR_ARG, "duplicate obs_idx within a step");
        mark[v] = k;
      }
  }
  return CAKF_OK;
}

bool same_shape(const cakf_ctx* c, const cakf_problem* p) {
  if (c->n != p->n || c->T != p->T || c->budget != p->budget_i || c->rank_r != p->rank_r ||
      c->precision != p->precision || c->has_mu != (p->prior_mean != nullptr) || c->replay != (p->replay_actions != nullptr) ||
      c->storage != p->factor_storage || c->ckpt_req != p->checkpoint_every || c->policy != p->policy ||
      c->dprime != (p->temporal == CAKF_TEMPORAL_MATERN32 ? 2 : 1))
    return false;
  for (int k = 0; k <= p->T; ++k)
    if (c->obs_ptr[k] != p->obs_ptr[k]) return false;
  if (c->replay)
    for (int k = 0; k <= p->T; ++k)
      if (c->replay_counts[k] != p->replay_counts[k]) return false;
  return true;
}

double nu_scale(int kernel) { return kernel == 0 ? 1.0 : (kernel == 1 ? std::sqrt(3.0) : std::sqrt(5.0)); }

const char* numeric_error_text(int e) {
  switch (e) {
    case kErrNllChol: return "a step's projected Gram S^T G S (or S^T S) is not positive definite in the NLL term";
    case kErrBatchChol: return "the batch update's projected Gram S^T G S is not positive definite";
    case kErrSecular: return "a secular equation of the truncation eigensolver did not converge";
    case kErrNonFinite: return "non-finite value in the outputs";
    case kErrGradChol: return "a step's projected Gram is not positive definite in the gradient pass";
    default: return "non-finite value or non-positive-definite action Gram";
  }
}

int sync_and_check(cakf_ctx* c, cudaStream_t st, const char* what) {
  cudaError_t ce = cudaStreamSynchronize(st);
  if (ce != cudaSuccess) return fail(CAKF_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(ce));
  int e = 0;
  cudaMemcpy(&e, c->err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e == kErrTimeout) return fail(CAKF_ERR_TIMEOUT, std::string(what) + ": a device-side wait exceeded its limit");
  if (e != 0) return fail(CAKF_ERR_NUMERIC, std::string(what) + ": " + numeric_error_text(e));
  return CAKF_OK;
}

void collect_profile(cakf_ctx* c) {
  auto sum = [](std::vector<std::pair<cudaEvent_t, cudaEvent_t>>& v) {
    double tot = 0;
    for (auto& pr : v) { float ms = 0; cudaEventElapsedTime(&ms, pr.first, pr.second); tot += ms; }
    return tot;
  };
  c->stats.gram_block_ms += sum(c->prof_gb);
  c->stats.gram_block_launches += (int64_t)c->prof_gb.size();
  for (double f : c->prof_gb_flops) c->stats.gram_block_flops += f;
  for (double f : c->prof_gb_evals) c->stats.gram_block_evals += f;
  c->stats.cg_matvec_ms += sum(c->prof_mv);
  c->stats.cg_matvec_launches += (int64_t)c->prof_mv.size();
  for (double f : c->prof_mv_evals) c->stats.cg_matvec_evals += f;
  c->stats.eig_ms += sum(c->prof_eig);
  c->stats.eig_phase_ms[0] += sum(c->prof_eig_tri);
  c->stats.eig_phase_ms[1] += sum(c->prof_eig_dc);
  c->stats.eig_phase_ms[2] += sum(c->prof_eig_bt);
  for (auto& ph : c->prof_phase) {
    float ms = 0;
    cudaEventElapsedTime(&ms, ph.second.first, ph.second.second);
    c->stats.phase_ms[ph.first] += ms;
  }
  c->prof_phase.clear();
  c->prof_gb.clear(); c->prof_gb_flops.clear(); c->prof_gb_evals.clear();
  c->prof_mv.clear(); c->prof_mv_evals.clear(); c->prof_eig.clear();
  c->prof_eig_tri.clear(); c->prof_eig_dc.clear(); c->prof_eig_bt.clear();
  c->ev_used = 0;
}

template <class T>
Runner<T> make_runner(cakf_ctx* c, cudaStream_t st) {
  // plain FP32 factor products: own SIMT kernels; tensor-core modes: own split-TF32 tcgen05 kernels
  set_gemm_mode(c->precision == CAKF_FP64 ? 0 : (c->precision == CAKF_FP32 ? 1 : 2));
  set_gemm_err(c->err);
  Runner<T> r;
  r.c = c;
  r.st = st;
  r.tc = tc_kind_of(c->precision) >= 0;
  r.tc_kind = std::max(tc_kind_of(c->precision), 0);
  return r;
}

}  // namespace

// ============================================================================================ ABI
extern "C" {

int cakf_filter(const cakf_problem* p, cakf_ctx** ctx_inout, double* mean_out, double* var_out, void* cuda_stream) {
  if (!ctx_inout) return fail(CAKF_ERR_ARG, "ctx_inout is NULL");
  int rc = validate(p);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  cakf_ctx* c = *ctx_inout;
  bool fresh = false;
  if (p->freeze_truncation && (!c || !c->filtered || !same_shape(c, p) || c->rank_r <= 0))
    return fail(CAKF_ERR_STATE, "freeze_truncation needs a previous successful cakf_filter of the same sizes "
                                "(with truncation) on this context");
  if (c && !same_shape(c, p)) { c->release(); c->filtered = false; fresh = true; }
  if (!c) { c = new cakf_ctx(); *ctx_inout = c; fresh = true; }
  c->n = p->n; c->dim = p->dim; c->kernel = p->kernel; c->T = p->T; c->budget = p->budget_i; c->rank_r = p->rank_r;
  c->precision = p->precision; c->lx = std::exp(p->log_lx); c->lt = std::exp(p->log_lt); c->sf2 = std::exp(p->log_sf2);
  c->sn2 = std::exp(p->log_sn2); c->dt = p->dt; c->a = std::exp(-p->dt / c->lt); c->cg_rtol = p->cg_rtol;
  c->dprime = p->temporal == CAKF_TEMPORAL_MATERN32 ? 2 : 1;
  if (c->dprime == 2) {
    // A^t = expm(F dt) = exp(-lam dt) (I + dt (F + lam I)) (F + lam I is nilpotent),
    // P^t_inf = diag(1, lam^2), F = [[0, 1], [-lam^2, -2 lam]], lam = sqrt(3) / l_t
    const double lam = std::sqrt(3.0) / c->lt, e = std::exp(-lam * p->dt), h = p->dt;
    const double At[4] = {e * (1.0 + lam * h), e * h, -e * lam * lam * h, e * (1.0 - lam * h)};
    const double Pt[4] = {1.0, 0.0, 0.0, lam * lam};
    std::memcpy(c->At, At, sizeof(At));
    std::memcpy(c->Pt, Pt, sizeof(Pt));
  }
  c->has_mu = p->prior_mean != nullptr;
  c->replay = p->replay_actions != nullptr;
  c->freeze = p->freeze_truncation != 0;
  if (c->replay) c->replay_counts.assign(p->replay_counts, p->replay_counts + p->T + 1);
  c->filtered = false;
  if (fresh || c->bufs.empty()) {
    rc = plan_and_alloc(c, p);
    if (rc) { c->release(); return rc; }
  }
  c->stats = cakf_stats{};
  c->stats.device_bytes = (int64_t)c->dev_bytes;
  c->launch_base = cakf::launch_count();
  const size_t N = c->obs_ptr[c->T];
  const int n = c->n;
  if ((rc = copy_in(c->coords64, p->coords, (size_t)n * p->dim * sizeof(double), st))) return rc;
  if ((rc = copy_in(c->obs, p->obs_idx, N * sizeof(int), st))) return rc;
  if ((rc = copy_in(c->y, p->y, N * sizeof(double), st))) return rc;
  if (c->has_mu && (rc = copy_in(c->mu, p->prior_mean, (size_t)(c->T + 1) * n * sizeof(double), st))) return rc;
  if (c->replay) {
    // pack the replayed actions per step (host input, concatenated m_k x i_k blocks)
    if ((rc = copy_in(c->rep, p->replay_actions, c->off_rep[c->T + 1] * sizeof(double), st))) return rc;
  }
  // device inputs are checked for non-finite values before any work (host inputs were checked by
  // validate): a NaN observation would otherwise only end its step's update as a breakdown
  if (ptr_kind(p->y) != kHost || ptr_kind(p->coords) != kHost) {
    cudaMemsetAsync(c->err, 0, sizeof(int), st);
    check_finite(c->y, N, c->err, st);
    check_finite(c->coords64, (size_t)n * p->dim, c->err, st);
    int e = 0;
    cudaMemcpyAsync(&e, c->err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) return fail(CAKF_ERR_CUDA, "checking the inputs");
    if (e) return fail(CAKF_ERR_ARG, "non-finite coordinate or observation");
  }
  const double scale = nu_scale(c->kernel) / c->lx;
  cudaEventRecord(c->ev0, st);
  if (c->precision == CAKF_FP64) {
    prep_coords<double>(c->coords64, n, p->dim, scale, (C4<double>*)c->X, st);
    Runner<double> r = make_runner<double>(c, st);
    rc = r.filter();
  } else {
    prep_coords<float>(c->coords64, n, p->dim, scale, (C4<float>*)c->X, st);
    Runner<float> r = make_runner<float>(c, st);
    rc = r.filter();
  }
  cudaEventRecord(c->ev1, st);
  if (rc) return rc;
  check_finite(c->mf, (size_t)(c->T + 1) * c->mstride, c->err, st);
  check_finite(c->vf, (size_t)(c->T + 1) * n, c->err, st);
  if ((rc = sync_and_check(c, st, "cakf_filter"))) return rc;
  float ms = 0;
  cudaEventElapsedTime(&ms, c->ev0, c->ev1);
  c->stats.filter_ms = ms;
  if (c->profiling) collect_profile(c);
  if (c->mstride == n) {
    if ((rc = copy_out(mean_out, c->mf, (size_t)(c->T + 1) * n, st))) return rc;
  } else if (mean_out) {
    // the positions of the two-block state means
    const PtrKind kind = ptr_kind(mean_out);
    if (kind == kOtherDevice) return fail(CAKF_ERR_ARG, "an output array lives on another device than the current one");
    cudaError_t ce = cudaMemcpy2DAsync(mean_out, n * sizeof(double), c->mf, c->mstride * sizeof(double),
                                       n * sizeof(double), c->T + 1,
                                       kind == kDevice ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st);
    if (ce != cudaSuccess) return fail(CAKF_ERR_CUDA, std::string("copy out: ") + cudaGetErrorString(ce));
  }
  if ((rc = copy_out(var_out, c->vf, (size_t)(c->T + 1) * n, st))) return rc;
  cudaError_t ce = cudaStreamSynchronize(st);
  if (ce != cudaSuccess) return fail(CAKF_ERR_CUDA, cudaGetErrorString(ce));
  c->filtered = true;
  return CAKF_OK;
}

int cakf_smooth(cakf_ctx* c, double* mean_out, double* var_out, void* cuda_stream) {
  if (!c) return fail(CAKF_ERR_STATE, "cakf_smooth: no context (cakf_filter creates it)");
  if (!c->filtered) return fail(CAKF_ERR_STATE, "cakf_smooth needs a successful cakf_filter on this context");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const size_t tot = (size_t)(c->T + 1) * c->n;
  int rc;
  if (ptr_kind(mean_out) == kOtherDevice || ptr_kind(var_out) == kOtherDevice)
    return fail(CAKF_ERR_ARG, "cakf_smooth: an output array lives on another device than the current one");
  double* ms = is_device_ptr(mean_out) ? mean_out : nullptr;
  double* vs = is_device_ptr(var_out) ? var_out : nullptr;
  if (!ms || !vs) {
    if (!c->ms_dev) {
      if ((rc = c->alloc(c->ms_dev, tot * sizeof(double)))) return rc;
      if ((rc = c->alloc(c->vs_dev, tot * sizeof(double)))) return rc;
    }
    if (!ms) ms = c->ms_dev;
    if (!vs) vs = c->vs_dev;
  }
  cudaMemsetAsync(c->err, 0, sizeof(int), st);
  cudaEventRecord(c->ev0, st);
  if (c->precision == CAKF_FP64) {
    Runner<double> r = make_runner<double>(c, st);
    rc = r.smooth(ms, vs);
  } else {
    Runner<float> r = make_runner<float>(c, st);
    rc = r.smooth(ms, vs);
  }
  cudaEventRecord(c->ev1, st);
  if (rc) return rc;
  check_finite(ms, tot, c->err, st);
  check_finite(vs, tot, c->err, st);
  if ((rc = sync_and_check(c, st, "cakf_smooth"))) return rc;
  float msec = 0;
  cudaEventElapsedTime(&msec, c->ev0, c->ev1);
  c->stats.smooth_ms = msec;
  if (c->profiling) collect_profile(c);
  if (mean_out && ms != mean_out && (rc = copy_out(mean_out, ms, tot, st))) return rc;
  if (var_out && vs != var_out && (rc = copy_out(var_out, vs, tot, st))) return rc;
  cudaError_t ce = cudaStreamSynchronize(st);
  return ce == cudaSuccess ? CAKF_OK : fail(CAKF_ERR_CUDA, cudaGetErrorString(ce));
}

int cakf_nll(cakf_ctx* c, double* nll_out) {
  if (!nll_out) return fail(CAKF_ERR_ARG, "cakf_nll: nll_out is NULL");
  if (!c) return fail(CAKF_ERR_STATE, "cakf_nll: no context (cakf_filter creates it)");
  if (!c->filtered) return fail(CAKF_ERR_STATE, "cakf_nll needs a successful cakf_filter on this context");
  std::vector<double> v(c->T + 1);
  if (cudaMemcpy(v.data(), c->nll, (c->T + 1) * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
    return fail(CAKF_ERR_CUDA, "reading NLL terms");
  double s = 0;
  for (double x : v) s += x;
  *nll_out = s;
  return CAKF_OK;
}

int cakf_get_actions(cakf_ctx* c, double* actions_out, int32_t* counts_out) {
  if (!counts_out) return fail(CAKF_ERR_ARG, "cakf_get_actions: counts_out is NULL");
  if (!c) return fail(CAKF_ERR_STATE, "cakf_get_actions: no context (cakf_filter creates it)");
  if (!c->filtered) return fail(CAKF_ERR_STATE, "no filter run on this context");
  std::vector<int> cnt(c->T + 1);
  cudaMemcpy(cnt.data(), c->count, (c->T + 1) * sizeof(int), cudaMemcpyDeviceToHost);
  for (int k = 0; k <= c->T; ++k) counts_out[k] = (k == 0) ? 0 : cnt[k];
  if (!actions_out) return CAKF_OK;
  size_t off = 0;
  const size_t es = elem_size(c->precision);
  for (int k = 1; k <= c->T; ++k) {
    const int m = c->obs_ptr[k] - c->obs_ptr[k - 1];
    const size_t cnt_el = (size_t)m * cnt[k];
    if (cnt_el == 0) continue;
    if (es == 8) {
      cudaMemcpy(actions_out + off, (double*)c->Spool + c->off_S[k], cnt_el * 8, cudaMemcpyDeviceToHost);
    } else {
      std::vector<float> tmp(cnt_el);
      cudaMemcpy(tmp.data(), (float*)c->Spool + c->off_S[k], cnt_el * 4, cudaMemcpyDeviceToHost);
      for (size_t q = 0; q < cnt_el; ++q) actions_out[off + q] = tmp[q];
    }
    off += cnt_el;
  }
  return CAKF_OK;
}

int cakf_interpolate(cakf_ctx* c, int32_t nq, const double* tq, const double* mu_q, double* fmean, double* fvar,
                     double* smean, double* svar, void* cuda_stream) {
  if (!c) return fail(CAKF_ERR_STATE, "cakf_interpolate: no context (cakf_filter creates it)");
  if (!c->filtered) return fail(CAKF_ERR_STATE, "cakf_interpolate needs a successful cakf_filter on this context");
  if (c->dprime != 1) return fail(CAKF_ERR_ARG, "cakf_interpolate: Ornstein-Uhlenbeck temporal factor only");
  if (nq < 1 || !tq) return fail(CAKF_ERR_ARG, "cakf_interpolate: nq >= 1 query times are needed");
  if (ptr_kind(tq) != kHost) return fail(CAKF_ERR_ARG, "cakf_interpolate: tq must be a host array");
  if (c->has_mu && !mu_q) return fail(CAKF_ERR_ARG, "cakf_interpolate: the problem has a prior mean, so mu_q is needed");
  const int n = c->n, T = c->T;
  const size_t tot = (size_t)nq * n;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  double* buf = nullptr;
  double* mq = nullptr;
  if (cudaMalloc(&buf, 4 * tot * sizeof(double)) != cudaSuccess ||
      (mu_q && cudaMalloc(&mq, tot * sizeof(double)) != cudaSuccess)) {
    cudaGetLastError();
    if (buf) cudaFree(buf);
    return fail(CAKF_ERR_OOM, "cakf_interpolate: workspace allocation failed");
  }
  int rc = mu_q ? copy_in(mq, mu_q, tot * sizeof(double), st) : CAKF_OK;
  double* ms = nullptr;
  double* vs = nullptr;
  if (!rc && !c->ms_dev) {
    if ((rc = c->alloc(c->ms_dev, (size_t)(T + 1) * n * sizeof(double))) == CAKF_OK)
      rc = c->alloc(c->vs_dev, (size_t)(T + 1) * n * sizeof(double));
  }
  if (!rc) {
    ms = c->ms_dev;
    vs = c->vs_dev;
    cudaMemsetAsync(c->err, 0, sizeof(int), st);
    auto run = [&](auto* runner) {
      using R = std::remove_pointer_t<decltype(runner)>;
      typename R::Queries Q;
      Q.at_k.assign(T + 1, {});
      Q.tq.assign(tq, tq + nq);
      for (int q = 0; q < nq; ++q) {
        const double t = tq[q];
        int k = (int)std::floor(t / c->dt + 1e-12);
        k = std::max(0, std::min(k, T));
        Q.at_k[k].push_back(q);
      }
      Q.mu_q = mq;
      Q.fm = buf; Q.fv = buf + tot; Q.sm = buf + 2 * tot; Q.sv = buf + 3 * tot;
      runner->qs = &Q;
      return runner->smooth(ms, vs);
    };
    for (int q = 0; q < nq && !rc; ++q)
      if (!(tq[q] >= 0.0) || !std::isfinite(tq[q])) rc = fail(CAKF_ERR_ARG, "cakf_interpolate: query times must be >= 0");
    if (!rc) {
      if (c->precision == CAKF_FP64) {
        Runner<double> r = make_runner<double>(c, st);
        rc = run(&r);
      } else {
        Runner<float> r = make_runner<float>(c, st);
        rc = run(&r);
      }
    }
  }
  if (!rc) rc = sync_and_check(c, st, "cakf_interpolate");
  double* outs[4] = {fmean, fvar, smean, svar};
  for (int j = 0; j < 4 && !rc; ++j) rc = copy_out(outs[j], buf + j * tot, tot, st);
  if (!rc) {
    cudaError_t ce = cudaStreamSynchronize(st);
    if (ce != cudaSuccess) rc = fail(CAKF_ERR_CUDA, cudaGetErrorString(ce));
  }
  cudaFree(buf);
  if (mq) cudaFree(mq);
  return rc;
}

int cakf_sample(cakf_ctx* c, int32_t n_samples, const double* x0, const double* q, const double* eps,
                double* filter_out, double* smoother_out, void* cuda_stream) {
  if (!c) return fail(CAKF_ERR_STATE, "cakf_sample: no context (cakf_filter creates it)");
  if (!c->filtered) return fail(CAKF_ERR_STATE, "cakf_sample needs a successful cakf_filter on this context");
  if (c->dprime != 1) return fail(CAKF_ERR_ARG, "cakf_sample: Ornstein-Uhlenbeck temporal factor only");
  if (n_samples < 1 || n_samples > 1024 || !x0 || !q || !eps)
    return fail(CAKF_ERR_ARG, "cakf_sample: 1 <= n_samples <= 1024 and x0, q, eps must be given");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const int S = n_samples, n = c->n, T = c->T;
  const size_t blk = (size_t)n * S, tot = (size_t)(T + 1) * blk, Ne = (size_t)c->obs_ptr[T] * S;
  const size_t es = elem_size(c->precision);
  const size_t lS = (size_t)c->ldn * S, mS = (size_t)std::max(c->mmax, 1) * S;
  const size_t work_elems = 5 * lS + 2 * mS;
  const size_t ii = (size_t)std::max(c->imax, 1) * S;
  const size_t small_elems = (size_t)(T + 2) * ii + (size_t)std::max(c->rmax, 1) * S + 2 * ii + 64;
  double *xf = nullptr, *xs = nullptr, *qd = nullptr, *ed = nullptr, *small = nullptr;
  void* work = nullptr;
  auto release = [&]() {
    for (void* p : {(void*)xf, (void*)xs, (void*)qd, (void*)ed, (void*)small, work}) if (p) cudaFree(p);
  };
  if (cudaMalloc(&xf, tot * 8) != cudaSuccess || cudaMalloc(&xs, tot * 8) != cudaSuccess ||
      cudaMalloc(&qd, tot * 8) != cudaSuccess || cudaMalloc(&ed, std::max<size_t>(Ne, 1) * 8) != cudaSuccess ||
      cudaMalloc(&small, small_elems * 8) != cudaSuccess || cudaMalloc(&work, work_elems * es) != cudaSuccess) {
    cudaGetLastError();
    release();
    return fail(CAKF_ERR_OOM, "cakf_sample: workspace allocation failed");
  }
  int rc;
  if ((rc = copy_in(xf, x0, blk * 8, st)) || (rc = copy_in(qd, q, tot * 8, st)) || (rc = copy_in(ed, eps, Ne * 8, st))) {
    release();
    return rc;
  }
  cudaMemsetAsync(c->err, 0, sizeof(int), st);
  if (c->precision == CAKF_FP64) {
    Runner<double> r = make_runner<double>(c, st);
    rc = r.sample(S, xf, xs, qd, ed, (double*)work, work_elems, small, small_elems);
  } else {
    Runner<float> r = make_runner<float>(c, st);
    rc = r.sample(S, xf, xs, qd, ed, (float*)work, work_elems, small, small_elems);
  }
  if (!rc) rc = sync_and_check(c, st, "cakf_sample");
  if (!rc && filter_out) rc = copy_out(filter_out, xf, tot, st);
  if (!rc && smoother_out) rc = copy_out(smoother_out, xs, tot, st);
  if (!rc) {
    cudaError_t ce = cudaStreamSynchronize(st);
    if (ce != cudaSuccess) rc = fail(CAKF_ERR_CUDA, cudaGetErrorString(ce));
  }
  release();
  return rc;
}

int cakf_get_diagnostics(const cakf_ctx* c, int32_t* actions, double* rel_residual, double* min_eta,
                         double* dropped_filter, double* dropped_smoother) {
  if (!c) return fail(CAKF_ERR_STATE, "cakf_get_diagnostics: no context (cakf_filter creates it)");
  if (!c->filtered) return fail(CAKF_ERR_STATE, "cakf_get_diagnostics: no filter run on this context");
  const int T = c->T, B = std::max(c->budget, c->imax);
  std::vector<int> cnt(T + 1);
  std::vector<double> r0(T + 1), rf(T + 1), eta((size_t)(T + 1) * B), df(T + 1), ds(T + 1);
  if (cudaMemcpy(cnt.data(), c->count, (T + 1) * sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(r0.data(), c->r0sq, (T + 1) * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(rf.data(), c->rfin, (T + 1) * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(eta.data(), c->eta, eta.size() * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(df.data(), c->dropped_f, (T + 1) * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(ds.data(), c->dropped_s, (T + 1) * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
    return fail(CAKF_ERR_CUDA, "cakf_get_diagnostics: reading the per-step records");
  for (int k = 0; k <= T; ++k) {
    const int ik = k == 0 ? 0 : cnt[k];
    if (actions) actions[k] = ik;
    if (rel_residual) rel_residual[k] = (ik > 0 && r0[k] > 0) ? std::sqrt(rf[k] / r0[k]) : 0.0;
    if (min_eta) {
      double mn = ik > 0 ? eta[(size_t)k * B] : 0.0;
      for (int j = 1; j < ik; ++j) mn = std::min(mn, eta[(size_t)k * B + j]);
      min_eta[k] = mn;
    }
    if (dropped_filter) dropped_filter[k] = df[k];
    if (dropped_smoother) dropped_smoother[k] = ds[k];
  }
  return CAKF_OK;
}

int cakf_set_wait_limit(int64_t iterations) {
  if (iterations < 0) return fail(CAKF_ERR_ARG, "cakf_set_wait_limit: negative limit");
  cakf::set_wait_limit((long long)iterations);
  return CAKF_OK;
}

int cakf_set_device_memory_limit(uint64_t bytes) {
  g_mem_limit.store(bytes);
  return CAKF_OK;
}

int cakf_get_stats(const cakf_ctx* c, cakf_stats* out) {
  if (!c || !out) return fail(CAKF_ERR_ARG, "NULL argument");
  *out = c->stats;
  out->kernel_launches = (int64_t)(cakf::launch_count() - c->launch_base);
  out->device_bytes = (int64_t)c->dev_bytes;
  return CAKF_OK;
}

int cakf_set_profiling(cakf_ctx* c, int on) {
  if (!c) return fail(CAKF_ERR_ARG, "ctx is NULL");
  c->profiling = on != 0;
  return CAKF_OK;
}

void cakf_free(cakf_ctx* c) { delete c; }

const char* cakf_last_error(void) { return g_err.c_str(); }

}  // extern "C"

// Lets the other translation units of the library report through cakf_last_error.
int cakf::set_last_error(int code, const char* msg) { return fail(code, msg); }

// Scratch of cakf_gram_matmul: kept per thread, grown on demand.
namespace {
struct GramScratch {
  void* coords = nullptr;
  size_t coords_bytes = 0;
  void* stage = nullptr;
  size_t stage_bytes = 0;
  int* err = nullptr;
  ~GramScratch() {
    if (coords) cudaFree(coords);
    if (stage) cudaFree(stage);
    if (err) cudaFree(err);
  }
};
thread_local GramScratch g_gs;

int ensure(void*& p, size_t& have, size_t need) {
  if (have >= need) return CAKF_OK;
  if (p) cudaFree(p);
  p = nullptr;
  have = 0;
  if (cudaMalloc(&p, need) != cudaSuccess) { cudaGetLastError(); return fail(CAKF_ERR_OOM, "scratch allocation failed"); }
  have = need;
  return CAKF_OK;
}
}  // namespace

extern "C" int cakf_gram_matmul(int32_t kernel, double log_lx, double log_sf2, int32_t dim, const double* Xr, int32_t nr,
                                const double* Xc, int32_t nc, const void* B, int32_t ldb, int32_t width, void* Out,
                                int32_t ldo, int32_t precision, void* cuda_stream) {
  if (kernel < 0 || kernel > 2 || dim < 1 || dim > 3 || nr < 1 || nc < 1 || width < 1 || ldb < nc || ldo < nr)
    return fail(CAKF_ERR_ARG, "cakf_gram_matmul: invalid sizes or kernel");
  if (!Xr || !Xc || !B || !Out) return fail(CAKF_ERR_ARG, "cakf_gram_matmul: NULL pointer");
  if (!is_device_ptr(Xr) || !is_device_ptr(Xc) || !is_device_ptr(B) || !is_device_ptr(Out))
    return fail(CAKF_ERR_ARG, "cakf_gram_matmul: all arrays must be device arrays of the current device");
  if (precision < CAKF_FP64 || precision > CAKF_TF32X3)
    return fail(CAKF_ERR_ARG, "cakf_gram_matmul: unknown precision");
  const bool tcp = tc_kind_of(precision) >= 0;
  if (tcp && (width < 2 || width > gram_tc_max_width()))
    return fail(CAKF_ERR_ARG, "cakf_gram_matmul: the tensor-core paths need 2 <= width <= 513");
  if (!std::isfinite(log_lx) || !std::isfinite(log_sf2)) return fail(CAKF_ERR_ARG, "non-finite hyperparameters");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const size_t es = precision == CAKF_FP64 ? 8 : 4;
  const double scale = nu_scale(kernel) / std::exp(log_lx);
  const double sf2 = std::exp(log_sf2);
  int rc;
  if ((rc = ensure(g_gs.coords, g_gs.coords_bytes, (size_t)(nr + nc) * 4 * es + 256))) return rc;
  if (!g_gs.err) {
    if (cudaMalloc(&g_gs.err, sizeof(int)) != cudaSuccess) return fail(CAKF_ERR_OOM, "scratch allocation failed");
  }
  cudaMemsetAsync(g_gs.err, 0, sizeof(int), st);
  if (precision == CAKF_FP64) {
    C4<double>* xr = (C4<double>*)g_gs.coords;
    C4<double>* xc = xr + nr;
    prep_coords<double>(Xr, nr, dim, scale, xr, st);
    prep_coords<double>(Xc, nc, dim, scale, xc, st);
    gram_block_simt<double>(kernel, xr, nr, xc, nc, (const double*)B, ldb, width, sf2, (double*)Out, ldo, st);
  } else {
    C4<float>* xr = (C4<float>*)g_gs.coords;
    C4<float>* xc = xr + nr;
    prep_coords<float>(Xr, nr, dim, scale, xr, st);
    prep_coords<float>(Xc, nc, dim, scale, xc, st);
    if (precision == CAKF_FP32) {
      gram_block_simt<float>(kernel, xr, nr, xc, nc, (const float*)B, ldb, width, (float)sf2, (float*)Out, ldo, st);
    } else {
      const int kind = tc_kind_of(precision);
      if ((rc = ensure(g_gs.stage, g_gs.stage_bytes, gram_tc_staging_bytes(nc, width, kind) + 4096))) return rc;
      const int ldp = (int)gram_tc_packed_ld(nc);
      int r2 = gram_tc_pack_b(kind, (const float*)B, ldb, nc, width, g_gs.stage, ldp, st);
      if (!r2) r2 = gram_block_tc(kernel, kind, xr, nr, xc, nc, g_gs.stage, ldp, width, (float)sf2, (float*)Out, ldo,
                                  g_gs.err, st);
      if (r2) return fail(CAKF_ERR_CUDA, "tensor-core Gram x block launch failed (code " + std::to_string(r2) + ")");
    }
  }
  cudaError_t ce = cudaStreamSynchronize(st);
  if (ce != cudaSuccess) return fail(CAKF_ERR_CUDA, std::string("cakf_gram_matmul: ") + cudaGetErrorString(ce));
  int e = 0;
  cudaMemcpy(&e, g_gs.err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e == kErrTimeout) return fail(CAKF_ERR_TIMEOUT, "cakf_gram_matmul: a device-side wait exceeded its limit");
  if (e) return fail(CAKF_ERR_NUMERIC, "cakf_gram_matmul: numeric error");
  (void)es;
  return CAKF_OK;
}

extern "C" int cakf_factor_gemm(int32_t trans_a, int32_t M, int32_t N, int32_t K, double alpha, const float* A,
                                int32_t lda, const float* B, int32_t ldb, double beta, float* C, int32_t ldc,
                                int32_t precision, void* cuda_stream) {
  if ((trans_a != 0 && trans_a != 1) || M < 1 || N < 1 || K < 0 || ldb < K || ldc < M ||
      lda < (trans_a ? K : M) || !A || !B || !C)
    return fail(CAKF_ERR_ARG, "cakf_factor_gemm: invalid sizes or NULL pointer");
  if (!is_device_ptr(A) || !is_device_ptr(B) || !is_device_ptr(C))
    return fail(CAKF_ERR_ARG, "cakf_factor_gemm: all arrays must be device arrays of the current device");
  if (precision != CAKF_FP32 && tc_kind_of(precision) < 0)
    return fail(CAKF_ERR_ARG, "cakf_factor_gemm: precision must be CAKF_FP32 or a tensor-core mode");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const int mode = precision == CAKF_FP32 ? 1 : 2;
  const size_t part_elems = std::max<size_t>(size_t(1) << 24, (size_t)M * N * 2);
  // workspace kept per thread (grown when needed), like cakf_gram_matmul's scratch
  static thread_local GramScratch ws;
  int rc;
  if ((rc = ensure(ws.stage, ws.stage_bytes, part_elems * sizeof(double) + (size_t)M * N * sizeof(double) + 256)))
    return rc;
  if (!ws.err && cudaMalloc(&ws.err, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    return fail(CAKF_ERR_OOM, "cakf_factor_gemm: workspace allocation failed");
  }
  double* part = reinterpret_cast<double*>(ws.stage);
  double* c64 = part + part_elems;
  int* err = ws.err;
  cudaMemsetAsync(err, 0, sizeof(int), st);
  const int saved = gemm_mode();
  set_gemm_mode(mode);
  set_gemm_err(err);
  if (trans_a) {
    // C = alpha A^T B + beta C through the FP64-output product, converted back to FP32
    convert_to_f64(C, ldc, M, N, c64, M, st);
    gemm_tn<float>(A, lda, M, B, ldb, N, K, alpha, beta, c64, M, part, part_elems, st);
    convert_from_f64<float>(c64, M, M, N, C, ldc, st);
  } else {
    gemm_nn<float, float>(M, N, K, (float)alpha, A, lda, B, ldb, (float)beta, C, ldc, st);
  }
  set_gemm_mode(saved);
  cudaError_t ce = cudaStreamSynchronize(st);
  int e = 0;
  if (ce == cudaSuccess) cudaMemcpy(&e, err, sizeof(int), cudaMemcpyDeviceToHost);
  if (ce != cudaSuccess) return fail(CAKF_ERR_CUDA, std::string("cakf_factor_gemm: ") + cudaGetErrorString(ce));
  if (e == kErrTimeout) return fail(CAKF_ERR_TIMEOUT, "cakf_factor_gemm: a device-side wait exceeded its limit");
  if (e) return fail(CAKF_ERR_NUMERIC, "cakf_factor_gemm: numeric error");
  return CAKF_OK;
}

static int eig_topk_entry(const double* A, int32_t N, int32_t keep, double* w_out, double* U_out, void* cuda_stream,
                          int assembly) {
  if (!A || !w_out || !U_out || N < 1 || keep < 1 || keep > N) return fail(CAKF_ERR_ARG, "cakf_eig_topk: invalid arguments");
  if (!is_device_ptr(A) || !is_device_ptr(w_out) || !is_device_ptr(U_out))
    return fail(CAKF_ERR_ARG, "cakf_eig_topk: all arrays must be device arrays of the current device");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const size_t wb = eig_workspace_bytes(N);
  double* Aw = nullptr;
  void* work = nullptr;
  int* err = nullptr;
  auto release = [&]() { if (Aw) cudaFree(Aw); if (work) cudaFree(work); if (err) cudaFree(err); };
  if (cudaMalloc(&Aw, (size_t)N * N * sizeof(double)) != cudaSuccess || cudaMalloc(&work, wb) != cudaSuccess ||
      cudaMalloc(&err, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    release();
    return fail(CAKF_ERR_OOM, "cakf_eig_topk: workspace allocation failed");
  }
  cudaMemsetAsync(err, 0, sizeof(int), st);
  cudaMemcpyAsync(Aw, A, (size_t)N * N * sizeof(double), cudaMemcpyDeviceToDevice, st);
  int rc = eig_sym_topk<double>(Aw, N, N, keep, w_out, U_out, N, work, wb, err, st, nullptr, assembly);
  cudaError_t ce = cudaStreamSynchronize(st);
  int e = 0;
  if (ce == cudaSuccess) cudaMemcpy(&e, err, sizeof(int), cudaMemcpyDeviceToHost);
  release();
  if (rc) return fail(CAKF_ERR_CUDA, "cakf_eig_topk: eigensolver launch failed (code " + std::to_string(rc) + ")");
  if (ce != cudaSuccess) return fail(CAKF_ERR_CUDA, std::string("cakf_eig_topk: ") + cudaGetErrorString(ce));
  if (e == kErrTimeout) return fail(CAKF_ERR_TIMEOUT, "cakf_eig_topk: a device-side wait exceeded its limit");
  if (e) return fail(CAKF_ERR_NUMERIC, "cakf_eig_topk: numeric error");
  return CAKF_OK;
}

extern "C" int cakf_eig_topk(const double* A, int32_t N, int32_t keep, double* w_out, double* U_out, void* cuda_stream) {
  return eig_topk_entry(A, N, keep, w_out, U_out, cuda_stream, kAssemblyFP64);
}

extern "C" int cakf_eig_topk_mixed(const double* A, int32_t N, int32_t keep, double* w_out, double* U_out,
                                   void* cuda_stream) {
  return eig_topk_entry(A, N, keep, w_out, U_out, cuda_stream, kAssemblyFF);
}

extern "C" int cakf_nll_backward(cakf_ctx* c, double* grad_out) {
  if (!grad_out) return fail(CAKF_ERR_ARG, "cakf_nll_backward: grad_out is NULL");
  if (!c) return fail(CAKF_ERR_STATE, "cakf_nll_backward: no context (cakf_filter creates it)");
  if (!c->filtered) return fail(CAKF_ERR_STATE, "cakf_nll_backward needs a successful cakf_filter on this context");
  if (c->dprime != 1) return fail(CAKF_ERR_ARG, "cakf_nll_backward: Ornstein-Uhlenbeck temporal factor only");
  cudaStream_t st = nullptr;
  int rc;
  const size_t es = elem_size(c->precision);
  const size_t ldn = c->ldn;
  const size_t NP = 4;
  if (!c->dMa) {
    const size_t msz = ldn * std::max(c->rmax, 1) * NP * es;
    const size_t mm = std::max(c->mmax, 1), ii = std::max(c->imax, 1);
    if ((rc = c->alloc(c->dMa, msz))) return rc;
    if ((rc = c->alloc(c->dMb, msz))) return rc;
    if ((rc = c->alloc(c->Eg, NP * ldn * (ii + 1) * es))) return rc;
    if ((rc = c->alloc(c->KS, mm * ii * es))) return rc;
    if ((rc = c->alloc(c->KlS, mm * ii * es))) return rc;
    if ((rc = c->alloc(c->dmo, mm * NP * es))) return rc;
    if ((rc = c->alloc(c->tvec, NP * ldn * es))) return rc;
    if ((rc = c->alloc(c->dmA, NP * c->n * sizeof(double)))) return rc;
    if ((rc = c->alloc(c->dmB, NP * c->n * sizeof(double)))) return rc;
    if ((rc = c->alloc(c->dmpred, NP * c->n * sizeof(double)))) return rc;
    c->gsmall_elems = 24 * ii * ii + 12 * (size_t)std::max(c->rmax, 1) * (ii + 1) + 24 * ii + 1024;
    if ((rc = c->alloc(c->gsmall, c->gsmall_elems * sizeof(double)))) return rc;
    if ((rc = c->alloc(c->grad, 8 * sizeof(double)))) return rc;
  }
  std::vector<int> cnt(c->T + 1, 0);
  cudaMemcpy(cnt.data(), c->count, (c->T + 1) * sizeof(int), cudaMemcpyDeviceToHost);
  cudaMemsetAsync(c->err, 0, sizeof(int), st);
  if (c->precision == CAKF_FP64) {
    Runner<double> r = make_runner<double>(c, st);
    rc = r.nll_grad(cnt);
  } else {
    Runner<float> r = make_runner<float>(c, st);
    rc = r.nll_grad(cnt);
  }
  if (rc) return rc;
  if ((rc = sync_and_check(c, st, "cakf_nll_backward"))) return rc;
  if (cudaMemcpy(grad_out, c->grad, 4 * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
    return fail(CAKF_ERR_CUDA, "reading the gradient");
  for (int p = 0; p < 4; ++p)
    if (!std::isfinite(grad_out[p])) return fail(CAKF_ERR_NUMERIC, "non-finite gradient");
  return CAKF_OK;
}
