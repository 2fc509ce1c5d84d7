"""Thin Python binding of libcakf.so (the C ABI in include/cakf.h).

Argument marshalling only: every step of the filter, smoother and likelihood
runs inside the library's CUDA kernels.  Arrays may be numpy arrays (host) or
torch tensors (host or CUDA); device tensors are passed by pointer.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libcakf.so")

ABI_VERSION = 3
OK, ERR_ARG, ERR_CUDA, ERR_OOM, ERR_NUMERIC, ERR_TIMEOUT, ERR_STATE = range(7)
MATERN12, MATERN32, MATERN52 = 0, 1, 2
TEMPORAL = {"ou": 0, "matern32": 1}
STORE_FP32, STORE_BF16, RECOMPUTE = 0, 1, 2
STORAGE = {"fp32": STORE_FP32, "bf16": STORE_BF16, "recompute": RECOMPUTE}
POLICY_CG, POLICY_COORDINATE, POLICY_BATCH = 0, 1, 2
POLICIES = {"cg": POLICY_CG, "coordinate": POLICY_COORDINATE, "batch": POLICY_BATCH}
FP64, FP32, TF32, BF16, FP16X3, TF32X3 = 0, 1, 2, 3, 4, 5
PRECISIONS = {"fp64": FP64, "fp32": FP32, "tf32": TF32, "bf16": BF16, "fp16x3": FP16X3, "tf32x3": TF32X3}
STATUS = {0: "OK", 1: "ERR_ARG", 2: "ERR_CUDA", 3: "ERR_OOM", 4: "ERR_NUMERIC", 5: "ERR_TIMEOUT", 6: "ERR_STATE"}


class cakf_problem(C.Structure):
    _fields_ = [
        ("abi_version", C.c_int32), ("n", C.c_int32), ("dim", C.c_int32), ("coords", C.c_void_p),
        ("kernel", C.c_int32), ("log_lx", C.c_double), ("log_lt", C.c_double), ("log_sf2", C.c_double),
        ("log_sn2", C.c_double), ("T", C.c_int32), ("dt", C.c_double), ("obs_ptr", C.c_void_p),
        ("obs_idx", C.c_void_p), ("y", C.c_void_p), ("prior_mean", C.c_void_p), ("budget_i", C.c_int32),
        ("rank_r", C.c_int32), ("cg_rtol", C.c_double), ("precision", C.c_int32),
        ("replay_actions", C.c_void_p), ("replay_counts", C.c_void_p), ("factor_storage", C.c_int32),
        ("checkpoint_every", C.c_int32), ("policy", C.c_int32), ("freeze_truncation", C.c_int32),
        ("temporal", C.c_int32),
    ]


class cakf_stats(C.Structure):
    _fields_ = [
        ("filter_ms", C.c_double), ("smooth_ms", C.c_double), ("gram_block_ms", C.c_double),
        ("gram_block_launches", C.c_int64), ("gram_block_flops", C.c_double), ("gram_block_evals", C.c_double),
        ("cg_matvec_ms", C.c_double), ("cg_matvec_launches", C.c_int64), ("cg_matvec_evals", C.c_double),
        ("eig_ms", C.c_double), ("eig_calls", C.c_int64), ("kernel_launches", C.c_int64),
        ("device_bytes", C.c_int64), ("phase_ms", C.c_double * 8), ("eig_phase_ms", C.c_double * 3),
        ("eig_flops", C.c_double * 2),
    ]


class CakfError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


_lib = None


def lib():
    """Load libcakf.so (fails loudly when it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libcakf.so not built ({LIB_PATH}); run paper_2405_08971_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        vp, i32p = C.c_void_p, C.POINTER(C.c_int32)
        L.cakf_filter.argtypes = [C.POINTER(cakf_problem), C.POINTER(vp), vp, vp, vp]
        L.cakf_smooth.argtypes = [vp, vp, vp, vp]
        L.cakf_nll.argtypes = [vp, C.POINTER(C.c_double)]
        L.cakf_nll_backward.argtypes = [vp, C.POINTER(C.c_double)]
        L.cakf_get_actions.argtypes = [vp, vp, i32p]
        L.cakf_get_stats.argtypes = [vp, C.POINTER(cakf_stats)]
        L.cakf_set_profiling.argtypes = [vp, C.c_int]
        L.cakf_gram_matmul.argtypes = [C.c_int32, C.c_double, C.c_double, C.c_int32, vp, C.c_int32, vp, C.c_int32,
                                       vp, C.c_int32, C.c_int32, vp, C.c_int32, C.c_int32, vp]
        L.cakf_gram_matmul.restype = C.c_int
        L.cakf_gram_matmul_noalloc.argtypes = L.cakf_gram_matmul.argtypes
        L.cakf_eig_topk.argtypes = [vp, C.c_int32, C.c_int32, vp, vp, vp]
        L.cakf_eig_topk.restype = C.c_int
        L.cakf_eig_topk_mixed.argtypes = [vp, C.c_int32, C.c_int32, vp, vp, vp]
        L.cakf_eig_topk_mixed.restype = C.c_int
        L.cakf_gram_matmul_noalloc.restype = C.c_int
        L.cakf_factor_gemm.argtypes = [C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_double, vp, C.c_int32, vp,
                                       C.c_int32, C.c_double, vp, C.c_int32, C.c_int32, vp]
        L.cakf_factor_gemm.restype = C.c_int
        L.cakf_probe_peaks.argtypes = [C.POINTER(C.c_double), C.POINTER(C.c_double), vp]
        L.cakf_probe_peaks.restype = C.c_int
        L.cakf_interpolate.argtypes = [vp, C.c_int32, vp, vp, vp, vp, vp, vp, vp]
        L.cakf_interpolate.restype = C.c_int
        L.cakf_sample.argtypes = [vp, C.c_int32, vp, vp, vp, vp, vp, vp]
        L.cakf_sample.restype = C.c_int
        L.cakf_get_diagnostics.argtypes = [vp, vp, vp, vp, vp, vp]
        L.cakf_get_diagnostics.restype = C.c_int
        L.cakf_set_wait_limit.argtypes = [C.c_int64]
        L.cakf_set_wait_limit.restype = C.c_int
        L.cakf_set_device_memory_limit.argtypes = [C.c_uint64]
        L.cakf_set_device_memory_limit.restype = C.c_int
        L.cakf_free.argtypes = [vp]
        L.cakf_free.restype = None
        L.cakf_last_error.restype = C.c_char_p
        for f in ("cakf_filter", "cakf_smooth", "cakf_nll", "cakf_nll_backward", "cakf_get_actions",
                  "cakf_get_stats", "cakf_set_profiling"):
            getattr(L, f).restype = C.c_int
        _lib = L
    return _lib


def _check(code):
    if code != OK:
        raise CakfError(code, lib().cakf_last_error().decode())


def _ptr(x, dtype):
    """(pointer, keepalive) for a numpy array / torch tensor, converting host data as needed."""
    if x is None:
        return None, None
    try:
        import torch
        if isinstance(x, torch.Tensor):
            want = {np.float64: torch.float64, np.int32: torch.int32}[dtype]
            t = x if (x.dtype == want and x.is_contiguous()) else x.to(want).contiguous()
            return t.data_ptr(), t
    except ImportError:
        pass
    a = np.ascontiguousarray(x, dtype=dtype)
    return a.ctypes.data, a


class Context:
    """Owns a cakf_ctx (the stored per-step factors of a filter run)."""

    def __init__(self):
        self.handle = C.c_void_p(None)
        self.T = None
        self.n = None

    def close(self):
        if self.handle:
            lib().cakf_free(self.handle)
            self.handle = C.c_void_p(None)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def make_problem(coords, kernel, log_lx, log_lt, log_sf2, log_sn2, T, dt, obs_ptr, obs_idx, y, budget_i, rank_r,
                 precision="fp32", prior_mean=None, cg_rtol=0.0, replay_actions=None, replay_counts=None,
                 factor_storage="fp32", checkpoint_every=0, policy="cg", freeze_truncation=False, temporal=0):
    """Build a cakf_problem; returns (struct, keepalive list).  temporal: 0 / "ou" (Ornstein-Uhlenbeck)
    or 1 / "matern32" (Matern-3/2 temporal factor, state of values and time derivatives)."""
    keep = []
    p = cakf_problem()
    p.abi_version = ABI_VERSION
    cp, k1 = _ptr(coords, np.float64)
    keep.append(k1)
    shape = tuple(k1.shape) if hasattr(k1, "shape") else None
    p.n = int(shape[0])
    p.dim = int(shape[1]) if len(shape) > 1 else 1
    p.coords = cp
    p.kernel = int(kernel)
    p.log_lx, p.log_lt, p.log_sf2, p.log_sn2 = float(log_lx), float(log_lt), float(log_sf2), float(log_sn2)
    p.T = int(T)
    p.dt = float(dt)
    op = np.ascontiguousarray(obs_ptr, dtype=np.int32)
    keep.append(op)
    p.obs_ptr = op.ctypes.data
    ip, k2 = _ptr(obs_idx, np.int32)
    yp, k3 = _ptr(y, np.float64)
    mp, k4 = _ptr(prior_mean, np.float64)
    keep += [k2, k3, k4]
    p.obs_idx, p.y, p.prior_mean = ip, yp, mp
    p.budget_i, p.rank_r = int(budget_i), int(rank_r)
    p.cg_rtol = float(cg_rtol)
    p.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    p.factor_storage = STORAGE[factor_storage] if isinstance(factor_storage, str) else int(factor_storage)
    p.checkpoint_every = int(checkpoint_every)
    p.policy = POLICIES[policy] if isinstance(policy, str) else int(policy)
    p.freeze_truncation = 1 if freeze_truncation else 0
    p.temporal = TEMPORAL[temporal] if isinstance(temporal, str) else int(temporal)
    if replay_actions is not None:
        ra = np.ascontiguousarray(replay_actions, dtype=np.float64)
        rc = np.ascontiguousarray(replay_counts, dtype=np.int32)
        keep += [ra, rc]
        p.replay_actions, p.replay_counts = ra.ctypes.data, rc.ctypes.data
    return p, keep


def problem_from_workload(w, precision="fp32", cg_rtol=0.0, replay=None, budget_i=None, rank_r=None,
                          factor_storage="fp32", checkpoint_every=0, policy="cg", freeze_truncation=False,
                          temporal=None, **hp):
    """cakf_problem of a `synth.Workload`-like object (any object with the same fields)."""
    ra = rc = None
    if replay is not None:
        ra, rc = replay
    return make_problem(w.coords, w.kernel, hp.get("log_lx", w.log_lx), hp.get("log_lt", w.log_lt),
                        hp.get("log_sf2", w.log_sf2), hp.get("log_sn2", w.log_sn2), w.T, w.dt, w.obs_ptr,
                        w.obs_idx, w.y, w.budget_i if budget_i is None else budget_i,
                        w.rank_r if rank_r is None else rank_r, precision=precision, prior_mean=w.prior_mean,
                        cg_rtol=cg_rtol, replay_actions=ra, replay_counts=rc, factor_storage=factor_storage,
                        checkpoint_every=checkpoint_every, policy=policy, freeze_truncation=freeze_truncation,
                        temporal=getattr(w, "temporal", 0) if temporal is None else temporal)


def _out(arr, shape):
    """Output buffer: numpy (host) or a provided torch tensor / numpy array."""
    if arr is None:
        arr = np.empty(shape, dtype=np.float64)
    try:
        import torch
        if isinstance(arr, torch.Tensor):
            assert arr.dtype == torch.float64 and arr.is_contiguous() and tuple(arr.shape) == shape
            return arr.data_ptr(), arr
    except ImportError:
        pass
    assert arr.dtype == np.float64 and arr.flags.c_contiguous and arr.shape == shape
    return arr.ctypes.data, arr


def cakf_filter(problem, ctx: Optional[Context] = None, mean_out=None, var_out=None, stream=None,
                want_outputs=True):
    """Run the CAKF (Alg. 1).  Returns (ctx, means, variances) with (T+1, n) outputs."""
    p, keep = problem
    ctx = ctx or Context()
    shape = (p.T + 1, p.n)
    mo = vo = None
    mp = vp = None
    if want_outputs:
        mp, mo = _out(mean_out, shape)
        vp, vo = _out(var_out, shape)
    _check(lib().cakf_filter(C.byref(p), C.byref(ctx.handle), mp, vp, stream))
    ctx.T, ctx.n = p.T, p.n
    return ctx, mo, vo


def cakf_smooth(ctx: Context, mean_out=None, var_out=None, stream=None):
    """Run the CAKS (Alg. 3) on the context's filter state.  Returns (means, variances)."""
    if ctx.T is None:   # no filter run: let the library report the state error
        _check(lib().cakf_smooth(ctx.handle, None, None, stream))
    shape = (ctx.T + 1, ctx.n)
    mp, mo = _out(mean_out, shape)
    vp, vo = _out(var_out, shape)
    _check(lib().cakf_smooth(ctx.handle, mp, vp, stream))
    return mo, vo


def cakf_nll(ctx: Context) -> float:
    v = C.c_double()
    _check(lib().cakf_nll(ctx.handle, C.byref(v)))
    return v.value


def cakf_nll_backward(ctx: Context) -> np.ndarray:
    g = (C.c_double * 4)()
    _check(lib().cakf_nll_backward(ctx.handle, g))
    return np.array(list(g))


def cakf_get_actions(ctx: Context, obs_ptr):
    """Actions of the last filter run: (list of per-step m_k x i_k arrays, counts)."""
    counts = np.zeros(ctx.T + 1, dtype=np.int32)
    _check(lib().cakf_get_actions(ctx.handle, None, counts.ctypes.data_as(C.POINTER(C.c_int32))))
    obs_ptr = np.asarray(obs_ptr)
    sizes = [(int(obs_ptr[k] - obs_ptr[k - 1]), int(counts[k])) for k in range(1, ctx.T + 1)]
    flat = np.zeros(sum(a * b for a, b in sizes), dtype=np.float64)
    _check(lib().cakf_get_actions(ctx.handle, flat.ctypes.data, counts.ctypes.data_as(C.POINTER(C.c_int32))))
    out = [np.zeros((0, 0))]
    off = 0
    for m, c in sizes:
        out.append(flat[off:off + m * c].reshape(c, m).T.copy())
        off += m * c
    return out, counts


def pack_actions(S_list, T):
    """Concatenated column-major action blocks + counts, the replay format of cakf_problem."""
    counts = np.zeros(T + 1, dtype=np.int32)
    parts = []
    for k in range(1, T + 1):
        S = np.asarray(S_list[k], dtype=np.float64)
        counts[k] = S.shape[1] if S.ndim == 2 else 0
        if counts[k]:
            parts.append(S.T.ravel())
    flat = np.concatenate(parts) if parts else np.zeros(0)
    return flat, counts


def cakf_get_stats(ctx: Context) -> dict:
    s = cakf_stats()
    _check(lib().cakf_get_stats(ctx.handle, C.byref(s)))
    out = {f: getattr(s, f) for f, _ in cakf_stats._fields_}
    out["phase_ms"] = list(out["phase_ms"])
    out["eig_phase_ms"] = list(out["eig_phase_ms"])
    out["eig_flops"] = list(out["eig_flops"])
    return out


def _gram_args(name, Xr, Xc, B, out, dt):
    """Shape, dtype and device checks shared by the two Gram x matrix wrappers (raise ValueError
    before anything reaches the library): Xr (nr, dim) and Xc (nc, dim) float64 with 1 <= dim <= 3,
    B (width, nc) and out (width, nr) of the precision's element type, all contiguous CUDA tensors
    on the current device.  Returns (nr, nc, dim, width)."""
    import torch
    tensors = (("Xr", Xr, torch.float64), ("Xc", Xc, torch.float64), ("B", B, dt), ("out", out, dt))
    for nm, t, want in tensors:
        if not isinstance(t, torch.Tensor):
            raise ValueError(f"{name}: {nm} must be a torch tensor")
        if t.dtype != want or not t.is_contiguous():
            raise ValueError(f"{name}: {nm} must be a contiguous {want} tensor")
    if Xr.dim() != 2 or Xc.dim() != 2 or B.dim() != 2 or out.dim() != 2:
        raise ValueError(f"{name}: Xr, Xc, B and out must be 2-D")
    nr, dim = Xr.shape
    nc = Xc.shape[0]
    width = B.shape[0]
    if not 1 <= dim <= 3 or Xc.shape[1] != dim:
        raise ValueError(f"{name}: Xr must be (nr, dim) and Xc (nc, dim) with the same dim in 1..3")
    if nr < 1 or nc < 1 or width < 1:
        raise ValueError(f"{name}: empty operand")
    if tuple(B.shape) != (width, nc):
        raise ValueError(f"{name}: B must have shape (width, nc) = ({width}, {nc})")
    if tuple(out.shape) != (width, nr):
        raise ValueError(f"{name}: out must have shape (width, nr) = ({width}, {nr})")
    dev = Xr.device
    if dev.type != "cuda":
        raise ValueError(f"{name}: the operands must be CUDA tensors")
    if dev.index != torch.cuda.current_device():
        raise ValueError(f"{name}: the operands must be on the current CUDA device")
    for nm, t, _ in tensors:
        if t.device != dev:
            raise ValueError(f"{name}: {nm} is on {t.device}, Xr on {dev}")
    return nr, nc, dim, width


def _stream_of(stream, dev):
    """The caller's stream handle, or torch's current stream on dev (so that the call is ordered
    after the work that produced its inputs)."""
    if stream is not None:
        return stream
    import torch
    return torch.cuda.current_stream(dev).cuda_stream


def cakf_gram_matmul(kernel, log_lx, log_sf2, Xr, Xc, B, out=None, precision="fp32", stream=None):
    """Out = K(Xr, Xc) B on the device (torch CUDA tensors; B and Out column-major, i.e. stored as
    (width, rows) row-major tensors).  Xr, Xc are converted to contiguous float64 and B to the
    precision's element type.  Runs on `stream` (a cudaStream_t handle), by default torch's current
    stream.  Returns Out with shape (width, nr)."""
    import torch
    prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    dt = torch.float64 if prec == FP64 else torch.float32
    Xr = Xr.to(torch.float64).contiguous()
    Xc = Xc.to(torch.float64).contiguous()
    B = B.to(dt).contiguous()
    if out is None:
        out = torch.empty((B.shape[0], Xr.shape[0]), dtype=dt, device=Xr.device)
    nr, nc, dim, width = _gram_args("cakf_gram_matmul", Xr, Xc, B, out, dt)
    _check(lib().cakf_gram_matmul(int(kernel), float(log_lx), float(log_sf2), int(dim), Xr.data_ptr(), int(nr),
                                  Xc.data_ptr(), int(nc), B.data_ptr(), int(nc), int(width), out.data_ptr(), int(nr),
                                  prec, _stream_of(stream, Xr.device)))
    return out


def cakf_gram_matmul_noalloc(kernel, log_lx, log_sf2, Xr, Xc, B, out, precision="fp32", stream=None):
    """cakf_gram_matmul into a caller-provided `out`, with no device allocation by the library or
    by this binding: Xr, Xc must be contiguous float64 CUDA tensors of shapes (nr, dim), (nc, dim),
    B and out contiguous CUDA tensors of the precision's element type (float64 for fp64, float32
    otherwise) of shapes (width, nc) and (width, nr) (column-major blocks), all on the current
    device.  Runs on `stream`, by default torch's current stream.  Returns out."""
    import torch
    prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    dt = torch.float64 if prec == FP64 else torch.float32
    nr, nc, dim, width = _gram_args("cakf_gram_matmul_noalloc", Xr, Xc, B, out, dt)
    _check(lib().cakf_gram_matmul_noalloc(int(kernel), float(log_lx), float(log_sf2), int(dim), Xr.data_ptr(),
                                          int(nr), Xc.data_ptr(), int(nc), B.data_ptr(), int(nc), int(width),
                                          out.data_ptr(), int(nr), prec, _stream_of(stream, Xr.device)))
    return out


def cakf_eig_topk(A, keep, stream=None, mixed=False):
    """Top `keep` eigenpairs of the symmetric CUDA float64 tensor A (N x N) through the library's
    FP64 eigensolver.  Returns (w, U): w descending (keep,), U with shape (keep, N) (column-major
    N x keep, i.e. row q of U is the q-th eigenvector).  mixed=True calls cakf_eig_topk_mixed (the
    eigenvector assembly in double-FP32, as the FP32-based modes run it)."""
    import torch
    if A.dtype != torch.float64 or not A.is_cuda:
        raise ValueError("cakf_eig_topk: A must be a CUDA float64 tensor")
    N = A.shape[0]
    if A.dim() != 2 or A.shape[1] != N or not 1 <= int(keep) <= N:
        raise ValueError("cakf_eig_topk: A must be square and 1 <= keep <= N")
    Ac = A.t().contiguous()          # column-major copy (A is symmetric: same values)
    w = torch.empty(keep, dtype=torch.float64, device=A.device)
    U = torch.empty((keep, N), dtype=torch.float64, device=A.device)
    fn = lib().cakf_eig_topk_mixed if mixed else lib().cakf_eig_topk
    _check(fn(Ac.data_ptr(), int(N), int(keep), w.data_ptr(), U.data_ptr(), _stream_of(stream, A.device)))
    return w, U


def cakf_factor_gemm(A, B, C=None, trans_a=False, alpha=1.0, beta=0.0, precision="fp32", stream=None):
    """C = alpha op(A) B + beta C on the device with the library's factor-product kernels.  A, B, C
    are CUDA float32 tensors holding column-major matrices as transposed row-major tensors: A of
    shape (K, M) for op(A) = A (M x K) or (M, K) for op(A) = A^T (A is K x M), B of shape (N, K),
    C of shape (N, M).  Returns C."""
    import torch
    for nm, t in (("A", A), ("B", B)):
        if not isinstance(t, torch.Tensor) or t.dtype != torch.float32 or not t.is_contiguous() or not t.is_cuda:
            raise ValueError(f"cakf_factor_gemm: {nm} must be a contiguous CUDA float32 tensor")
    if trans_a:
        M, K = A.shape
    else:
        K, M = A.shape
    N = B.shape[0]
    if tuple(B.shape) != (N, K):
        raise ValueError("cakf_factor_gemm: B must have shape (N, K)")
    if C is None:
        C = torch.zeros((N, M), dtype=torch.float32, device=A.device)
    if tuple(C.shape) != (N, M) or C.dtype != torch.float32 or not C.is_contiguous():
        raise ValueError("cakf_factor_gemm: C must be a contiguous float32 tensor of shape (N, M)")
    prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    _check(lib().cakf_factor_gemm(1 if trans_a else 0, M, N, K, float(alpha), A.data_ptr(), K if trans_a else M,
                                  B.data_ptr(), K, float(beta), C.data_ptr(), M, prec, _stream_of(stream, A.device)))
    return C


def cakf_probe_peaks(stream=None) -> dict:
    """Measured MUFU (sqrt + exp2 pair) and FP64 FMA throughputs of the current device."""
    mufu, fp64 = C.c_double(), C.c_double()
    _check(lib().cakf_probe_peaks(C.byref(mufu), C.byref(fp64), stream))
    return {"mufu_ops_per_s": mufu.value, "fp64_flops_per_s": fp64.value}


def cakf_interpolate(ctx: Context, tq, mu_q=None, stream=None):
    """Filter and smoother marginals at the query times tq (host): returns (filter means, filter
    variances, smoother means, smoother variances), each (len(tq), n)."""
    tq = np.ascontiguousarray(tq, dtype=np.float64)
    nq, n = tq.size, ctx.n
    outs = [np.empty((nq, n)) for _ in range(4)]
    mq = None if mu_q is None else np.ascontiguousarray(mu_q, dtype=np.float64)
    _check(lib().cakf_interpolate(ctx.handle, nq, tq.ctypes.data, None if mq is None else mq.ctypes.data,
                                  *[o.ctypes.data for o in outs], stream))
    return tuple(outs)


def cakf_sample(ctx: Context, x0, q, eps, obs_ptr, stream=None):
    """Posterior draws with the context's filter factors.  x0: (n, S); q: list of T+1 arrays (n, S)
    (entry 0 unused); eps: list of T+1 arrays (m_k, S) (entry 0 unused).  Returns (filter draws,
    smoother draws), each (T+1, n, S) numpy arrays."""
    n, T = ctx.n, ctx.T
    x0 = np.asarray(x0, dtype=np.float64)
    S = x0.shape[1]
    x0c = np.ascontiguousarray(x0.T)                                        # (S, n): column s at s*n
    qc = np.ascontiguousarray(np.stack([np.zeros((S, n))] + [np.asarray(q[k]).T for k in range(1, T + 1)]))
    ec = np.ascontiguousarray(np.concatenate([np.asarray(eps[k], dtype=np.float64).T.ravel()
                                              for k in range(1, T + 1)] or [np.zeros(0)]))
    fo = np.empty((T + 1, S, n))
    so = np.empty((T + 1, S, n))
    _check(lib().cakf_sample(ctx.handle, S, x0c.ctypes.data, qc.ctypes.data, ec.ctypes.data, fo.ctypes.data,
                             so.ctypes.data, stream))
    return fo.transpose(0, 2, 1), so.transpose(0, 2, 1)


def cakf_get_diagnostics(ctx: Context) -> dict:
    """Per-step records of the last run: actions used, relative final residual, smallest eta,
    discarded truncation mass of the filter and of the smoother (arrays of T+1 entries)."""
    T = ctx.T if ctx.T is not None else 0
    acts = np.zeros(T + 1, dtype=np.int32)
    arrs = [np.zeros(T + 1) for _ in range(4)]
    _check(lib().cakf_get_diagnostics(ctx.handle, acts.ctypes.data, *[a.ctypes.data for a in arrs]))
    return {"actions": acts, "rel_residual": arrs[0], "min_eta": arrs[1], "dropped_filter": arrs[2],
            "dropped_smoother": arrs[3]}


def cakf_set_wait_limit(iterations: int):
    _check(lib().cakf_set_wait_limit(int(iterations)))


def cakf_set_device_memory_limit(nbytes: int):
    _check(lib().cakf_set_device_memory_limit(int(nbytes)))


def cakf_set_profiling(ctx: Context, on: bool):
    _check(lib().cakf_set_profiling(ctx.handle, 1 if on else 0))
