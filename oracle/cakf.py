"""Plain FP64 reference of the computation-aware Kalman filter (CAKF) and smoother (CAKS).

TEST INFRASTRUCTURE ONLY -- the oracle.  Slow, literal, numpy float64.  Only
`tests/`, `__graft_entry__.smoke()` and `bench.py`'s CPU-baseline legs use it.
It shares no code with the CUDA path.

What it follows (arXiv 2405.08971, "Computation-Aware Kalman Filtering and
Smoothing"):

* Model: the space-time separable Gauss-Markov lemma (appendix, "Space-time
  separable Gauss-Markov processes"): A = A^t (x) I, Q = Q^t (x) K.  With an
  Ornstein-Uhlenbeck temporal factor (D'=1) this is A = a I, Q = (1-a^2) K,
  a = exp(-dt/l_t), and the stationary prior covariance Sigma_k = K for all k.
  A known prior mean mu_k enters as b_{k-1} = mu_k - a mu_{k-1}.  With a
  Matern-3/2 temporal factor (D'=2; the remark after the lemma: Matern(p + 1/2)
  kernels have a state-space form) the state is (f, df/dt) at every grid point,
  A^t = expm(F dt), Sigma = P^t_inf (x) K and Q^t = P^t_inf - A^t P^t_inf A^t^T.
* Filter: Alg. 1 (CAKF) with the iterative update step (appendix algorithm
  "CAKF Update Step (Iterative Version)"), CG policy = the current residual
  (Sec. 3.3).  Predict / update in downdate form (Prop. "Downdate-form Kalman
  filter"): P^- = Sigma - M^- M^-T, M = (M^-, P^- W).
* Truncate: Sec. 3.2 -- keep the top-r eigen-directions of M M^T (computed from
  the small Gram M^T M, same eigenvectors up to the map u -> M u).
* Smoother: Alg. 3 (CAKS), the inverse-free RTS recursion in downdate form
  (Prop. "Inverse-free RTS smoother").
* Block policies: the batch update (Alg. 2, "CAKF Update Step"): the actions S are chosen once
  per step, Ghat = S^T (H P^- H^T + R) S, W = H^T S lsqrt(Ghat^+), w = H^T S Ghat^+ S^T (y - H m^-),
  with coordinate actions (unit vectors at a space-filling subset of the observations) or given
  actions (e.g. Gaussian sketches drawn by the caller) -- the policy appendix.
* Posterior sampler: the CAKF/CAKS sampler algorithm of the appendix (Matheron's rule in the
  modified model, inverse-free smoother form): given a prior draw x_0, dynamics noise q_{k-1} and
  observation noise eps_k, x^-_k = A x_{k-1} + b + q, w_k = H^T V_k V_k^T (y_k - H x^-_k - eps_k),
  x_k = x^-_k + P^-_k w_k, then ws_k = w_k + (I - W_k W_k^T P^-_k) A^T ws_{k+1} and
  x^s_k = x_k + P_k A^T ws_{k+1}.  The projected noise S^T eps has the law the algorithm draws
  (N(0, S^T R S)), so the draw is made in observation space.
* NLL: not in the paper (named as future work at the end of the conclusion).
  Defined here as the negative log density of the projected data S_k^T y_k
  under the modified observation model (eq. proj-observation), in Euclidean-
  normalised coordinates:
      nll_k = 1/2 logdet(2 pi S^T G S) + 1/2 (S^T r0)^T (S^T G S)^{-1} (S^T r0)
              - 1/2 logdet(S^T S),
  G = H P^- H^T + sigma_n^2 I, r0 = y - H m^-.  At full budget it is the exact
  Kalman-filter NLL term.
* Gradient: central finite differences of the NLL with the actions S_k and the
  truncation rotations U_k frozen (exact inference in a fixed modified model).

Readings taken where the paper is ambiguous, garbled or silent:
  R1 residual/action order in the iterative update: per iteration
     r = r0 - G v; s = r; alpha = s^T r; d = (I - V V^T G) s; eta = s^T G d;
     v += (alpha/eta) d; V <- (V, d/sqrt(eta)).
  R2 stopping: i = min(budget, m_k); stop early if cg_rtol > 0 and
     ||r|| <= cg_rtol ||r0||, or on breakdown (eta not finite, or
     eta <= 1e-12 * s^T G s).
  R4 truncation by eig of M^T M, descending; no truncation when #cols <= r.
  R5 smoother truncation: same rank r, Euclidean eig of Ws^T Ws.
  R6 the smoother uses the untruncated filter factor M_k (filter covariance
     P_k = K - M_k M_k^T) and the predicted P^-_k = K - a^2 M+_{k-1} M+_{k-1}^T.
  R7 smoother loop k = T-1 .. 0 with w_0 = 0, W_0 empty.
  R9 Matern kernels in the Rasmussen-Williams form, output scale = variance.
  R20 Matern-3/2 temporal factor: the state stacks the positions above the velocities; the
     temporal factor has unit variance (sigma_f^2 stays in K); a prior mean mu_k of the
     positions enters as the state mean (mu_k, 0) -- the model is the zero-mean Matern process
     of the deviation f - mu, so b_{k-1} = (mu_k, 0) - A (mu_{k-1}, 0); H observes positions.
  R18 coordinate policy: the space-filling subset is read as i observations evenly spaced through
     the step's observation list (sorted grid indices, i.e. raster order of the grid): positions
     floor((q + 1/2) m_k / i), q = 0..i-1; the left square root of Ghat^+ is L^-T with
     L L^T = Ghat (Cholesky; Ghat is positive definite for distinct coordinates and noise > 0).
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

MATERN12, MATERN32, MATERN52 = 0, 1, 2
_BLOCK_BYTES = 256 << 20


# ----------------------------------------------------------------------------- kernel
def matern(u: np.ndarray, kernel: int) -> np.ndarray:
    """Unit-variance Matern correlation of the scaled distance u = d / l (R9)."""
    if kernel == MATERN12:
        return np.exp(-u)
    if kernel == MATERN32:
        s = math.sqrt(3.0) * u
        return (1.0 + s) * np.exp(-s)
    if kernel == MATERN52:
        s = math.sqrt(5.0) * u
        return (1.0 + s + s * s / 3.0) * np.exp(-s)
    raise ValueError(f"unknown kernel {kernel}")


def kernel_matrix(Xa: np.ndarray, Xb: np.ndarray, kernel: int, lx: float, sf2: float) -> np.ndarray:
    """Dense Gram matrix sigma_f^2 k(|x_a - x_b| / l_x) between two coordinate sets."""
    diff = Xa[:, None, :] - Xb[None, :, :]
    d = np.sqrt(np.sum(diff * diff, axis=-1))
    return sf2 * matern(d / lx, kernel)


@dataclasses.dataclass
class Model:
    """Separable state-space model on a fixed grid (appendix lemma on STSGMPs): A = A^t (x) I_n,
    Q = Q^t (x) K, stationary prior covariance Sigma = P^t_inf (x) K.

    temporal 0: Ornstein-Uhlenbeck factor (D' = 1): A^t = a = exp(-dt/l_t), P^t_inf = 1.
    temporal 1: Matern-3/2 factor (D' = 2, state (f, df/dt) stacked as [positions; velocities]):
      the SDE dx = F x dt + L dW with F = [[0, 1], [-lam^2, -2 lam]], lam = sqrt(3)/l_t, whose
      stationary covariance is P^t_inf = diag(1, lam^2) (unit temporal variance; sigma_f^2 sits in K);
      A^t = expm(F dt) and Q^t = P^t_inf - A^t P^t_inf A^t^T (Lemma: Sigma_{k+1} = A Sigma_k A^T + Q).
    """
    X: np.ndarray
    kernel: int
    lx: float
    sf2: float
    a: float
    sn2: float
    mu: Optional[np.ndarray]   # (T+1, n) prior mean of the positions, or None
    temporal: int = 0
    At: Optional[np.ndarray] = None     # (D', D') temporal transition over one step
    Pinf: Optional[np.ndarray] = None   # (D', D') stationary temporal covariance

    def __post_init__(self):
        if self.At is None:
            self.At = np.array([[self.a]])
            self.Pinf = np.array([[1.0]])

    @property
    def n(self):
        return self.X.shape[0]

    @property
    def dprime(self):
        return self.At.shape[0]

    @property
    def D(self):
        """State dimension n D'."""
        return self.n * self.dprime

    def K_times(self, B: np.ndarray, rows: Optional[np.ndarray] = None,
                cols: Optional[np.ndarray] = None) -> np.ndarray:
        """K(X[rows], X[cols]) @ B without holding the full Gram matrix (row blocks)."""
        Xr = self.X if rows is None else self.X[rows]
        Xc = self.X if cols is None else self.X[cols]
        B2 = B.reshape(B.shape[0], -1)
        out = np.empty((Xr.shape[0], B2.shape[1]))
        step = max(1, _BLOCK_BYTES // (8 * max(1, Xc.shape[0]) * (2 + Xc.shape[1])))
        for lo in range(0, Xr.shape[0], step):
            hi = min(lo + step, Xr.shape[0])
            out[lo:hi] = kernel_matrix(Xr[lo:hi], Xc, self.kernel, self.lx, self.sf2) @ B2
        return out.reshape((Xr.shape[0],) + B.shape[1:])

    def _blocks(self, B):
        n = self.n
        return [B[q * n:(q + 1) * n] for q in range(self.dprime)]

    def _kron_times(self, C: np.ndarray, B: np.ndarray) -> np.ndarray:
        """(C (x) I_n) B for a D' x D' matrix C and a D-row B."""
        Bq = self._blocks(B)
        return np.concatenate([sum(C[p, q] * Bq[q] for q in range(self.dprime)) for p in range(self.dprime)],
                              axis=0)

    def A_times(self, B: np.ndarray) -> np.ndarray:
        return self._kron_times(self.At, B)

    def AT_times(self, B: np.ndarray) -> np.ndarray:
        return self._kron_times(self.At.T, B)

    def sigma_times(self, B: np.ndarray) -> np.ndarray:
        """Sigma B = (P^t_inf (x) K) B."""
        KB = [self.K_times(Bq) for Bq in self._blocks(B)]
        return np.concatenate([sum(self.Pinf[p, q] * KB[q] for q in range(self.dprime)) for p in range(self.dprime)],
                              axis=0)

    def sigma_Ht_times(self, V: np.ndarray, obs: np.ndarray) -> np.ndarray:
        """Sigma H^T V with H selecting the positions obs: blocks P^t_inf[p, 0] K(X, X_obs) V."""
        KV = self.K_times(V, cols=obs)
        return np.concatenate([self.Pinf[p, 0] * KV for p in range(self.dprime)], axis=0)

    def H_sigma_Ht(self, obs: np.ndarray) -> np.ndarray:
        """H Sigma H^T = P^t_inf[0, 0] K(X_obs, X_obs)."""
        return self.Pinf[0, 0] * self.K_times(np.eye(len(obs)), rows=obs, cols=obs)

    def prior_var(self) -> np.ndarray:
        """diag(Sigma) (D)."""
        return np.concatenate([np.full(self.n, self.Pinf[p, p] * self.sf2) for p in range(self.dprime)])

    def _mean_state(self, k: int) -> np.ndarray:
        """Prior mean of the state at step k: the position mean mu_k, zero velocities (reading R20)."""
        out = np.zeros(self.D)
        if self.mu is not None:
            out[:self.n] = self.mu[k]
        return out

    def b(self, k: int) -> np.ndarray:
        """Dynamics offset b_{k-1} so that the prior mean at step k is mu_k."""
        return self._mean_state(k) - self.A_times(self._mean_state(k - 1))

    def m0(self) -> np.ndarray:
        return self._mean_state(0)


def matern32_temporal(lt: float, dt: float):
    """(A^t, P^t_inf) of the Matern-3/2 temporal factor over a step dt.  F + lam I is nilpotent
    ((F + lam I)^2 = 0), so expm(F dt) = exp(-lam dt) (I + dt (F + lam I))."""
    lam = math.sqrt(3.0) / lt
    F = np.array([[0.0, 1.0], [-lam * lam, -2.0 * lam]])
    At = math.exp(-lam * dt) * (np.eye(2) + dt * (F + lam * np.eye(2)))
    return At, np.diag([1.0, lam * lam])


def model_from(w, log_lx=None, log_lt=None, log_sf2=None, log_sn2=None) -> Model:
    """Model of a `synth.Workload` (hyperparameters optionally overridden, in log space)."""
    lx = math.exp(w.log_lx if log_lx is None else log_lx)
    lt = math.exp(w.log_lt if log_lt is None else log_lt)
    sf2 = math.exp(w.log_sf2 if log_sf2 is None else log_sf2)
    sn2 = math.exp(w.log_sn2 if log_sn2 is None else log_sn2)
    temporal = int(getattr(w, "temporal", 0))
    At = Pinf = None
    if temporal == 1:
        At, Pinf = matern32_temporal(lt, w.dt)
    elif temporal != 0:
        raise ValueError(f"unknown temporal factor {temporal}")
    return Model(X=np.asarray(w.coords, dtype=np.float64), kernel=w.kernel, lx=lx, sf2=sf2,
                 a=math.exp(-w.dt / lt), sn2=sn2, mu=w.prior_mean, temporal=temporal, At=At, Pinf=Pinf)


# ----------------------------------------------------------------------------- truncation
def truncate(M: np.ndarray, r: int):
    """Truncate (Sec. 3.2): M M^T = M+ M+^T + N N^T keeping the top-r eigen-directions.

    Returns (M_plus, U_r or None, eigenvalues kept, eigenvalues dropped).  U_r
    holds the eigenvectors of M^T M for the r largest eigenvalues (descending),
    so M+ = M U_r.  No truncation when r <= 0 or #cols <= r (R4)."""
    if r <= 0 or M.shape[1] <= r:
        return M, None, None, None
    lam, U = np.linalg.eigh(M.T @ M)
    order = np.argsort(lam)[::-1]
    lam, U = lam[order], U[:, order]
    return M @ U[:, :r], U[:, :r], lam[:r], lam[r:]


# ----------------------------------------------------------------------------- filter
@dataclasses.dataclass
class FilterResult:
    m: np.ndarray                 # (T+1, D) filter means (D = n D' state dimension)
    var: np.ndarray               # (T+1, D) filter marginal variances (pre-truncation)
    M_hat: List[np.ndarray]       # updated factor per step (untruncated); [0] is D x 0
    M_pred: List[np.ndarray]      # predictive factor A M+_{k-1} per step; [0] is D x 0
    w: List[np.ndarray]           # filter message w_k = H^T v (dense D-vector); [0] zeros
    W: List[np.ndarray]           # filter message W_k = H^T V (dense D x j); [0] empty
    S: List[np.ndarray]           # actions per step (m_k x j)
    U: List[Optional[np.ndarray]] # truncation rotations per step (None: not truncated)
    nll: np.ndarray               # (T+1,) per-step NLL terms, [0] = 0
    iters: np.ndarray             # (T+1,) actions used per step
    dropped: np.ndarray           # (T+1,) discarded truncation mass sum(dropped eigenvalues)
    G: List[Optional[np.ndarray]] # dense projected innovation Grams (kept for tests)
    r0: List[Optional[np.ndarray]]


def update_iterative(model: Model, m_pred, M_pred, obs, y, budget, cg_rtol=0.0, S_replay=None):
    """CAKF update step, iterative version (appendix algorithm, reading R1/R2).

    Forms G = H P^- H^T + sigma_n^2 I densely (m x m; this is the oracle) and
    runs the G-orthogonalised projected update with CG actions s = current
    residual.  Returns (m, M_hat, w, W, S, V, G, r0)."""
    D = model.D
    mo = len(obs)
    Ko = model.H_sigma_Ht(obs)
    Mo = M_pred[obs]                                  # H M^-: the positions come first in the state
    G = Ko - Mo @ Mo.T + model.sn2 * np.eye(mo)
    r0 = y - m_pred[obs]
    v = np.zeros(mo)
    V = np.zeros((mo, 0))
    S = []
    nmax = min(budget, mo) if S_replay is None else S_replay.shape[1]
    r0n = np.linalg.norm(r0)
    for it in range(nmax):
        r = r0 - G @ v
        if S_replay is None and cg_rtol > 0 and np.linalg.norm(r) <= cg_rtol * r0n:
            break
        s = r if S_replay is None else S_replay[:, it]
        alpha = s @ r
        Gs = G @ s
        d = s - V @ (V.T @ Gs)
        eta = s @ (G @ d)
        if not np.isfinite(eta) or eta <= 1e-12 * (s @ Gs):
            break
        v = v + (alpha / eta) * d
        V = np.concatenate([V, (d / math.sqrt(eta))[:, None]], axis=1)
        S.append(s)
    S = np.stack(S, axis=1) if S else np.zeros((mo, 0))
    # w = H^T v, W = H^T V; P^- [W w] = Sigma H^T [V v] - M^- (M_o^T [V v])
    Vv = np.concatenate([V, v[:, None]], axis=1)
    PVv = model.sigma_Ht_times(Vv, obs) - M_pred @ (Mo.T @ Vv)
    m_new = m_pred + PVv[:, -1]
    M_hat = np.concatenate([M_pred, PVv[:, :-1]], axis=1)
    w = np.zeros(D)
    w[obs] = v
    W = np.zeros((D, V.shape[1]))
    W[obs] = V
    return m_new, M_hat, w, W, S, V, G, r0


def coordinate_actions(m: int, i: int) -> np.ndarray:
    """Coordinate policy (policy appendix, reading R18): m x i unit vectors at observation positions
    floor((q + 1/2) m / i), q = 0..i-1 (i <= m)."""
    i = min(i, m)
    S = np.zeros((m, i))
    for q in range(i):
        S[int((q + 0.5) * m / i), q] = 1.0
    return S


def update_batch(model: Model, m_pred, M_pred, obs, y, S):
    """CAKF update step, batch version (Alg. 2) with the actions S (m x i) chosen up front.

    Ghat = S^T G S with G = H P^- H^T + sigma_n^2 I (dense here), W = H^T S L^-T (L L^T = Ghat),
    w = H^T S Ghat^-1 S^T r0.  Returns the same tuple as update_iterative."""
    D = model.D
    mo = len(obs)
    Ko = model.H_sigma_Ht(obs)
    Mo = M_pred[obs]
    G = Ko - Mo @ Mo.T + model.sn2 * np.eye(mo)
    r0 = y - m_pred[obs]
    Gh = S.T @ G @ S
    L = np.linalg.cholesky(Gh)
    V = np.linalg.solve(L, S.T).T                     # S L^-T: lsqrt of Ghat^+ applied to S
    v = S @ np.linalg.solve(Gh, S.T @ r0)
    Vv = np.concatenate([V, v[:, None]], axis=1)
    PVv = model.sigma_Ht_times(Vv, obs) - M_pred @ (Mo.T @ Vv)
    m_new = m_pred + PVv[:, -1]
    M_hat = np.concatenate([M_pred, PVv[:, :-1]], axis=1)
    w = np.zeros(D)
    w[obs] = v
    W = np.zeros((D, V.shape[1]))
    W[obs] = V
    return m_new, M_hat, w, W, S, V, G, r0


def _nll_step(G, S, r0):
    """Per-step NLL of the projected data (definition in the module docstring)."""
    j = S.shape[1]
    if j == 0:
        return 0.0
    Gh = S.T @ G @ S
    yh = S.T @ r0
    L = np.linalg.cholesky(Gh)
    Ls = np.linalg.cholesky(S.T @ S)
    z = np.linalg.solve(L, yh)
    return (0.5 * j * math.log(2 * math.pi) + np.sum(np.log(np.diag(L))) + 0.5 * z @ z
            - np.sum(np.log(np.diag(Ls))))


def filter_run(w, model: Optional[Model] = None, budget=None, rank_r=None, cg_rtol=0.0,
               S_replay=None, U_replay=None, keep_G=False, policy="cg", S_given=None) -> FilterResult:
    """Alg. 1 (CAKF) over steps k = 1..T of a `synth.Workload`.

    policy "cg": iterative update with CG actions (or S_replay); "coordinate": batch update (Alg. 2)
    with coordinate actions; "given": batch update with the actions S_given[k] (m_k x i_k)."""
    model = model or model_from(w)
    budget = w.budget_i if budget is None else budget
    rank_r = w.rank_r if rank_r is None else rank_r
    D, T = model.D, w.T
    pvar = model.prior_var()
    m = np.zeros((T + 1, D))
    var = np.zeros((T + 1, D))
    m[0] = model.m0()
    var[0] = pvar
    Mplus = np.zeros((D, 0))
    res = FilterResult(m=m, var=var, M_hat=[Mplus], M_pred=[Mplus], w=[np.zeros(D)],
                       W=[np.zeros((D, 0))], S=[np.zeros((0, 0))], U=[None], nll=np.zeros(T + 1),
                       iters=np.zeros(T + 1, dtype=np.int64), dropped=np.zeros(T + 1), G=[None], r0=[None])
    for k in range(1, T + 1):
        # predict (Alg. 1): m^- = A m + b, M^- = A M+
        m_pred = model.A_times(m[k - 1]) + model.b(k)
        M_pred = model.A_times(Mplus)
        obs = w.obs(k)
        if len(obs) == 0:   # IsMissing
            m_new, M_hat = m_pred, M_pred
            wk, Wk, S, G, r0 = np.zeros(D), np.zeros((D, 0)), np.zeros((0, 0)), None, None
        else:
            if policy == "cg":
                Srep = None if S_replay is None else S_replay[k]
                m_new, M_hat, wk, Wk, S, V, G, r0 = update_iterative(
                    model, m_pred, M_pred, obs, w.yk(k), budget, cg_rtol, Srep)
            else:
                Sb = coordinate_actions(len(obs), budget) if policy == "coordinate" else S_given[k]
                m_new, M_hat, wk, Wk, S, V, G, r0 = update_batch(model, m_pred, M_pred, obs, w.yk(k), Sb)
            res.nll[k] = _nll_step(G, S, r0)
        m[k] = m_new
        var[k] = pvar - np.sum(M_hat * M_hat, axis=1)
        if U_replay is not None:   # frozen truncation: None = the base run kept the factor
            U, lam_drop = U_replay[k], None
            Mplus = M_hat if U is None else M_hat @ U
        else:
            Mplus, U, _, lam_drop = truncate(M_hat, rank_r)
        res.M_hat.append(M_hat)
        res.M_pred.append(M_pred)
        res.w.append(wk)
        res.W.append(Wk)
        res.S.append(S)
        res.U.append(U)
        res.iters[k] = S.shape[1]
        res.dropped[k] = 0.0 if lam_drop is None else float(np.sum(lam_drop))
        res.G.append(G if keep_G else None)
        res.r0.append(r0 if keep_G else None)
    return res


# ----------------------------------------------------------------------------- smoother
def smoother_run(w, filt: FilterResult, model: Optional[Model] = None, rank_r=None, U_replay=None):
    """Alg. 3 (CAKS): backward pass k = T-1 .. 0 (readings R5-R7).

    Returns (means, variances, per-step smoother truncation rotations)."""
    model = model or model_from(w)
    rank_r = w.rank_r if rank_r is None else rank_r
    T, D = w.T, model.D
    ms = np.zeros((T + 1, D))
    vs = np.zeros((T + 1, D))
    ms[T] = filt.m[T]
    vs[T] = filt.var[T]
    ws = filt.w[T]
    Ws = filt.W[T]
    Us: List[Optional[np.ndarray]] = [None] * (T + 1)
    for k in range(T - 1, -1, -1):
        X = model.AT_times(np.concatenate([Ws, ws[:, None]], axis=1))   # A^T [Ws ws]
        Mk = filt.M_hat[k]
        SX = model.sigma_times(X)
        PX = SX - Mk @ (Mk.T @ X)                                    # P_k A^T [Ws ws]
        ms[k] = filt.m[k] + PX[:, -1]
        E = PX[:, :-1]
        vs[k] = filt.var[k] - np.sum(E * E, axis=1)                 # M^s_k = (M_k, P_k A^T Ws)
        if k == 0:
            break
        Mp = filt.M_pred[k]
        PmX = SX - Mp @ (Mp.T @ X)                                   # P^-_k A^T [Ws ws]
        Wk = filt.W[k]
        Y2 = X - Wk @ (Wk.T @ PmX)                                   # (I - W W^T P^-) A^T [Ws ws]
        ws = filt.w[k] + Y2[:, -1]
        Wfull = np.concatenate([Wk, Y2[:, :-1]], axis=1)
        if U_replay is not None:
            Us[k] = U_replay[k]
            Ws = Wfull if Us[k] is None else Wfull @ Us[k]
        else:
            Ws, Us[k], _, _ = truncate(Wfull, rank_r)
    return ms, vs, Us


# ----------------------------------------------------------------------------- posterior sampler
def sample_run(w, filt: FilterResult, x0, q, eps, model: Optional[Model] = None):
    """The CAKF/CAKS sampler (appendix algorithm) for S draws at once, with the filter's actions,
    factors and G-orthonormal directions V_k = W_k[obs] of `filt`.

    x0 (n, S) initial draw; q[k] (n, S) dynamics noise of the transition into step k; eps[k] (m_k, S)
    observation noise.  Per step: x^-_k = a x_{k-1} + b_{k-1} + q[k];
    w_k = H^T V_k V_k^T (y_k - H x^-_k - eps_k)  (= W_k lsqrt(Ghat)^T (S^T y - S^T H x^- - S^T eps));
    x_k = x^-_k + P^-_k w_k.  Smoother: ws_T = w_T; for k = T-1..0:
    x^s_k = x_k + P_k (a ws_{k+1}); ws_k = w_k + a ws_{k+1} - W_k W_k^T P^-_k (a ws_{k+1}).
    Returns (filter draws (T+1, n, S), smoother draws (T+1, n, S))."""
    model = model or model_from(w)
    if model.dprime != 1:
        raise NotImplementedError("sample_run: Ornstein-Uhlenbeck temporal factor only")
    T, n, a = w.T, model.n, model.a
    S = x0.shape[1]
    xf = np.zeros((T + 1, n, S))
    wk_all = [np.zeros((n, S))]
    xf[0] = x0
    for k in range(1, T + 1):
        xp = a * xf[k - 1] + model.b(k)[:, None] + q[k]
        obs = w.obs(k)
        Mp = filt.M_pred[k]
        if len(obs) == 0 or filt.W[k].shape[1] == 0:
            xf[k] = xp
            wk_all.append(np.zeros((n, S)))
            continue
        V = filt.W[k][obs]
        c = V.T @ (w.yk(k)[:, None] - xp[obs] - eps[k])
        wk = np.zeros((n, S))
        wk[obs] = V @ c
        Pw = model.K_times(wk) - Mp @ (Mp.T @ wk)                  # P^-_k w_k
        xf[k] = xp + Pw
        wk_all.append(wk)
    xs = np.zeros_like(xf)
    xs[T] = xf[T]
    ws = wk_all[T]
    for k in range(T - 1, -1, -1):
        t = a * ws
        Mh = filt.M_hat[k]
        xs[k] = xf[k] + model.K_times(t) - Mh @ (Mh.T @ t)       # x_k + P_k A^T ws_{k+1}
        if k == 0:
            break
        Mp = filt.M_pred[k]
        Pt = model.K_times(t) - Mp @ (Mp.T @ t)                   # P^-_k A^T ws_{k+1}
        Wk = filt.W[k]
        ws = wk_all[k] + t - Wk @ (Wk.T @ Pt)
    return xf, xs


# ----------------------------------------------------------------------------- temporal interpolation
def interpolate_run(w, filt: FilterResult, smooth_W, smooth_w, tq, mu_q=None, model: Optional[Model] = None):
    """Filter and smoother marginals at query times between the steps (the interpolation corollary of
    the appendix, in downdate form), for the OU prior A(t, s) = exp(-(t - s)/l_t) I.

    For t_k <= t < t_{k+1} (t_k = k dt; k = T for t >= t_T): a_tau = A(t, t_k),
      filter:   m(t) = a_tau m_k + b(t, t_k),  P(t) = K - a_tau^2 M_k M_k^T  (M_k the updated factor),
      smoother: m^s(t) = m(t) + P(t) A(t_{k+1}, t)^T ws_{k+1},
                P^s(t) = P(t) - P(t) A^T Ws_{k+1} (P(t) A^T Ws_{k+1})^T   (t < t_T; else = filter),
    with b(t, t_k) = mu(t) - a_tau mu_k (mu_q[q] the prior mean at tq[q], or zero).  smooth_W[k],
    smooth_w[k] are the smoother messages Ws_k, ws_k of Alg. 3 (smoother_messages).
    Returns (filter means, filter variances, smoother means, smoother variances), each (len(tq), n)."""
    model = model or model_from(w)
    if model.dprime != 1:
        raise NotImplementedError("interpolate_run: Ornstein-Uhlenbeck temporal factor only")
    T, n = w.T, model.n
    lt = -w.dt / math.log(model.a)
    out = [np.zeros((len(tq), n)) for _ in range(4)]
    for q, t in enumerate(tq):
        k = min(int(math.floor(t / w.dt + 1e-12)), T)
        tau = t - k * w.dt
        at = math.exp(-tau / lt)
        mu_t = np.zeros(n) if mu_q is None else mu_q[q]
        mu_k = np.zeros(n) if model.mu is None else model.mu[k]
        m = at * filt.m[k] + (mu_t - at * mu_k)
        Mt = at * filt.M_hat[k]
        v = model.sf2 - np.sum(Mt * Mt, axis=1)
        out[0][q], out[1][q] = m, v
        if k == T:
            out[2][q], out[3][q] = m, v
            continue
        a2 = math.exp(-(w.dt - tau) / lt)
        X = a2 * np.concatenate([smooth_W[k + 1], smooth_w[k + 1][:, None]], axis=1)
        PX = model.K_times(X) - Mt @ (Mt.T @ X)
        out[2][q] = m + PX[:, -1]
        E = PX[:, :-1]
        out[3][q] = v - np.sum(E * E, axis=1)
    return out


def smoother_messages(w, filt: FilterResult, model: Optional[Model] = None, rank_r=None):
    """The smoother messages (Ws_k, ws_k), k = 1..T, of Alg. 3 with its truncation (the factors the
    smoother carries from step k + 1 to step k); entry k holds the message after step k's update."""
    model = model or model_from(w)
    rank_r = w.rank_r if rank_r is None else rank_r
    T = w.T
    Wm = [None] * (T + 1)
    wm = [None] * (T + 1)
    ws, Ws = filt.w[T], filt.W[T]
    Wm[T], wm[T] = Ws, ws
    for k in range(T - 1, 0, -1):
        X = model.AT_times(np.concatenate([Ws, ws[:, None]], axis=1))
        Mp = filt.M_pred[k]
        PmX = model.sigma_times(X) - Mp @ (Mp.T @ X)
        Wk = filt.W[k]
        Y2 = X - Wk @ (Wk.T @ PmX)
        ws = filt.w[k] + Y2[:, -1]
        Ws, _, _, _ = truncate(np.concatenate([Wk, Y2[:, :-1]], axis=1), rank_r)
        Wm[k], wm[k] = Ws, ws
    return Wm, wm


# ----------------------------------------------------------------------------- NLL and gradient
def nll_terms(filt: FilterResult) -> np.ndarray:
    return filt.nll.copy()


def nll_total(filt: FilterResult) -> float:
    return float(np.sum(filt.nll))


def nll_grad_fd(w, h=1e-4, budget=None, rank_r=None):
    """Central finite-difference gradient of the NLL w.r.t. (log l_x, log l_t, log sigma_f^2,
    log sigma_n^2) with the actions and truncation rotations of the base run frozen.

    Returns (nll at the base point, gradient[4])."""
    base = filter_run(w, budget=budget, rank_r=rank_r)
    theta0 = np.array([w.log_lx, w.log_lt, w.log_sf2, w.log_sn2])
    g = np.zeros(4)
    for p in range(4):
        vals = []
        for sgn in (+1, -1):
            th = theta0.copy()
            th[p] += sgn * h
            f = filter_run(w, model=model_from(w, *th), budget=budget, rank_r=rank_r,
                           S_replay=base.S, U_replay=base.U)
            vals.append(nll_total(f))
        g[p] = (vals[0] - vals[1]) / (2 * h)
    return nll_total(base), g
