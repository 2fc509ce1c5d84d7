"""Independent dense FP64 references used to pin the oracle (tests only).

None of this code is shared with `oracle/`: every routine is written from its
textbook / paper definition with dense matrices.

* `kf_rts`: the Kalman filter (Thm. "Kalman filter") and the RTS smoother
  (Thm. "RTS smoother") with dense covariances and an explicit smoother gain, on the dense
  state-space matrices A = A^t (x) I, Q, Sigma; for the Matern-3/2 temporal factor A^t and P^t_inf
  come from scipy's matrix exponential and Lyapunov solver (`_temporal`), not from the oracle.
* `batch_gp`: the iteratively approximated batch GP posterior (Def.
  "Iteratively approximated batch GP regression") with block-diagonal actions
  (Prop. "Connecting batch spatio-temporal GP regression and filtering and
  smoothing"), on the full space-time covariance a^|k-k'| K(x, x').
* `dense_truncated`: the CAKF / CAKS with dense covariance matrices and the
  truncation done on the n x n downdate (eig of Sigma - P, resp. of Ws Ws^T),
  i.e. the outer-product form of Alg. 1 / Alg. 3 without any factors.
* `batch_nll_grad`: the analytic gradient of the projected batch NLL with
  frozen actions, 1/2 tr(Gh^-1 S^T dKy S) - 1/2 b^T S^T dKy S b.
"""
from __future__ import annotations

import math

import numpy as np


def _kern(Xa, Xb, kernel, lx, sf2):
    d = np.sqrt(((Xa[:, None, :] - Xb[None, :, :]) ** 2).sum(-1))
    u = d / lx
    if kernel == 0:
        return sf2 * np.exp(-u)
    if kernel == 1:
        return sf2 * (1 + math.sqrt(3) * u) * np.exp(-math.sqrt(3) * u)
    return sf2 * (1 + math.sqrt(5) * u + 5 * u * u / 3) * np.exp(-math.sqrt(5) * u)


def _dkern_dloglx(Xa, Xb, kernel, lx, sf2):
    d = np.sqrt(((Xa[:, None, :] - Xb[None, :, :]) ** 2).sum(-1))
    u = d / lx
    if kernel == 0:
        dk = -np.exp(-u)
    elif kernel == 1:
        dk = -3 * u * np.exp(-math.sqrt(3) * u)
    else:
        dk = -(5.0 / 3.0) * u * (1 + math.sqrt(5) * u) * np.exp(-math.sqrt(5) * u)
    return sf2 * dk * (-u)        # d/dlog l of k(d/l) = k'(u) * (-u)


def _params(w):
    lx, lt, sf2, sn2 = (math.exp(w.log_lx), math.exp(w.log_lt), math.exp(w.log_sf2), math.exp(w.log_sn2))
    return lx, lt, sf2, sn2, math.exp(-w.dt / lt)


def _mu(w, k):
    return np.zeros(w.n) if w.prior_mean is None else w.prior_mean[k]


def _temporal(w):
    """Temporal factor (A^t, P^t_inf) of a workload, from library routines: the OU factor
    (a = exp(-dt/l_t), 1); for the Matern-3/2 factor the matrix exponential of the SDE drift
    F = [[0, 1], [-lam^2, -2 lam]] (scipy expm) and the stationary covariance from the continuous
    Lyapunov equation F P + P F^T + L q L^T = 0 with the Matern-3/2 spectral density q = 4 lam^3."""
    lx, lt, sf2, sn2, a = _params(w)
    if getattr(w, "temporal", 0) == 0:
        return np.array([[a]]), np.array([[1.0]])
    import scipy.linalg as sl
    lam = math.sqrt(3.0) / lt
    F = np.array([[0.0, 1.0], [-lam * lam, -2.0 * lam]])
    Pinf = sl.solve_continuous_lyapunov(F, -np.array([[0.0, 0.0], [0.0, 4.0 * lam ** 3]]))
    return sl.expm(F * w.dt), Pinf


def _tcorr(w, lag):
    """Temporal correlation between steps lag apart (closed form): a^|lag| for the OU factor,
    (1 + lam tau) exp(-lam tau), tau = |lag| dt, lam = sqrt(3)/l_t for the Matern-3/2 factor."""
    lx, lt, sf2, sn2, a = _params(w)
    lag = np.abs(lag)
    if getattr(w, "temporal", 0) == 0:
        return a ** lag
    u = math.sqrt(3.0) * lag * w.dt / lt
    return (1.0 + u) * np.exp(-u)


def _lgssm(w):
    """Dense (A, Q, Sigma, state prior means) of the state-space model: A = A^t (x) I,
    Sigma = P^t_inf (x) K, Q = Sigma - A Sigma A^T; the state mean stacks the prior mean of the
    positions above zero velocities."""
    lx, lt, sf2, sn2, a = _params(w)
    K = _kern(w.coords, w.coords, w.kernel, lx, sf2)
    At, Pinf = _temporal(w)
    dp = At.shape[0]
    A = np.kron(At, np.eye(w.n))
    Sig = np.kron(Pinf, K)
    Q = Sig - A @ Sig @ A.T

    def mu(k):
        out = np.zeros(dp * w.n)
        out[:w.n] = _mu(w, k)
        return out
    return A, Q, Sig, mu


def kf_rts(w):
    """Dense Kalman filter + RTS smoother over the whole state (D = n D'); returns dict of
    means/vars (T+1, D) and per-step NLL."""
    lx, lt, sf2, sn2, a = _params(w)
    A, Q, Sig, mu = _lgssm(w)
    T = w.T
    m, P = mu(0), Sig.copy()
    mf, Pf, mp, Pp = [m], [P], [None], [None]
    nll = np.zeros(T + 1)
    for k in range(1, T + 1):
        mpk = A @ m + (mu(k) - A @ mu(k - 1))
        Ppk = A @ P @ A.T + Q
        o = w.obs(k)
        if len(o):
            G = Ppk[np.ix_(o, o)] + sn2 * np.eye(len(o))
            r = w.yk(k) - mpk[o]
            gain = np.linalg.solve(G, Ppk[o, :]).T
            m = mpk + gain @ r
            P = Ppk - gain @ Ppk[o, :]
            sign, ld = np.linalg.slogdet(2 * np.pi * G)
            nll[k] = 0.5 * ld + 0.5 * r @ np.linalg.solve(G, r)
        else:
            m, P = mpk, Ppk
        mf.append(m); Pf.append(P); mp.append(mpk); Pp.append(Ppk)
    ms, Ps = [None] * (T + 1), [None] * (T + 1)
    ms[T], Ps[T] = mf[T], Pf[T]
    for k in range(T - 1, -1, -1):
        J = np.linalg.solve(Pp[k + 1].T, (Pf[k] @ A.T).T).T      # P_k A^T (P^-_{k+1})^{-1}
        ms[k] = mf[k] + J @ (ms[k + 1] - mp[k + 1])
        Ps[k] = Pf[k] + J @ (Ps[k + 1] - Pp[k + 1]) @ J.T
    return dict(mf=np.array(mf), vf=np.array([np.diag(p) for p in Pf]),
                ms=np.array(ms), vs=np.array([np.diag(p) for p in Ps]), nll=nll)


def _spacetime(w, upto=None):
    """Observation list Z=(step, index) and the space-time prior blocks."""
    lx, lt, sf2, sn2, a = _params(w)
    K = _kern(w.coords, w.coords, w.kernel, lx, sf2)
    T = w.T if upto is None else upto
    steps = np.concatenate([np.full(len(w.obs(k)), k) for k in range(1, T + 1)]) if T > 0 else np.zeros(0, int)
    idx = np.concatenate([w.obs(k) for k in range(1, T + 1)]) if T > 0 else np.zeros(0, int)
    return K, steps.astype(int), idx.astype(int), sn2


def batch_gp(w, S_list, upto=None, k_eval=None):
    """Iteratively approximated batch GP posterior marginals at all grid points of step k_eval,
    using data of steps 1..upto and block-diagonal actions S = diag(S_1, ..., S_upto)."""
    K, st, ix, sn2 = _spacetime(w, upto)
    T = w.T if upto is None else upto
    N = ix.size
    Kzz = _tcorr(w, st[:, None] - st[None, :]) * K[np.ix_(ix, ix)]
    Ky = Kzz + sn2 * np.eye(N)
    cols = sum(S_list[k].shape[1] for k in range(1, T + 1))
    S = np.zeros((N, cols))
    r0 = c0 = 0
    for k in range(1, T + 1):
        Sk = S_list[k]
        S[r0:r0 + Sk.shape[0], c0:c0 + Sk.shape[1]] = Sk
        r0 += Sk.shape[0]
        c0 += Sk.shape[1]
    ybar = np.concatenate([w.yk(k) - _mu(w, k)[w.obs(k)] for k in range(1, T + 1)])
    C = S @ np.linalg.solve(S.T @ Ky @ S, S.T)
    kk = T if k_eval is None else k_eval
    Kxz = _tcorr(w, kk - st)[None, :] * K[:, ix]
    mean = _mu(w, kk) + Kxz @ (C @ ybar)
    var = np.diag(K) - np.einsum("ij,jk,ik->i", Kxz, C, Kxz)
    Gh = S.T @ Ky @ S
    yh = S.T @ ybar
    nll = (0.5 * cols * math.log(2 * math.pi) + 0.5 * np.linalg.slogdet(Gh)[1]
           + 0.5 * yh @ np.linalg.solve(Gh, yh) - 0.5 * np.linalg.slogdet(S.T @ S)[1])
    return mean, var, nll


def batch_nll_grad(w, S_list):
    """Analytic d NLL / d(log l_x, log l_t, log sf2, log sn2) of the projected batch NLL, frozen S."""
    lx, lt, sf2, sn2, a = _params(w)
    assert getattr(w, "temporal", 0) == 0, "batch_nll_grad: OU temporal factor"
    K, st, ix, sn2 = _spacetime(w)
    N = ix.size
    dk = np.abs(st[:, None] - st[None, :])
    At = a ** dk
    Kzz = At * K[np.ix_(ix, ix)]
    Ky = Kzz + sn2 * np.eye(N)
    cols = sum(S_list[k].shape[1] for k in range(1, w.T + 1))
    S = np.zeros((N, cols))
    r0 = c0 = 0
    for k in range(1, w.T + 1):
        Sk = S_list[k]
        S[r0:r0 + Sk.shape[0], c0:c0 + Sk.shape[1]] = Sk
        r0 += Sk.shape[0]
        c0 += Sk.shape[1]
    ybar = np.concatenate([w.yk(k) - _mu(w, k)[w.obs(k)] for k in range(1, w.T + 1)])
    Gh = S.T @ Ky @ S
    b = np.linalg.solve(Gh, S.T @ ybar)
    Ghi = np.linalg.inv(Gh)
    dK = [
        At * _dkern_dloglx(w.coords[ix], w.coords[ix], w.kernel, lx, sf2),
        Kzz * dk * (w.dt / lt),
        Kzz,
        sn2 * np.eye(N),
    ]
    g = np.zeros(4)
    for p, D in enumerate(dK):
        SDS = S.T @ D @ S
        g[p] = 0.5 * np.trace(Ghi @ SDS) - 0.5 * b @ SDS @ b
    return g


def dense_truncated(w, S_list, r):
    """Outer-product (dense covariance) CAKF + CAKS with truncation on the D x D downdates.

    Filter: P^-_k = A P~_{k-1} A^T + Q; update with the given actions S_k;
    truncation P~_k = Sigma - best_rank_r(Sigma - P_k).  Smoother (Alg. 3 in outer-product
    form): Omega_k = W_k W_k^T + B Omega~_{k+1} B^T with B = (I - W W^T P^-_k) A^T and
    Omega~ = best_rank_r(Omega); mean m^s_k = m_k + P_k A^T ws_{k+1};
    cov P^s_k = P_k - P_k A^T Omega~_{k+1} A P_k."""
    lx, lt, sf2, sn2, a = _params(w)
    A, Q, Sig, mu = _lgssm(w)
    D, T = Sig.shape[0], w.T

    def rank_r(Dm):
        if r <= 0:
            return Dm
        lam, U = np.linalg.eigh(Dm)
        o = np.argsort(lam)[::-1][:r]
        return (U[:, o] * lam[o]) @ U[:, o].T

    m, Pt = mu(0), Sig.copy()
    mf, Pf, Pm, Ww, ww = [m], [Sig.copy()], [Sig.copy()], [np.zeros((D, D))], [np.zeros(D)]
    for k in range(1, T + 1):
        mpk = A @ m + (mu(k) - A @ mu(k - 1))
        Ppk = A @ Pt @ A.T + Q
        o = w.obs(k)
        Sk = S_list[k]
        if len(o) and Sk.shape[1]:
            H = np.zeros((len(o), D))
            H[np.arange(len(o)), o] = 1.0
            Hs = Sk.T @ H
            Gh = Hs @ Ppk @ Hs.T + sn2 * Sk.T @ Sk
            Ginv = np.linalg.inv(Gh)
            wk = Hs.T @ Ginv @ (Sk.T @ (w.yk(k) - mpk[o]))
            WW = Hs.T @ Ginv @ Hs
            m = mpk + Ppk @ wk
            P = Ppk - Ppk @ WW @ Ppk
        else:
            wk, WW, m, P = np.zeros(D), np.zeros((D, D)), mpk, Ppk
        mf.append(m); Pf.append(P); Pm.append(Ppk); Ww.append(WW); ww.append(wk)
        Pt = Sig - rank_r(Sig - P)
    ms, vs = [None] * (T + 1), [None] * (T + 1)
    ms[T], vs[T] = mf[T], np.diag(Pf[T])
    ws, Om = ww[T], Ww[T]
    for k in range(T - 1, -1, -1):
        ms[k] = mf[k] + Pf[k] @ A.T @ ws
        vs[k] = np.diag(Pf[k] - Pf[k] @ A.T @ Om @ A @ Pf[k])
        if k == 0:
            break
        B = (np.eye(D) - Ww[k] @ Pm[k]) @ A.T
        ws = ww[k] + B @ ws
        Om = rank_r(Ww[k] + B @ Om @ B.T)
    return dict(mf=np.array(mf), vf=np.array([np.diag(p) for p in Pf]), ms=np.array(ms), vs=np.array(vs))


def _chol_sym(A):
    """Cholesky factor L (A = L L^T) of a symmetric matrix without conjugation: analytic in the
    entries of A, so it can carry a complex-step perturbation."""
    n = A.shape[0]
    L = np.zeros_like(A)
    for j in range(n):
        L[j, j] = np.sqrt(A[j, j] - np.sum(L[j, :j] * L[j, :j]))
        for i in range(j + 1, n):
            L[i, j] = (A[i, j] - np.sum(L[i, :j] * L[j, :j])) / L[j, j]
    return L


def frozen_truncated_nll(w, S_list, U_list, theta):
    """NLL of the projected data in the modified model with frozen actions S_k and frozen
    truncation rotations U_k, at log-hyperparameters theta = (log l_x, log l_t, log sf2, log sn2).

    Written with factors and the batch form of the update (V_k = S_k L_k^-T with
    L_k L_k^T = S_k^T G_k S_k, the G-orthonormalisation of the actions): M^-_k = a M+_{k-1},
    [P^-W_k, P^-w_k] = K[:, o] [V_k v_k] - M^-_k (M^-_k[o]^T [V_k v_k]), M_k = (M^-_k, P^-W_k),
    M+_k = M_k U_k (U_k None: no truncation).  Every operation is analytic in theta (no
    conjugation, no absolute values, no eigendecomposition), so theta may be complex: the
    complex-step derivative Im f(theta + i h e_p) / h is then the exact gradient."""
    lx, lt, sf2, sn2 = (np.exp(theta[0]), np.exp(theta[1]), np.exp(theta[2]), np.exp(theta[3]))
    a = np.exp(-w.dt / lt)
    X = w.coords
    d = np.sqrt(((X[:, None, :] - X[None, :, :]) ** 2).sum(-1))
    u = d / lx
    if w.kernel == 0:
        K = sf2 * np.exp(-u)
    elif w.kernel == 1:
        K = sf2 * (1 + math.sqrt(3) * u) * np.exp(-math.sqrt(3) * u)
    else:
        K = sf2 * (1 + math.sqrt(5) * u + 5 * u * u / 3) * np.exp(-math.sqrt(5) * u)
    n = w.n
    m = _mu(w, 0).astype(complex)
    Mp = np.zeros((n, 0), dtype=complex)
    nll = 0.0 + 0.0j
    for k in range(1, w.T + 1):
        mpk = a * m + (_mu(w, k) - a * _mu(w, k - 1))
        Mm = a * Mp
        o = w.obs(k)
        Sk = S_list[k]
        if len(o) == 0 or Sk.shape[1] == 0:
            m, Mk = mpk, Mm
        else:
            Mo = Mm[o]
            G = K[np.ix_(o, o)] - Mo @ Mo.T + sn2 * np.eye(len(o))
            r0 = w.yk(k) - mpk[o]
            L = _chol_sym(Sk.T @ G @ Sk)
            V = np.linalg.solve(L, Sk.T).T                     # S L^-T
            yh = Sk.T @ r0
            z = np.linalg.solve(L, yh)
            v = V @ z
            Ls = _chol_sym((Sk.T @ Sk).astype(complex))
            j = Sk.shape[1]
            nll += 0.5 * j * math.log(2 * math.pi) + np.sum(np.log(np.diag(L))) + 0.5 * z @ z \
                - np.sum(np.log(np.diag(Ls)))
            Vv = np.concatenate([V, v[:, None]], axis=1)
            PVv = K[:, o] @ Vv - Mm @ (Mo.T @ Vv)
            m = mpk + PVv[:, -1]
            Mk = np.concatenate([Mm, PVv[:, :-1]], axis=1)
        Mp = Mk if U_list[k] is None else Mk @ U_list[k]
    return nll


def frozen_truncated_nll_grad(w, S_list, U_list, h=1e-30):
    """Exact gradient of frozen_truncated_nll by the complex step (no subtraction, no h error)."""
    th = np.array([w.log_lx, w.log_lt, w.log_sf2, w.log_sn2], dtype=complex)
    g = np.zeros(4)
    for p in range(4):
        t = th.copy()
        t[p] += 1j * h
        g[p] = frozen_truncated_nll(w, S_list, U_list, t).imag / h
    return float(frozen_truncated_nll(w, S_list, U_list, th).real), g
