"""Seeded synthetic workloads for the computation-aware Kalman filter / smoother.

This module is shared by the FP64 oracle, the tests and the benchmark.  It holds
only input generation: grids, observation index sets, and data drawn from an
approximate prior sample.  It contains none of the filter's or smoother's
arithmetic (no kernel matrices, no Kalman recursions).

Model shape (paper, Sec. 2.2 and the space-time separable Gauss-Markov lemma in
the appendix): a spatial Matern kernel on a fixed grid X (n points), an
Ornstein-Uhlenbeck temporal factor with decay a = exp(-dt / l_t), and at each
step k = 1..T a set of m_k observed grid indices with i.i.d. Gaussian noise.

Data are drawn from random Fourier features (RFF) of the Matern spectral
density (a multivariate Student-t with 2*nu degrees of freedom, scale 1/l_x),
with OU dynamics on the feature weights (or, for the Matern-3/2 temporal
factor, weight paths drawn from that kernel's covariance over the step times),
so that the sample is (up to the feature count) a draw from the same separable
prior.  The paper's ERA5 data are
not available here; configs "sphere-*" stand in for them with the ERA5 grid
shape (lat-lon grid mapped to the unit sphere, extrinsic Matern on chordal
distance).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

MATERN12, MATERN32, MATERN52 = 0, 1, 2
NU = {MATERN12: 0.5, MATERN32: 1.5, MATERN52: 2.5}


@dataclasses.dataclass
class Workload:
    name: str
    coords: np.ndarray            # (n, dim) float64, row-major
    kernel: int                   # MATERN12 | MATERN32 | MATERN52
    log_lx: float
    log_lt: float
    log_sf2: float
    log_sn2: float
    T: int
    dt: float
    obs_ptr: np.ndarray           # (T+1,) int32; step k (1-based) owns [obs_ptr[k-1], obs_ptr[k])
    obs_idx: np.ndarray           # (N,) int32, sorted and distinct within a step
    y: np.ndarray                 # (N,) float64
    budget_i: int
    rank_r: int                   # <= 0: no truncation
    prior_mean: Optional[np.ndarray] = None   # (T+1, n) float64 or None (zero mean)
    truth: Optional[np.ndarray] = None        # (T+1, n) latent sample when kept
    temporal: int = 0                         # temporal factor: 0 Ornstein-Uhlenbeck, 1 Matern-3/2

    @property
    def n(self) -> int:
        return int(self.coords.shape[0])

    @property
    def dim(self) -> int:
        return int(self.coords.shape[1])

    def obs(self, k: int) -> np.ndarray:
        """Observed grid indices at step k (1-based)."""
        return self.obs_idx[self.obs_ptr[k - 1]:self.obs_ptr[k]]

    def yk(self, k: int) -> np.ndarray:
        return self.y[self.obs_ptr[k - 1]:self.obs_ptr[k]]

    def with_(self, **kw) -> "Workload":
        return dataclasses.replace(self, **kw)


# ----------------------------------------------------------------------------- grids
def grid_1d(n: int) -> np.ndarray:
    return (np.arange(n, dtype=np.float64) / max(n - 1, 1))[:, None]


def grid_2d(nx: int, ny: int) -> np.ndarray:
    gx = (np.arange(nx) + 0.5) / nx
    gy = (np.arange(ny) + 0.5) / ny
    xx, yy = np.meshgrid(gx, gy, indexing="ij")
    return np.stack([xx.ravel(), yy.ravel()], axis=1).astype(np.float64)


def grid_sphere(nlat: int, nlon: int) -> np.ndarray:
    """Cell-centred lat-lon grid mapped to the unit sphere (x, y, z)."""
    lat = -math.pi / 2 + (np.arange(nlat) + 0.5) * math.pi / nlat
    lon = 2 * math.pi * np.arange(nlon) / nlon
    la, lo = np.meshgrid(lat, lon, indexing="ij")
    xyz = np.stack([np.cos(la) * np.cos(lo), np.cos(la) * np.sin(lo), np.sin(la)], axis=-1)
    return xyz.reshape(-1, 3).astype(np.float64)


# ----------------------------------------------------------------------------- observations
def obs_uniform(rng: np.random.Generator, n: int, m: int, T: int, missing=()) -> tuple:
    ptr = [0]
    idx = []
    for k in range(1, T + 1):
        if k in missing:
            sel = np.zeros(0, dtype=np.int64)
        else:
            sel = np.sort(rng.choice(n, size=m, replace=False))
        idx.append(sel)
        ptr.append(ptr[-1] + sel.size)
    return np.asarray(ptr, dtype=np.int32), np.concatenate(idx).astype(np.int32)


def obs_stations(rng: np.random.Generator, n: int, m: int, T: int, frac: float = 0.7) -> tuple:
    """floor(frac*m) fixed station indices plus fresh distinct random others per step."""
    ns = int(math.floor(frac * m))
    stations = rng.choice(n, size=ns, replace=False)
    mask = np.ones(n, dtype=bool)
    mask[stations] = False
    others = np.nonzero(mask)[0]
    ptr = [0]
    idx = []
    for _ in range(T):
        extra = rng.choice(others, size=m - ns, replace=False)
        sel = np.sort(np.concatenate([stations, extra]))
        idx.append(sel)
        ptr.append(ptr[-1] + sel.size)
    return np.asarray(ptr, dtype=np.int32), np.concatenate(idx).astype(np.int32)


# ----------------------------------------------------------------------------- data
def seasonal_mean(coords: np.ndarray, T: int, dt: float) -> np.ndarray:
    """Deterministic mean 0.5 sin(2 pi t / 5) cos(2 pi x_1) on steps 0..T."""
    t = np.arange(T + 1) * dt
    return 0.5 * np.sin(2 * np.pi * t / 5.0)[:, None] * np.cos(2 * np.pi * coords[:, 0])[None, :]


def rff_draw(rng, coords, kernel, lx, lt, sf2, sn2, T, dt, obs_ptr, obs_idx,
             n_features=1024, keep_truth=False, prior_mean=None, device=None, temporal=0):
    """Observations y from an RFF prior sample with OU feature weights (temporal = 0) or with
    Matern-3/2 feature weights (temporal = 1: each weight's path over the step times t_k = k dt is
    drawn from the closed-form temporal covariance (1 + sqrt(3) |t - t'| / l_t) exp(-sqrt(3) |t - t'| / l_t)
    through its Cholesky factor).

    Returns (y, truth-or-None).  The bulk cos() evaluation runs through torch on
    `device` when given (data generation only; never timed).
    """
    nu = NU[kernel]
    d = coords.shape[1]
    z = rng.standard_normal((n_features, d))
    g = rng.chisquare(2 * nu, size=n_features)
    omega = z / lx * np.sqrt(2 * nu / g)[:, None]
    phase = rng.uniform(0, 2 * np.pi, size=n_features)
    if temporal == 1:
        tt = np.arange(T + 1) * dt
        u = math.sqrt(3.0) * np.abs(tt[:, None] - tt[None, :]) / lt
        Ct = (1.0 + u) * np.exp(-u)
        Lt = np.linalg.cholesky(Ct + 1e-12 * np.eye(T + 1))
        w = Lt @ rng.standard_normal((T + 1, n_features))
    else:
        a = math.exp(-dt / lt)
        w = np.empty((T + 1, n_features))
        w[0] = rng.standard_normal(n_features)
        for k in range(1, T + 1):
            w[k] = a * w[k - 1] + math.sqrt(1 - a * a) * rng.standard_normal(n_features)
    scale = math.sqrt(2.0 * sf2 / n_features)
    noise = rng.standard_normal(obs_idx.size) * math.sqrt(sn2)

    import torch
    dev = torch.device(device) if device is not None else torch.device("cpu")
    Xt = torch.as_tensor(coords, dtype=torch.float64, device=dev)
    Om = torch.as_tensor(omega, dtype=torch.float64, device=dev)
    Ph = torch.as_tensor(phase, dtype=torch.float64, device=dev)
    Wt = torch.as_tensor(w, dtype=torch.float64, device=dev)

    y = np.empty(obs_idx.size)
    truth = np.empty((T + 1, coords.shape[0])) if keep_truth else None
    if keep_truth:
        feats = torch.cos(Xt @ Om.T + Ph) * scale
        truth[:] = (Wt @ feats.T).cpu().numpy()
    for k in range(1, T + 1):
        lo, hi = int(obs_ptr[k - 1]), int(obs_ptr[k])
        if hi == lo:
            continue
        ix = torch.as_tensor(obs_idx[lo:hi].astype(np.int64), device=dev)
        f = (torch.cos(Xt[ix] @ Om.T + Ph) * scale) @ Wt[k]
        y[lo:hi] = f.cpu().numpy()
    y += noise
    if prior_mean is not None:
        for k in range(1, T + 1):
            lo, hi = int(obs_ptr[k - 1]), int(obs_ptr[k])
            y[lo:hi] += prior_mean[k, obs_idx[lo:hi]]
        if truth is not None:
            truth += prior_mean
    return y, truth


def make(name, coords, kernel, lx, lt, sf2, sn2, T, dt, m, budget_i, rank_r, seed,
         stations=False, seasonal=False, missing=(), n_features=1024, keep_truth=False,
         device=None, temporal=0) -> Workload:
    rng = np.random.default_rng(seed)
    n = coords.shape[0]
    if stations:
        ptr, idx = obs_stations(rng, n, m, T)
    else:
        ptr, idx = obs_uniform(rng, n, m, T, missing=missing)
    pm = seasonal_mean(coords, T, dt) if seasonal else None
    y, truth = rff_draw(rng, coords, kernel, lx, lt, sf2, sn2, T, dt, ptr, idx,
                        n_features=n_features, keep_truth=keep_truth, prior_mean=pm, device=device,
                        temporal=temporal)
    return Workload(name=name, coords=coords, kernel=kernel, log_lx=math.log(lx), log_lt=math.log(lt),
                    log_sf2=math.log(sf2), log_sn2=math.log(sn2), T=T, dt=dt, obs_ptr=ptr, obs_idx=idx,
                    y=y, budget_i=budget_i, rank_r=rank_r, prior_mean=pm, truth=truth, temporal=temporal)


# ----------------------------------------------------------------------------- named configs
def tiny_1d(T=50, seed=0, **kw) -> Workload:
    """n=256 1-D grid, Matern-3/2 (l=0.1), OU l_t=0.5, dt=0.1, m=32, sn2=0.01, full budget, no truncation."""
    return make("tiny-1d-n256", grid_1d(256), MATERN32, 0.1, 0.5, 1.0, 0.01, T, 0.1, 32,
                budget_i=32, rank_r=0, seed=seed, **kw)


def grid2d_16k(T=200, seed=1, side=128, m=2000, budget_i=32, rank_r=256, **kw) -> Workload:
    """128x128 grid on [0,1]^2 (n=16384), Matern-5/2 (l=0.05), OU l_t=1, dt=0.1, m=2000, i=32, r=256,
    seasonal prior mean."""
    return make(f"grid2d-n{side*side}", grid_2d(side, side), MATERN52, 0.05, 1.0, 1.0, 0.01, T, 0.1, m,
                budget_i=budget_i, rank_r=rank_r, seed=seed, seasonal=True, **kw)


def sphere_65k(T=500, seed=2, nlat=256, nlon=256, m=8192, budget_i=64, rank_r=512, **kw) -> Workload:
    """256x256 lat-lon grid on the unit sphere (n=65536), extrinsic Matern-3/2 (chordal l=0.1), OU l_t=1,
    dt=0.1, m=8192 (70% fixed stations), sn2=0.05, i=64, r=512."""
    return make(f"sphere-n{nlat*nlon}", grid_sphere(nlat, nlon), MATERN32, 0.1, 1.0, 1.0, 0.05, T, 0.1, m,
                budget_i=budget_i, rank_r=rank_r, seed=seed, stations=True, **kw)


def fd_grid2d_1k(T=20, seed=3, **kw) -> Workload:
    """The 16k-grid model on a 32x32 grid (n=1024), T=20, m=128, i=32, r=256 (gradient checks)."""
    return make("grid2d-n1024", grid_2d(32, 32), MATERN52, 0.05, 1.0, 1.0, 0.01, T, 0.1, 128,
                budget_i=32, rank_r=256, seed=seed, seasonal=True, **kw)


def sphere_262k(T=300, seed=4, **kw) -> Workload:
    """512x512 sphere grid (n=262144), Matern-3/2 (l=0.05), m=16384, sn2=0.05, i=128, r=256."""
    return make("sphere-n262144", grid_sphere(512, 512), MATERN32, 0.05, 1.0, 1.0, 0.05, T, 0.1, 16384,
                budget_i=128, rank_r=256, seed=seed, stations=True, **kw)


def small(n=200, dim=2, m=40, T=6, budget_i=8, rank_r=0, kernel=MATERN32, lx=0.3, lt=0.7, sf2=1.3,
          sn2=0.05, dt=0.1, seed=11, seasonal=False, missing=(), sphere=False, **kw) -> Workload:
    """Small randomized problem for parity tests (scattered points in the unit cube / on the sphere)."""
    rng = np.random.default_rng(seed + 1000)
    if sphere:
        v = rng.standard_normal((n, 3))
        coords = v / np.linalg.norm(v, axis=1, keepdims=True)
    else:
        coords = rng.uniform(0, 1, size=(n, dim))
    return make(f"small-n{n}", coords, kernel, lx, lt, sf2, sn2, T, dt, m, budget_i=budget_i,
                rank_r=rank_r, seed=seed, seasonal=seasonal, missing=missing, **kw)


def gaussian_actions(w: Workload, seed: int = 0, budget_i: Optional[int] = None) -> list:
    """Randomized actions of the policy appendix: for each step k an m_k x i_k matrix of i.i.d.
    standard normal entries (i_k = min(budget, m_k)); entry [0] is an empty placeholder.  The
    draws are inputs of the method, made here once and passed to both the oracle and the device."""
    rng = np.random.default_rng(seed)
    i = w.budget_i if budget_i is None else budget_i
    out = [np.zeros((0, 0))]
    for k in range(1, w.T + 1):
        m = int(w.obs_ptr[k] - w.obs_ptr[k - 1])
        out.append(rng.standard_normal((m, min(i, m))) if m else np.zeros((0, 0)))
    return out


def sampler_inputs(w: Workload, n_samples: int, seed: int = 0, n_features: int = 1024):
    """Random inputs of the posterior sampler (the sampling algorithm of the paper's appendix), drawn
    once and passed to both the oracle and the device: an approximate prior sample of the initial
    state x0 ~ N(mu_0, K) and of the OU dynamics noise q_{k-1} ~ N(0, (1 - a^2) K) by random Fourier
    features (as the paper suggests), and observation noise eps_k ~ N(0, sn2 I).

    Returns (x0, q, eps): x0 (n, S); q[k] (n, S) for k = 1..T (q[0] unused); eps[k] (m_k, S)."""
    rng = np.random.default_rng(seed)
    nu = NU[w.kernel]
    lx, lt, sf2, sn2 = (math.exp(w.log_lx), math.exp(w.log_lt), math.exp(w.log_sf2), math.exp(w.log_sn2))
    d = w.coords.shape[1]
    z = rng.standard_normal((n_features, d))
    g = rng.chisquare(2 * nu, size=n_features)
    omega = z / lx * np.sqrt(2 * nu / g)[:, None]
    phase = rng.uniform(0, 2 * np.pi, size=n_features)
    feats = np.cos(w.coords @ omega.T + phase) * math.sqrt(2.0 * sf2 / n_features)   # (n, F)
    a = math.exp(-w.dt / lt)
    mu0 = np.zeros(w.n) if w.prior_mean is None else w.prior_mean[0]
    x0 = mu0[:, None] + feats @ rng.standard_normal((n_features, n_samples))
    q = [np.zeros((w.n, n_samples))]
    eps = [np.zeros((0, n_samples))]
    for k in range(1, w.T + 1):
        q.append(math.sqrt(1 - a * a) * (feats @ rng.standard_normal((n_features, n_samples))))
        m = int(w.obs_ptr[k] - w.obs_ptr[k - 1])
        eps.append(rng.standard_normal((m, n_samples)) * math.sqrt(sn2))
    return x0, q, eps
