"""Pins of the oracle's Matern-3/2 temporal factor (D' = 2: state (f, df/dt) per grid point) against
independent computations (CPU only).

* The temporal factor (A^t, P^t_inf) against scipy's matrix exponential of the SDE drift and its
  continuous Lyapunov equation, and its position covariance against the closed-form Matern-3/2
  kernel (the remark after the space-time separable lemma: Matern(p + 1/2) kernels have an exact
  state-space form).
* Full action budget, no truncation: the CAKF / CAKS equal the dense Kalman filter / RTS smoother
  on the whole 2n-dimensional state (positions and velocities), NLL included.
* Any budget, no truncation: the positions equal the iteratively approximated batch GP on the
  closed-form space-time covariance k_t(t - t') K(x, x').
* With truncation: the factor form equals the dense outer-product form on the 2n x 2n downdates.
"""
import math

import numpy as np
import pytest

import dense_ref
import oracle
import synth
from oracle import cakf as oc

pytest.importorskip("scipy")


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.max(np.abs(a - b)) / max(1e-300, np.max(np.abs(b))))


def m32(**kw):
    return synth.small(temporal=1, **kw)


@pytest.mark.parametrize("lt,dt", [(0.5, 0.1), (2.0, 0.3), (0.1, 0.05)])
def test_temporal_factor_against_expm_lyapunov_and_the_kernel(lt, dt):
    w = m32(n=4, m=2, T=2, lt=lt, dt=dt, seed=1)
    At, Pinf = oc.matern32_temporal(lt, dt)
    At_ref, Pinf_ref = dense_ref._temporal(w)
    assert rel(At, At_ref) < 1e-13
    assert rel(Pinf, Pinf_ref) < 1e-12
    lam = math.sqrt(3.0) / lt
    for lag in range(0, 6):
        tau = lag * dt
        cov = (np.linalg.matrix_power(At, lag) @ Pinf)[0, 0]      # Cov(f(t + tau), f(t))
        assert abs(cov - (1 + lam * tau) * math.exp(-lam * tau)) < 1e-13
    Qt = Pinf - At @ Pinf @ At.T
    assert np.min(np.linalg.eigvalsh(Qt)) > 0


@pytest.mark.parametrize("seasonal", [False, True])
def test_full_budget_equals_dense_kf_rts_on_the_whole_state(seasonal):
    w = m32(n=20, dim=1, m=6, T=6, budget_i=6, rank_r=0, seasonal=seasonal, missing=(3,), seed=31)
    f = oracle.filter_run(w)
    ms, vs, _ = oracle.smoother_run(w, f)
    ref = dense_ref.kf_rts(w)
    assert f.m.shape == (w.T + 1, 2 * w.n)
    assert rel(f.m, ref["mf"]) < 1e-9
    assert rel(f.var, ref["vf"]) < 1e-9
    assert rel(ms, ref["ms"]) < 1e-9
    assert rel(vs, ref["vs"]) < 1e-9
    assert np.allclose(f.nll, ref["nll"], rtol=1e-9, atol=1e-10)


@pytest.mark.parametrize("budget", [1, 4])
def test_partial_budget_positions_equal_batch_gp(budget):
    w = m32(n=24, dim=2, m=8, T=5, budget_i=budget, rank_r=0, seasonal=True, seed=33)
    f = oracle.filter_run(w)
    ms, vs, _ = oracle.smoother_run(w, f)
    n = w.n
    for k in range(1, w.T + 1):
        mb, vb, _ = dense_ref.batch_gp(w, f.S, upto=k, k_eval=k)
        assert rel(f.m[k, :n], mb) < 1e-9
        assert rel(f.var[k, :n], vb) < 1e-9
    for k in range(0, w.T + 1):
        mb, vb, nb = dense_ref.batch_gp(w, f.S, upto=w.T, k_eval=k)
        assert rel(ms[k, :n], mb) < 1e-9, k
        assert rel(vs[k, :n], vb) < 1e-9, k
    assert abs(oracle.nll_total(f) - nb) < 1e-9 * abs(nb)


def test_truncated_run_matches_dense_outer_product():
    w = m32(n=18, dim=2, m=8, T=6, budget_i=3, rank_r=5, seasonal=True, seed=35)
    f = oracle.filter_run(w)
    ms, vs, _ = oracle.smoother_run(w, f)
    ref = dense_ref.dense_truncated(w, f.S, w.rank_r)
    assert rel(f.m, ref["mf"]) < 1e-9
    assert rel(f.var, ref["vf"]) < 1e-9
    assert rel(ms, ref["ms"]) < 1e-9
    assert rel(vs, ref["vs"]) < 1e-9


@pytest.mark.parametrize("mistake", ["drift_sign", "velocity_variance", "transpose"])
def test_pins_catch_planted_mistakes_in_the_temporal_factor(monkeypatch, mistake):
    real = oc.matern32_temporal

    def planted(lt, dt):
        At, Pinf = real(lt, dt)
        if mistake == "drift_sign":
            At = At.copy(); At[1, 0] = -At[1, 0]
        elif mistake == "velocity_variance":
            Pinf = Pinf.copy(); Pinf[1, 1] *= 1.5
        else:
            At = At.T.copy()
        return At, Pinf
    monkeypatch.setattr(oc, "matern32_temporal", planted)
    w = m32(n=16, dim=1, m=6, T=5, budget_i=6, rank_r=0, seed=37)
    f = oracle.filter_run(w)
    ms, vs, _ = oracle.smoother_run(w, f)
    ref = dense_ref.kf_rts(w)
    bad = max(rel(f.m, ref["mf"]), rel(f.var, ref["vf"]), rel(ms, ref["ms"]), rel(vs, ref["vs"]))
    assert bad > 1e-6
