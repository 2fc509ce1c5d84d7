"""Pins of the FP64 oracle against results the paper and the mathematics fix (CPU only).

Every check compares the oracle with an independent computation:
* the scalar Kalman filter written out by hand (n = 1);
* the dense Kalman filter / RTS smoother at full action budget (the projection
  then loses nothing, Sec. 3.1; Prop. "Downdate-form Kalman filter"; Prop.
  "Inverse-free RTS smoother");
* the iteratively approximated batch GP with block-diagonal actions for any
  budget without truncation (Prop. "Connecting ... filtering and smoothing");
* the dense outer-product form of the filter and smoother with truncation on
  the n x n downdates (Sec. 3.2, Alg. 3);
* Eckart-Young via a direct SVD of the factor (Sec. 3.2);
* the analytic gradient of the projected batch NLL with frozen actions;
* the Matern kernels against scikit-learn's implementation when available.
"""
import math

import numpy as np
import pytest

import dense_ref
import oracle
import synth
from oracle import cakf as oc


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.max(np.abs(a - b)) / max(1e-300, np.max(np.abs(b))))


def test_scalar_kalman_closed_form():
    """n = 1: the CAKF reduces to the scalar Kalman filter (textbook recursion by hand)."""
    w = synth.small(n=1, m=1, T=7, budget_i=1, rank_r=0, seed=5)
    f = oracle.filter_run(w)
    lx, lt, sf2, sn2 = math.exp(w.log_lx), math.exp(w.log_lt), math.exp(w.log_sf2), math.exp(w.log_sn2)
    a = math.exp(-w.dt / lt)
    m, P = 0.0, sf2
    nll = 0.0
    for k in range(1, w.T + 1):
        mp, Pp = a * m, a * a * P + (1 - a * a) * sf2
        y = float(w.yk(k)[0])
        g = Pp + sn2
        m = mp + Pp / g * (y - mp)
        P = Pp - Pp * Pp / g
        nll += 0.5 * math.log(2 * math.pi * g) + 0.5 * (y - mp) ** 2 / g
        assert abs(f.m[k, 0] - m) < 1e-12 * max(1, abs(m))
        assert abs(f.var[k, 0] - P) < 1e-12
    assert abs(oracle.nll_total(f) - nll) < 1e-10 * abs(nll)


@pytest.mark.parametrize("kernel,seasonal", [(synth.MATERN32, True), (synth.MATERN52, False), (synth.MATERN12, False)])
def test_full_budget_equals_kf_rts(kernel, seasonal):
    """i_k = m_k, no truncation: CAKF/CAKS = dense KF/RTS (means, variances, NLL)."""
    w = synth.small(n=36, dim=1, m=9, T=6, budget_i=9, rank_r=0, kernel=kernel, seasonal=seasonal,
                    missing=(3,), seed=21)
    f = oracle.filter_run(w)
    ms, vs, _ = oracle.smoother_run(w, f)
    ref = dense_ref.kf_rts(w)
    assert rel(f.m, ref["mf"]) < 1e-9
    assert rel(f.var, ref["vf"]) < 1e-9
    assert rel(ms, ref["ms"]) < 1e-9
    assert rel(vs, ref["vs"]) < 1e-9
    assert np.allclose(f.nll, ref["nll"], rtol=1e-9, atol=1e-10)


@pytest.mark.parametrize("budget", [1, 3, 5])
def test_partial_budget_equals_batch_gp(budget):
    """Any budget, no truncation: filter at k = batch GP on data 1..k; smoother = batch GP on all
    data; sum of NLL terms = projected batch NLL."""
    w = synth.small(n=30, dim=2, m=10, T=5, budget_i=budget, rank_r=0, seasonal=True, seed=7)
    f = oracle.filter_run(w)
    ms, vs, _ = oracle.smoother_run(w, f)
    for k in range(1, w.T + 1):
        mb, vb, _ = dense_ref.batch_gp(w, f.S, upto=k, k_eval=k)
        assert rel(f.m[k], mb) < 1e-9
        assert rel(f.var[k], vb) < 1e-9
    for k in range(0, w.T + 1):
        mb, vb, nb = dense_ref.batch_gp(w, f.S, upto=w.T, k_eval=k)
        assert rel(ms[k], mb) < 1e-9, k
        assert rel(vs[k], vb) < 1e-9, k
    assert abs(oracle.nll_total(f) - nb) < 1e-9 * abs(nb)


def test_update_internal_identities():
    """V^T G V = I per step, CG actions mutually orthogonal, and the batch update (Alg. 2) with the
    recorded actions gives the same w and W W^T (Prop. on the equivalence of the two updates)."""
    w = synth.small(n=50, dim=2, m=15, T=4, budget_i=6, rank_r=0, seed=9)
    f = oracle.filter_run(w, keep_G=True)
    for k in range(1, w.T + 1):
        o = w.obs(k)
        V = f.W[k][o]
        G = f.G[k]
        assert np.allclose(V.T @ G @ V, np.eye(V.shape[1]), atol=1e-10)
        S = f.S[k]
        SS = S.T @ S
        assert np.allclose(SS - np.diag(np.diag(SS)), 0, atol=1e-9 * np.max(np.diag(SS)))
        Gh = S.T @ G @ S
        v_batch = S @ np.linalg.solve(Gh, S.T @ f.r0[k])
        assert rel(f.w[k][o], v_batch) < 1e-9
        assert rel(V @ V.T, S @ np.linalg.solve(Gh, S.T)) < 1e-9


def test_truncate_eckart_young():
    """Truncate keeps the best rank-r part: M+ M+^T equals the rank-r SVD truncation of M M^T and
    M M^T = M+ M+^T + N N^T with N N^T PSD (Sec. 3.2)."""
    rng = np.random.default_rng(3)
    M = rng.standard_normal((40, 12)) @ np.diag(np.logspace(0, -3, 12))
    Mp, U, lk, ld = oracle.truncate(M, 7)
    Us, s, _ = np.linalg.svd(M, full_matrices=False)
    best = (Us[:, :7] * s[:7] ** 2) @ Us[:, :7].T
    assert rel(Mp @ Mp.T, best) < 1e-12
    NN = M @ M.T - Mp @ Mp.T
    assert np.min(np.linalg.eigvalsh(NN)) > -1e-12
    assert np.allclose(np.sort(np.concatenate([lk, ld]))[::-1], s ** 2, rtol=1e-10)
    same, U2, _, _ = oracle.truncate(M, 12)
    assert U2 is None and same is M


def test_truncated_run_matches_dense_outer_product():
    """With truncation: oracle (factors, small Gram eig) = dense outer-product form (n x n eig)."""
    w = synth.small(n=34, dim=2, m=10, T=7, budget_i=4, rank_r=6, seasonal=True, seed=13)
    f = oracle.filter_run(w)
    ms, vs, _ = oracle.smoother_run(w, f)
    ref = dense_ref.dense_truncated(w, f.S, w.rank_r)
    assert rel(f.m, ref["mf"]) < 1e-9
    assert rel(f.var, ref["vf"]) < 1e-9
    assert rel(ms, ref["ms"]) < 1e-9
    assert rel(vs, ref["vs"]) < 1e-9


def test_truncation_is_conservative_and_rank_large_is_identity():
    """Same actions: truncation never lowers a marginal variance (Sec. 3.2, computational noise);
    a rank above the number of columns changes nothing."""
    w = synth.small(n=40, dim=2, m=12, T=6, budget_i=4, rank_r=5, seed=17)
    ft = oracle.filter_run(w)
    fu = oracle.filter_run(w, rank_r=0, S_replay=ft.S, U_replay=[None] * (w.T + 1))
    assert np.all(ft.var >= fu.var - 1e-12)
    mst, vst, _ = oracle.smoother_run(w, ft)
    msu, vsu, _ = oracle.smoother_run(w, fu, rank_r=0)
    assert np.all(vst >= vsu - 1e-12)
    fbig = oracle.filter_run(w, rank_r=10 ** 6)
    f0 = oracle.filter_run(w, rank_r=0)
    assert rel(fbig.var, f0.var) < 1e-14 and rel(fbig.m, f0.m) < 1e-14


def test_fd_gradient_matches_batch_analytic():
    """Central FD of the oracle NLL (frozen actions) = analytic gradient of the projected batch NLL."""
    w = synth.small(n=25, dim=2, m=8, T=4, budget_i=3, rank_r=0, seasonal=True, seed=19)
    nll, g_fd = oracle.nll_grad_fd(w, h=1e-5)
    f = oracle.filter_run(w)
    g_an = dense_ref.batch_nll_grad(w, f.S)
    assert np.allclose(g_fd, g_an, rtol=1e-6, atol=1e-6 * np.max(np.abs(g_an)))


def test_fd_gradient_with_truncation_matches_complex_step():
    """The oracle's truncated NLL with frozen actions and rotations (the U_replay path of
    filter_run), pinned by an independent factor-form implementation of the same modified model
    (batch update V = S L^-T, frozen M+_k = M_k U_k) differentiated by the complex step: its NLL
    at the base point equals the oracle's and its exact gradient equals the oracle's central FD.
    Truncation is active (rank 5 < 3 columns per step accumulated over 4 steps), so a rotation
    replayed at the wrong step changes the function and fails the comparison."""
    w = synth.small(n=30, dim=2, m=9, T=4, budget_i=3, rank_r=5, seasonal=True, seed=23)
    f = oracle.filter_run(w)
    assert sum(u is not None for u in f.U) >= 2
    nll0, g_fd = oracle.nll_grad_fd(w, h=1e-5)
    nll_ref, g_cs = dense_ref.frozen_truncated_nll_grad(w, f.S, f.U)
    assert abs(nll0 - nll_ref) <= 1e-10 * abs(nll_ref)
    assert np.allclose(g_fd, g_cs, rtol=1e-6, atol=1e-7 * np.max(np.abs(g_cs))), (g_fd, g_cs)
    # the rotation of the next step replayed in place of this one (same shape) is a different
    # model: its gradient moves visibly (the last step's rotation feeds no NLL term, so a later
    # step's is taken for an earlier one)
    shifted = list(f.U)
    for k in range(1, w.T):
        if f.U[k] is not None and f.U[k + 1] is not None and f.U[k].shape == f.U[k + 1].shape:
            shifted[k] = f.U[k + 1]
            break
    assert any(shifted[k] is not f.U[k] for k in range(1, w.T + 1))
    _, g_bad = dense_ref.frozen_truncated_nll_grad(w, f.S, shifted)
    assert not np.allclose(g_bad, g_cs, rtol=1e-4)


def test_breakdown_exit_stops_at_a_repeated_action():
    """A replayed action that repeats an earlier one has d = (I - V V^T G) s = 0, so eta falls
    below 1e-12 s^T G s: the update stops there (R2), keeps only the actions before it, and the
    result equals the run given just those actions."""
    w = synth.small(n=40, dim=2, m=12, T=2, budget_i=4, rank_r=0, seed=29)
    base = oracle.filter_run(w)
    s1, s2 = base.S[1][:, 0], base.S[1][:, 1]
    rep = [None, np.stack([s1, s2, s1, base.S[1][:, 2]], axis=1), base.S[2]]
    f = oracle.filter_run(w, S_replay=rep)
    assert f.iters[1] == 2 and f.iters[2] == base.S[2].shape[1]
    g = oracle.filter_run(w, S_replay=[None, np.stack([s1, s2], axis=1), base.S[2]])
    assert np.array_equal(f.m, g.m) and np.array_equal(f.var, g.var)
    assert f.nll[1] == g.nll[1]


def test_coordinate_policy_is_exact_conditioning_on_the_chosen_points():
    """Batch update (Alg. 2) with coordinate actions: conditioning on the chosen subset of each
    step's observations exactly, so without truncation it equals the dense Kalman filter / RTS
    smoother run on the data of those points only (means, variances, NLL terms); with i = m it is the
    full Kalman filter."""
    w = synth.small(n=60, dim=2, m=14, T=4, budget_i=5, rank_r=0, seasonal=True, seed=51)
    f = oracle.filter_run(w, policy="coordinate")
    ms, vs, _ = oracle.smoother_run(w, f)
    # the workload restricted to the coordinates the policy picks
    idx, ys, ptr = [], [], [0]
    for k in range(1, w.T + 1):
        o, yk = w.obs(k), w.yk(k)
        pos = np.nonzero(oracle.coordinate_actions(len(o), w.budget_i).sum(axis=1))[0]
        idx.append(o[pos]); ys.append(yk[pos]); ptr.append(ptr[-1] + len(pos))
    sub = w.with_(obs_idx=np.concatenate(idx).astype(np.int32), y=np.concatenate(ys),
                  obs_ptr=np.array(ptr, dtype=np.int32))
    ref = dense_ref.kf_rts(sub)
    for got, exp in ((f.m, ref["mf"]), (f.var, ref["vf"]), (ms, ref["ms"]), (vs, ref["vs"])):
        assert rel(got, exp) < 1e-9
    assert np.allclose(f.nll, ref["nll"], rtol=1e-9, atol=1e-12)
    full = oracle.filter_run(w.with_(budget_i=w.n), policy="coordinate")
    kf = dense_ref.kf_rts(w)
    assert rel(full.m, kf["mf"]) < 1e-9 and rel(full.var, kf["vf"]) < 1e-9


def test_batch_update_equals_iterative_update_with_the_same_actions():
    """Alg. 2 and the iterative update give the same filter (and NLL) for the same actions (the
    paper's proposition on their equivalence): Gaussian actions drawn once, truncation active."""
    w = synth.small(n=70, dim=2, m=16, T=5, budget_i=6, rank_r=10, seed=52)
    S = synth.gaussian_actions(w, seed=7)
    fb = oracle.filter_run(w, policy="given", S_given=S)
    fi = oracle.filter_run(w, S_replay=S)
    assert rel(fb.m, fi.m) < 1e-9 and rel(fb.var, fi.var) < 1e-9
    assert np.allclose(fb.nll, fi.nll, rtol=1e-9, atol=1e-12)
    mb, vb, _ = oracle.smoother_run(w, fb)
    mi, vi, _ = oracle.smoother_run(w, fi)
    assert rel(mb, mi) < 1e-9 and rel(vb, vi) < 1e-9


def test_sampler_without_noise_returns_the_posterior_means():
    """The sampler's recursions with the prior mean as initial draw and no dynamics or observation
    noise are the filter's and the smoother's mean recursions (Matheron's rule at zero noise)."""
    w = synth.small(n=60, dim=2, m=15, T=5, budget_i=4, rank_r=7, seasonal=True, seed=53)
    f = oracle.filter_run(w)
    ms, _, _ = oracle.smoother_run(w, f)
    x0 = w.prior_mean[0][:, None].copy()
    q = [np.zeros((w.n, 1))] * (w.T + 1)
    eps = [np.zeros((int(w.obs_ptr[k] - w.obs_ptr[k - 1]) if k else 0, 1)) for k in range(w.T + 1)]
    xf, xs = oracle.sample_run(w, f, x0, q, eps)
    assert rel(xf[:, :, 0], f.m) < 1e-12
    assert rel(xs[:, :, 0], ms) < 1e-11


def test_sampler_at_full_budget_is_exact_matheron():
    """At full budget without truncation the modified model is the original one, so each draw is
    Matheron's rule for the space-time GP: x_prior + C(x, z) (C(z, z) + sn2 I)^-1 (y - x_prior[z] - eps),
    with the prior trajectory x_prior built from the same x0 and dynamics noise; the filter draw of
    step k conditions on the data of steps 1..k only."""
    w = synth.small(n=30, dim=2, m=8, T=4, budget_i=8, rank_r=0, seasonal=True, seed=54)
    f = oracle.filter_run(w)
    x0, q, eps = synth.sampler_inputs(w, 3, seed=9)
    xf, xs = oracle.sample_run(w, f, x0, q, eps)
    m = oracle.model_from(w)
    xp = [x0]
    for k in range(1, w.T + 1):
        xp.append(m.a * xp[-1] + m.b(k)[:, None] + q[k])
    K = oracle.kernel_matrix(w.coords, w.coords, w.kernel, m.lx, m.sf2)
    for upto in range(1, w.T + 1):
        steps = np.concatenate([np.full(len(w.obs(k)), k) for k in range(1, upto + 1)])
        idx = np.concatenate([w.obs(k) for k in range(1, upto + 1)])
        Czz = (m.a ** np.abs(steps[:, None] - steps[None, :])) * K[np.ix_(idx, idx)] + m.sn2 * np.eye(idx.size)
        d = np.concatenate([w.yk(k)[:, None] - xp[k][w.obs(k)] - eps[k] for k in range(1, upto + 1)])
        sol = np.linalg.solve(Czz, d)
        kk = range(0, upto + 1) if upto == w.T else [upto]
        for k in kk:
            exact = xp[k] + ((m.a ** np.abs(k - steps))[None, :] * K[:, idx]) @ sol
            got = xs[k] if upto == w.T else xf[k]
            assert rel(got, exact) < 1e-9, (upto, k)


def test_interpolation_at_full_budget_is_the_exact_gp_posterior():
    """Filter and smoother marginals at times between the steps (interpolation corollary) equal the
    exact space-time GP posterior at those times when the budget is full and nothing is truncated:
    the filter conditions on the data up to the last step before t, the smoother on all data.  The
    seasonal prior mean is evaluated at the query times.  At the step times themselves the
    interpolation returns the filter and smoother outputs."""
    w = synth.small(n=30, dim=2, m=8, T=4, budget_i=8, rank_r=0, seasonal=True, seed=55)
    f = oracle.filter_run(w)
    Wm, wm = oracle.smoother_messages(w, f)
    m = oracle.model_from(w)
    tq = np.array([0.03, 0.1, 0.17, 0.25, 0.31, 0.399, 0.4, 0.47])
    mu_q = np.stack([0.5 * np.sin(2 * np.pi * t / 5.0) * np.cos(2 * np.pi * w.coords[:, 0]) for t in tq])
    mf, vf, ms, vs = oracle.interpolate_run(w, f, Wm, wm, tq, mu_q=mu_q)
    K = oracle.kernel_matrix(w.coords, w.coords, w.kernel, m.lx, m.sf2)
    lt = math.exp(w.log_lt)
    for q, t in enumerate(tq):
        k = min(int(np.floor(t / w.dt + 1e-12)), w.T)
        for upto, gm, gv in ((k, mf[q], vf[q]), (w.T, ms[q], vs[q])):
            if upto == 0:
                exp_m, exp_v = mu_q[q], np.diag(K)
            else:
                st = np.concatenate([np.full(len(w.obs(j)), j) for j in range(1, upto + 1)])
                ix = np.concatenate([w.obs(j) for j in range(1, upto + 1)])
                Czz = np.exp(-np.abs(st[:, None] - st[None, :]) * w.dt / lt) * K[np.ix_(ix, ix)] \
                    + m.sn2 * np.eye(ix.size)
                Ctz = np.exp(-np.abs(t - st * w.dt) / lt)[None, :] * K[:, ix]
                resid = np.concatenate([w.yk(j) - w.prior_mean[j][w.obs(j)] for j in range(1, upto + 1)])
                exp_m = mu_q[q] + Ctz @ np.linalg.solve(Czz, resid)
                exp_v = np.diag(K) - np.einsum("ij,ji->i", Ctz, np.linalg.solve(Czz, Ctz.T))
            assert rel(gm, exp_m) < 1e-9, (t, upto)
            assert rel(gv, exp_v) < 1e-9, (t, upto)
    # at the step times the interpolation is the filter / smoother output
    ms_o, vs_o, _ = oracle.smoother_run(w, f)
    tk = np.arange(w.T + 1) * w.dt
    o = oracle.interpolate_run(w, f, Wm, wm, tk, mu_q=w.prior_mean)
    assert rel(o[0], f.m) < 1e-13 and rel(o[2], ms_o) < 1e-13 and rel(o[3], vs_o) < 1e-13


def test_matern_against_sklearn():
    sk = pytest.importorskip("sklearn.gaussian_process.kernels")
    rng = np.random.default_rng(0)
    X = rng.uniform(size=(20, 3))
    for code, nu in [(0, 0.5), (1, 1.5), (2, 2.5)]:
        ours = oracle.kernel_matrix(X, X, code, 0.37, 1.0)
        ref = sk.Matern(length_scale=0.37, nu=nu)(X)
        assert np.allclose(ours, ref, rtol=1e-12, atol=1e-14)


def test_pins_catch_planted_mistakes(monkeypatch):
    """A dropped term in the kernel, or a wrong smoother sign, makes the pins fail."""
    w = synth.small(n=20, dim=1, m=6, T=4, budget_i=6, rank_r=0, seed=23)
    ref = dense_ref.kf_rts(w)

    def bad_matern(u, kernel):
        return np.exp(-math.sqrt(3.0) * u)          # Matern-3/2 without its (1 + sqrt(3) u) factor
    monkeypatch.setattr(oc, "matern", bad_matern)
    f = oracle.filter_run(w)
    assert rel(f.m, ref["mf"]) > 1e-3
    monkeypatch.undo()

    orig = oc.Model.K_times

    def sign_flip(self, B, rows=None, cols=None):
        out = orig(self, B, rows, cols)
        return -out if (rows is None and cols is None) else out   # only the smoother's K X products
    monkeypatch.setattr(oc.Model, "K_times", sign_flip)
    f = oracle.filter_run(w)
    ms, vs, _ = oracle.smoother_run(w, f)
    assert rel(vs, ref["vs"]) > 1e-3


def test_smoother_kernel_products_follow_the_recursion():
    """Alg. 3 needs P^-_k X with X = a [Ws ws]; its expensive part K X can be carried through the
    smoother's own linear recursion: every column of [Ws ws] is a combination of earlier [Ws ws]
    columns and of the filter's W_k = H^T V_k, so K [Ws ws] obeys the same recursion with K W_k in
    place of W_k.  Checked here in FP64 against K applied directly, step by step (truncation
    included), on the oracle's own filter run."""
    w = synth.small(n=150, dim=2, m=30, T=6, budget_i=6, rank_r=14, seed=51)
    model = oc.model_from(w)
    f = oracle.filter_run(w)
    a, T = model.a, w.T
    Ws, ws = f.W[T], f.w[T]
    KWs, Kws = model.K_times(Ws), model.K_times(ws)
    for k in range(T - 1, 0, -1):
        X = a * np.concatenate([Ws, ws[:, None]], axis=1)
        KX = a * np.concatenate([KWs, Kws[:, None]], axis=1)            # recursion, no K evaluation
        assert rel(KX, model.K_times(X)) < 1e-11
        Mp = f.M_pred[k]
        PmX = KX - Mp @ (Mp.T @ X)
        Wk = f.W[k]
        KWk, Kwk = model.K_times(Wk), model.K_times(f.w[k])            # the filter's stored products
        Z = Wk.T @ PmX
        Y2 = X - Wk @ Z
        KY2 = KX - KWk @ Z
        ws, Kws = f.w[k] + Y2[:, -1], Kwk + KY2[:, -1]
        Wfull = np.concatenate([Wk, Y2[:, :-1]], axis=1)
        KWfull = np.concatenate([KWk, KY2[:, :-1]], axis=1)
        Ws, U, _, _ = oc.truncate(Wfull, w.rank_r)
        KWs = KWfull if U is None else KWfull @ U
        assert rel(KWs, model.K_times(Ws)) < 1e-11
        assert rel(Kws, model.K_times(ws)) < 1e-11


def test_cg_policy_is_krylov_galerkin_and_rtol_stops_at_the_first_small_residual():
    """With the CG policy (action = current residual) the actions span the Krylov space
    K_j(G, r0), so the update's coefficient vector after j actions is the Galerkin solution of
    G v = r0 on that space (the exact conjugate-gradient iterate) and the filter mean is
    m^- + K(X, X_o) v_j; with cg_rtol the step stops at the first j whose residual norm is at most
    cg_rtol ||r0|| (reading R2).  Reference: an orthonormal Krylov basis built with full
    re-orthogonalisation and the projected solve (textbook CG recurrences lose orthogonality after
    a dozen iterations here and would not be an FP64 reference)."""
    w = synth.small(n=80, dim=2, m=24, T=1, budget_i=24, rank_r=0, seed=52)
    model = oc.model_from(w)
    obs = w.obs(1)
    G = model.K_times(np.eye(len(obs)), rows=obs, cols=obs) + model.sn2 * np.eye(len(obs))
    mp = model.a * model.m0()
    r0 = w.yk(1) - mp[obs]
    r0n = np.linalg.norm(r0)
    Q = np.zeros((len(obs), 0))
    q = r0 / r0n
    xs, norms = [np.zeros_like(r0)], [r0n]
    for _ in range(len(obs) - 4):
        Q = np.concatenate([Q, q[:, None]], axis=1)
        x = Q @ np.linalg.solve(Q.T @ G @ Q, Q.T @ r0)
        xs.append(x)
        norms.append(np.linalg.norm(r0 - G @ x))
        z = G @ q
        for _ in range(2):
            z = z - Q @ (Q.T @ z)
        q = z / np.linalg.norm(z)
    for rtol in (1e-1, 1e-3):
        j = next(k for k, nr in enumerate(norms) if nr <= rtol * r0n)
        f = oracle.filter_run(w, cg_rtol=rtol)
        assert f.iters[1] == j, (rtol, f.iters[1], j)
        want = mp + model.K_times(xs[j], cols=obs)
        assert rel(f.m[1], want) < 1e-9
