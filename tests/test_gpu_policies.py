"""Block policies (the batch update, Alg. 2) through the C ABI against the oracle.

* CAKF_POLICY_COORDINATE: unit-vector actions at a space-filling subset of each step's observations
  (the oracle's coordinate_actions, reading R18), projected Gram S^T G S from one Gram x block
  product K(X_o, X_o)[S r0] (tensor cores in the tensor-core modes), Cholesky in FP64.
* CAKF_POLICY_BATCH: the same update with given actions (Gaussian sketches drawn once by
  synth.gaussian_actions and passed to both sides).
Tolerances as in test_gpu_parity: FP64 1e-10; FP32 and split FP16 1e-3 (means normwise per step,
variances elementwise, NLL).  The gradient of the NLL with the batch policy's frozen actions is
checked against central differences of the oracle's frozen-action NLL (1e-6).
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2405_08971_gb300 as ck  # noqa: E402


def mean_err(got, ref):
    return max(float(np.linalg.norm(got[k] - ref[k]) / np.linalg.norm(ref[k])) for k in range(ref.shape[0])
               if np.linalg.norm(ref[k]) > 0)


def var_err(got, ref):
    return float(np.max(np.abs(got - ref) / np.abs(ref)))


def errors(got, f, ms, vs):
    return dict(mf=mean_err(got["mf"], f.m), vf=var_err(got["vf"], f.var), ms=mean_err(got["ms"], ms),
                vs=var_err(got["vs"], vs), nll=abs(got["nll"] - oracle.nll_total(f)) / abs(oracle.nll_total(f)))


def run_gpu(w, precision, policy, actions=None):
    replay = None if actions is None else ck.pack_actions(actions, w.T)
    prob = ck.problem_from_workload(w, precision=precision, policy=policy, replay=replay)
    ctx, mf, vf = ck.cakf_filter(prob)
    ms, vs = ck.cakf_smooth(ctx)
    out = dict(mf=mf, vf=vf, ms=ms, vs=vs, nll=ck.cakf_nll(ctx), stats=ck.cakf_get_stats(ctx))
    out["S"], out["counts"] = ck.cakf_get_actions(ctx, w.obs_ptr)
    ctx.close()
    return out


CASES = {
    "grid2d-trunc": lambda: synth.small(n=900, dim=2, m=200, T=6, budget_i=24, rank_r=60, seed=71, seasonal=True),
    "sphere-trunc": lambda: synth.small(n=700, m=150, T=5, budget_i=16, rank_r=40, seed=72, sphere=True, lx=0.4),
    "missing-m52": lambda: synth.small(n=300, dim=1, m=40, T=6, budget_i=8, rank_r=20, seed=73,
                                       kernel=synth.MATERN52, missing=(2, 4)),
    "one-obs": lambda: synth.small(n=50, dim=2, m=1, T=3, budget_i=4, rank_r=2, seed=74),
}


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("fp32", 1e-3), ("fp16x3", 1e-3)])
@pytest.mark.parametrize("name", list(CASES))
def test_coordinate_policy_against_oracle(name, precision, tol):
    w = CASES[name]()
    f = oracle.filter_run(w, policy="coordinate")
    ms, vs, _ = oracle.smoother_run(w, f)
    got = run_gpu(w, precision, "coordinate")
    e = errors(got, f, ms, vs)
    print(name, precision, {k: f"{v:.2e}" for k, v in e.items()})
    assert np.array_equal(got["counts"][1:], f.iters[1:])
    for k in range(1, w.T + 1):     # the same unit vectors
        if f.S[k].size:
            assert np.array_equal(got["S"][k], f.S[k])
    for k, v in e.items():
        assert v < tol, (k, v)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("fp16x3", 1e-3)])
def test_batch_policy_with_gaussian_actions(precision, tol):
    w = CASES["grid2d-trunc"]()
    S = synth.gaussian_actions(w, seed=5)
    f = oracle.filter_run(w, policy="given", S_given=S)
    ms, vs, _ = oracle.smoother_run(w, f)
    got = run_gpu(w, precision, "batch", actions=S)
    e = errors(got, f, ms, vs)
    print("gaussian", precision, {k: f"{v:.2e}" for k, v in e.items()})
    for k, v in e.items():
        assert v < tol, (k, v)


def test_coordinate_policy_gradient_against_frozen_fd():
    w = synth.small(n=150, dim=2, m=40, T=4, budget_i=8, rank_r=14, seed=75, seasonal=True)
    base = oracle.filter_run(w, policy="coordinate")
    theta0 = np.array([w.log_lx, w.log_lt, w.log_sf2, w.log_sn2])
    h, g_fd = 1e-5, np.zeros(4)
    for p in range(4):
        vals = []
        for sgn in (1, -1):
            th = theta0.copy()
            th[p] += sgn * h
            fk = oracle.filter_run(w, model=oracle.model_from(w, *th), S_replay=base.S, U_replay=base.U)
            vals.append(oracle.nll_total(fk))
        g_fd[p] = (vals[0] - vals[1]) / (2 * h)
    prob = ck.problem_from_workload(w, precision="fp64", policy="coordinate")
    ctx, _, _ = ck.cakf_filter(prob, want_outputs=False)
    g = ck.cakf_nll_backward(ctx)
    ctx.close()
    print("coordinate gradient fd", g_fd, "gpu", g)
    assert np.max(np.abs(g - g_fd)) < 1e-6 * np.max(np.abs(g_fd))


def test_coordinate_policy_sphere65k_three_steps():
    """The 65,536-state workload with the coordinate policy: split FP16 against the device FP64 mode
    over three steps (1e-3); the projected Gram comes from one Gram x block launch per step."""
    w = synth.sphere_65k(T=3)
    ref = run_gpu(w, "fp64", "coordinate")
    got = run_gpu(w, "fp16x3", "coordinate")
    e = dict(mf=mean_err(got["mf"][1:], ref["mf"][1:]), vf=var_err(got["vf"], ref["vf"]),
             ms=mean_err(got["ms"], ref["ms"]), vs=var_err(got["vs"], ref["vs"]),
             nll=abs(got["nll"] - ref["nll"]) / abs(ref["nll"]))
    print("65k coordinate", {k: f"{v:.2e}" for k, v in e.items()})
    for k, v in e.items():
        assert v < 1e-3, (k, v)


def test_policy_arguments_are_validated():
    w = synth.small(n=50, dim=2, m=10, T=2, budget_i=3, rank_r=4, seed=76)
    for kw in (dict(policy="batch"), dict(policy=9), dict(policy="coordinate", budget_i=161)):
        with pytest.raises(ck.CakfError) as ei:
            ck.cakf_filter(ck.problem_from_workload(w, precision="fp32", **kw))
        assert ei.value.code == ck.binding.ERR_ARG
