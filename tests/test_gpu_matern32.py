"""The Matern-3/2 temporal factor (D' = 2: values and time derivatives at every grid point, state
dimension 2n) on the device against the FP64 oracle on identical seeded inputs.

The outputs are the positions' marginals (the oracle's first n state entries).  Tolerances as in
test_gpu_parity: FP64 within 1e-10 (means normwise per step, variances elementwise, NLL); the
FP32 and split tensor-core modes replay the oracle's actions (the same projected model) and are
held to 1e-3.  Cases cover truncation (filter 576 -> r style, here small), a ragged n (not a
multiple of the 128-row blocks), a step without data, the coordinate policy, and full size
(n = 65,536, a 131,072-dimensional state) for three steps against the device FP64 mode.
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
    scale = max(float(np.linalg.norm(ref[k])) for k in range(ref.shape[0]))
    return max(float(np.linalg.norm(got[k] - ref[k]) / (np.linalg.norm(ref[k]) or scale)) for k in range(ref.shape[0]))


def var_err(got, ref):
    return float(np.max(np.abs(got - ref) / np.abs(ref)))


CASES = {
    "trunc-seasonal": lambda: synth.small(n=500, dim=2, m=100, T=6, budget_i=10, rank_r=30, seasonal=True,
                                          seed=201, temporal=1),
    "ragged-missing-no-trunc": lambda: synth.small(n=333, dim=2, m=60, T=6, budget_i=8, rank_r=0, missing=(3,),
                                                   seed=202, temporal=1, lt=0.4),
    "sphere-trunc-m52": lambda: synth.small(n=640, m=120, T=5, budget_i=12, rank_r=24, sphere=True, lx=0.4,
                                            kernel=synth.MATERN52, seed=203, temporal=1),
}


def oracle_run(w, **kw):
    f = oracle.filter_run(w, **kw)
    ms, vs, _ = oracle.smoother_run(w, f)
    n = w.n
    return dict(mf=f.m[:, :n], vf=f.var[:, :n], ms=ms[:, :n], vs=vs[:, :n], nll=oracle.nll_total(f), f=f)


def gpu_run(w, precision, **kw):
    prob = ck.problem_from_workload(w, precision=precision, **kw)
    ctx, mf, vf = ck.cakf_filter(prob)
    ms, vs = ck.cakf_smooth(ctx)
    nll = ck.cakf_nll(ctx)
    ctx.close()
    return dict(mf=mf, vf=vf, ms=ms, vs=vs, nll=nll)


def errors(got, ref):
    return [mean_err(got["mf"], ref["mf"]), var_err(got["vf"], ref["vf"]), mean_err(got["ms"], ref["ms"]),
            var_err(got["vs"], ref["vs"]), abs(got["nll"] - ref["nll"]) / abs(ref["nll"])]


@pytest.mark.parametrize("case", list(CASES))
def test_fp64_against_oracle(case):
    w = CASES[case]()
    ref = oracle_run(w)
    got = gpu_run(w, "fp64")
    e = errors(got, ref)
    print(case, "fp64", [f"{v:.2e}" for v in e])
    assert max(e) < 1e-10, e


@pytest.mark.parametrize("precision", ["fp32", "fp16x3", "tf32x3"])
@pytest.mark.parametrize("case", list(CASES))
def test_mixed_modes_with_the_oracle_actions(case, precision):
    w = CASES[case]()
    ref = oracle_run(w)
    flat, counts = ck.pack_actions(ref["f"].S, w.T)
    got = gpu_run(w, precision, replay=(flat, counts))
    e = errors(got, ref)
    print(case, precision, [f"{v:.2e}" for v in e])
    tol = 3e-3 if precision == "tf32x3" else 1e-3
    assert max(e) < tol, e


def test_coordinate_policy_fp64():
    w = CASES["trunc-seasonal"]()
    ref = oracle_run(w, policy="coordinate")
    got = gpu_run(w, "fp64", policy="coordinate")
    e = errors(got, ref)
    assert max(e) < 1e-10, e


def test_ou_path_unchanged_by_the_temporal_field():
    """temporal = 0 on a Matern-3/2-generated workload runs the OU model the oracle runs with
    temporal = 0."""
    w = CASES["trunc-seasonal"]().with_(temporal=0)
    ref = oracle_run(w)
    got = gpu_run(w, "fp64")
    assert max(errors(got, ref)) < 1e-10


def test_unsupported_calls_are_rejected():
    w = synth.small(n=100, dim=2, m=20, T=3, budget_i=4, rank_r=8, seed=204, temporal=1)
    ctx, _, _ = ck.cakf_filter(ck.problem_from_workload(w, precision="fp32"))
    with pytest.raises(ck.CakfError) as ei:
        ck.cakf_nll_backward(ctx)
    assert ei.value.code == ck.binding.ERR_ARG
    ctx.close()
    with pytest.raises(ck.CakfError) as ei:
        ck.cakf_filter(ck.problem_from_workload(w, precision="fp32", factor_storage="bf16", checkpoint_every=2))
    assert ei.value.code == ck.binding.ERR_ARG


def test_sphere65k_three_steps_against_fp64_mode():
    """n = 65,536 (state 131,072), m = 8,192, i = 64: the split-FP16 mode with the FP64 mode's
    actions replayed against the FP64 mode, filter and smoother over three steps."""
    w = synth.sphere_65k(T=3, temporal=1, device="cuda")
    ref = gpu_run(w, "fp64")
    prob = ck.problem_from_workload(w, precision="fp64")
    ctx, _, _ = ck.cakf_filter(prob)
    acts, counts = ck.cakf_get_actions(ctx, w.obs_ptr)
    ctx.close()
    flat, cnt = ck.pack_actions(acts, w.T)
    got = gpu_run(w, "fp16x3", replay=(flat, cnt))
    e = errors(got, ref)
    print("sphere65k m32 fp16x3 vs fp64", [f"{v:.2e}" for v in e])
    assert max(e) < 1e-3, e
