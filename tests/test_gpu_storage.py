"""Factor storage between the filter and the smoother / gradient pass (cakf_problem.factor_storage).

* CAKF_RECOMPUTE keeps only M+_k (and its eigenvalues) every checkpoint_every steps plus the actions
  of every step; the smoother and the gradient pass re-run each filter segment with the stored
  actions.  The same kernels on the same inputs give the same factors, so every output -- filter,
  smoother, NLL, gradient -- must equal the all-resident run exactly (bit for bit), in every
  precision, for segment lengths that do and do not divide T.
* CAKF_STORE_BF16 keeps BF16 copies of every step's factors: the filter outputs are untouched, the
  smoother reads factors rounded to 8 significant bits, which moves its outputs by up to a few
  1e-2 relative on these ill-conditioned cases (bounds below); the context holds fewer bytes.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2405_08971_gb300 as ck  # noqa: E402


def run(w, precision, storage, every=0, grad=True):
    prob = ck.problem_from_workload(w, precision=precision, factor_storage=storage, checkpoint_every=every)
    ctx, mf, vf = ck.cakf_filter(prob)
    ms, vs = ck.cakf_smooth(ctx)
    out = dict(mf=mf, vf=vf, ms=ms, vs=vs, nll=ck.cakf_nll(ctx))
    if grad:
        out["g"] = ck.cakf_nll_backward(ctx)
    out["bytes"] = ck.cakf_get_stats(ctx)["device_bytes"]
    ctx.close()
    return out


CASE = dict(n=600, dim=2, m=120, T=11, budget_i=8, rank_r=30, seasonal=True, seed=61)


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16x3"])
@pytest.mark.parametrize("every", [1, 3, 7])
def test_recompute_reproduces_the_resident_run(precision, every):
    w = synth.small(**CASE)
    ref = run(w, precision, "fp32")
    got = run(w, precision, "recompute", every)
    for key in ("mf", "vf", "ms", "vs"):
        assert np.array_equal(got[key], ref[key]), key
    assert got["nll"] == ref["nll"]
    assert np.array_equal(got["g"], ref["g"])
    assert got["bytes"] < ref["bytes"]


def test_recompute_with_missing_steps_and_no_truncation():
    w = synth.small(n=200, dim=1, m=40, T=9, budget_i=6, rank_r=0, seed=62, kernel=synth.MATERN12, missing=(2, 5))
    ref = run(w, "fp32", "fp32")
    got = run(w, "fp32", "recompute", 4)
    for key in ("mf", "vf", "ms", "vs", "g"):
        assert np.array_equal(got[key], ref[key]), key


def test_bf16_store_moves_only_the_smoother():
    w = synth.small(**CASE)
    ref = run(w, "fp16x3", "fp32", grad=False)
    got = run(w, "fp16x3", "bf16", 4, grad=False)
    assert np.array_equal(got["mf"], ref["mf"]) and np.array_equal(got["vf"], ref["vf"])
    assert got["nll"] == ref["nll"]
    em = max(np.linalg.norm(got["ms"][k] - ref["ms"][k]) / np.linalg.norm(ref["ms"][k]) for k in range(w.T + 1))
    ev = float(np.max(np.abs(got["vs"] - ref["vs"]) / ref["vs"]))
    print(f"bf16 store: smoother mean {em:.2e} variance {ev:.2e}")
    assert em < 2e-2 and ev < 5e-2
    assert np.all(np.isfinite(got["vs"])) and np.all(got["vs"] > 0)
    assert got["bytes"] < ref["bytes"]


def test_storage_arguments_are_validated():
    w = synth.small(n=50, dim=2, m=10, T=3, budget_i=3, rank_r=4, seed=63)
    for kw in (dict(precision="fp64", factor_storage="bf16"), dict(precision="fp32", factor_storage=7),
               dict(precision="fp32", factor_storage="recompute", checkpoint_every=-1)):
        with pytest.raises(ck.CakfError) as ei:
            ck.cakf_filter(ck.problem_from_workload(w, **kw))
        assert ei.value.code == ck.binding.ERR_ARG
