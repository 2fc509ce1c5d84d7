"""The posterior sampler (cakf_sample) against the oracle's sampler on identical random inputs.

The draws are deterministic functions of the inputs (initial draw, dynamics noise, observation
noise), so they are compared elementwise: FP64 within 1e-10 (normwise per step and draw), FP32 and
split FP16 within 1e-3.  Truncation is active, steps without data are included, and the factors
are also restored by recomputation (CAKF_RECOMPUTE) for the sampler's passes.
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


def draw_err(got, ref):
    err = 0.0
    for k in range(ref.shape[0]):
        for s in range(ref.shape[2]):
            err = max(err, float(np.linalg.norm(got[k, :, s] - ref[k, :, s]) / np.linalg.norm(ref[k, :, s])))
    return err


CASES = {
    "grid2d-trunc": lambda: synth.small(n=600, dim=2, m=120, T=6, budget_i=10, rank_r=30, seasonal=True, seed=91),
    "missing-m12": lambda: synth.small(n=200, dim=1, m=40, T=7, budget_i=6, rank_r=14, seed=92,
                                       kernel=synth.MATERN12, missing=(2, 5)),
}


@pytest.mark.parametrize("storage", ["fp32", "recompute"])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("fp32", 1e-3), ("fp16x3", 1e-3)])
@pytest.mark.parametrize("name", list(CASES))
def test_sampler_against_oracle(name, precision, tol, storage):
    w = CASES[name]()
    f = oracle.filter_run(w)
    x0, q, eps = synth.sampler_inputs(w, 3, seed=13)
    xf_o, xs_o = oracle.sample_run(w, f, x0, q, eps)
    flat, counts = ck.pack_actions(f.S, w.T)
    prob = ck.problem_from_workload(w, precision=precision, replay=(flat, counts), factor_storage=storage,
                                    checkpoint_every=3)
    ctx, _, _ = ck.cakf_filter(prob)
    xf, xs = ck.cakf_sample(ctx, x0, q, eps, w.obs_ptr)
    ctx.close()
    ef, es = draw_err(xf, xf_o), draw_err(xs, xs_o)
    print(name, precision, storage, f"filter draws {ef:.2e} smoother draws {es:.2e}")
    assert ef < tol and es < tol


def test_sampler_without_noise_gives_the_means():
    w = CASES["grid2d-trunc"]()
    prob = ck.problem_from_workload(w, precision="fp64")
    ctx, mf, _ = ck.cakf_filter(prob)
    ms, _ = ck.cakf_smooth(ctx)
    x0 = w.prior_mean[0][:, None]
    q = [np.zeros((w.n, 1))] * (w.T + 1)
    eps = [np.zeros((int(w.obs_ptr[k] - w.obs_ptr[k - 1]) if k else 0, 1)) for k in range(w.T + 1)]
    xf, xs = ck.cakf_sample(ctx, x0, q, eps, w.obs_ptr)
    ctx.close()
    assert np.max(np.abs(xf[:, :, 0] - mf)) < 1e-10 * np.max(np.abs(mf))
    assert np.max(np.abs(xs[:, :, 0] - ms)) < 1e-10 * np.max(np.abs(ms))
