"""Temporal interpolation (cakf_interpolate) against the oracle's interpolation on identical inputs.

Queries fall inside the steps' intervals, on the steps themselves, before the first observation
and after the last step.  FP64 within 1e-10 (means normwise per query, variances elementwise), the
FP32 and split-FP16 modes (with the oracle's actions replayed: the same projected model) within
1e-3.  The seasonal prior mean is passed at the query times.
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
    # normwise per query; a query whose mean is exactly zero (the seasonal prior mean vanishes at
    # t = 0, before any observation) is measured against the largest query norm instead
    scale = max(float(np.linalg.norm(ref[q])) for q in range(ref.shape[0]))
    return max(float(np.linalg.norm(got[q] - ref[q]) / (np.linalg.norm(ref[q]) or scale))
               for q in range(ref.shape[0]))


def var_err(got, ref):
    return float(np.max(np.abs(got - ref) / np.abs(ref)))


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("fp32", 1e-3), ("fp16x3", 1e-3)])
@pytest.mark.parametrize("storage", ["fp32", "recompute"])
def test_interpolation_against_oracle(precision, tol, storage):
    w = synth.small(n=500, dim=2, m=100, T=6, budget_i=10, rank_r=30, seasonal=True, seed=101)
    f = oracle.filter_run(w)
    Wm, wm = oracle.smoother_messages(w, f)
    tq = np.array([0.0, 0.04, 0.1, 0.13, 0.25, 0.33, 0.5, 0.59, 0.6, 0.75])
    mu_q = np.stack([0.5 * np.sin(2 * np.pi * t / 5.0) * np.cos(2 * np.pi * w.coords[:, 0]) for t in tq])
    ref = oracle.interpolate_run(w, f, Wm, wm, tq, mu_q=mu_q)
    flat, counts = ck.pack_actions(f.S, w.T)
    prob = ck.problem_from_workload(w, precision=precision, replay=(flat, counts), factor_storage=storage,
                                    checkpoint_every=4)
    ctx, _, _ = ck.cakf_filter(prob)
    got = ck.cakf_interpolate(ctx, tq, mu_q=mu_q)
    ctx.close()
    e = [mean_err(got[0], ref[0]), var_err(got[1], ref[1]), mean_err(got[2], ref[2]), var_err(got[3], ref[3])]
    print(precision, storage, [f"{v:.2e}" for v in e])
    assert max(e) < tol, e


def test_interpolation_needs_the_prior_mean_at_the_queries():
    w = synth.small(n=100, dim=2, m=20, T=3, budget_i=4, rank_r=8, seasonal=True, seed=102)
    ctx, _, _ = ck.cakf_filter(ck.problem_from_workload(w, precision="fp32"))
    with pytest.raises(ck.CakfError) as ei:
        ck.cakf_interpolate(ctx, np.array([0.05]))
    assert ei.value.code == ck.binding.ERR_ARG
    ctx.close()
