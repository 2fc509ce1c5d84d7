"""Failure detection without a GPU fault (the failures are made on the host or by a bounded wait):

* a bounded device-side wait that runs out -- the iteration limit lowered with cakf_set_wait_limit so
  that the tensor-core Gram x block's mbarrier waits, the tensor-core factor GEMM's waits and the
  tridiagonalisation's exchange polling give up -- returns CAKF_ERR_TIMEOUT, and the next call with
  the default limit succeeds with correct results (the kernels stopped cleanly);
* non-finite inputs (host or device arrays) are rejected with CAKF_ERR_ARG before any work, and the
  context is reused successfully afterwards;
* a replayed action that repeats an earlier one ends the step's update there (breakdown, R2): the
  per-step diagnostics report fewer actions than the budget;
* a cap on the context's device memory returns CAKF_ERR_OOM before any allocation;
* the per-step diagnostics of a normal run: relative residuals in (0, 1], positive eta, discarded
  truncation mass >= 0 and > 0 once truncation starts.
"""
import math

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2405_08971_gb300 as ck  # noqa: E402


@pytest.fixture(autouse=True)
def _defaults():
    yield
    ck.cakf_set_wait_limit(0)
    ck.cakf_set_device_memory_limit(0)


def gram_inputs(nr=3000, nc=2000, width=65):
    g = torch.Generator().manual_seed(3)
    d = torch.device("cuda:0")
    Xr = torch.rand((nr, 2), generator=g, dtype=torch.float64).to(d)
    Xc = torch.rand((nc, 2), generator=g, dtype=torch.float64).to(d)
    B = torch.randn((width, nc), generator=g, dtype=torch.float64).to(torch.float32).to(d)
    return Xr, Xc, B


@pytest.mark.parametrize("precision", ["bf16", "fp16x3", "tf32x3"])
def test_gram_wait_timeout_then_recovery(precision):
    Xr, Xc, B = gram_inputs()
    ref = ck.cakf_gram_matmul(1, math.log(0.2), 0.0, Xr, Xc, B, precision=precision)
    torch.cuda.synchronize()
    ck.cakf_set_wait_limit(1)
    with pytest.raises(ck.CakfError) as ei:
        ck.cakf_gram_matmul(1, math.log(0.2), 0.0, Xr, Xc, B, precision=precision)
    assert ei.value.code == ck.binding.ERR_TIMEOUT
    ck.cakf_set_wait_limit(0)
    again = ck.cakf_gram_matmul(1, math.log(0.2), 0.0, Xr, Xc, B, precision=precision)
    assert torch.equal(again, ref)


def test_factor_gemm_wait_timeout_then_recovery():
    g = torch.Generator().manual_seed(4)
    d = torch.device("cuda:0")
    A = torch.randn((576, 20000), generator=g).to(d)     # column-major 20000 x 576
    Bm = torch.randn((512, 576), generator=g).to(d)
    ref = ck.cakf_factor_gemm(A, Bm, precision="tf32x3")
    ck.cakf_set_wait_limit(1)
    with pytest.raises(ck.CakfError) as ei:
        ck.cakf_factor_gemm(A, Bm, precision="tf32x3")
    assert ei.value.code == ck.binding.ERR_TIMEOUT
    ck.cakf_set_wait_limit(0)
    assert torch.equal(ck.cakf_factor_gemm(A, Bm, precision="tf32x3"), ref)


def test_eigensolver_poll_timeout_then_recovery():
    rng = np.random.default_rng(5)
    X = rng.standard_normal((576, 576))
    A = torch.as_tensor(X @ X.T, device="cuda:0")
    w0, _ = ck.cakf_eig_topk(A, 512)
    ck.cakf_set_wait_limit(1)
    with pytest.raises(ck.CakfError) as ei:
        ck.cakf_eig_topk(A, 512)
    assert ei.value.code == ck.binding.ERR_TIMEOUT
    ck.cakf_set_wait_limit(0)
    w1, _ = ck.cakf_eig_topk(A, 512)
    assert torch.equal(w0, w1)


def test_non_finite_inputs():
    w = synth.small(n=200, dim=2, m=40, T=4, budget_i=6, rank_r=12, seed=81)
    good = ck.problem_from_workload(w, precision="fp32")
    ctx, mf, _ = ck.cakf_filter(good)
    y = w.y.copy()
    y[5] = np.nan
    with pytest.raises(ck.CakfError) as ei:
        ck.cakf_filter(ck.problem_from_workload(w.with_(y=y), precision="fp32"), ctx)
    assert ei.value.code == ck.binding.ERR_ARG
    coords = w.coords.copy()
    coords[3, 1] = np.inf
    with pytest.raises(ck.CakfError) as ei:
        ck.cakf_filter(ck.problem_from_workload(w.with_(coords=coords), precision="fp32"), ctx)
    assert ei.value.code == ck.binding.ERR_ARG
    d = torch.device("cuda:0")
    prob = ck.make_problem(torch.as_tensor(w.coords, device=d), w.kernel, w.log_lx, w.log_lt, w.log_sf2, w.log_sn2,
                           w.T, w.dt, w.obs_ptr, torch.as_tensor(w.obs_idx, device=d), torch.as_tensor(y, device=d),
                           w.budget_i, w.rank_r, precision="fp32")
    with pytest.raises(ck.CakfError) as ei:
        ck.cakf_filter(prob, ctx)
    assert ei.value.code == ck.binding.ERR_ARG
    ctx, mf2, _ = ck.cakf_filter(good, ctx)     # the context is usable again
    assert np.array_equal(mf, mf2)
    ctx.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_repeated_replayed_action_breaks_down(precision):
    w = synth.small(n=120, dim=2, m=30, T=3, budget_i=5, rank_r=0, seed=82)
    base = oracle.filter_run(w)
    S = [np.zeros((0, 0))] + [base.S[k].copy() for k in range(1, w.T + 1)]
    S[2] = np.concatenate([S[2][:, :2], S[2][:, :1], S[2][:, 2:4]], axis=1)    # action 3 repeats action 1
    prob = ck.problem_from_workload(w, precision=precision, replay=ck.pack_actions(S, w.T))
    ctx, _, _ = ck.cakf_filter(prob)
    diag = ck.cakf_get_diagnostics(ctx)
    ctx.close()
    assert diag["actions"][2] == 2
    assert diag["actions"][1] == base.S[1].shape[1] and diag["actions"][3] == base.S[3].shape[1]
    ref = oracle.filter_run(w, S_replay=S)
    assert ref.iters[2] == 2


def test_memory_cap_returns_oom():
    w = synth.small(n=500, dim=2, m=80, T=5, budget_i=8, rank_r=20, seed=83)
    ck.cakf_set_device_memory_limit(1 << 20)
    with pytest.raises(ck.CakfError) as ei:
        ck.cakf_filter(ck.problem_from_workload(w, precision="fp32"))
    assert ei.value.code == ck.binding.ERR_OOM
    ck.cakf_set_device_memory_limit(0)
    ctx, mf, _ = ck.cakf_filter(ck.problem_from_workload(w, precision="fp32"))
    assert np.all(np.isfinite(mf))
    ctx.close()


@pytest.mark.parametrize("policy", ["cg", "coordinate"])
def test_diagnostics_of_a_normal_run(policy):
    w = synth.small(n=800, dim=2, m=150, T=6, budget_i=12, rank_r=30, seed=84)
    ctx, _, _ = ck.cakf_filter(ck.problem_from_workload(w, precision="fp64", policy=policy))
    ck.cakf_smooth(ctx)
    d = ck.cakf_get_diagnostics(ctx)
    ctx.close()
    f = oracle.filter_run(w, policy=policy)
    assert np.array_equal(d["actions"], f.iters)
    assert np.all(d["rel_residual"][1:] > 0) and np.all(d["rel_residual"][1:] < 10)   # not monotone in general
    assert np.all(d["min_eta"][1:] > 0)
    assert np.all(d["dropped_filter"] >= -1e-9) and d["dropped_filter"][-1] > 0
    # the filter's discarded mass is the oracle's sum of dropped eigenvalues
    assert np.allclose(d["dropped_filter"], f.dropped, rtol=1e-8, atol=1e-10 * np.max(f.dropped))
    assert np.all(d["dropped_smoother"] >= -1e-9)
