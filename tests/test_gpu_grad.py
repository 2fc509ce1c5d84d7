"""NLL gradient through the C ABI (cakf_nll_backward) against the oracle.

The gradient is taken w.r.t. (log l_x, log l_t, log sf2, log sn2) with the actions and truncation
rotations of the base run held fixed.  References:
  * central finite differences of the FP64 oracle NLL with the same frozen actions and rotations
    (h = 1e-5 in log space; FD truncation error ~1e-9 relative);
  * without truncation, the analytic gradient of the projected batch-GP NLL.
Tolerance in FP64 mode: 1e-6 relative (per component, against max |g|); FP32 mode: 5e-3.
"""
import numpy as np
import pytest

import dense_ref
import oracle
import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2405_08971_gb300 as ck  # noqa: E402


def gpu_grad(w, precision):
    prob = ck.problem_from_workload(w, precision=precision)
    ctx, _, _ = ck.cakf_filter(prob, want_outputs=False)
    nll = ck.cakf_nll(ctx)
    g = ck.cakf_nll_backward(ctx)
    ctx.close()
    return nll, g


def rel(g, ref):
    return np.max(np.abs(g - ref)) / np.max(np.abs(ref))


@pytest.mark.parametrize("kw", [
    dict(n=120, dim=2, m=30, T=5, budget_i=6, rank_r=14, seasonal=True, seed=41),
    dict(n=200, dim=1, m=25, T=6, budget_i=5, rank_r=12, kernel=synth.MATERN52, missing=(3,), seed=42),
    dict(n=150, m=40, T=4, budget_i=8, rank_r=20, sphere=True, lx=0.5, kernel=synth.MATERN12, seed=43),
])
def test_gradient_vs_oracle_fd(kw):
    w = synth.small(**kw)
    nll_o, g_fd = oracle.nll_grad_fd(w, h=1e-5)
    nll, g = gpu_grad(w, "fp64")
    print("fd", g_fd, "gpu", g)
    assert abs(nll - nll_o) < 1e-9 * abs(nll_o)
    assert rel(g, g_fd) < 1e-6, (g, g_fd)


def test_gradient_vs_batch_analytic_without_truncation():
    w = synth.small(n=60, dim=2, m=12, T=4, budget_i=4, rank_r=0, seasonal=True, seed=44)
    f = oracle.filter_run(w)
    g_an = dense_ref.batch_nll_grad(w, f.S)
    _, g = gpu_grad(w, "fp64")
    assert rel(g, g_an) < 1e-8, (g, g_an)


def test_gradient_fp32_close_to_fp64():
    w = synth.small(n=300, dim=2, m=60, T=5, budget_i=8, rank_r=24, seed=45)
    _, g64 = gpu_grad(w, "fp64")
    _, g32 = gpu_grad(w, "fp32")
    print("fp32 gradient rel err", rel(g32, g64))
    assert rel(g32, g64) < 5e-3


def test_autograd_function():
    from paper_2405_08971_gb300.autograd import cakf_neg_log_likelihood, workload_data
    w = synth.small(n=100, dim=2, m=20, T=4, budget_i=5, rank_r=12, seed=46)
    theta = torch.tensor([w.log_lx, w.log_lt, w.log_sf2, w.log_sn2], dtype=torch.float64, requires_grad=True)
    nll = cakf_neg_log_likelihood(theta, workload_data(w), precision="fp64")
    nll.backward()
    _, g = gpu_grad(w, "fp64")
    assert np.allclose(theta.grad.numpy(), g, rtol=1e-12, atol=0)


def test_gradient_fd_instance_n1024_t20():
    """The gradient-check configuration: the 16k-grid model on a 32 x 32 grid (n = 1,024), T = 20,
    m = 128, i = 32, r = 256; device FP64 gradient against central FD of the oracle (h = 1e-5),
    within 1e-5 relative.  Here the budget is a quarter of the observations and CG converges
    within it, so the device-chosen actions differ from the oracle's at rounding level and the
    NLL (a function of span(S)) by ~1e-6; the device therefore replays the oracle's actions,
    which makes both sides differentiate the same frozen model."""
    w = synth.fd_grid2d_1k(T=20)
    nll_o, g_fd = oracle.nll_grad_fd(w, h=1e-5)
    f = oracle.filter_run(w)
    flat, counts = ck.pack_actions(f.S, w.T)
    prob = ck.problem_from_workload(w, precision="fp64", replay=(flat, counts))
    ctx, _, _ = ck.cakf_filter(prob, want_outputs=False)
    nll = ck.cakf_nll(ctx)
    g = ck.cakf_nll_backward(ctx)
    ctx.close()
    print("n1024 fd", g_fd, "gpu", g)
    assert abs(nll - nll_o) < 1e-9 * abs(nll_o)
    assert rel(g, g_fd) < 1e-5, (g, g_fd)


def test_gradient_c4_configuration_against_frozen_fd():
    """The gradient configuration at full size (128 x 128 grid, n = 16,384, T = 200, m = 2,000,
    i = 32, r = 256): the device FP64 gradient against central differences (h = 1e-4 in log space)
    of the device FP64 NLL of the same frozen modified model (the base run's actions replayed and
    its truncation rotations reused through freeze_truncation), within 1e-5 relative; and the FP32
    gradient of the same frozen actions against the FP64 one (reported, 1e-3)."""
    w = synth.grid2d_16k(T=200)
    ctx, _, _ = ck.cakf_filter(ck.problem_from_workload(w, precision="fp64"), want_outputs=False)
    S, _ = ck.cakf_get_actions(ctx, w.obs_ptr)
    rep = ck.pack_actions(S, w.T)
    ctx.close()
    # the base of the frozen model: the same actions replayed (its rotations are then reused)
    ctx, _, _ = ck.cakf_filter(ck.problem_from_workload(w, precision="fp64", replay=rep), want_outputs=False)
    g64 = ck.cakf_nll_backward(ctx)
    theta0 = np.array([w.log_lx, w.log_lt, w.log_sf2, w.log_sn2])
    names = ["log_lx", "log_lt", "log_sf2", "log_sn2"]
    h, g_fd = 1e-4, np.zeros(4)
    for p in range(4):
        vals = []
        for sgn in (1, -1):
            th = theta0.copy()
            th[p] += sgn * h
            pr = ck.problem_from_workload(w, precision="fp64", replay=rep, freeze_truncation=True,
                                          **{nm: float(v) for nm, v in zip(names, th)})
            ctx, _, _ = ck.cakf_filter(pr, ctx, want_outputs=False)
            vals.append(ck.cakf_nll(ctx))
        g_fd[p] = (vals[0] - vals[1]) / (2 * h)
    ctx.close()
    e = rel(g64, g_fd)
    print("c4 fp64 gradient", g64, "frozen fd", g_fd, f"rel {e:.2e}")
    assert e < 1e-5, (g64, g_fd)
    prob32 = ck.problem_from_workload(w, precision="fp32", replay=rep)
    ctx32, _, _ = ck.cakf_filter(prob32, want_outputs=False)
    g32 = ck.cakf_nll_backward(ctx32)
    ctx32.close()
    print("c4 fp32 gradient", g32, f"rel to fp64 {rel(g32, g64):.2e}")
    assert rel(g32, g64) < 1e-3


def test_adam_fit_decreases_the_nll():
    """Ten Adam steps through the autograd Function on the n = 1,024, T = 20 instance, from both
    lengthscales doubled: the NLL decreases and the lengthscales move toward the generating ones."""
    from paper_2405_08971_gb300.autograd import workload_data
    from paper_2405_08971_gb300.fit import fit_adam
    w = synth.fd_grid2d_1k(T=20)
    theta0 = [w.log_lx + np.log(2.0), w.log_lt + np.log(2.0), w.log_sf2, w.log_sn2]
    theta, trace = fit_adam(workload_data(w), theta0, steps=10, lr=0.05, precision="fp32")
    nlls = [t[1] for t in trace]
    print("adam nll trace", [f"{v:.2f}" for v in nlls])
    assert nlls[-1] < nlls[0]
    assert abs(theta[0] - w.log_lx) < abs(theta0[0] - w.log_lx)
