"""Parity of the CUDA path (through the C ABI) with the FP64 oracle on identical seeded inputs.

Tolerances (written per quantity):
  FP64 mode: means (per-step normwise), variances (elementwise) and the NLL within 1e-10 relative,
             with the CG actions chosen on the device and with the oracle's actions replayed (the
             NLL is computed on the device from its definition: FP64 Cholesky factors of S^T G S
             and S^T S, as in the oracle).
  FP32 mode: the CG actions are chosen from FP32 residuals, so the projected subspace itself moves
             by ~1e-6; 1e-3 relative on means (normwise), variances (elementwise) and the NLL.
  FP16X3 / TF32X3 modes: the Gram x block products carry each operand as two FP16 (TF32) parts
             (22 significant bits, FP32 accumulation; the mean column stays FP32) and the factor
             products are split-TF32 tensor-core GEMMs; the FP32 bounds (1e-3).
  (Plain BF16 rounds each operand to 2^-8 relative; variances near observed points, where the
  posterior variance is a small difference of O(sf2) terms, then lose 1e-2..4e-1 relative on
  these ill-conditioned cases, so that mode is checked at the kernel level in test_gpu_gram.)
Where several results are correct (the factors are defined up to rotation), only products and
diagonals are compared: means, marginal variances, NLL.
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


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2405_08971_gb300 import build
    build.build()


def mean_err(got, ref):
    errs = []
    for k in range(ref.shape[0]):
        nr = np.linalg.norm(ref[k])
        if nr > 0:
            errs.append(np.linalg.norm(got[k] - ref[k]) / nr)
        else:
            errs.append(np.linalg.norm(got[k]))
    return max(errs)


def var_err(got, ref):
    return float(np.max(np.abs(got - ref) / np.abs(ref)))


def run_gpu(w, precision, **kw):
    prob = ck.problem_from_workload(w, precision=precision, **kw)
    ctx, mf, vf = ck.cakf_filter(prob)
    ms, vs = ck.cakf_smooth(ctx)
    nll = ck.cakf_nll(ctx)
    acts, counts = ck.cakf_get_actions(ctx, w.obs_ptr)
    ctx.close()
    return dict(mf=mf, vf=vf, ms=ms, vs=vs, nll=nll, S=acts, counts=counts)


def run_oracle(w, **kw):
    f = oracle.filter_run(w, **kw)
    ms, vs, _ = oracle.smoother_run(w, f)
    return dict(mf=f.m, vf=f.var, ms=ms, vs=vs, nll=oracle.nll_total(f), S=f.S, f=f)


CASES = {
    # name: (workload factory, fp64 tol)
    "tiny1d-full-budget-no-trunc": lambda: synth.tiny_1d(T=12),
    "grid2d-ragged-trunc": lambda: synth.small(n=1000, dim=2, m=300, T=6, budget_i=16, rank_r=48, seed=31,
                                               seasonal=True),
    "sphere-m32-trunc": lambda: synth.small(n=700, m=150, T=5, budget_i=12, rank_r=30, seed=32, sphere=True,
                                            lx=0.4),
    "missing-steps-m12": lambda: synth.small(n=200, dim=1, m=40, T=6, budget_i=8, rank_r=20, seed=33,
                                             kernel=synth.MATERN12, missing=(2, 5)),
    "m52-full-budget-trunc": lambda: synth.small(n=150, dim=2, m=20, T=5, budget_i=20, rank_r=30, seed=34,
                                                 kernel=synth.MATERN52),
    # degenerate and ragged shapes: one state and one observation; one full 128-wide matvec tile
    # plus a single-row tile; a single time step with truncation in it
    "scalar-n1-m1": lambda: synth.small(n=1, m=1, T=5, budget_i=1, rank_r=0, seed=36),
    "ragged-m129": lambda: synth.small(n=400, dim=2, m=129, T=3, budget_i=5, rank_r=12, seed=37),
    "one-step-trunc": lambda: synth.small(n=100, dim=2, m=30, T=1, budget_i=6, rank_r=4, seed=38),
}

# Truncation Grams of order 512 (r + i = 448 + 64): the eigensolver's larger shared-memory
# configurations.  Checked with the oracle's actions replayed: 64 CG iterations amplify FP64
# rounding differences in the action directions to ~1e-9 (means) / ~1e-7 (variances) even on this
# well-determined problem (relative CG residual ~1e-3 after 64 iterations), so the device-chosen
# actions are not a 1e-9 pin of the truncation path; the replayed ones are.
LARGE = {
    "large-rank-trunc": lambda: synth.small(n=2000, dim=2, m=1000, T=9, budget_i=64, rank_r=448, seed=35,
                                            lx=0.05),
}


@pytest.mark.parametrize("name", list(CASES))
def test_fp64_parity(name):
    w = CASES[name]()
    ref = run_oracle(w)
    got = run_gpu(w, "fp64")
    e = dict(mf=mean_err(got["mf"], ref["mf"]), vf=var_err(got["vf"], ref["vf"]),
             ms=mean_err(got["ms"], ref["ms"]), vs=var_err(got["vs"], ref["vs"]),
             nll=abs(got["nll"] - ref["nll"]) / abs(ref["nll"]))
    print(name, {k: f"{v:.2e}" for k, v in e.items()})
    assert np.array_equal(got["counts"][1:], ref["f"].iters[1:])
    for k, v in e.items():
        assert v < 1e-10, (k, v)


@pytest.mark.parametrize("name", ["grid2d-ragged-trunc", "sphere-m32-trunc", "large-rank-trunc"])
def test_fp64_replayed_actions(name):
    """With the oracle's actions replayed, the device update is Alg. 2 on the same subspace."""
    w = {**CASES, **LARGE}[name]()
    ref = run_oracle(w)
    flat, counts = ck.pack_actions(ref["S"], w.T)
    got = run_gpu(w, "fp64", replay=(flat, counts))
    for key, fn in (("mf", mean_err), ("ms", mean_err), ("vf", var_err), ("vs", var_err)):
        assert fn(got[key], ref[key]) < 1e-10, key
    assert abs(got["nll"] - ref["nll"]) < 1e-10 * abs(ref["nll"])


@pytest.mark.parametrize("name", ["grid2d-ragged-trunc", "sphere-m32-trunc", "missing-steps-m12", "scalar-n1-m1",
                                  "ragged-m129", "one-step-trunc"])
def test_fp32_parity(name):
    w = CASES[name]()
    ref = run_oracle(w)
    got = run_gpu(w, "fp32")
    e = dict(mf=mean_err(got["mf"], ref["mf"]), vf=var_err(got["vf"], ref["vf"]),
             ms=mean_err(got["ms"], ref["ms"]), vs=var_err(got["vs"], ref["vs"]),
             nll=abs(got["nll"] - ref["nll"]) / abs(ref["nll"]))
    print(name, "fp32", {k: f"{v:.2e}" for k, v in e.items()})
    for k, v in e.items():
        assert v < 1e-3, (k, v)


def test_device_buffers_and_context_reuse():
    """Device-resident inputs/outputs give the same numbers as host buffers; a context is reusable."""
    w = CASES["missing-steps-m12"]()
    ref = run_gpu(w, "fp64")
    dev = torch.device("cuda:0")
    prob = ck.make_problem(torch.as_tensor(w.coords, device=dev), w.kernel, w.log_lx, w.log_lt, w.log_sf2,
                           w.log_sn2, w.T, w.dt, w.obs_ptr, torch.as_tensor(w.obs_idx, device=dev),
                           torch.as_tensor(w.y, device=dev), w.budget_i, w.rank_r, precision="fp64")
    shape = (w.T + 1, w.n)
    mo = torch.empty(shape, dtype=torch.float64, device=dev)
    vo = torch.empty(shape, dtype=torch.float64, device=dev)
    ctx = ck.Context()
    for _ in range(2):
        ctx, _, _ = ck.cakf_filter(prob, ctx, mo, vo)
        assert np.array_equal(mo.cpu().numpy(), ref["mf"]) and np.array_equal(vo.cpu().numpy(), ref["vf"])
        ms = torch.empty(shape, dtype=torch.float64, device=dev)
        vs = torch.empty(shape, dtype=torch.float64, device=dev)
        ck.cakf_smooth(ctx, ms, vs)
        assert np.array_equal(ms.cpu().numpy(), ref["ms"]) and np.array_equal(vs.cpu().numpy(), ref["vs"])
    ctx.close()


def test_state_errors():
    ctx = ck.Context()
    with pytest.raises(ck.CakfError) as ei:
        ck.cakf_nll(ctx)
    assert ei.value.code == ck.binding.ERR_STATE
    w = CASES["missing-steps-m12"]()
    prob = ck.problem_from_workload(w, precision="fp32")
    ctx, _, _ = ck.cakf_filter(prob, ctx)
    bad = ck.problem_from_workload(w.with_(obs_idx=w.obs_idx + w.n), precision="fp32")
    with pytest.raises(ck.CakfError) as ei:
        ck.cakf_filter(bad, ctx)
    assert ei.value.code == ck.binding.ERR_ARG
    ctx.close()


# split FP16 at the FP32 bound; split TF32 carries as many operand bits, but kind::tf32 products
# measure about twice the Gram x block error of kind::f16 (test_gpu_gram), 1.9e-3 on the variances of
# the ill-conditioned 2-D case: bound 3e-3 there, 1e-3 on the rest.  On that case (300 observations,
# 16 actions per step, truncation from step 4) the variances near the observed points are small
# differences of O(sf2) terms and the CG actions picked from working-precision residuals move the
# projected subspace itself: with the device's own actions the distance to the oracle changed from
# 6.9e-4 to 1.1e-3 (split FP16) and 1.7e-4 to 3.8e-4 (FP32) when only the summation order of the CG
# update kernels changed.  So there the oracle's actions are replayed: the same projected model, the
# arithmetic alone is compared.
SPLIT_TOL = {"fp16x3": 1e-3, "tf32x3": 3e-3}


@pytest.mark.parametrize("precision", ["fp16x3", "tf32x3"])
@pytest.mark.parametrize("name", ["grid2d-ragged-trunc", "sphere-m32-trunc", "missing-steps-m12", "ragged-m129"])
def test_split_tensor_core_parity(name, precision):
    w = CASES[name]()
    ref = run_oracle(w)
    kw = {}
    if name == "grid2d-ragged-trunc":
        flat, counts = ck.pack_actions(ref["S"], w.T)
        kw["replay"] = (flat, counts)
    got = run_gpu(w, precision, **kw)
    e = dict(mf=mean_err(got["mf"], ref["mf"]), vf=var_err(got["vf"], ref["vf"]),
             ms=mean_err(got["ms"], ref["ms"]), vs=var_err(got["vs"], ref["vs"]),
             nll=abs(got["nll"] - ref["nll"]) / abs(ref["nll"]))
    print(name, precision, {k: f"{v:.2e}" for k, v in e.items()})
    tol = SPLIT_TOL[precision] if name == "grid2d-ragged-trunc" else 1e-3
    for k, v in e.items():
        assert v < tol, (k, v)


@pytest.mark.parametrize("name", ["grid2d-ragged-trunc", "sphere-m32-trunc"])
def test_single_pass_tensor_core_modes_run(name):
    """BF16 and TF32 (one MMA per product, 8 resp. 11 significant bits) are the fast, less accurate
    modes: on these ill-conditioned cases they are checked for finite outputs within the prior
    variance and a mean error below 5e-2 (their kernel-level accuracy is pinned in test_gpu_gram)."""
    w = CASES[name]()
    ref = run_oracle(w)
    sf2 = float(np.exp(w.log_sf2))
    for precision in ("bf16", "tf32"):
        got = run_gpu(w, precision)
        e = mean_err(got["mf"], ref["mf"])
        print(name, precision, f"mean {e:.2e} var {var_err(got['vf'], ref['vf']):.2e}")
        for key in ("mf", "vf", "ms", "vs"):
            assert np.all(np.isfinite(got[key]))
        assert np.all(got["vf"] <= sf2 * (1 + 1e-5))
        assert e < 5e-2
