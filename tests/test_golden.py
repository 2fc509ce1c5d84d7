"""Stored expected values (tests/golden/tiny_1d_T8.json, written by tests/golden/make_golden.py from
the FP64 oracle) for the 1-D full-budget configuration over 8 steps.

* CPU: the stored values equal the exact Kalman filter / RTS smoother computed densely here (at
  full budget the method loses nothing, Sec. 3.1), and the oracle still reproduces them.
* GPU: the CUDA path reproduces them through the C ABI -- FP64 mode within 1e-10 (relative to the
  largest magnitude of each quantity), FP32 within 1e-4 for means, variances and the
  NLL (the FP32 path on this well-conditioned 1-D case).
"""
import json
import os

import numpy as np
import pytest

import dense_ref
import oracle
import synth

HERE = os.path.dirname(os.path.abspath(__file__))
GOLD = os.path.join(HERE, "golden", "tiny_1d_T8.json")


def load():
    with open(GOLD) as fh:
        g = json.load(fh)
    return g, synth.tiny_1d(T=g["T"], seed=g["seed"])


def rel(a, b):
    a, b = np.asarray(a, dtype=float), np.asarray(b, dtype=float)
    return float(np.max(np.abs(a - b)) / max(1e-300, np.max(np.abs(b))))


def test_golden_equals_dense_kf_rts():
    g, w = load()
    ref = dense_ref.kf_rts(w)
    cols = g["grid_points"]
    assert rel(g["filter_mean"], ref["mf"][:, cols]) < 1e-10
    assert rel(g["filter_var"], ref["vf"][:, cols]) < 1e-10
    assert rel(g["smoother_mean"], ref["ms"][:, cols]) < 1e-10
    assert rel(g["smoother_var"], ref["vs"][:, cols]) < 1e-10
    assert rel(g["nll_terms"], ref["nll"]) < 1e-10


def test_oracle_reproduces_golden():
    g, w = load()
    f = oracle.filter_run(w)
    ms, vs, _ = oracle.smoother_run(w, f)
    cols = g["grid_points"]
    assert rel(np.asarray(f.m)[:, cols], g["filter_mean"]) < 1e-12
    assert rel(np.asarray(f.var)[:, cols], g["filter_var"]) < 1e-12
    assert rel(np.asarray(ms)[:, cols], g["smoother_mean"]) < 1e-12
    assert rel(np.asarray(vs)[:, cols], g["smoother_var"]) < 1e-12
    assert rel(oracle.nll_terms(f), g["nll_terms"]) < 1e-12


@pytest.mark.gpu
@pytest.mark.parametrize("precision,tol,tol_nll", [("fp64", 1e-10, 1e-10), ("fp32", 1e-4, 1e-4)])
def test_cuda_path_reproduces_golden(precision, tol, tol_nll):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_2405_08971_gb300 as ck
    g, w = load()
    prob = ck.problem_from_workload(w, precision=precision)
    ctx, mf, vf = ck.cakf_filter(prob)
    ms, vs = ck.cakf_smooth(ctx)
    nll = ck.cakf_nll(ctx)
    ctx.close()
    cols = g["grid_points"]
    errs = dict(mf=rel(mf[:, cols], g["filter_mean"]), vf=rel(vf[:, cols], g["filter_var"]),
                ms=rel(ms[:, cols], g["smoother_mean"]), vs=rel(vs[:, cols], g["smoother_var"]))
    print(precision, {k: f"{v:.1e}" for k, v in errs.items()})
    for k, v in errs.items():
        assert v < tol, (k, v)
    tot = float(np.sum(g["nll_terms"]))
    assert abs(nll - tot) / abs(tot) < tol_nll
