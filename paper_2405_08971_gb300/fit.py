"""Hyperparameter fitting by Adam through the differentiable CAKF negative log likelihood.

theta = (log l_x, log l_t, log sf2, log sn2); every step runs cakf_filter + cakf_nll (forward) and
cakf_nll_backward (gradient with that run's actions and truncation rotations held fixed) through
the torch.autograd.Function of `autograd.py`.  All compute happens in libcakf.so.

    python -m paper_2405_08971_gb300.fit [--config grid2d-16k] [--steps 50] [--lr 0.05]

runs the gradient configuration of the 2-D model (128 x 128 grid, n = 16,384, T = 200, m = 2,000,
i = 32, r = 256, FP32 contractions) from both lengthscales doubled and prints the NLL trace.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys
import time

import torch

from .autograd import cakf_neg_log_likelihood, workload_data


def fit_adam(data: dict, theta0, steps: int = 50, lr: float = 0.05, precision: str = "fp32", log=None):
    """Adam on theta from theta0; returns (final theta, list of (step, nll, theta, seconds))."""
    theta = torch.tensor(theta0, dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([theta], lr=lr)
    trace = []
    for it in range(steps):
        t0 = time.perf_counter()
        opt.zero_grad()
        nll = cakf_neg_log_likelihood(theta, data, precision=precision)
        nll.backward()
        opt.step()
        rec = (it, float(nll.detach()), [float(v) for v in theta.detach()], time.perf_counter() - t0)
        trace.append(rec)
        if log:
            log(rec)
    return theta.detach().numpy(), trace


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--config", default="grid2d-16k", choices=["grid2d-16k", "grid2d-1k"])
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--lr", type=float, default=0.05)
    ap.add_argument("--precision", default="fp32")
    args = ap.parse_args()
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import synth
    from . import build
    build.build()
    w = synth.grid2d_16k(T=200) if args.config == "grid2d-16k" else synth.fd_grid2d_1k(T=20)
    truth = [w.log_lx, w.log_lt, w.log_sf2, w.log_sn2]
    theta0 = [w.log_lx + math.log(2.0), w.log_lt + math.log(2.0), w.log_sf2, w.log_sn2]
    print(json.dumps({"config": args.config, "truth": truth, "start": theta0, "precision": args.precision}), flush=True)
    _, trace = fit_adam(workload_data(w), theta0, args.steps, args.lr, args.precision,
                        log=lambda r: print(json.dumps({"step": r[0], "nll": r[1], "theta": r[2], "s": round(r[3], 3)}),
                                            flush=True))


if __name__ == "__main__":
    main()
