"""Writes the stored expected values of tests/golden/ from the FP64 oracle (and nothing else).

    python tests/golden/make_golden.py

tiny_1d_T8.json: the 1-D configuration (n = 256 grid points on [0, 1], Matern-3/2 l = 0.1,
OU l_t = 0.5, dt = 0.1, m = 32 observations per step, noise 0.01, full action budget, no
truncation; seed 0) over T = 8 steps: filter and smoother means and variances at every 16th grid
point, and the per-step NLL terms.  At full budget the method equals the exact Kalman filter and
RTS smoother (Sec. 3.1), which tests/test_golden.py checks the stored values against.
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
import synth  # noqa: E402

T, SEED, STRIDE = 8, 0, 16


def main():
    w = synth.tiny_1d(T=T, seed=SEED)
    f = oracle.filter_run(w)
    ms, vs, _ = oracle.smoother_run(w, f)
    cols = list(range(0, w.n, STRIDE))
    out = {
        "workload": "synth.tiny_1d(T=8, seed=0)", "T": T, "seed": SEED, "grid_points": cols,
        "filter_mean": np.asarray(f.m)[:, cols].tolist(), "filter_var": np.asarray(f.var)[:, cols].tolist(),
        "smoother_mean": np.asarray(ms)[:, cols].tolist(), "smoother_var": np.asarray(vs)[:, cols].tolist(),
        "nll_terms": np.asarray(oracle.nll_terms(f)).tolist(),
    }
    with open(os.path.join(HERE, "tiny_1d_T8.json"), "w") as fh:
        json.dump(out, fh, indent=0)


if __name__ == "__main__":
    main()
