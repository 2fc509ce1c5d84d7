"""Writes tests/golden/sphere65k_T12.json from the FP64 oracle (and nothing else).

    python tests/golden/make_sphere65k.py        # about an hour on 8 host cores

The workload is the 65,536-state sphere configuration (256 x 256 lat-lon grid on the unit sphere,
Matern-3/2 on chordal distance with l_x = 0.1, OU l_t = 1, dt = 0.1, sigma_n^2 = 0.05, m = 8,192
observations per step of which 5,734 are fixed stations, i = 64 CG actions, truncation rank
r = 512; seed 2) over a horizon of T' = 12 steps.  The downdate factor reaches the rank r after
eight steps, so the filter truncates at steps 9..12 (576 -> 512 columns) and the smoother, whose
factor grows by 64 columns per step backwards, truncates at steps 4..1.

Stored: filter and smoother means and variances at 128 grid points (64 station points, where
the posterior variance is smallest and the cancellation in sigma_f^2 - rowsumsq(M) largest, and
64 other points drawn with a fixed seed), the per-step NLL terms and the CG action counts.  The
CUDA path is compared with these values in tests/test_gpu_fullsize.py.
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
import synth  # noqa: E402

T = 12
OUT = os.path.join(HERE, "sphere65k_T12.json")


def sample_points(w):
    """64 station points (observed at every step) and 64 other grid points, sorted."""
    stations = set(w.obs(1).tolist())
    for k in range(2, w.T + 1):
        stations &= set(w.obs(k).tolist())
    rng = np.random.default_rng(12345)
    st = np.sort(rng.choice(np.array(sorted(stations)), 64, replace=False))
    rest = np.setdiff1d(np.arange(w.n), np.array(sorted(stations)))
    ot = np.sort(rng.choice(rest, 64, replace=False))
    return np.sort(np.concatenate([st, ot])), st


def main():
    t0 = time.time()
    w = synth.sphere_65k(T=T)
    cols, st = sample_points(w)
    f = oracle.filter_run(w)
    print(f"filter done in {time.time() - t0:.0f} s", file=sys.stderr, flush=True)
    ms, vs, _ = oracle.smoother_run(w, f)
    print(f"smoother done in {time.time() - t0:.0f} s", file=sys.stderr, flush=True)
    out = {
        "workload": "synth.sphere_65k(T=12) (seed 2)", "T": T, "grid_points": cols.tolist(),
        "station_points": st.tolist(),
        "filter_mean": np.asarray(f.m)[:, cols].tolist(), "filter_var": np.asarray(f.var)[:, cols].tolist(),
        "smoother_mean": np.asarray(ms)[:, cols].tolist(), "smoother_var": np.asarray(vs)[:, cols].tolist(),
        "nll_terms": np.asarray(oracle.nll_terms(f)).tolist(), "actions": np.asarray(f.iters).tolist(),
        "dropped": np.asarray(f.dropped).tolist(),
    }
    with open(OUT, "w") as fh:
        json.dump(out, fh)
    print(f"wrote {OUT} in {time.time() - t0:.0f} s", file=sys.stderr)


if __name__ == "__main__":
    main()
