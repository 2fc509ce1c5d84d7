"""Benchmark: filter + smoother time steps per second of the computation-aware Kalman filter/smoother.

One bench "step" is a full pass of the hot path over the whole series: cakf_filter (CG actions,
Gram x block finalize, truncation) over k = 1..T followed by cakf_smooth over k = T-1..0, on a
seeded synthetic workload (default: the 256 x 256 lat-lon sphere grid, n = 65,536, m = 8,192
observations per step, i = 64 actions, truncation rank r = 512, T = 500 steps).

Prints ONE JSON line on rank 0.  `value` is whole-job time steps per second (sum over ranks of
T * K / the slowest rank's timed region).  Multi-GPU runs are independent replicas (one series
per rank, different seeds): the method's recursion is sequential in time and the paper runs on a
single GPU, so there is no data-path collective.

The default precision is fp16x3 (Gram tiles x blocks on the tensor cores with split FP16 operands,
FP32-class products: the mixed-precision mode that holds the 1e-3 relative error target on means
and variances); bf16 is the single-MMA mode (faster, 2^-8 operand rounding), fp32 the plain SIMT
path, fp64 the reference mode.

  python bench.py [--steps K] [--warmup W] [--precision fp16x3|bf16|fp32|fp64] [--T T] [--config NAME]
  python bench.py --impl reference ...      # the FP64 oracle on the host cores (bounded sample)
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

DTYPE_NAME = {"fp16x3": "fp16x3", "tf32x3": "tf32x3", "tf32": "tf32", "bf16": "bf16", "fp32": "f32", "fp64": "f64"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp16x3", choices=list(DTYPE_NAME))
    ap.add_argument("--config", default="sphere-65k")
    ap.add_argument("--storage", default="fp32", choices=["fp32", "bf16", "recompute"],
                    help="factor storage between the filter and the smoother (cakf_problem.factor_storage)")
    ap.add_argument("--checkpoint-every", type=int, default=0,
                    help="segment length of the bf16 / recompute storage (0: the library default, 20)")
    ap.add_argument("--grad", action="store_true",
                    help="after the timed passes, time one cakf_nll_backward (NLL gradient) on the last filter")
    ap.add_argument("--T", type=int, default=None, help="override the number of time steps")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp32-compare", action="store_true",
                    help="skip the plain-FP32 comparison pass (one untimed + one timed pass at fp32)")
    ap.add_argument("--cpu-row-frac", type=int, default=16,
                    help="the CPU baseline's smoother kernel products are timed on 1/N of the rows and scaled")
    ap.add_argument("--no-accuracy", action="store_true",
                    help="skip the untimed FP64 passes that give the accuracy of the timed precision")
    ap.add_argument("--accuracy-steps", type=int, default=100,
                    help="time steps of the accuracy passes (a prefix of the benched series)")
    return ap.parse_args()


def workload(name, T, seed_offset=0, device=None):
    import synth
    if name == "sphere-65k":
        return synth.sphere_65k(T=T or 500, seed=2 + seed_offset, device=device), \
            "sphere-n65536-m8192-i64-r512 (256x256 lat-lon grid on S^2, extrinsic Matern-3/2 l=0.1, OU l_t=1, dt=0.1, sn2=0.05)"
    if name == "grid2d-16k":
        return synth.grid2d_16k(T=T or 200, seed=1 + seed_offset, device=device), \
            "grid2d-n16384-m2000-i32-r256 (128x128 grid, Matern-5/2 l=0.05, OU l_t=1, dt=0.1, sn2=0.01, seasonal mean)"
    if name == "sphere-262k":
        return synth.sphere_262k(T=T or 300, seed=4 + seed_offset, device=device), \
            "sphere-n262144-m16384-i128-r256 (512x512 sphere grid, Matern-3/2 l=0.05)"
    if name == "small":
        return synth.small(n=4096, dim=2, m=512, T=T or 20, budget_i=16, rank_r=64, seed=5 + seed_offset,
                           device=device), "small-n4096-m512-i16-r64"
    raise SystemExit(f"unknown config {name}")


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return d, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}, \
            "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def allmax(ws, x):
    """Maximum of x over the ranks (the slowest rank's time); a CPU tensor under gloo."""
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cpu" if dist.get_backend() == "gloo" else "cuda"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(ws, T, steps, ms_max):
    """Whole-job time steps per second: every rank filters and smooths its own series of T steps
    (independent replicas), so the job processes ws * T * steps time steps in the slowest rank's time."""
    return ws * T * steps / (ms_max / 1e3)


# --------------------------------------------------------------------------------------- CPU leg
def oracle_sample(w, row_frac=16):
    """Time the FP64 oracle on one steady-state step pair of the workload (host cores).

    Filter: the oracle's update (iterative version, CG actions) and Truncate on a prior factor of
    the steady-state width r (random columns with decaying norms, the shapes the filter reaches
    after r / i steps), measured in full.  Smoother: the oracle's step costs two products
    K [Ws ws] of width r + i + 1 over all n x n kernel entries (P_k A^T X and P^-_k A^T X) plus
    low-rank terms; the K products are timed on 1/row_frac of the rows and scaled by row_frac,
    the low-rank terms in full.  Returns (seconds per time step, description)."""
    import oracle
    model = oracle.model_from(w)
    n, r, i = w.n, max(w.rank_r, 0), w.budget_i
    rng = np.random.default_rng(0)
    # a valid downdate factor of the steady-state width: the update of the prior by r noisy point
    # values, K(X, X_s) (K_ss + sn2 I)^(-1/2), so that K - M M^T stays positive definite
    pts = np.sort(rng.choice(n, r, replace=False))
    Ks = model.K_times(np.eye(r), cols=pts)
    lam, Q = np.linalg.eigh(Ks[pts] + model.sn2 * np.eye(r))
    Mp = Ks @ (Q / np.sqrt(lam)[None, :])
    obs = w.obs(1)
    m_pred = np.zeros(n)
    t0 = time.perf_counter()
    m_new, M_hat, *_ = oracle.update_iterative(model, m_pred, model.a * Mp, obs, w.yk(1), i)
    var = model.sf2 - np.sum(M_hat * M_hat, axis=1)
    oracle.truncate(M_hat, r)
    t_f = time.perf_counter() - t0
    c = M_hat.shape[1]
    X = model.a * rng.standard_normal((n, c + 1)) / math.sqrt(n)
    rows = np.arange(0, n, row_frac)
    t0 = time.perf_counter()
    for _ in range(2):                                    # P_k A^T X and P^-_k A^T X
        model.K_times(X, rows=rows)
    t_k = (time.perf_counter() - t0) * (n / rows.size)
    t0 = time.perf_counter()
    for M in (M_hat, model.a * Mp):
        M @ (M.T @ X)
    t_l = time.perf_counter() - t0
    del var, m_new
    desc = (f"one steady-state step pair of the oracle (n={n}, m={len(obs)}, i={i}, r={r}): filter update + "
            f"Truncate measured in full ({t_f:.1f} s); smoother: the two n x n x {c + 1} kernel products timed on "
            f"1/{row_frac} of the rows and scaled ({t_k:.1f} s), its low-rank products in full ({t_l:.1f} s)")
    return t_f + t_k + t_l, desc


def cpu_model():
    try:
        with open("/proc/cpuinfo") as fh:
            for ln in fh:
                if ln.lower().startswith(("model name", "cpu part", "hardware")):
                    return ln.split(":", 1)[1].strip() + f" ({os.cpu_count()} cores)"
    except Exception:
        pass
    return f"{os.cpu_count()} cores"


def cpu_cores():
    # an explicit BLAS / OpenMP thread limit in the environment (e.g. a single-thread timing) wins
    for var in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        v = os.environ.get(var)
        if v and v.isdigit():
            return min(int(v), os.cpu_count() or int(v))
    try:
        import threadpoolctl
        info = threadpoolctl.threadpool_info()
        n = max((d.get("num_threads", 1) for d in info), default=os.cpu_count())
        return int(n)
    except Exception:
        return os.cpu_count()


def run_untimed(ck, w, coords, obs_idx, y, mu, precision, stream, replay=None, want_actions=False):
    """One untimed filter + smoother pass at `precision` on workload w (device inputs coords, obs_idx,
    y, mu); returns its four (T+1) x n outputs and the NLL (and the actions when asked)."""
    import torch
    ra, rc = replay if replay is not None else (None, None)
    prob = ck.make_problem(coords, w.kernel, w.log_lx, w.log_lt, w.log_sf2, w.log_sn2, w.T, w.dt, w.obs_ptr,
                           obs_idx, y, w.budget_i, w.rank_r, precision=precision, prior_mean=mu,
                           replay_actions=ra, replay_counts=rc)
    outs = [torch.empty((w.T + 1, w.n), dtype=torch.float64, device=coords.device) for _ in range(4)]
    ctx = ck.Context()
    ck.cakf_filter(prob, ctx, outs[0], outs[1], stream=stream.cuda_stream)
    ck.cakf_smooth(ctx, outs[2], outs[3], stream=stream.cuda_stream)
    outs.append(ck.cakf_nll(ctx))
    acts = ck.cakf_get_actions(ctx, w.obs_ptr) if want_actions else None
    ctx.close()
    torch.cuda.synchronize()
    return (outs, acts) if want_actions else outs


def accuracy_passes(ck, w, coords, obs_idx, y, mu, precision, steps, stream):
    """Errors of `precision` and of plain FP32 against the device FP64 mode over the first `steps`
    steps of the workload: with the FP64 run's actions replayed (arithmetic error) and with their
    own CG actions (the method's sensitivity to the action choice)."""
    wa = w.with_(T=steps, obs_ptr=w.obs_ptr[:steps + 1],
                 prior_mean=None if w.prior_mean is None else w.prior_mean[:steps + 1])
    mua = None if mu is None else mu[:steps + 1]
    ref, (S, _) = run_untimed(ck, wa, coords, obs_idx, y, mua, "fp64", stream, want_actions=True)
    rep = ck.pack_actions(S, steps)
    res = {}
    for key, prec in (("timed", precision), ("fp32", "fp32")):
        got = run_untimed(ck, wa, coords, obs_idx, y, mua, prec, stream, replay=rep)
        own = run_untimed(ck, wa, coords, obs_idx, y, mua, prec, stream)
        res[key] = accuracy(got, ref, f"fp64 device mode, steps 1..{steps}, fp64 actions replayed")
        res[key]["own_actions"] = accuracy(own, ref, f"fp64 device mode, steps 1..{steps}, own CG actions")
    return res


def accuracy(got, ref, against):
    """Errors of one pass against a reference pass, per result, max over the steps 1..T (state 0 is
    the prior): means normwise relative per step, variances elementwise relative."""
    out = {"against": against}
    for name, i, kind in (("filter_mean", 0, "m"), ("filter_var", 1, "v"), ("smoother_mean", 2, "m"),
                          ("smoother_var", 3, "v")):
        a, b = got[i][1:], ref[i][1:]
        if kind == "m":
            e = (a - b).norm(dim=1) / b.norm(dim=1).clamp_min(1e-300)
        else:
            e = ((a - b).abs() / b.abs().clamp_min(1e-300)).amax(dim=1)
        out[name] = float(e.max())
        out[name + "_worst_step"] = int(e.argmax()) + 1
    if len(got) > 4 and len(ref) > 4:
        out["nll"] = abs(got[4] - ref[4]) / abs(ref[4])
    return out


# --------------------------------------------------------------------------------------- main
def main():
    args = parse()
    ws, rank, local = dist_setup()
    if args.impl == "reference":
        return run_reference(args, ws, rank)
    import torch
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import paper_2405_08971_gb300 as ck
    from paper_2405_08971_gb300 import build
    build.build()
    w, desc = workload(args.config, args.T, seed_offset=rank, device=dev)
    T, n = w.T, w.n
    stream = torch.cuda.current_stream(dev)
    coords = torch.as_tensor(w.coords, device=dev)
    obs_idx = torch.as_tensor(w.obs_idx, device=dev)
    y = torch.as_tensor(w.y, device=dev)
    mu = None if w.prior_mean is None else torch.as_tensor(w.prior_mean, device=dev)
    prob = ck.make_problem(coords, w.kernel, w.log_lx, w.log_lt, w.log_sf2, w.log_sn2, T, w.dt, w.obs_ptr,
                           obs_idx, y, w.budget_i, w.rank_r, precision=args.precision, prior_mean=mu,
                           factor_storage=args.storage, checkpoint_every=args.checkpoint_every)
    shape = (T + 1, n)
    outs = [torch.empty(shape, dtype=torch.float64, device=dev) for _ in range(4)]
    ctx = ck.Context()

    def one_step():
        ck.cakf_filter(prob, ctx, outs[0], outs[1], stream=stream.cuda_stream)
        ck.cakf_smooth(ctx, outs[2], outs[3], stream=stream.cuda_stream)

    for _ in range(max(args.warmup, 1)):   # at least one untimed pass creates the context
        one_step()
    ck.cakf_set_profiling(ctx, True)
    launches = 0
    sampler = ClockSampler(local)
    barrier(ws)
    torch.cuda.synchronize(dev)
    sampler.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    prof = {"gram_block_ms": 0.0, "gram_block_launches": 0, "gram_block_flops": 0.0, "gram_block_evals": 0.0,
            "cg_matvec_ms": 0.0, "cg_matvec_launches": 0, "cg_matvec_evals": 0.0, "eig_ms": 0.0, "eig_calls": 0}
    phases = [0.0] * 8
    eig_parts = [0.0] * 3
    eig_flops = [0.0] * 2
    for _ in range(args.steps):
        one_step()
        st = ck.cakf_get_stats(ctx)
        launches += int(st["kernel_launches"])
        for k in prof:
            prof[k] += st[k]
        phases = [a + b for a, b in zip(phases, st["phase_ms"])]
        eig_parts = [a + b for a, b in zip(eig_parts, st["eig_phase_ms"])]
        eig_flops = [a + b for a, b in zip(eig_flops, st["eig_flops"])]
    phases_launches_cg = 8.0   # the matvec is timed on every 8th CG iteration: total ~ 8 x the sampled time
    e1.record(stream)
    torch.cuda.synchronize(dev)
    clocks = sampler.stop()
    barrier(ws)
    ms = e0.elapsed_time(e1)
    ms_max = allmax(ws, ms)
    value = job_value(ws, T, args.steps, ms_max)

    # ---- rooflines from live CUDA events (per kernel class), the dominant one reported as `roofline`
    pk, pk_src = peaks()
    clk_mhz = clocks.get("sm_mhz") or pk.get("sm_max_mhz", 2070.0)
    clk = clk_mhz * 1e6
    nsm = 152
    # MUFU (sqrt + exp2 pair) and FP64 FMA throughputs measured by the library's probe kernels on
    # this device right after the timed region (MEASURED_PEAKS.json holds only copy and GEMM rates)
    probe = ck.cakf_probe_peaks(stream.cuda_stream)
    fp64_peak = probe["fp64_flops_per_s"] / 1e12
    mufu_peak = probe["mufu_ops_per_s"] / 1e12
    peak_note = "measured by cakf_probe_peaks ({})"
    kernels = {}
    # DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from one ncu capture of
    # each kernel as it is now, on the shapes of this workload (summaries under profiles/):
    # k_tridiag at N = 576, k_gram_matvec_f2 at m = 8,192 (a launch of the first step, without the
    # M^T s blocks), k_gram_tc (split FP16) at 65,536 x 8,192 x 65.  Only the sphere-65k split-FP16
    # configuration has them; other runs report null.
    ncu_traffic = {"k_tridiag": 2705664.0, "k_gram_matvec": 197376.0, "k_gram_tc": 8160000.0} \
        if (args.config == "sphere-65k" and args.precision == "fp16x3") else {}
    # FP64 tridiagonalisation (the eigensolver's dominant part): (4/3) N^3 flops per call
    tri_ms = eig_parts[0]
    if prof["eig_calls"] and tri_ms > 0:
        ach = eig_flops[0] / (tri_ms / 1e3) / 1e12
        kernels["k_tridiag"] = {"bound": "alu", "achieved": ach, "peak": fp64_peak, "unit": "TFLOP/s",
                                "frac": ach / fp64_peak, "traffic": ncu_traffic.get("k_tridiag"),
                                "peak_source": peak_note.format("FP64 FMA chains, 2 flops each"),
                                "launches": prof["eig_calls"], "avg_ms": tri_ms / prof["eig_calls"],
                                "ms_total": tri_ms,
                                "note": "one cross-block exchange per Householder column (epoch-tagged word pairs, no grid barrier): bound by its latency chain, not by FP64 throughput"}
    # tensor-core / SIMT Gram x block (filter finalize): kernel entries on MUFU (sqrt + exp2 each)
    if prof["gram_block_launches"]:
        gb_ms = prof["gram_block_ms"]
        evals = prof["gram_block_evals"] / (gb_ms / 1e3) / 1e12
        tfl = prof["gram_block_flops"] / (gb_ms / 1e3) / 1e12
        ent = {"bound": "alu", "achieved": 2 * evals, "peak": mufu_peak, "unit": "TMUFU-op/s",
               "frac": 2 * evals / mufu_peak, "traffic": ncu_traffic.get("k_gram_tc"),
               "peak_source": peak_note.format("sqrt.approx + ex2.approx chains"),
               "launches": prof["gram_block_launches"], "avg_ms": gb_ms / prof["gram_block_launches"],
               "ms_total": gb_ms, "tensor_tflops": tfl}
        tc_modes = ("bf16", "fp16x3", "tf32", "tf32x3")
        if args.precision in tc_modes:
            tpk = float(pk.get("bf16_tflops_sustained", pk.get("bf16_tflops")))
            # TF32 MMAs: the measured BF16 rate times the nominal TF32 / BF16 dense ratio (1.1 / 2.25)
            tf32 = args.precision in ("tf32", "tf32x3")
            if tf32:
                tpk *= 1.1 / 2.25
            mmas = 3 if args.precision in ("fp16x3", "tf32x3") else 1
            ent["tensor_frac"] = mmas * tfl / tpk
            ent["tensor_peak_source"] = (f"{pk_src} bf16_tflops_sustained" + (" x 1.1/2.25 (nominal TF32/BF16)" if tf32 else "")
                                         + f"; {mmas} MMA(s) per algorithmic flop")
        kernels["k_gram_tc" if args.precision in tc_modes else "k_gram_block_simt"] = ent
    # CG Gram matvec (sampled every 8th iteration): m (m + 1) / 2 unique kernel entries per launch
    # (the symmetric Gram is evaluated once per entry pair), 2 MUFU operations each
    if prof["cg_matvec_launches"]:
        mv_ms = prof["cg_matvec_ms"]
        evals = prof["cg_matvec_evals"] / (mv_ms / 1e3) / 1e12
        kernels["k_gram_matvec"] = {"bound": "alu", "achieved": 2 * evals, "peak": mufu_peak,
                                    "unit": "TMUFU-op/s", "frac": 2 * evals / mufu_peak,
                                    "traffic": ncu_traffic.get("k_gram_matvec"),
                                    "peak_source": peak_note.format("sqrt.approx + ex2.approx chains"),
                                    "launches_sampled": prof["cg_matvec_launches"],
                                    "avg_ms": mv_ms / prof["cg_matvec_launches"],
                                    "ms_total": mv_ms * phases_launches_cg}
    dominant = max(kernels, key=lambda k: kernels[k]["ms_total"]) if kernels else None
    roof = dict(kernels[dominant], kernel=dominant) if dominant else None
    share = roof["ms_total"] / ms if roof and ms > 0 else None

    line = {
        "metric": "filter+smoother time steps/sec",
        "value": value, "unit": "time steps/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": DTYPE_NAME[args.precision], "data": "synthetic (seeded RFF prior sample; ERA5-shaped grid)",
        "config": {"workload": desc, "n": n, "m_per_step": int(w.obs_ptr[1] - w.obs_ptr[0]), "T": T,
                   "i": w.budget_i, "r": w.rank_r, "precision": args.precision, "factor_storage": args.storage,
                   "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
                   "l2": "working set larger than L2 (stored factors ~%.0f GB)" % (
                       (n * (w.rank_r + w.budget_i) * T * (8 if args.precision == 'fp64' else 4)) / 1e9)},
        "roofline": roof,
        "dominant_kernel_share_of_step": share,
        "roofline_kernels": kernels,
        "cg_matvec": {"avg_ms": prof["cg_matvec_ms"] / max(1, prof["cg_matvec_launches"]),
                      "evals_per_launch": prof["cg_matvec_evals"] / max(1, prof["cg_matvec_launches"])},
        "eig": {"calls": prof["eig_calls"], "avg_ms": prof["eig_ms"] / max(1, prof["eig_calls"]),
                "avg_ms_parts": dict(zip(["tridiagonalisation", "divide_conquer", "back_transform"],
                                         [p / max(1, prof["eig_calls"]) for p in eig_parts]))},
        "phase_ms": {"filter": st["filter_ms"], "smooth": st["smooth_ms"]},
        "phase_ms_per_pass": dict(zip(["filter_cg", "filter_finalize", "filter_truncate", "smooth_products",
                                       "smooth_combine", "smooth_truncate", "nll", "reserved"],
                                      [p / max(1, args.steps) for p in phases])),
        "clocks": clocks,
        "gpu_launches": launches,
        "probed_peaks": {"mufu_tops": mufu_peak, "fp64_tflops": fp64_peak,
                         "mufu_per_sm_per_clk": probe["mufu_ops_per_s"] / (nsm * clk),
                         "fp64_fma_per_sm_per_clk": probe["fp64_flops_per_s"] / 2 / (nsm * clk)},
    }

    # ---- end to end through the C ABI with pinned host buffers (copies inside the timed region)
    if not args.no_e2e:
        pin = lambda a, dt: torch.as_tensor(a).to(dt).pin_memory()
        hc = pin(w.coords, torch.float64)
        ho = pin(w.obs_idx, torch.int32)
        hy = pin(w.y, torch.float64)
        hm = None if w.prior_mean is None else pin(w.prior_mean, torch.float64)
        hprob = ck.make_problem(hc, w.kernel, w.log_lx, w.log_lt, w.log_sf2, w.log_sn2, T, w.dt, w.obs_ptr, ho, hy,
                                w.budget_i, w.rank_r, precision=args.precision, prior_mean=hm)
        houts = [torch.empty(shape, dtype=torch.float64).pin_memory() for _ in range(4)]
        ck.cakf_set_profiling(ctx, False)
        barrier(ws)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            ck.cakf_filter(hprob, ctx, houts[0], houts[1], stream=stream.cuda_stream)
            ck.cakf_smooth(ctx, houts[2], houts[3], stream=stream.cuda_stream)
        torch.cuda.synchronize(dev)
        te = allmax(ws, time.perf_counter() - t0)
        h2d = hc.numel() * 8 + ho.numel() * 4 + hy.numel() * 8 + (0 if hm is None else hm.numel() * 8)
        d2h = 4 * (T + 1) * n * 8
        line["e2e"] = {"value": ws * T * args.steps / te, "unit": "time steps/s", "h2d_bytes_per_step": h2d,
                       "d2h_bytes_per_step": d2h}

    # ---- NLL gradient on the last filter run (untimed by the steps/s figure; cakf_nll_backward runs on
    # the legacy default stream, timed with events there)
    if args.grad:
        torch.cuda.synchronize(dev)
        g0 = torch.cuda.Event(enable_timing=True)
        g1 = torch.cuda.Event(enable_timing=True)
        legacy = torch.cuda.default_stream(dev)
        g0.record(legacy)
        grad = ck.cakf_nll_backward(ctx)
        g1.record(legacy)
        torch.cuda.synchronize(dev)
        line["grad"] = {"ms": g0.elapsed_time(g1), "value": [float(x) for x in grad],
                        "wrt": ["log_lx", "log_lt", "log_sf2", "log_sn2"], "nll": ck.cakf_nll(ctx)}

    # ---- CPU baseline: the FP64 oracle on a bounded sample (rank 0, N = 1 only)
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        secs, sample = oracle_sample(w, args.cpu_row_frac)
        line["cpu_baseline"] = {"value": 1.0 / secs, "unit": "time steps/s", "cores": cpu_cores(), "kind": "oracle",
                                "sample": sample, "cpu": cpu_model()}
    ctx.close()

    # ---- accuracy of the timed precision against the device FP64 mode (untimed passes over the
    # first accuracy_steps steps; the FP64 mode's parity with the oracle is pinned by the tests).
    # The CG actions of this configuration are chaotic in the inputs (an FP64 run on data changed by
    # 1e-12 relative ends up as far from the unperturbed one as the FP32 run), so the arithmetic
    # error of a precision is measured on the same projected model: the FP64 run's actions
    # replayed.  The distance of the precision's own-action run is reported beside it.
    acc = None
    if not args.no_accuracy and args.precision != "fp64":
        acc = accuracy_passes(ck, w, coords, obs_idx, y, mu, args.precision, min(T, args.accuracy_steps), stream)
        line["accuracy"] = acc["timed"]
    # ---- the same workload through the plain FP32 path (SIMT Gram x block, FP32 factors), for the
    # mixed-vs-FP32 comparison the metric names: one untimed and three timed passes (median), events
    # on the stream
    if not args.no_fp32_compare and args.precision != "fp32":
        prob32 = ck.make_problem(coords, w.kernel, w.log_lx, w.log_lt, w.log_sf2, w.log_sn2, T, w.dt, w.obs_ptr,
                                 obs_idx, y, w.budget_i, w.rank_r, precision="fp32", prior_mean=mu)
        ctx32 = ck.Context()
        ck.cakf_filter(prob32, ctx32, outs[0], outs[1], stream=stream.cuda_stream)
        ck.cakf_smooth(ctx32, outs[2], outs[3], stream=stream.cuda_stream)
        times32 = []
        for _ in range(3):
            barrier(ws)
            torch.cuda.synchronize(dev)
            f0 = torch.cuda.Event(enable_timing=True)
            f1 = torch.cuda.Event(enable_timing=True)
            f0.record(stream)
            ck.cakf_filter(prob32, ctx32, outs[0], outs[1], stream=stream.cuda_stream)
            ck.cakf_smooth(ctx32, outs[2], outs[3], stream=stream.cuda_stream)
            f1.record(stream)
            torch.cuda.synchronize(dev)
            times32.append(allmax(ws, f0.elapsed_time(f1)))
        ms32 = statistics.median(times32)
        v32 = ws * T / (ms32 / 1e3)
        line["fp32_plain"] = {"value": v32, "unit": "time steps/s", "timed_passes": len(times32),
                              "ms_per_pass_median": ms32, "ms_per_pass_all": times32,
                              "mixed_over_fp32": value / v32}
        ctx32.close()
        if acc is not None:
            line["fp32_plain"]["accuracy"] = acc["fp32"]
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_reference(args, ws, rank):
    """The reference arm: the FP64 oracle (numpy, host cores) on a bounded sample of the same workload."""
    if rank != 0:
        return
    w, desc = workload(args.config, args.T, device=None)
    if args.warmup > 0:                       # one untimed sample (page-in, BLAS thread start)
        oracle_sample(w, args.cpu_row_frac)
    times = []
    sample = ""
    for _ in range(max(1, args.steps)):
        secs, sample = oracle_sample(w, args.cpu_row_frac)
        times.append(secs)
    tot = sum(times)
    value = len(times) / tot
    line = {"metric": "filter+smoother time steps/sec", "value": value, "unit": "time steps/s", "n_gpus": ws,
            "steps": len(times), "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": desc, "precision": "fp64 oracle"},
            "cpu_baseline": {"value": value, "unit": "time steps/s", "cores": cpu_cores(), "kind": "oracle",
                             "sample": sample, "cpu": cpu_model()},
            "e2e": {"value": value, "unit": "time steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
