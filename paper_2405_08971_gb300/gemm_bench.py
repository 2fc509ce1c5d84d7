"""Time the factor product primitive (cakf_factor_gemm) on one shape.

    python -m paper_2405_08971_gb300.gemm_bench --m 65536 --n 512 --k 576              # M+ = M U
    python -m paper_2405_08971_gb300.gemm_bench --m 512 --n 577 --k 65536 --trans-a    # M^T X

A and B are standard normal FP32, created on the device before timing.  Each repetition is one
cakf_factor_gemm call (C = op(A) B, beta = 0), timed with CUDA events on the launching stream.
Prints one JSON line: the mean time per call and the algorithmic rate 2 M N K flops per call.
"""
import argparse
import json

import torch

from . import binding


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--m", type=int, default=65536)
    ap.add_argument("--n", type=int, default=512)
    ap.add_argument("--k", type=int, default=576)
    ap.add_argument("--trans-a", action="store_true", help="op(A) = A^T (A stored K x M)")
    ap.add_argument("--precision", default="tf32x3", choices=["fp32", "tf32x3"])
    ap.add_argument("--reps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    a = ap.parse_args()
    dev = torch.device("cuda", 0)
    g = torch.Generator(device=dev).manual_seed(0)
    A = torch.randn((a.m, a.k) if a.trans_a else (a.k, a.m), generator=g, device=dev)
    B = torch.randn((a.n, a.k), generator=g, device=dev)
    C = torch.zeros((a.n, a.m), device=dev)
    st = torch.cuda.current_stream(dev)
    call = lambda: binding.cakf_factor_gemm(A, B, C, trans_a=a.trans_a, precision=a.precision,
                                            stream=st.cuda_stream)
    for _ in range(a.warmup):
        call()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(a.reps):
        call()
    e1.record(st)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / a.reps
    flops = 2.0 * a.m * a.n * a.k
    print(json.dumps({"m": a.m, "n": a.n, "k": a.k, "trans_a": a.trans_a, "precision": a.precision,
                      "ms_per_call": ms, "tflops": flops / (ms / 1e3) / 1e12}))


if __name__ == "__main__":
    main()
