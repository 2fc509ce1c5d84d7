"""Time the kernel-Gram x block primitive (cakf_gram_matmul) on one shape.

    python -m paper_2405_08971_gb300.gram_bench --nr 65536 --nc 65536 --width 513 --precision bf16
    python -m paper_2405_08971_gb300.gram_bench --nr 65536 --nc 8192 --width 65 --precision fp16x3

Coordinates are uniform on the unit sphere (the layout of the 256 x 256 lat-lon workload), B is
standard normal; all inputs are created on the device before timing.  Each repetition is one
cakf_gram_matmul call (operand packing + Gram x block kernel), timed with CUDA events on the
launching stream.  Prints one JSON line: the mean time per call and the algorithmic rate
2 * nr * nc * (width - 1) flops per call (the last column, accumulated on the CUDA cores, is
not counted).
"""
import argparse
import json
import math

import torch

from . import binding


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--nr", type=int, default=65536)
    ap.add_argument("--nc", type=int, default=65536)
    ap.add_argument("--width", type=int, default=513)
    ap.add_argument("--kernel", type=int, default=1, help="0, 1, 2: Matern 1/2, 3/2, 5/2")
    ap.add_argument("--lx", type=float, default=0.1)
    ap.add_argument("--precision", default="bf16", choices=["fp64", "fp32", "bf16", "fp16x3"])
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=2)
    a = ap.parse_args()
    dev = torch.device("cuda", 0)
    g = torch.Generator(device=dev).manual_seed(0)
    dt = torch.float64 if a.precision == "fp64" else torch.float32

    def sphere(n):
        x = torch.randn((n, 3), generator=g, device=dev, dtype=torch.float64)
        return (x / x.norm(dim=1, keepdim=True)).contiguous()

    Xr, Xc = sphere(a.nr), sphere(a.nc)
    B = torch.randn((a.width, a.nc), generator=g, device=dev, dtype=torch.float64).to(dt)
    out = torch.empty((a.width, a.nr), device=dev, dtype=dt)
    st = torch.cuda.current_stream(dev)
    call = lambda: binding.cakf_gram_matmul(a.kernel, math.log(a.lx), 0.0, Xr, Xc, B, out=out,
                                            precision=a.precision, stream=st.cuda_stream)
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
    flops = 2.0 * a.nr * a.nc * (a.width - 1)
    print(json.dumps({"nr": a.nr, "nc": a.nc, "width": a.width, "precision": a.precision, "ms_per_call": ms,
                      "tflops": flops / (ms / 1e3) / 1e12, "kernel_evals_per_s": a.nr * a.nc / (ms / 1e3)}))


if __name__ == "__main__":
    main()
