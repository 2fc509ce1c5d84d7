"""cakf_gram_matmul_noalloc (static device scratch, no allocation in the call) against
cakf_gram_matmul, the entry point that allocates its scratch.

Both run the same kernels on the same inputs, so each no-alloc result must match the allocating
one within the tolerance of the path (FP64 1e-13, FP32 / BF16 1e-6 relative; the kernels are
deterministic, so equality is expected).  Each case calls the no-alloc entry point twice in a row
into separate outputs: the second call must not see anything left by the first.  The file is
collected last so that it also runs after every other test has used the device; it holds no
state of its own and passes alone as well.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2405_08971_gb300 as ck  # noqa: E402

SCRATCH = 64 << 20
TOL = {"fp64": 1e-13, "fp32": 1e-6, "bf16": 1e-6, "fp16x3": 1e-6}


def inputs(nr, nc, width, dim, precision, seed):
    g = torch.Generator().manual_seed(seed)
    d = torch.device("cuda:0")
    dt = torch.float64 if precision == "fp64" else torch.float32
    Xr = torch.rand((nr, dim), generator=g, dtype=torch.float64).to(d)
    Xc = torch.rand((nc, dim), generator=g, dtype=torch.float64).to(d)
    B = torch.randn((width, nc), generator=g, dtype=torch.float64).to(dt).to(d)
    outs = [torch.full((width, nr), float("nan"), dtype=dt, device=d) for _ in range(3)]
    return Xr, Xc, B, outs


def rel(a, b):
    a, b = a.double(), b.double()
    return float((a - b).norm() / b.norm().clamp_min(1e-300))


CASES = [
    (1000, 777, 2, 2, 1, "fp64"), (513, 1000, 65, 1, 0, "fp32"), (300, 257, 17, 3, 2, "bf16"),
    (384, 300, 513, 2, 1, "bf16"), (4096, 32768, 513, 3, 1, "bf16"), (2000, 65536, 257, 2, 1, "bf16"),
    # split FP16: two packed operand parts plus the per-column scales in the staging area
    (700, 1000, 33, 2, 1, "fp16x3"), (4096, 32768, 257, 3, 1, "fp16x3"),
]


@pytest.mark.parametrize("nr,nc,width,dim,kernel,precision", CASES)
def test_noalloc_matches_allocating_entry_point(nr, nc, width, dim, kernel, precision):
    Xr, Xc, B, (ref, o1, o2) = inputs(nr, nc, width, dim, precision, seed=nr + nc + width)
    llx, lsf2 = math.log(0.2), math.log(1.3)
    ck.cakf_gram_matmul(kernel, llx, lsf2, Xr, Xc, B, out=ref, precision=precision)
    ck.cakf_gram_matmul_noalloc(kernel, llx, lsf2, Xr, Xc, B, o1, precision=precision)
    ck.cakf_gram_matmul_noalloc(kernel, llx, lsf2, Xr, Xc, B, o2, precision=precision)
    torch.cuda.synchronize()
    assert torch.isfinite(o1).all() and torch.isfinite(o2).all()
    e1, e2 = rel(o1, ref), rel(o2, ref)
    assert e1 <= TOL[precision], e1
    assert e2 <= TOL[precision], e2


@pytest.mark.parametrize("nc,width,precision", [(65536, 513, "bf16"), (32768, 513, "fp16x3")])
def test_noalloc_rejects_calls_beyond_the_scratch(nc, width, precision):
    """BF16 with nc = 65536 and width 513 needs the packed operand (64 MiB) plus coordinates; split
    FP16 needs twice the operand bytes, so nc = 32768 at width 513 is over the limit as well."""
    Xr, Xc, B, (out, _, _) = inputs(256, nc, width, 2, precision, seed=7)
    with pytest.raises(ck.CakfError) as ei:
        ck.cakf_gram_matmul_noalloc(1, 0.0, 0.0, Xr, Xc, B, out, precision=precision)
    assert ei.value.code == ck.binding.ERR_ARG
    assert "bytes of scratch" in str(ei.value) and str(SCRATCH) in str(ei.value)
    assert torch.isnan(out).all()          # rejected before any device work


def test_noalloc_leaves_free_device_memory_unchanged():
    """After a first call has loaded the kernels, further calls change the device's free memory by
    nothing: the call takes no device memory."""
    cases = [inputs(nr, nc, w, dim, p, seed=11) + (k, p) for nr, nc, w, dim, k, p in CASES[:5]]
    for Xr, Xc, B, outs, k, p in cases:
        ck.cakf_gram_matmul_noalloc(k, 0.1, 0.2, Xr, Xc, B, outs[0], precision=p)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for Xr, Xc, B, outs, k, p in cases:
        ck.cakf_gram_matmul_noalloc(k, 0.1, 0.2, Xr, Xc, B, outs[1], precision=p)
        ck.cakf_gram_matmul_noalloc(k, 0.1, 0.2, Xr, Xc, B, outs[2], precision=p)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    for Xr, Xc, B, outs, k, p in cases:
        assert torch.equal(outs[1], outs[2])
