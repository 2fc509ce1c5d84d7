"""The Gram x matrix primitive (cakf_gram_matmul) against the oracle's dense definition.

Out = K(Xr, Xc) B with the Gram matrix never stored.  Sizes are ragged (rows not a multiple of the
128-row tile, columns not a multiple of the 64-column slice) and widths cover one MMA chunk, two
chunks and the 512-column TMEM limit; one case has more row tiles than the GPU has SMs, so the
persistent tensor-core grid splits tiles between CTAs.  Tolerances:
  FP64 SIMT   1e-12 relative (per column, normwise)
  FP32 SIMT   2e-5 relative
  BF16 tcgen05 columns 0..w-2: within 2e-4 of the exact product of the BF16-rounded operands
               (correlations and B rounded to bf16, FP64 accumulation, times sf2 after the
               contraction), i.e. the kernel adds only
               FP32 accumulation-order rounding to the BF16 operand rounding; and within 3e-2 of
               the exact product (the bf16 rounding itself, ~2^-9 per operand);
               the last column is accumulated in FP32 on the CUDA cores: 2e-5 relative.
  FP16X3      fp16 hi + lo parts of both operands (B scaled per column), three MMAs: within
               1e-4 of the exact product.  The operand parts carry 22 bits (2^-22 per product
               term); what remains is the tensor core's own FP32 accumulation, which measures
               1e-6..2e-5 on these cases (the same order as the BF16 path's distance from its
               exactly-accumulated BF16 emulation).
  TF32        kind::tf32, operands rounded to TF32 (round to nearest, 2^-11): within 2e-4 of the
               exact product of the TF32-rounded operands, and within 5e-3 of the exact product.
  TF32X3      tf32 hi + lo parts (no scaling), three kind::tf32 MMAs: within 1e-4 of the exact
               product, as FP16X3.
"""
import math

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2405_08971_gb300 as ck  # noqa: E402


def colwise_rel(got, ref):
    num = np.linalg.norm(got - ref, axis=1)
    den = np.maximum(np.linalg.norm(ref, axis=1), 1e-300)
    return num / den


def case(nr, nc, width, dim, kernel, seed, lx=0.3, sf2=1.7):
    rng = np.random.default_rng(seed)
    Xr = rng.uniform(size=(nr, dim))
    Xc = rng.uniform(size=(nc, dim))
    B = rng.standard_normal((width, nc))          # stored as (width, nc): column-major nc x width
    C = oracle.kernel_matrix(Xr, Xc, kernel, lx, 1.0)     # correlations; K = sf2 * C
    ref = sf2 * (C @ B.T).T
    bf = lambda a: torch.tensor(a, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    ref_bf16 = sf2 * (bf(C) @ bf(B).T).T
    return Xr, Xc, B, ref, ref_bf16, math.log(lx), math.log(sf2)


def tf32(a):
    """FP32 -> TF32 round to nearest (ties away from zero) on the magnitude bits, as cvt.rna.tf32."""
    bits = np.asarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    bits = ((bits + 0x1000) & 0xFFFFE000).astype(np.uint32)
    return bits.view(np.float32).astype(np.float64)


@pytest.mark.parametrize("nr,nc,width,dim,kernel", [
    (1000, 777, 2, 2, 1), (300, 257, 17, 3, 2), (513, 1000, 65, 1, 0), (257, 640, 257, 3, 1),
    (384, 300, 513, 2, 1), (130, 70, 100, 3, 2),
    (19500, 1000, 129, 2, 1),   # 153 row tiles: the persistent grid shares tiles between CTAs
])
def test_gram_matmul_all_precisions(nr, nc, width, dim, kernel):
    Xr, Xc, B, ref, ref_bf16, llx, lsf2 = case(nr, nc, width, dim, kernel, seed=nr + width)
    d = torch.device("cuda:0")
    tXr, tXc = torch.as_tensor(Xr, device=d), torch.as_tensor(Xc, device=d)
    out64 = ck.cakf_gram_matmul(kernel, llx, lsf2, tXr, tXc, torch.as_tensor(B, device=d), precision="fp64")
    e64 = colwise_rel(out64.cpu().numpy(), ref)
    assert e64.max() < 1e-12, e64.max()
    out32 = ck.cakf_gram_matmul(kernel, llx, lsf2, tXr, tXc, torch.as_tensor(B, device=d), precision="fp32")
    e32 = colwise_rel(out32.cpu().double().numpy(), ref)
    assert e32.max() < 2e-5, e32.max()
    outbf = ck.cakf_gram_matmul(kernel, llx, lsf2, tXr, tXc, torch.as_tensor(B, device=d), precision="bf16")
    got = outbf.cpu().double().numpy()
    ebf = colwise_rel(got, ref)
    emu = colwise_rel(got[:-1], ref_bf16[:-1])
    print(f"nr={nr} nc={nc} w={width}: fp64 {e64.max():.1e} fp32 {e32.max():.1e} "
          f"bf16 tc {ebf[:-1].max():.1e} (vs bf16-rounded operands {emu.max():.1e}) last-col {ebf[-1]:.1e}")
    assert emu.max() < 2e-4, emu.max()
    assert ebf[:-1].max() < 3e-2, ebf[:-1].max()
    assert ebf[-1] < 2e-5, ebf[-1]
    outx3 = ck.cakf_gram_matmul(kernel, llx, lsf2, tXr, tXc, torch.as_tensor(B, device=d), precision="fp16x3")
    ex3 = colwise_rel(outx3.cpu().double().numpy(), ref)
    print(f"   fp16x3 {ex3[:-1].max():.1e} last-col {ex3[-1]:.1e}")
    assert ex3[:-1].max() < 1e-4, ex3[:-1].max()
    assert ex3[-1] < 2e-5, ex3[-1]
    C = oracle.kernel_matrix(Xr, Xc, kernel, math.exp(llx), 1.0)
    ref_tf32 = math.exp(lsf2) * (tf32(C) @ tf32(B).T).T
    outtf = ck.cakf_gram_matmul(kernel, llx, lsf2, tXr, tXc, torch.as_tensor(B, device=d), precision="tf32")
    got = outtf.cpu().double().numpy()
    etf, emt = colwise_rel(got, ref), colwise_rel(got[:-1], ref_tf32[:-1])
    outt3 = ck.cakf_gram_matmul(kernel, llx, lsf2, tXr, tXc, torch.as_tensor(B, device=d), precision="tf32x3")
    et3 = colwise_rel(outt3.cpu().double().numpy(), ref)
    print(f"   tf32 {etf[:-1].max():.1e} (vs tf32-rounded operands {emt.max():.1e}) tf32x3 {et3[:-1].max():.1e} "
          f"last-col {etf[-1]:.1e} {et3[-1]:.1e}")
    assert emt.max() < 2e-4, emt.max()
    assert etf[:-1].max() < 5e-3, etf[:-1].max()
    assert et3[:-1].max() < 1e-4, et3[:-1].max()
    assert etf[-1] < 2e-5 and et3[-1] < 2e-5


def test_gram_matmul_rejects_host_pointers():
    """Host tensors are refused by the binding (ValueError) and, passed straight to the C ABI, by
    the library (CAKF_ERR_ARG) before any launch."""
    Xr = torch.zeros((4, 2), dtype=torch.float64)
    B = torch.zeros((3, 4), dtype=torch.float32)
    out = torch.zeros((3, 4), dtype=torch.float32)
    with pytest.raises(ValueError):
        ck.cakf_gram_matmul(1, 0.0, 0.0, Xr, Xr, B, out=out, precision="fp32")
    for fn in (ck.lib().cakf_gram_matmul, ck.lib().cakf_gram_matmul_noalloc):
        rc = fn(1, 0.0, 0.0, 2, Xr.data_ptr(), 4, Xr.data_ptr(), 4, B.data_ptr(), 4, 3, out.data_ptr(), 4,
                ck.FP32, None)
        assert rc == ck.binding.ERR_ARG
