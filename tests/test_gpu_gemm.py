"""The tall-skinny factor products (cakf_factor_gemm) against FP64 products of the same FP32 inputs.

These are the products of the downdate factors in the filter's finalize and Truncate (Sec. 3.2) and in
the smoother (Alg. 3): a tall factor times a small coefficient block (NN: n x K times K x N) and the
projection of one tall block onto another (TN: n x M transposed times n x N), with n up to the
65,536-state workload's size.  Shapes are ragged (rows not a multiple of the 128-row tile, K not a
multiple of the 16-wide slice, N above the 256-column chunk so that it is split into chunks).  NN
products with at least 64 row tiles take B pre-split into its stage layout (one bulk copy per
stage); the others split B in the producers.

Tolerance, per output column normwise relative to the exact product of the FP32 inputs:
  FP32 SIMT            1e-5 (FP32 accumulation over K up to 65,536 terms)
  split TF32 tcgen05   5e-5: hi + lo TF32 parts carry about 22 bits per operand (2^-21 per product
                       term after dropping lo * lo), FP32 accumulation in TMEM over at most 1,024
                       K values, partial tiles summed in FP64 (TN).  Measured: NN 6.7e-6, TN up
                       to 3e-5 on sums of 65,536 random-sign terms (the tensor core's FP32
                       accumulation inside an MMA is the larger part).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2405_08971_gb300 as ck  # noqa: E402

TOL = {"fp32": 1e-5, "tf32x3": 5e-5}


def colwise_rel(got, ref):
    return np.linalg.norm(got - ref, axis=1) / np.maximum(np.linalg.norm(ref, axis=1), 1e-300)


def factors(rows, cols, rng, decay=6.0):
    """A tall block whose columns span several orders of magnitude, like a downdate factor."""
    scale = np.exp(-decay * np.arange(cols) / max(cols, 1))
    return (rng.standard_normal((rows, cols)) * scale[None, :]).astype(np.float32)


@pytest.mark.parametrize("precision", ["fp32", "tf32x3"])
@pytest.mark.parametrize("M,K,N", [(5000, 576, 512), (65536, 576, 512), (4097, 512, 577), (300000 // 7, 64, 65),
                                   (2000, 17, 33), (20000, 100, 300)])
def test_nn_tall_times_small(precision, M, K, N):
    rng = np.random.default_rng(M + K + N)
    A = factors(M, K, rng)                                    # column-major M x K = row-major (K, M)^T
    B = rng.standard_normal((K, N)).astype(np.float32)
    C0 = rng.standard_normal((M, N)).astype(np.float32)
    d = torch.device("cuda:0")
    tA = torch.as_tensor(np.ascontiguousarray(A.T), device=d)
    tB = torch.as_tensor(np.ascontiguousarray(B.T), device=d)
    tC = torch.as_tensor(np.ascontiguousarray(C0.T), device=d)
    ck.cakf_factor_gemm(tA, tB, tC, alpha=-0.7, beta=1.0, precision=precision)
    ref = -0.7 * (A.astype(np.float64) @ B.astype(np.float64)) + C0.astype(np.float64)
    e = colwise_rel(tC.cpu().double().numpy(), ref.T)
    print(f"NN {precision} M={M} K={K} N={N}: {e.max():.2e}")
    assert e.max() < TOL[precision], e.max()


@pytest.mark.parametrize("precision", ["fp32", "tf32x3"])
@pytest.mark.parametrize("K,M,N", [(65536, 512, 577), (65536, 512, 64), (8191, 64, 577), (70000, 64, 64),
                                   (1000, 40, 3)])
def test_tn_projection(precision, K, M, N):
    rng = np.random.default_rng(K + M + N)
    A = factors(K, M, rng)
    B = factors(K, N, rng, decay=2.0)
    d = torch.device("cuda:0")
    tA = torch.as_tensor(np.ascontiguousarray(A.T), device=d)   # (M, K): column-major K x M
    tB = torch.as_tensor(np.ascontiguousarray(B.T), device=d)
    tC = ck.cakf_factor_gemm(tA, tB, trans_a=True, precision=precision)
    ref = A.astype(np.float64).T @ B.astype(np.float64)
    e = colwise_rel(tC.cpu().double().numpy(), ref.T)
    print(f"TN {precision} K={K} M={M} N={N}: {e.max():.2e}")
    assert e.max() < TOL[precision], e.max()
