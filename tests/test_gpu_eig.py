"""The FP64 eigensolver of Truncate (cakf_eig_topk) against LAPACK (numpy.linalg.eigh).

Matrices: dense random PSD Grams, the structured Gram the filter truncation meets
([diag(a^2 lambda), B; B^T, C] with the leading block diagonal), and spectra with clusters and
exact repeats (the deflation paths of divide & conquer).  Orders span the shared-memory
configurations of the kernels (40 .. 640, around 512).

Bounds (FP64, backward stable algorithms): eigenvalues within 1e-12 * ||A||_2 of LAPACK's;
residual ||A U - U diag(w)||_F <= 1e-12 * ||A||_2 * sqrt(keep); ||U^T U - I||_max <= 1e-12.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2405_08971_gb300 as ck  # noqa: E402


def random_gram(N, seed):
    rng = np.random.default_rng(seed)
    M = rng.standard_normal((N + 7, N)) * np.exp(-np.arange(N) / (N / 6.0))
    return M.T @ M


def filter_gram(N, i, seed):
    """[diag(d), B; B^T, C]: the Gram of [a M+ (orthogonal columns), P^-W] the filter truncates."""
    rng = np.random.default_rng(seed)
    r = N - i
    d = np.sort(np.exp(-np.arange(r) / 40.0) * rng.uniform(0.5, 1.5, r))[::-1]
    n = 3 * N
    Q, _ = np.linalg.qr(rng.standard_normal((n, r)))
    Mp = Q * np.sqrt(d)
    W = rng.standard_normal((n, i)) * 0.3
    F = np.concatenate([Mp, W], axis=1)
    return F.T @ F


def clustered(N, seed):
    rng = np.random.default_rng(seed)
    lam = np.repeat(np.linspace(1.0, 4.0, N // 8 + 1), 8)[:N]
    lam[: N // 4] += 1e-13 * rng.standard_normal(N // 4)
    Q, _ = np.linalg.qr(rng.standard_normal((N, N)))
    return (Q * lam) @ Q.T


CASES = []
for N in (40, 300, 511, 512, 513, 576, 640):
    CASES.append(("random", N, N - 64 if N > 64 else N // 2))
for N in (512, 576, 640):
    CASES.append(("filter", N, N - 64))
for N in (96, 576):
    CASES.append(("clustered", N, N // 2))


def case_matrix(kind, N):
    if kind == "random":
        A = random_gram(N, seed=N)
    elif kind == "filter":
        A = filter_gram(N, 64, seed=N)
    else:
        A = clustered(N, seed=N)
    return 0.5 * (A + A.T)


@pytest.mark.parametrize("kind,N,keep", CASES)
def test_eig_topk_against_lapack(kind, N, keep):
    A = case_matrix(kind, N)
    nrm = np.linalg.norm(A, 2)
    w_ref = np.linalg.eigvalsh(A)[::-1][:keep]
    w, U = ck.cakf_eig_topk(torch.as_tensor(A, device="cuda"), keep)
    w = w.cpu().numpy()
    U = U.cpu().numpy().T            # N x keep
    ew = np.max(np.abs(w - w_ref)) / nrm
    res = np.linalg.norm(A @ U - U * w) / (nrm * np.sqrt(keep))
    orth = np.max(np.abs(U.T @ U - np.eye(keep)))
    print(kind, N, keep, f"eigvals {ew:.1e} residual {res:.1e} orthogonality {orth:.1e}")
    assert ew <= 1e-12, ew
    assert res <= 1e-12, res
    assert orth <= 1e-12, orth


@pytest.mark.parametrize("kind,N,keep", CASES)
def test_eig_topk_mixed_assembly(kind, N, keep):
    """The eigensolver as the FP32-based modes run it: eigenvalues from the same FP64 code (equal
    bit for bit), eigenvectors assembled in double-FP32 -- within 1e-12 of the FP64 assembly entry
    by entry, and held to the same LAPACK bounds."""
    A = case_matrix(kind, N)
    nrm = np.linalg.norm(A, 2)
    At = torch.as_tensor(A, device="cuda")
    w, U = ck.cakf_eig_topk(At, keep)
    wm, Um = ck.cakf_eig_topk(At, keep, mixed=True)
    assert torch.equal(w, wm)
    du = float((Um - U).abs().max())
    Um = Um.cpu().numpy().T
    wm = wm.cpu().numpy()
    res = np.linalg.norm(A @ Um - Um * wm) / (nrm * np.sqrt(keep))
    orth = np.max(np.abs(Um.T @ Um - np.eye(keep)))
    print(kind, N, keep, f"assembly {du:.1e} residual {res:.1e} orthogonality {orth:.1e}")
    assert du <= 1e-12, du
    assert res <= 1e-12, res
    assert orth <= 1e-12, orth
