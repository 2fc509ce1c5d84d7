"""A model of the CG matvec's tiling (no GPU), following k_gram_matvec / k_gram_matvec_f2: the
symmetric K(X_o, X_o) is cut into T x T tiles; block b decodes to the tile pair (I, J), I <= J, by
walking the upper triangle row by row; it writes the row sums of tile (I, J) (weights s_J) to slot
J of the rows of I and, for I < J, the column sums (weights s_I) to slot I of the rows of J.  The
model checks that every (slot, row) is written exactly once -- so the combine's fixed-order sum is
deterministic and needs no zeroing -- and that the slot sums equal K s, for ragged m."""
import numpy as np
import pytest


def decode(b, nb):
    idx, I = b, 0
    while idx >= nb - I:
        idx -= nb - I
        I += 1
    return I, I + idx


@pytest.mark.parametrize("m,T", [(1, 128), (127, 128), (128, 128), (129, 128), (300, 128), (1000, 64)])
def test_slots_written_once_and_sum_to_the_product(m, T):
    rng = np.random.default_rng(m)
    A = rng.standard_normal((m, m))
    K = A @ A.T                                   # any symmetric matrix
    s = rng.standard_normal(m)
    nb = max(1, (m + T - 1) // T)
    part = np.full((nb, m), np.nan)
    written = np.zeros((nb, m), dtype=int)
    for b in range(nb * (nb + 1) // 2):
        I, J = decode(b, nb)
        assert 0 <= I <= J < nb
        ri = np.arange(I * T, min(m, (I + 1) * T))
        rj = np.arange(J * T, min(m, (J + 1) * T))
        if ri.size == 0 or rj.size == 0:
            continue
        blk = K[np.ix_(ri, rj)]
        part[J, ri] = blk @ s[rj]
        written[J, ri] += 1
        if I != J:
            part[I, rj] = blk.T @ s[ri]
            written[I, rj] += 1
    assert np.all(written == 1)
    np.testing.assert_allclose(part.sum(axis=0), K @ s, rtol=1e-12, atol=1e-12 * np.abs(K @ s).max())
