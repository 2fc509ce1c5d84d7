"""Models (no GPU) of index arithmetic in the device kernels, checked against plain definitions:

* the merge of two ascending child spectra by rank in divide & conquer (k_dc_prep): entry t of
  child 1 goes to t + #(child-2 keys < key_t), entry u of child 2 to u + #(child-1 keys <= key_u);
  the result must be a permutation equal to a stable merge (child 1 first on ties);
* the butterfly reduce-scatter of the CG matvec (k_gram_matvec_f2): 32 lanes, each with 32
  per-column partial sums, exchange halves over offsets 16, 8, 4, 2, 1; lane l must end with the
  sum over lanes of column l;
* the order-preserving integer key of a double used by the sorts (negative values mirrored).
"""
import struct

import numpy as np
import pytest


def order_key(x):
    b = struct.unpack("<q", struct.pack("<d", x))[0]
    return b if b >= 0 else b ^ 0x7FFFFFFFFFFFFFFF


def merge_by_rank(k1, k2):
    n1, K = len(k1), len(k1) + len(k2)
    keys = list(k1) + list(k2)
    perm = [None] * K
    for t in range(K):
        kt = keys[t]
        if t < n1:
            a, b = n1, K                      # first child-2 index with key >= kt
            while a < b:
                m = (a + b) >> 1
                if keys[m] < kt:
                    a = m + 1
                else:
                    b = m
            pos = t + (a - n1)
        else:
            a, b = 0, n1                      # first child-1 index with key > kt
            while a < b:
                m = (a + b) >> 1
                if keys[m] <= kt:
                    a = m + 1
                else:
                    b = m
            pos = (t - n1) + a
        assert perm[pos] is None
        perm[pos] = t
    return perm


@pytest.mark.parametrize("seed", range(10))
def test_merge_by_rank_is_a_stable_merge(seed):
    rng = np.random.default_rng(seed)
    n1, n2 = int(rng.integers(1, 40)), int(rng.integers(1, 40))
    pool = rng.normal(size=8)                 # few distinct values: many ties within and across
    v1 = np.sort(rng.choice(pool, n1))
    v2 = np.sort(rng.choice(pool, n2))
    perm = merge_by_rank([order_key(x) for x in v1], [order_key(x) for x in v2])
    vals = np.concatenate([v1, v2])
    stable = sorted(range(n1 + n2), key=lambda t: (vals[t], 0 if t < n1 else 1, t))
    assert perm == stable


def test_order_key_is_monotone():
    rng = np.random.default_rng(1)
    x = np.sort(np.concatenate([rng.normal(size=200) * 10.0 ** rng.integers(-30, 30, 200),
                                [0.0, 1e-310, -1e-310, np.inf, -np.inf]]))
    keys = [order_key(v) for v in x]
    assert all(a <= b for a, b in zip(keys, keys[1:]))


def test_butterfly_reduce_scatter():
    rng = np.random.default_rng(2)
    v = rng.normal(size=(32, 32))             # v[lane, column]
    want = v.sum(axis=0)
    cur = v.copy()
    o = 16
    while o >= 1:
        new = cur.copy()
        for lane in range(32):
            up = (lane & o) != 0
            partner = lane ^ o
            for q in range(o):
                send_partner = cur[partner, q] if ((partner & o) != 0) else cur[partner, q + o]
                keep = cur[lane, q + o] if up else cur[lane, q]
                new[lane, q] = keep + send_partner
        cur = new
        o >>= 1
    np.testing.assert_allclose(cur[:, 0], want, rtol=1e-12)
