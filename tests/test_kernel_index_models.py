"""Models (no GPU) of index arithmetic in the device kernels, checked against plain definitions:

* the merge of two ascending child spectra by rank in divide & conquer (k_dc_prep): entry t of
  child 1 goes to t + #(child-2 keys < key_t), entry u of child 2 to u + #(child-1 keys <= key_u);
  the result must be a permutation equal to a stable merge (child 1 first on ties);
* the butterfly reduce-scatter of the CG matvec (k_gram_matvec_f2): 32 lanes, each with 32
  per-column partial sums, exchange halves over offsets 16, 8, 4, 2, 1; lane l must end with the
  sum over lanes of column l;
* the order-preserving integer key of a double used by the sorts (negative values mirrored);
* the close-pole deflation of k_dc_prep (pair tests on the merged values, sequential scan only from
  the first pair that fires) against the full sequential scan, on clustered poles with tiny z
  components, and the grouped, register-carried rotation application of k_dc_rot against applying
  the rotations one by one;
* the merge product of k_dc_gemm, whose row tiles skip the kept columns supported on the other
  child only, against the full product;
* the stream-K partition of the tcgen05 Gram x block over (row tile, K slice) units: a tile is
  shared by at most two CTAs, so its atomic accumulation onto zeros is order-independent;
* the split-FP16 operands (hi + lo parts, B columns scaled by a power of two, three exact products
  per pair) against exact products: about 22 significant bits (one FP16 part alone: ~11);
* the compensated FP32 row sums of squares (row_sumsq) against exact sums, and the epoch tag of
  the tridiagonalisation's exchange words (at most 3 ulps of change).
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


# ---- divide & conquer deflation (k_dc_prep, k_dc_rot)
def scan_full(D, Z, small, tol):
    """Sequential close-pole scan over all entries (the definition)."""
    D, Z = D.copy(), Z.copy()
    stat = [1 if s else 0 for s in small]
    rots, last = [], -1
    for j in range(len(D)):
        if stat[j]:
            continue
        if last >= 0:
            zl, zj, dl, dj = Z[last], Z[j], D[last], D[j]
            t2 = zl * zl + zj * zj
            if abs(dj - dl) * abs(zl * zj) <= tol * t2:
                t = np.sqrt(t2)
                c, s = zj / t, -zl / t
                rots.append((last, j, c, s))
                D[last], D[j] = c * c * dl + s * s * dj, s * s * dl + c * c * dj
                Z[last], Z[j] = 0.0, t
                stat[last] = 2
        last = j
    return D, Z, stat, rots


def scan_from_first_firing(D, Z, small, tol):
    """The kernel's form: test consecutive candidate pairs on the merged values (in parallel),
    then scan sequentially from the first pair that fires."""
    cand = [j for j in range(len(D)) if not small[j]]
    fires = [u for u in range(1, len(cand))
             if abs(D[cand[u]] - D[cand[u - 1]]) * abs(Z[cand[u - 1]] * Z[cand[u]])
             <= tol * (Z[cand[u - 1]] ** 2 + Z[cand[u]] ** 2)]
    D, Z = D.copy(), Z.copy()
    stat = [1 if s else 0 for s in small]
    rots = []
    if fires:
        first = fires[0]
        last = cand[first - 1]
        for u in range(first, len(cand)):
            j = cand[u]
            zl, zj, dl, dj = Z[last], Z[j], D[last], D[j]
            t2 = zl * zl + zj * zj
            if abs(dj - dl) * abs(zl * zj) <= tol * t2:
                t = np.sqrt(t2)
                c, s = zj / t, -zl / t
                rots.append((last, j, c, s))
                D[last], D[j] = c * c * dl + s * s * dj, s * s * dl + c * c * dj
                Z[last], Z[j] = 0.0, t
                stat[last] = 2
            last = j
    return D, Z, stat, rots


def apply_sequential(Q, rots):
    Q = Q.copy()
    for a, b, c, s in rots:
        qa, qb = Q[:, a].copy(), Q[:, b].copy()
        Q[:, a], Q[:, b] = c * qa + s * qb, -s * qa + c * qb
    return Q


def apply_grouped(Q, rots, RG=8):
    """k_dc_rot per row: groups of RG rotations load their operands first; the a_q = b_{q-1}
    chain is carried in a register."""
    Q = Q.copy()
    for row in range(Q.shape[0]):
        carry, carry_col = 0.0, -1
        for q0 in range(0, len(rots), RG):
            grp = rots[q0:q0 + RG]
            xa, xb = [], []
            for u, (a, b, _, _) in enumerate(grp):
                prev = carry_col if u == 0 else grp[u - 1][1]
                xb.append(Q[row, b])
                xa.append(0.0 if a == prev else Q[row, a])
            for u, (a, b, c, s) in enumerate(grp):
                prev = carry_col if u == 0 else grp[u - 1][1]
                av = carry if a == prev else xa[u]
                na, nb = c * av + s * xb[u], -s * av + c * xb[u]
                Q[row, a], Q[row, b] = na, nb
                carry, carry_col = nb, b
    return Q


@pytest.mark.parametrize("seed", range(12))
def test_deflation_scan_and_rotation_application(seed):
    rng = np.random.default_rng(100 + seed)
    K = int(rng.integers(4, 60))
    D = np.sort(rng.choice(np.round(rng.normal(size=K // 3 + 2), 1), K)
                + 1e-15 * rng.normal(size=K))                 # clusters of near-equal poles
    Z = rng.normal(size=K)
    Z[rng.random(K) < 0.2] *= 1e-17                            # some tiny components
    Z /= np.linalg.norm(Z)
    rho, tol = 1.3, 8 * 2.22e-16 * 3.0
    small = [rho * abs(z) <= tol for z in Z]
    ref = scan_full(D, Z, small, tol)
    got = scan_from_first_firing(D, Z, small, tol)
    assert ref[2] == got[2] and len(ref[3]) == len(got[3])
    np.testing.assert_array_equal(ref[0], got[0])
    np.testing.assert_array_equal(ref[1], got[1])
    Q = rng.normal(size=(K, K))
    np.testing.assert_allclose(apply_grouped(Q, ref[3]), apply_sequential(Q, ref[3]), rtol=0, atol=1e-13)


# ---- divide & conquer merge product (k_dc_gemm with the support grouping of k_dc_prep)
@pytest.mark.parametrize("seed", range(6))
def test_merge_product_skips_only_zero_blocks(seed):
    """The child eigenvector matrix of a merge is block diagonal; columns mixed by a deflation
    rotation have both supports.  Kept columns are ordered child-1-only, mixed, child-2-only (gperm,
    counts g1, g2); a 32-row tile inside child 1 sums over [0, g1 + g2), inside child 2 over
    [g1, Kp), a straddling tile over all -- the same product as the full sum."""
    rng = np.random.default_rng(200 + seed)
    K = int(rng.integers(40, 130))
    n1 = K // 2
    Q = np.zeros((K, K))
    Q[:n1, :n1] = rng.normal(size=(n1, n1))
    Q[n1:, n1:] = rng.normal(size=(K - n1, K - n1))
    typ = np.array([1] * n1 + [3] * (K - n1))
    for _ in range(int(rng.integers(0, 6))):                  # a few mixing rotations
        a, b = int(rng.integers(0, n1)), int(rng.integers(n1, K))
        c, s = np.cos(0.3), np.sin(0.3)
        qa, qb = Q[:, a].copy(), Q[:, b].copy()
        Q[:, a], Q[:, b] = c * qa + s * qb, -s * qa + c * qb
        typ[a] = typ[b] = 2
    keep = np.sort(rng.choice(K, size=int(0.8 * K), replace=False))  # kept columns (pole order)
    Kp = len(keep)
    U = rng.normal(size=(Kp, Kp))
    gperm = [q for t in (1, 2, 3) for q in range(Kp) if typ[keep[q]] == t]
    g1 = sum(typ[keep[q]] == 1 for q in range(Kp))
    g2 = sum(typ[keep[q]] == 2 for q in range(Kp))
    full = Q[:, keep] @ U
    out = np.zeros_like(full)
    for r0 in range(0, K, 32):
        rows = slice(r0, min(K, r0 + 32))
        kb, ke = 0, Kp
        if r0 + 32 <= n1:
            ke = g1 + g2
        elif r0 >= n1:
            kb = g1
        idx = gperm[kb:ke]
        out[rows] = Q[rows][:, keep[idx]] @ U[idx]
    np.testing.assert_allclose(out, full, rtol=1e-12, atol=1e-12 * np.abs(full).max())


# ---- tcgen05 Gram x block: stream-K partition of (row tile, K slice) units (gram_tc launch)
@pytest.mark.parametrize("ntiles,nk,slots", [(1, 2048, 152), (3, 7, 152), (512, 256, 152), (152, 1, 152),
                                             (153, 5, 152), (2048, 33, 304), (600, 1, 152)])
def test_stream_k_splits_a_tile_over_at_most_two_ctas(ntiles, nk, slots):
    """grid = min(#tiles, resident slots); CTA b takes units [total b / grid, total (b+1) / grid).
    Every range then holds at least one tile's worth of units, so a tile is shared by at most two
    CTAs -- its two partial sums added with atomics onto zeros are order-independent."""
    grid = min(ntiles, slots)
    total = ntiles * nk
    owners = [set() for _ in range(ntiles)]
    for b in range(grid):
        u0, u1 = total * b // grid, total * (b + 1) // grid
        assert u1 - u0 >= nk
        for u in range(u0, u1):
            owners[u // nk].add(b)
    assert max(len(o) for o in owners) <= 2
    assert set().union(*owners) == set(range(grid))


# ---- split-FP16 operands of the tcgen05 Gram x block (k_col_scale, k_pack_b, producers)
def split16(x):
    hi = x.astype(np.float16)
    lo = (x - hi.astype(np.float32)).astype(np.float16)
    return hi.astype(np.float32), lo.astype(np.float32)


@pytest.mark.parametrize("seed", range(4))
def test_split_fp16_products_carry_about_22_bits(seed):
    """Each kernel value k in (0, 1] and each B entry (column scaled by a power of two so that its
    largest magnitude is in [0.5, 1)) is written as hi + lo FP16 parts; the three products
    hi*hi + hi*lo + lo*hi are exact in FP32.  Against the exact product sum the error stays below
    4 * 2^-22 of sum |k| |b| per output -- the split's ~22 significant bits."""
    rng = np.random.default_rng(300 + seed)
    rows, cols = 512, 8
    k = np.exp(-rng.uniform(0, 8, size=rows)).astype(np.float32)            # correlations
    B = (rng.normal(size=(rows, cols)) * 10.0 ** rng.uniform(-3, 3, size=cols)).astype(np.float32)
    e = np.frexp(np.abs(B).max(axis=0))[1]
    sc = np.ldexp(1.0, -e).astype(np.float32)                                 # k_col_scale
    Bs = (B * sc).astype(np.float32)
    kh, kl = split16(k)
    bh, bl = split16(Bs)
    approx = (kh[:, None].astype(np.float64) * bh + kh[:, None] * bl + kl[:, None] * bh).sum(axis=0)
    approx = approx / sc                                                       # epilogue scale back
    exact = (k.astype(np.float64)[:, None] * B.astype(np.float64)).sum(axis=0)
    scale = (np.abs(k.astype(np.float64))[:, None] * np.abs(B.astype(np.float64))).sum(axis=0)
    assert np.all(np.abs(approx - exact) <= 4 * 2.0 ** -22 * scale)


# ---- compensated FP32 row sums of squares (row_sumsq) and the epoch tag of the exchange words
def kahan4(v):
    """row_sumsq for FP32 data: four compensated FP32 sums over interleaved columns, combined in FP64."""
    s = np.zeros(4, dtype=np.float32)
    e = np.zeros(4, dtype=np.float32)
    n4 = len(v) - len(v) % 4
    for c in range(0, n4, 4):
        for u in range(4):
            x = np.float32(v[c + u])
            y = np.float32(np.float32(x * x) - e[u])     # the kernel fuses x*x - e in one fma
            t = np.float32(s[u] + y)
            e[u] = np.float32(np.float32(t - s[u]) - y)
            s[u] = t
    for c in range(n4, len(v)):
        x = np.float32(v[c])
        y = np.float32(np.float32(x * x) - e[0])
        t = np.float32(s[0] + y)
        e[0] = np.float32(np.float32(t - s[0]) - y)
        s[0] = t
    return float(np.sum(s.astype(np.float64) - e.astype(np.float64)))


def test_compensated_row_sums_keep_fp32_accuracy():
    rng = np.random.default_rng(5)
    for cols in (3, 64, 511, 2048):
        v = (rng.normal(size=cols) * np.exp(rng.normal(size=cols))).astype(np.float32)
        exact = float(np.sum(v.astype(np.float64) ** 2))
        assert abs(kahan4(v) - exact) <= 4 * 2.0 ** -24 * exact


def test_epoch_tag_changes_a_word_by_at_most_three_ulps():
    rng = np.random.default_rng(6)
    x = rng.normal(size=1000) * 10.0 ** rng.integers(-200, 200, 1000)
    bits = x.view(np.int64)
    for ep in range(4):
        tagged = ((bits & ~np.int64(3)) | np.int64(ep)).view(np.float64)
        assert np.all(np.abs(tagged - x) <= 3 * np.spacing(np.abs(x)))
        assert np.all((tagged.view(np.int64) & 3) == ep)
