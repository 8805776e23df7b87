"""Pins for the oracle's tuple sampling (Sec. 5.3: k domains of distinct
fingers chosen at random; Alg. 2: (p_i, n_i) <- Random(D_i))."""
import numpy as np

import oracle


def _draws(seed, i, tau, n):
    key = [seed & 0xFFFFFFFF, seed >> 32]
    out = []
    for blk in range((n + 3) // 4):
        out.extend(int(x) for x in oracle.philox4x32_10([i, tau, blk, 0], key))
    return out[:n]


def test_sampled_tuples_are_set_bits_of_distinct_nonempty_fingers():
    rng = np.random.default_rng(4)
    P, F, N, T, k = 20, 5, 300, 16, 3
    W = (N + 31) // 32
    bits = (rng.random((P, F, W * 32)) < 0.05)
    bits[:, :, N:] = False
    bits[3, :3] = False          # pose 3: only 2 non-empty fingers -> invalid tuples
    bits[5, 1] = False
    masks = np.packbits(bits, axis=2, bitorder="little").view(np.uint32).copy()
    counts = bits.sum(axis=2).astype(np.uint32)
    tup, fin = oracle.sample_tuples(masks, counts, N, T, k, seed=77)
    for i in range(P):
        nonempty = [f for f in range(F) if counts[i, f] > 0]
        for t in range(T):
            if len(nonempty) < k:
                assert (tup[i, t] == -1).all() and (fin[i, t] == 255).all()
                continue
            assert len(set(fin[i, t].tolist())) == k
            for d in range(k):
                f = int(fin[i, t, d])
                assert f in nonempty
                assert bits[i, f, tup[i, t, d]]


def test_sampling_follows_the_stated_draws():
    """Finger choice = partial Fisher-Yates with floor(u * m / 2^32); point = the
    r-th set bit with r = floor(u * count / 2^32) (numpy nonzero as the check)."""
    rng = np.random.default_rng(8)
    P, F, N, T, k, seed = 6, 4, 200, 10, 3, 2**40 + 5
    W = (N + 31) // 32
    bits = rng.random((P, F, W * 32)) < 0.1
    bits[:, :, N:] = False
    masks = np.packbits(bits, axis=2, bitorder="little").view(np.uint32).copy()
    counts = bits.sum(axis=2).astype(np.uint32)
    tup, fin = oracle.sample_tuples(masks, counts, N, T, k, seed)
    for i in range(P):
        nonempty = [f for f in range(F) if counts[i, f] > 0]
        m = len(nonempty)
        for t in range(T):
            u = _draws(seed, i, t, 2 * k)
            idx = list(nonempty)
            for d in range(k):
                j = d + (u[d] * (m - d) >> 32)
                idx[d], idx[j] = idx[j], idx[d]
            for d in range(k):
                f = idx[d]
                r = u[k + d] * int(counts[i, f]) >> 32
                assert fin[i, t, d] == f
                assert tup[i, t, d] == np.nonzero(bits[i, f])[0][r]


def test_rank_draw_is_uniform_over_a_domain():
    N, T = 64, 4000
    bits = np.zeros((1, 3, 64), bool)
    bits[0, 0, ::3] = True      # 22 points
    bits[0, 1, 5] = True
    bits[0, 2, 7] = True
    masks = np.packbits(bits, axis=2, bitorder="little").view(np.uint32).copy()
    counts = bits.sum(axis=2).astype(np.uint32)
    tup, fin = oracle.sample_tuples(masks, counts, N, T, 3, seed=3)
    pts = tup[0][fin[0] == 0]
    h = np.bincount(pts // 3, minlength=22)
    e = pts.size / 22
    assert ((h - e) ** 2 / e).sum() < 46.8  # chi-square df=21, 99.9%


def test_finger_choice_is_a_uniform_ordered_k_subset():
    """Sec. 5.3 draws k distinct fingers at random.  With all F = 5 domains
    non-empty, every ordered triple of distinct fingers has probability
    1 / (5 * 4 * 3).  A shuffle that swaps with any position (not only the
    not-yet-chosen ones) still yields distinct fingers but puts up to 2.4x the
    mass on some triples, which this chi-square test rejects."""
    P, F, N, T, k = 4, 5, 64, 2000, 3
    bits = np.zeros((P, F, 64), bool)
    bits[:, :, 0] = True
    masks = np.packbits(bits, axis=2, bitorder="little").view(np.uint32).copy()
    counts = bits.sum(axis=2).astype(np.uint32)
    _, fin = oracle.sample_tuples(masks, counts, N, T, k, seed=11)
    code = (fin[..., 0].astype(int) * F + fin[..., 1]) * F + fin[..., 2]
    h = np.bincount(code.ravel(), minlength=F ** 3)
    triples = [(a * F + b) * F + c for a in range(F) for b in range(F) for c in range(F)
               if len({a, b, c}) == 3]
    assert h.sum() == h[triples].sum() == P * T
    e = P * T / len(triples)
    assert ((h[triples] - e) ** 2 / e).sum() < 98.3  # chi-square df=59, 99.9%
