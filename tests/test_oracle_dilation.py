"""Pins of theta-dilated bins (the leaf normal test -x^T n >= theta_hit of
Sec. 4.3 read as "the cell holds a bin within theta of the query's bin"):
no dilation = the same-bin test, full dilation = the cell-occupancy test,
masks grow with the angle, and the indexed query equals the literal
existential check."""
import math

import numpy as np
import pytest

import oracle
import synth


@pytest.fixture(scope="module")
def small():
    w = synth.workload("tiny_sphere", P=6, S=512)
    return w, w.obj.soa()


def _deg_between_levels(bins, target_deg):
    """A dilation angle near target_deg that no pair of bins sits on."""
    d = bins.astype(np.float64)
    ang = np.unique(np.round(np.degrees(np.arccos(np.clip(d @ d.T, -1, 1))), 9))
    lo = ang[ang <= target_deg].max()
    hi = ang[ang > target_deg].min() if (ang > target_deg).any() else 180.0
    return float(np.float32(0.5 * (lo + hi)))


def test_dilation_masks_definition(small):
    w, _ = small
    assert np.array_equal(oracle.dilation_masks(w.bins, 0.0), np.uint32(1) << np.arange(w.B, dtype=np.uint32))
    full = oracle.dilation_masks(w.bins, 180.0)
    assert np.all(full == np.uint32((1 << w.B) - 1))
    deg = _deg_between_levels(w.bins, 80)
    m = oracle.dilation_masks(w.bins, deg)
    d = w.bins.astype(np.float64)
    for b in range(w.B):
        want = sum(1 << b2 for b2 in range(w.B) if np.degrees(np.arccos(np.clip(d[b] @ d[b2], -1, 1))) <= deg) | (1 << b)
        assert m[b] == want
        assert all(((m[b] >> b2) & 1) == ((m[b2] >> b) & 1) for b2 in range(w.B))  # symmetric


def test_no_and_full_dilation(small):
    w, soa = small
    base, _ = oracle.Field(w.hand, w.q, w.inv_h, w.bins).query(soa, w.poses)
    same, _ = oracle.Field(w.hand, w.q, w.inv_h, w.bins, dilate_deg=0.0).query(soa, w.poses)
    assert np.array_equal(base, same)
    fd = oracle.Field(w.hand, w.q, w.inv_h, w.bins, dilate_deg=180.0)
    full, _ = fd.query(soa, w.poses)
    # full dilation: a hit iff the finger's field occupies the cell at all
    pi = np.repeat(np.arange(w.P), w.obj.N)
    xi = np.tile(np.arange(w.obj.N), w.P)
    codes = oracle.point_codes(soa, w.poses, pi, xi, w.inv_h, w.bins)
    for f in range(w.hand.F):
        cells = set(map(tuple, fd.codes(f)[:, :3].tolist()))
        hit = np.array([tuple(c[:3]) in cells for c in codes.tolist()])
        bits = (full[pi, f, xi >> 5] >> (xi & 31)) & 1
        assert np.array_equal(hit, bits.astype(bool))


def test_dilation_monotone_and_brute_force(small):
    w, soa = small
    prev = None
    for deg in (20, 70, 110):
        c = _deg_between_levels(w.bins, deg)
        m, _ = oracle.Field(w.hand, w.q, w.inv_h, w.bins, dilate_deg=c).query(soa, w.poses)
        if prev is not None:
            assert np.all((prev & ~m) == 0)  # a wider angle only adds hits
            assert (m & ~prev).any()         # and past the bin spacing it does add some
        prev = m
    c = _deg_between_levels(w.bins, 70)
    q = np.ascontiguousarray(w.q[:, :, :64])
    idx, _ = oracle.Field(w.hand, q, w.inv_h, w.bins, dilate_deg=c).query(soa, w.poses[:2])
    brute = oracle.query_masks_brute(w.hand, q, w.inv_h, w.bins, soa, w.poses[:2], dilate_deg=c)
    assert np.array_equal(idx, brute)
    assert idx.any()
