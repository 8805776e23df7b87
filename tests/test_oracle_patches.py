"""Pins of the oracle's fine-grained (per-patch) contact field (Sec. 4.4) and
the dependency-group merge of Sec. 5.3.  A patch is the surface points of one
link; the field of a finger is the union of its patches' fields, so the union
of a finger's patch codes must be exactly the finger field's codes, and the OR
of its patch domains exactly its domain (checked against the per-finger field,
itself pinned by the literal brute-force check)."""
import numpy as np

import oracle
import synth


def _sets(c):
    return set(map(tuple, np.asarray(c).tolist()))


def test_patch_codes_partition_the_finger_field():
    w = synth.workload("hand16_superquadric", P=2, S=512)
    pf = oracle.PatchFields(w.hand, w.q, w.inv_h, w.bins)
    fd = oracle.Field(w.hand, w.q, w.inv_h, w.bins)
    assert len(pf.slots) == 12  # 4 fingers x 3 links with surface points (the abduction link has none)
    assert [f for f, _ in pf.slots] == sorted(f for f, _ in pf.slots)
    for f in range(w.hand.F):
        union = set()
        for s, (ff, link) in enumerate(pf.slots):
            if ff == f:
                assert np.any(w.hand.surf_link[f] == link)
                union |= _sets(pf.codes(s))
        assert union == _sets(fd.codes(f))


def test_merged_patch_domains_equal_the_finger_domains():
    w = synth.workload("tiny_sphere", P=6, S=1024)
    pf = oracle.PatchFields(w.hand, w.q, w.inv_h, w.bins)
    fd = oracle.Field(w.hand, w.q, w.inv_h, w.bins)
    soa = w.obj.soa()
    pm, pc = pf.query(soa, w.poses)
    assert pm.shape[1] == len(pf.slots) == 9
    merged, mc = pf.merge(pm)
    m, c = fd.query(soa, w.poses)
    assert np.array_equal(merged, m)
    assert np.array_equal(mc, c)
    # a patch's domain lies inside its finger's domain; every finger hit comes from at least one patch
    for s, (f, _) in enumerate(pf.slots):
        assert np.all(pm[:, s] & ~m[:, f] == 0)
    assert c.sum() > 0 and pc.sum() >= c.sum()


def test_patch_query_against_brute_force_of_one_link():
    """One patch's domain by the literal existential check over that link's samples only."""
    w = synth.workload("tiny_sphere", P=2, N=256, S=256)
    pf = oracle.PatchFields(w.hand, w.q, w.inv_h, w.bins)
    soa = w.obj.soa()
    pm, _ = pf.query(soa, w.poses)
    for s in (0, 4, 8):
        f, link = pf.slots[s]
        sub = oracle._SubHand(w.hand, f, link)
        brute = oracle.query_masks_brute(sub, w.q[f:f + 1], w.inv_h, w.bins, soa, w.poses)
        assert np.array_equal(brute[:, 0], pm[:, s])
